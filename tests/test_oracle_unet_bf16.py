"""Pins of the BF16 network oracle and of its per-element spread (CPU only).

The learned path's precision is fixed (BF16 weights and activations, FP32
accumulation); the oracle computes that network exactly (FP64 sums, BF16
rounding at the same points) and, per element, the standard deviation sigma
of how far an implementation that accumulates in FP32 in another order may
lie from it (accumulation noise, and the BF16 rounding flips it causes near
rounding boundaries). Pinned here: the rounding against torch's BF16
conversion; the BF16 network against the finite-difference-pinned FP64
network (they differ only by BF16 rounding); and sigma against an
independent float32 implementation (numpy im2col GEMMs, another summation
order) that must stay within 8 sigma everywhere, while the same
implementation with one planted mistake must not."""
import numpy as np
import pytest
import torch

import oracle.unet as ou


def _tbf16(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


def _params(seed):
    rng = np.random.default_rng(seed)
    p = np.zeros(ou.param_count(), np.float32)
    for (ws, bs), ci in zip(ou.layer_slices(), ou.CIN):
        p[ws] = rng.normal(0, np.sqrt(2.0 / (9 * ci)), ws.stop - ws.start)
        p[bs] = rng.normal(0, 0.05, bs.stop - bs.start)
    ws, _ = ou.layer_slices()[0]
    p[ws].reshape(32, 9, 16)[:, :, 4:] = 0
    q = p.astype(np.float64)
    for ws, _ in ou.layer_slices():
        q[ws] = _tbf16(p[ws])  # the weights the implementation multiplies with
    return q


def test_rounding_matches_torch_bf16():
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.normal(0, 1, 20000), rng.normal(0, 1e-30, 2000), rng.normal(0, 1e30, 2000)])
    v = v.astype(np.float32)
    # exact ties: values halfway between two BF16 neighbours
    b = _tbf16(rng.normal(0, 1, 2000))
    ties = (b.view(np.uint32) + np.uint32(0x8000)).view(np.float32)
    v = np.concatenate([v, ties, np.float32([1e-40, -3e-39, 0.0])])
    assert np.array_equal(ou.bf16(v.astype(np.float64)), _tbf16(v).astype(np.float64))


def _conv(x, w, b, relu, rnd):
    """float32 conv3x3 (zero padding) by im2col + GEMM: w [Cout][9][Cin]."""
    N, H, W, C = x.shape
    xp = np.zeros((N, H + 2, W + 2, C), np.float32)
    xp[:, 1:-1, 1:-1] = x
    cols = np.concatenate([xp[:, dy:dy + H, dx:dx + W] for dy in range(3) for dx in range(3)], axis=3)
    Cout = w.shape[0]
    y = cols.reshape(-1, 9 * C) @ w.reshape(Cout, 9 * C).T.astype(np.float32) + b.astype(np.float32)
    y = y.reshape(N, H, W, Cout)
    if relu:
        y = np.maximum(y, 0)
    return _tbf16(y) if rnd else y


def _np_forward(q, x, bug=None):
    ls = ou.layer_slices()
    W = [q[ws].reshape(co, 9, ci).astype(np.float32) for (ws, _), ci, co in zip(ls, ou.CIN, ou.COUT)]
    Bv = [q[bs].astype(np.float32) for _, bs in ls]
    N, h, w, _ = x.shape
    xin = np.zeros((N, h, w, 16), np.float32)
    xin[..., :4] = _tbf16(x)
    pool = lambda a: _tbf16((a[:, 0::2, 0::2] + a[:, 0::2, 1::2] + a[:, 1::2, 0::2] + a[:, 1::2, 1::2]) * 0.25)
    up = lambda a: a.repeat(2, axis=1).repeat(2, axis=2)
    a1 = _conv(xin, W[0], Bv[0], 1, 1)
    e1 = _conv(a1, W[1], Bv[1], 1, 1)
    if bug == "row":
        e1 = e1.copy()
        e1[:, 3] = 0  # a lost row of one activation
    a2 = _conv(pool(e1), W[2], Bv[2], 1, 1)
    e2 = _conv(a2, W[3], Bv[3], 1, 1)
    a3 = _conv(pool(e2), W[4], Bv[4], 1, 1)
    b3 = _conv(a3, W[5], Bv[5], 1, 1)
    a4 = _conv(np.concatenate([up(b3), e2], 3), W[6], Bv[6], 1, 1)
    d2 = _conv(a4, W[7], Bv[7], 1, 1)
    a5 = _conv(np.concatenate([up(d2), e1], 3), W[8], Bv[8], 1, 1)
    d1 = _conv(a5, W[9], Bv[9], 1, 1)
    head = _conv(d1, W[10], Bv[10], 0, 0)
    out = ou.bilinear2x(x.astype(np.float32).astype(np.float64)).astype(np.float32)
    for c in range(4):
        for dy in range(2):
            for dx in range(2):
                out[:, dy::2, dx::2, c] += head[..., 4 * c + 2 * dy + dx]
    return out.astype(np.float64)


K = 8.0  # the tests' acceptance: |impl - oracle| <= K sigma


@pytest.fixture(scope="module")
def net():
    q = _params(5)
    rng = np.random.default_rng(7)
    x = rng.uniform(0, 1, (2, 16, 24, 4)).astype(np.float32).astype(np.float64)
    out, sigma = ou.bf16_forward(q, x)
    return q, x, out, sigma


def test_an_independent_float32_implementation_stays_within_8_sigma(net):
    q, x, out, sigma = net
    impl = _np_forward(q, x)
    ratio = np.abs(impl - out) / sigma
    assert ratio.max() <= K, f"{np.count_nonzero(ratio > K)} outputs beyond {K} sigma; worst {ratio.max():.2f}"
    # sigma reflects the BF16 rounding noise: well below a BF16 step of the
    # outputs (about 2e-3 at 0.5), and the implementation does differ
    assert np.median(sigma) < 2e-3 and ratio.max() > 0.5


def _planted(q, kind, L):
    q = q.copy()
    ws, bs = ou.layer_slices()[L]
    W = q[ws].reshape(ou.COUT[L], 9, ou.CIN[L])
    if kind == "bias":
        q[bs] *= 1.1
    elif kind == "channel":
        W[3] = 0
    elif kind == "tap":
        W[:, 4, :] *= 0.9
    return q


@pytest.mark.parametrize("kind,L", [("row", 0), ("bias", 1), ("bias", 7), ("bias", 10), ("channel", 9),
                                    ("tap", 2), ("tap", 6)])
def test_a_planted_mistake_leaves_8_sigma(net, kind, L):
    """A lost row of one activation, a bias 10% off, a zeroed output channel,
    the centre tap's weights 10% off: each puts many outputs beyond 8 sigma."""
    q, x, out, sigma = net
    impl = _np_forward(q, x, bug="row") if kind == "row" else _np_forward(_planted(q, kind, L), x)
    assert (np.abs(impl - out) > K * sigma).sum() > 10


def test_the_bf16_network_is_the_fp64_network_up_to_bf16_rounding(net):
    """Same loops in FP64, BF16 rounding at the activations: the outputs'
    residuals and every gradient agree with the FP64 network to a few BF16
    steps (relative 2e-2 / 5e-2), and the loss to 1e-2."""
    q, x, _, _ = net
    rng = np.random.default_rng(9)
    t = rng.uniform(0, 1, (2, 32, 48, 4))
    loss16, g16, eg16, out16, _ = ou.bf16_loss_grad(q, x, t)
    loss, g, out = ou.loss_grad(q, x, t)
    base = ou.bilinear2x(x)
    assert np.linalg.norm((out16 - base) - (out - base)) <= 2e-2 * np.linalg.norm(out - base)
    assert loss16 == pytest.approx(loss, rel=1e-2)
    for ws, bs in ou.layer_slices():
        for sl in (ws, bs):
            assert np.linalg.norm(g16[sl] - g[sl]) <= 5e-2 * np.linalg.norm(g[sl]) + 1e-12
    assert (eg16 >= 0).all() and np.isfinite(eg16).all()


def test_zero_head_bf16_network_is_the_bilinear_upsampling():
    q = _params(4)
    ws, bs = ou.layer_slices()[-1]
    q[ws] = 0
    q[bs] = 0
    x = np.random.default_rng(3).uniform(0, 1, (1, 8, 12, 4)).astype(np.float32).astype(np.float64)
    out, sigma = ou.bf16_forward(q, x)
    assert np.array_equal(out, ou.bilinear2x(x)) and sigma.max() < 1e-6
