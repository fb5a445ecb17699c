"""Pins of the FP64 network oracle: hand-derived gradients against central
finite differences, closed forms of the bilinear upsampling, and the
zero-head network being exactly that upsampling (CPU only)."""
import numpy as np
import pytest

import oracle.unet as ou


def _params(seed, scale=0.3, head=True):
    rng = np.random.default_rng(seed)
    p = np.zeros(ou.param_count())
    for (ws, bs), ci in zip(ou.layer_slices(), ou.CIN):
        p[ws] = rng.normal(0, scale * np.sqrt(2.0 / (9 * ci)), ws.stop - ws.start)
        p[bs] = rng.normal(0, 0.05, bs.stop - bs.start)
    if not head:
        ws, bs = ou.layer_slices()[-1]
        p[ws] = 0
        p[bs] = 0
    return p


def test_gradients_match_central_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, (1, 8, 8, 4))
    t = rng.uniform(0, 1, (1, 16, 16, 4))
    p = _params(2, scale=1.0)
    loss, g, _ = ou.loss_grad(p, x, t)
    eps = 1e-6
    checked = 0
    for L, (ws, bs) in enumerate(ou.layer_slices()):
        for idx in list(rng.integers(ws.start, ws.stop, 4)) + [bs.start]:
            q = p.copy()
            q[idx] += eps
            lp, _, _ = ou.loss_grad(q, x, t)
            q[idx] -= 2 * eps
            lm, _, _ = ou.loss_grad(q, x, t)
            fd = (lp - lm) / (2 * eps)
            assert g[idx] == pytest.approx(fd, rel=1e-4, abs=1e-9), (ou.NAMES[L], idx)
            checked += abs(fd) > 1e-9
    assert checked >= 20  # most sampled parameters influence the loss


def test_bilinear_reproduces_constants_and_interior_ramps():
    c = np.full((1, 6, 8, 4), 0.37)
    assert np.allclose(ou.bilinear2x(c), 0.37, atol=1e-15)
    # value a (x + 0.5) at half-res pixel x upsamples to a (X + 0.5) / 2 inside
    a = 0.01
    ramp = np.tile((a * (np.arange(8) + 0.5))[None, None, :, None], (1, 6, 1, 4))
    up = ou.bilinear2x(ramp)
    X = np.arange(16)
    assert np.allclose(up[0, 3, 1:15, 0], (a * (X + 0.5) / 2)[1:15], atol=1e-15)
    # edges clamp: the outermost full-res pixels take the edge values
    assert up[0, 0, 0, 0] == pytest.approx(ramp[0, 0, 0, 0])


def test_zero_head_network_is_the_bilinear_upsampling():
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (2, 8, 12, 4))
    out = ou.forward(_params(4, head=False), x)
    assert np.allclose(out, ou.bilinear2x(x), atol=1e-15)
