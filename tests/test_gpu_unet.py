"""Learned reconstruction on the GPU against the network oracle: every
output value and every weight and bias gradient of every convolution path
within 8 sigma of the BF16 network (sigma: the per-element spread of an
FP32-accumulating implementation, propagated by the oracle from the BF16
rounding points), the untrained (zero-head) network as exact bilinear
upsampling, the PSNR kernel's closed form, and a short training run that
must beat the method without the network."""
import numpy as np
import pytest

import oracle.unet as ou
import synth

pytestmark = pytest.mark.gpu


def _bf16(x):
    import torch
    return torch.from_numpy(np.asarray(x, np.float32)).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)


def _random_params(seed, n):
    rng = np.random.default_rng(seed)
    p = np.zeros(n, np.float32)
    for (ws, bs), ci in zip(ou.layer_slices(), ou.CIN):
        p[ws] = rng.normal(0, np.sqrt(2.0 / (9 * ci)), ws.stop - ws.start)
        p[bs] = rng.normal(0, 0.05, bs.stop - bs.start)
    ws, _ = ou.layer_slices()[0]
    w0 = p[ws].reshape(32, 9, 16)
    w0[:, :, 4:] = 0  # padding input channels
    return p


def _run(net, x, t=None):
    import torch
    from paper_1804_08197_b300 import sg
    N, h, w, _ = x.shape
    xin = [torch.from_numpy(np.ascontiguousarray(x[i], np.float32)).cuda() for i in range(N)]
    out = [torch.zeros((2 * h, 2 * w, 4), device="cuda") for _ in range(N)]
    sg.sg_unet_forward(net, xin, w * 4, h, w, out, 2 * w * 4)
    loss = None
    if t is not None:
        tt = [torch.from_numpy(np.ascontiguousarray(t[i], np.float32)).cuda() for i in range(N)]
        lb = torch.zeros(1, device="cuda")
        sg.sg_unet_backward(net, tt, 2 * w * 4, out, 2 * w * 4, loss=lb)
        torch.cuda.synchronize()
        loss = float(lb.item())
    torch.cuda.synchronize()
    return np.stack([o.cpu().numpy() for o in out]).astype(np.float64), loss


K = 8.0  # |gpu - oracle| <= K sigma, element by element


def _oracle_params(p):
    """the parameters as the tensor cores see them: BF16 weights, FP32 biases"""
    q = p.astype(np.float64).copy()
    for ws, _ in ou.layer_slices():
        q[ws] = _bf16(p[ws])
    return q


def check_elementwise(name, got, ref, sigma, record=None):
    """every element within K sigma; returns the achieved figures"""
    err = np.abs(np.asarray(got, np.float64) - ref)
    ratio = err / np.maximum(sigma, 1e-300)
    bad = ratio > K
    assert not bad.any(), (f"{name}: {int(bad.sum())} of {bad.size} elements beyond {K} sigma; worst "
                           f"{ratio.max():.2f} sigma (|err| {err.reshape(-1)[np.argmax(ratio)]:.3g})")
    fig = dict(max_abs_err=err.max(), max_sigma_ratio=ratio.max(), max_abs_ref=np.abs(ref).max(), n=err.size)
    if record:
        record(name, **fig)
    return fig


def check_network(gpu_out, gpu_loss, g_gpu, p, x, t, record=None, tag=""):
    """outputs, loss and every gradient against the BF16 network oracle"""
    q = _oracle_params(p)
    x32 = x.astype(np.float32).astype(np.float64)
    t32 = t.astype(np.float32).astype(np.float64)
    loss, g, sg, out, so = ou.bf16_loss_grad(q, x32, t32)
    check_elementwise(tag + "output", gpu_out, out, so, record)
    cnt = out.size
    sl = np.sqrt(np.sum((2.0 * (out - t32) * so / cnt) ** 2)) + 2.0 ** -23 * np.sqrt(cnt) * loss
    assert abs(gpu_loss - loss) <= K * sl, (gpu_loss, loss, sl)
    if record:
        record(tag + "loss", abs_err=abs(gpu_loss - loss), sigma=sl)
    for L, (ws, bs) in enumerate(ou.layer_slices()):
        check_elementwise(f"{tag}{ou.NAMES[L]}.dW", g_gpu[ws], g[ws], sg[ws], record)
        check_elementwise(f"{tag}{ou.NAMES[L]}.db", g_gpu[bs], g[bs], sg[bs], record)


def test_forward_and_gradients_match_the_oracle_element_by_element(record_error):
    from paper_1804_08197_b300 import sg
    net = sg.sg_unet_create(2, 16, 24, seed=3)
    try:
        n = sg.sg_unet_param_count(net)
        assert n == ou.param_count()
        p = _random_params(5, n)
        sg.sg_unet_set_params(net, p)
        rng = np.random.default_rng(7)
        x = rng.uniform(0, 1, (2, 16, 24, 4))
        t = rng.uniform(0, 1, (2, 32, 48, 4))
        gpu_out, gpu_loss = _run(net, x, t)
        sg.sg_unet_check(net)
        g_gpu = sg.sg_unet_get_params(net, which=1).astype(np.float64)
        check_network(gpu_out, gpu_loss, g_gpu, p, x, t, record_error)
    finally:
        sg.sg_unet_destroy(net)


def test_every_convolution_path_matches_the_oracle_element_by_element(record_error):
    """The tcgen05 paths (TMEM; implicit GEMM, halo reuse with cp.async or
    TMA row segments, the persistent warp-specialised kernel) and the
    mma.sync path compute the same BF16 products with FP32 sums in different
    orders: each is within 8 sigma of the BF16 network on every output and
    gradient. Two row segments of 128 pixels per row (140 columns)."""
    from paper_1804_08197_b300 import sg
    net = sg.sg_unet_create(2, 24, 140, seed=11)
    try:
        p = _random_params(12, sg.sg_unet_param_count(net))
        sg.sg_unet_set_params(net, p)
        rng = np.random.default_rng(13)
        x = rng.uniform(0, 1, (2, 24, 140, 4))
        t = rng.uniform(0, 1, (2, 48, 280, 4))
        res = {}
        for path in (0, 1, 2, 3, 4):
            sg.sg_unet_set_tensor_path(net, path)
            out, loss = _run(net, x, t)
            sg.sg_unet_check(net)
            res[path] = (out, loss, sg.sg_unet_get_params(net, which=1).astype(np.float64))
            check_network(out, loss, res[path][2], p, x, t, record_error if path == 4 else None, f"path{path}.")
        # TMA staging of the row segments moves the same bytes to the same
        # places: identical outputs to the cp.async halo path
        assert np.array_equal(res[3][0], res[2][0])
    finally:
        sg.sg_unet_destroy(net)


def test_persistent_convolution_over_many_tiles():
    """The persistent warp-specialised convolution walks several tiles per
    CTA (two TMEM accumulators in turn, the shared-memory ring wrapping
    within and across tiles); ragged rows and columns at every level: 404 x
    300 per image is 51 bands of 8 rows x 3 column segments (the last 44
    pixels wide) at full size, over 2 x 148 tiles in all. Outputs, loss and
    gradients agree with the mma.sync path to summation order."""
    from paper_1804_08197_b300 import sg
    net = sg.sg_unet_create(2, 404, 300, seed=21)
    try:
        p = _random_params(22, sg.sg_unet_param_count(net))
        sg.sg_unet_set_params(net, p)
        rng = np.random.default_rng(23)
        x = rng.uniform(0, 1, (2, 404, 300, 4))
        t = rng.uniform(0, 1, (2, 808, 600, 4))
        res = {}
        for path in (0, 4, 4):
            sg.sg_unet_set_tensor_path(net, path)
            out, loss = _run(net, x, t)
            sg.sg_unet_check(net)
            g = sg.sg_unet_get_params(net, which=1).astype(np.float64)
            if path in res:
                # a second run on the same inputs: the same products and sums
                assert np.array_equal(out, res[path][0])
            res[path] = (out, loss, g)
        base = ou.bilinear2x(x)
        r0, r1 = res[0][0] - base, res[4][0] - base
        assert np.linalg.norm(r1 - r0) <= 5e-3 * np.linalg.norm(r0)
        assert res[4][1] == pytest.approx(res[0][1], rel=1e-4)
        for ws, bs in ou.layer_slices():
            for sl in (ws, bs):
                g0, g1 = res[0][2][sl], res[4][2][sl]
                assert np.linalg.norm(g1 - g0) <= 2e-2 * np.linalg.norm(g0) + 1e-12
    finally:
        sg.sg_unet_destroy(net)


def test_tensor_core_weight_gradients_match_the_oracle_element_by_element(record_error):
    """With widths that are multiples of 8 at every level (32 x 64, 16 x 32,
    8 x 16) the weight and bias gradients run on tcgen05 (pixels as the
    contraction over transposed, row-padded operands, one TMEM accumulator
    per tap, pixel splits summed in a fixed order): every gradient is within
    8 sigma of the BF16 network's, for the tcgen05 and the mma.sync weight
    gradients alike, and repeats exactly on a second run."""
    from paper_1804_08197_b300 import sg
    net = sg.sg_unet_create(3, 32, 64, seed=31)
    try:
        p = _random_params(32, sg.sg_unet_param_count(net))
        sg.sg_unet_set_params(net, p)
        rng = np.random.default_rng(33)
        x = rng.uniform(0, 1, (3, 32, 64, 4))
        t = rng.uniform(0, 1, (3, 64, 128, 4))
        res = {}
        for path in (0, 4, 4):
            sg.sg_unet_set_tensor_path(net, path)
            out, loss = _run(net, x, t)
            sg.sg_unet_check(net)
            g = sg.sg_unet_get_params(net, which=1).astype(np.float64)
            if path in res:
                assert np.array_equal(g, res[path][1])
                continue
            res[path] = (loss, g)
            check_network(out, loss, g, p, x, t, record_error if path == 4 else None, f"wgrad_path{path}.")
    finally:
        sg.sg_unet_destroy(net)


def test_untrained_network_is_exactly_bilinear_upsampling():
    from paper_1804_08197_b300 import sg
    net = sg.sg_unet_create(3, 12, 20, seed=9)
    try:
        x = np.random.default_rng(2).uniform(0, 1, (3, 12, 20, 4))
        out, _ = _run(net, x)
        assert np.abs(out - ou.bilinear2x(x)).max() < 1e-6
    finally:
        sg.sg_unet_destroy(net)


def test_psnr_closed_form():
    import torch
    from paper_1804_08197_b300 import sg
    a = torch.zeros(1000, device="cuda")
    b = torch.full((1000,), 0.1, device="cuda")
    db = torch.zeros(1, device="cuda")
    sg.sg_psnr(a, b, 1000, db)
    assert float(db.item()) == pytest.approx(20.0, abs=1e-4)  # MSE 0.01
    b[:500] = 0.0
    sg.sg_psnr(a, b, 1000, db)
    assert float(db.item()) == pytest.approx(10 * np.log10(1 / 0.005), abs=1e-4)


def test_training_beats_the_method_without_the_network():
    import torch
    from paper_1804_08197_b300 import sg
    from paper_1804_08197_b300.learned import Learned
    dims = (192, 192, 192)
    a = synth.filaments_u16(dims, seed=41, ntubes=30)
    vol = sg.sg_volume_create(dims, sg.SG_U16, 32, 3, model=synth.volume_model(192, 0.5))
    try:
        d = torch.from_numpy(a.view(np.int16)).cuda()
        sg.sg_upload_volume_device(vol, 0, 0, d.data_ptr())
        sg.sg_set_transfer_function(vol, 0, synth.tf_piecewise(2002, zero_alpha_points=2), 300.0, 60000.0)
        W, H = 256, 288
        rec = Learned(vol, W, H, max_batch=8, crop=32, seed=5)
        try:
            train = synth.head_poses(40, seed=9100, width=W, height=H, dist=(0.35, 0.8))
            held = synth.head_poses(4, seed=9200, width=W, height=H, dist=(0.35, 0.8))
            before = [rec.evaluate(v, p) for v, p in held]
            for i in range(160):
                v, p = train[i % len(train)]
                rec.train_on_pair(v, p, steps=2, batch=8, lr=1e-3)
            after = [rec.evaluate(v, p) for v, p in held]
            assert np.mean(after) > np.mean(before) + 0.5, (before, after)
        finally:
            rec.close()
    finally:
        sg.sg_volume_destroy(vol)


def test_a_bounded_wait_that_runs_out_is_reported_and_the_context_survives():
    """Failure detection without a GPU fault: a wait on a barrier nothing
    arrives at gives up after its poll limit, raises the error word, and
    sg_unet_check reports SG_ERR_TIMEOUT once (then clears it). The CUDA
    context stays usable: a forward pass afterwards runs and checks clean."""
    import torch
    from paper_1804_08197_b300 import sg
    net = sg.sg_unet_create(1, 16, 32, seed=3)
    try:
        sg.sg_unet_check(net)  # clean to start with
        sg.sg_unet_wait_selftest(net, 4096)
        torch.cuda.synchronize()
        with pytest.raises(sg.SGError) as ei:
            sg.sg_unet_check(net)
        assert ei.value.status == sg.SG_ERR_TIMEOUT
        sg.sg_unet_check(net)  # reported once, then cleared
        x = [torch.rand((16, 32, 4), device="cuda")]
        out = [torch.zeros((32, 64, 4), device="cuda")]
        sg.sg_unet_forward(net, x, 32 * 4, 16, 32, out, 64 * 4)
        torch.cuda.synchronize()
        sg.sg_unet_check(net)
        assert torch.isfinite(out[0]).all()
    finally:
        sg.sg_unet_destroy(net)


def _learned_case(sg, torch, seed=41):
    dims = (192, 192, 192)
    a = synth.filaments_u16(dims, seed=seed, ntubes=30)
    vol = sg.sg_volume_create(dims, sg.SG_U16, 32, 3, model=synth.volume_model(192, 0.5))
    d = torch.from_numpy(a.view(np.int16)).cuda()
    sg.sg_upload_volume_device(vol, 0, 0, d.data_ptr())
    sg.sg_set_transfer_function(vol, 0, synth.tf_piecewise(2002, zero_alpha_points=2), 300.0, 60000.0)
    torch.cuda.synchronize()
    return vol


def test_learned_frame_is_the_reduced_render_through_the_network_and_judges_on_the_device():
    """sg_render_learned = select + render at half resolution and twice the
    step, then the network: identical to those calls made one by one. Judged,
    it writes the stereo PSNR 10 log10(1 / mean of the eyes' MSE) against the
    full-rate render (checked here from the downloaded images) and falls back
    to that render exactly when the PSNR is below the threshold."""
    import torch
    from paper_1804_08197_b300 import sg
    from paper_1804_08197_b300.learned import Learned
    vol = _learned_case(sg, torch)
    try:
        W, H = 256, 288
        rec = Learned(vol, W, H, max_batch=8, crop=32, seed=5)
        try:
            train = synth.head_poses(8, seed=9100, width=W, height=H, dist=(0.35, 0.8))
            for i in range(12):
                rec.train_on_pair(*train[i % 8], steps=2, batch=8, lr=1e-3)
            views, projs = synth.head_poses(1, seed=9200, width=W, height=H, dist=(0.35, 0.8))[0]
            # one by one
            rec.render_half(views, projs)
            rec.reconstruct()
            ref = [r.clone() for r in rec.recon]
            rec.render_full(views, projs)
            full = [f.clone() for f in rec.full]
            # one call, not judged: the same images
            for r in rec.recon:
                r.fill_(-1.0)
            rec.frame(views, projs)
            torch.cuda.synchronize()
            for e in range(2):
                assert torch.equal(rec.recon[e], ref[e])
            # judged: PSNR from the images, fallback both ways
            mse = [float(((ref[e].double() - full[e].double()) ** 2).mean()) for e in range(2)]
            want = 10 * np.log10(1.0 / np.mean(mse))
            for thr, falls in ((want - 1.0, False), (want + 1.0, True)):
                rec.frame(views, projs, judge=True, threshold_db=thr, index=3)
                torch.cuda.synchronize()
                got = rec.psnr_frames[3].cpu().numpy()
                assert got[2] == pytest.approx(want, abs=2e-3)
                assert got[0] == pytest.approx(10 * np.log10(1 / mse[0]), abs=2e-3)
                assert bool(rec.fell_back[3].item()) == falls
                for e in range(2):
                    assert torch.equal(rec.recon[e], full[e] if falls else ref[e])
        finally:
            rec.close()
    finally:
        sg.sg_volume_destroy(vol)


def test_checkpoint_resumes_training_exactly(tmp_path):
    """sg_unet_save / sg_unet_load carry the parameters, both Adam moments and
    the step: a network loaded from a checkpoint gives bit-identical outputs
    and, after one more identical training step, bit-identical parameters."""
    import torch
    from paper_1804_08197_b300 import sg
    a = sg.sg_unet_create(2, 16, 24, seed=3)
    b = sg.sg_unet_create(2, 16, 24, seed=99)
    try:
        rng = np.random.default_rng(7)
        x = rng.uniform(0, 1, (2, 16, 24, 4))
        t = rng.uniform(0, 1, (2, 32, 48, 4))
        for _ in range(3):
            _run(a, x, t)
            sg.sg_unet_adam_step(a, 1e-3)
        path = tmp_path / "net.ckpt"
        sg.sg_unet_save(a, path)
        sg.sg_unet_load(b, path)
        oa, la = _run(a, x, t)
        ob, lb = _run(b, x, t)
        assert np.array_equal(oa, ob) and lb == pytest.approx(la, rel=1e-6)  # the loss sums with atomics
        sg.sg_unet_adam_step(a, 1e-3)
        sg.sg_unet_adam_step(b, 1e-3)
        torch.cuda.synchronize()
        pa = sg.sg_unet_get_params(a, which=0)
        pb = sg.sg_unet_get_params(b, which=0)
        assert np.array_equal(pa, pb)
        # a file of another shape or a truncated one is refused
        open(tmp_path / "short.ckpt", "wb").write(open(path, "rb").read()[:1000])
        with pytest.raises(sg.SGError):
            sg.sg_unet_load(b, tmp_path / "short.ckpt")
    finally:
        sg.sg_unet_destroy(a)
        sg.sg_unet_destroy(b)
