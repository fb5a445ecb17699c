"""The bench's full-size stereo workload against the FP64 oracle on sampled
outputs: 1024^3 u16 filaments (200 tubes, seed 1002), 64^3 bricks, 4
levels, table seed 2002 over the window [300, 60000], head poses of seed
3002 at 2 x 1440 x 1600, step 0.5, tau 1 px, rendered in the launch shape
the autotuner picks (as bench.py times it). The selection is compared bit
for bit over the whole octree; the image on every 97th pixel of both eyes
(about 47 500 rays); the sample counts on the same pixels of the render
without empty-space skipping, which must equal the skipping one bit for
bit. Then all 64 poses: selections bit for bit and every 16th pixel."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import GpuCase, compare_image, compare_selection

pytestmark = pytest.mark.gpu

N_VOX, BRICK, LEVELS = 1024, 64, 4
W_EYE, H_EYE = 1440, 1600
WINDOW = (300.0, 60000.0)


@pytest.fixture(scope="module")
def bench_case():
    vol = synth.filaments_u16((N_VOX,) * 3, seed=1002, ntubes=200)
    case = GpuCase([vol], BRICK, LEVELS, model=synth.volume_model(N_VOX, 0.5))
    del vol
    case.set_tfs([synth.tf_piecewise(2002, zero_alpha_points=2)], [WINDOW])
    yield case
    case.close()


@pytest.mark.parametrize("pose_index", [0, 37])
def test_full_size_stereo_frame_on_sampled_pixels(bench_case, pose_index, record_error):
    import torch
    from paper_1804_08197_b300 import sg
    case = bench_case
    views, projs = synth.head_poses(pose_index + 1, seed=3002, width=W_EYE, height=H_EYE)[pose_index]
    pose, stats, gsel, ref = case.select(views, projs, W_EYE, H_EYE, tau=1.0)
    compare_selection(gsel, ref)
    assert stats["selected"] == ref["selected"] and stats["selected"] > 0
    # the launch shape the bench times
    outs = [torch.empty((H_EYE, W_EYE, 4), dtype=torch.float32, device="cuda") for _ in range(2)]
    sg.sg_autotune_render(case.vol, [pose], sg.render_params(step=0.5), outs, reps=1)
    # empty-space skipping on (the bench's setting): images only, since the
    # jumps change which zero-alpha samples are counted; skipping off: the
    # sample counts too, and the two images agree bit for bit
    imgs, _ = case.render(pose, step=0.5, counts=False)
    plain, cnts = case.render(pose, step=0.5, empty_skip=0)
    npix = W_EYE * H_EYE
    for e in range(2):
        assert np.array_equal(imgs[e], plain[e])
        pix = np.arange(13 * e + pose_index % 97, npix, 97)
        oref = case.ovol.render(case.otfs, ref["leaf"], views[e], projs[e], W_EYE, H_EYE, step=0.5, pixels=pix)
        st = compare_image(imgs[e][pix], oref)
        assert st["n"] == len(pix)
        compare_image(plain[e][pix], oref, cnts[e][pix])
        # max |gpu - oracle| per RGBA channel over the sampled pixels with no
        # ambiguous lattice point and no termination tie
        keep = np.ones(len(pix), bool)
        keep[oref["var_idx"]] = False
        keep &= (oref["flags"] & oracle.FL_TERM) == 0
        ch = np.abs(imgs[e][pix][keep] - oref["late"][keep]).max(axis=0)
        record_error(f"eye {e} image", max_abs_err_rgba=[float(v) for v in ch],
                     max_err_termination_bracket=st["max_err_termination_bracket"],
                     max_abs_err_ambiguous=st["max_err_ambiguous"], ambiguous_fraction=st["ambiguous"],
                     termination_ties=st["termination_ties"], pixels=st["n"])


def test_every_bench_pose_on_a_sixteenth_of_the_pixels(bench_case, record_error):
    """All 64 bench poses: each pose's selection bit for bit over the whole
    octree, and every 16th pixel of both eyes (a different offset per pose
    and eye, 288 000 rays per eye) against the oracle's ray casting, in the
    launch shape the autotuner picks on the first pose."""
    import torch
    from paper_1804_08197_b300 import sg
    case = bench_case
    poses = synth.head_poses(64, seed=3002, width=W_EYE, height=H_EYE)
    outs = [torch.empty((H_EYE, W_EYE, 4), dtype=torch.float32, device="cuda") for _ in range(2)]
    npix = W_EYE * H_EYE
    worst = dict(max_err=0.0, max_err_termination_bracket=0.0, max_err_ambiguous=0.0)
    amb, ties, n = 0.0, 0, 0
    for i, (views, projs) in enumerate(poses):
        pose, stats, gsel, ref = case.select(views, projs, W_EYE, H_EYE, tau=1.0)
        compare_selection(gsel, ref)
        if i == 0:
            sg.sg_autotune_render(case.vol, [pose], sg.render_params(step=0.5), outs, reps=1)
        imgs, _ = case.render(pose, step=0.5, counts=False)
        for e in range(2):
            pix = np.arange((5 * i + 3 * e) % 16, npix, 16)
            oref = case.ovol.render(case.otfs, ref["leaf"], views[e], projs[e], W_EYE, H_EYE, step=0.5, pixels=pix)
            st = compare_image(imgs[e][pix], oref)
            assert st["n"] == len(pix)
            for k in worst:
                worst[k] = max(worst[k], st[k])
            amb = max(amb, st["ambiguous"])
            ties += st["termination_ties"]
            n += st["n"]
    record_error("64 poses x 2 eyes, every 16th pixel", **worst, ambiguous_fraction_max=amb,
                 termination_ties=ties, pixels=n)


def test_full_size_batched_4d_on_sampled_pixels(record_error):
    """The batched 4D workload at full size, as bench.py times it: 16 time
    points of 512 x 512 x 256 u16 with 2 channels (blob seed 1003, tables 2003
    / 2004 over [200, 40000], additive blend), 3 stereo viewers at 1440 x
    1600, 1080 x 1200 and 720 x 800 (seeds 3003-3005): 96 images selected and
    rendered in one persistent launch, captured in a CUDA graph and replayed,
    in the autotuned launch shape. For time points 0, 9 and 15 every viewer's
    selection matches the oracle bit for bit and every 211th pixel of each
    eye matches the oracle's ray casting."""
    import torch
    import oracle
    from paper_1804_08197_b300 import sg
    dims, T, res = (512, 512, 256), 16, [(1440, 1600), (1080, 1200), (720, 800)]
    model = synth.volume_model(max(dims), 0.5)
    tabs = [synth.tf_piecewise(2003, zero_alpha_points=2, colour=(0.1, 0.9, 0.2)),
            synth.tf_piecewise(2004, zero_alpha_points=2, colour=(0.9, 0.1, 0.8))]
    vol = sg.sg_volume_create(dims, sg.SG_U16, BRICK, LEVELS, channels=2, timepoints=T, model=model)
    try:
        data = {}
        for t in range(T):
            for c in range(2):
                a = synth.blobs_u16(dims, seed=1003, channel=c, t=t, nblobs=40)
                if t in (0, 9, 15):
                    data[(t, c)] = a
                d = torch.from_numpy(a.view(np.int16)).cuda()
                sg.sg_upload_volume_device(vol, t, c, d.data_ptr())
                torch.cuda.synchronize()
                del d
        for c in range(2):
            sg.sg_set_transfer_function(vol, c, tabs[c], 200.0, 40000.0)
        viewers = [synth.head_poses(1, seed=3003 + i, width=w, height=h)[0] for i, (w, h) in enumerate(res)]
        poses, outs = [], []
        for t in range(T):
            for i, (w, h) in enumerate(res):
                poses.append(sg.make_pose(*viewers[i], w, h, pixel_error=1.0, t=t, slot=t * 3 + i))
                outs += [torch.empty((h, w, 4), dtype=torch.float32, device="cuda") for _ in range(2)]
        stream = torch.cuda.Stream()
        prm = sg.render_params(step=0.5)
        sg.sg_select_lod_batch(vol, poses, stream=stream)
        sg.sg_autotune_render(vol, poses, prm, outs, reps=1, stream=stream)
        g = torch.cuda.CUDAGraph()
        for o in outs:
            o.fill_(-1.0)
        with torch.cuda.graph(g, stream=stream):
            sg.sg_select_lod_batch(vol, poses, stream=stream)
            sg.sg_render_batch(vol, poses, prm, outs, stream=stream)
        with torch.cuda.stream(stream):
            g.replay()
        torch.cuda.synchronize()
        otfs = [oracle.make_tf(tb, 200.0, 40000.0) for tb in tabs]
        worst, amb = 0.0, []
        for t in (0, 9, 15):
            ovol = oracle.Volume([oracle.pyramid(data[(t, c)], LEVELS) for c in range(2)], BRICK, model=model)
            ranges = ovol.block_ranges()
            nb0 = ovol.blocks_per_axis(0)
            for i, (w, h) in enumerate(res):
                views, projs = viewers[i]
                ref = ovol.select(otfs, views, projs, h, tau=1.0, ranges=ranges)
                compare_selection(sg.sg_read_selection(vol, t * 3 + i, nb0[0] * nb0[1] * nb0[2], ovol.node_count), ref)
                for e in range(2):
                    pix = np.arange(7 * e + t + i, w * h, 211)
                    oref = ovol.render(otfs, ref["leaf"], views[e], projs[e], w, h, step=0.5, pixels=pix)
                    img = outs[2 * (t * 3 + i) + e].cpu().numpy().reshape(-1, 4)
                    st = compare_image(img[pix], oref)
                    worst = max(worst, st["max_err"])
                    amb.append(st["ambiguous"])
        record_error("96 images (time points 0, 9, 15 sampled)", max_abs_err=worst,
                     ambiguous_fraction_mean=float(np.mean(amb)))
    finally:
        sg.sg_volume_destroy(vol)


def test_full_size_learned_forward_on_sampled_crops(record_error):
    """The learned reconstruction's network at the bench's size (both eyes of
    720 x 800 -> 1440 x 1600, the persistent tcgen05 convolution over 1200
    tiles per layer) against the FP64 network oracle on sampled crops. The
    network is local: an output farther than its receptive radius (under 28
    input pixels: 3x3 convolutions at three levels, two 2x2 pools, two 2x
    upsamplings) from a crop's edge is the same computed on the crop or on
    the whole image, when the crop keeps the pooling grid (origin a multiple
    of 4). The oracle runs its BF16 network on 96 x 96 crops; their centres
    (and, for a corner crop, the region along the image edges) must match
    element by element within 8 sigma (the per-element spread of an
    FP32-accumulating implementation, from the oracle)."""
    import torch
    import oracle.unet as ou
    from paper_1804_08197_b300 import sg
    h, w, R, C = 800, 720, 28, 96
    net = sg.sg_unet_create(2, h, w, seed=41)
    try:
        rng = np.random.default_rng(42)
        p = np.zeros(ou.param_count(), np.float32)
        for (ws, bs), ci in zip(ou.layer_slices(), ou.CIN):
            p[ws] = rng.normal(0, np.sqrt(2.0 / (9 * ci)), ws.stop - ws.start)
            p[bs] = rng.normal(0, 0.05, bs.stop - bs.start)
        ws0, _ = ou.layer_slices()[0]
        p[ws0].reshape(32, 9, 16)[:, :, 4:] = 0  # padding input channels
        sg.sg_unet_set_params(net, p)
        x = rng.uniform(0, 1, (2, h, w, 4)).astype(np.float32)
        xin = [torch.from_numpy(np.ascontiguousarray(x[i])).cuda() for i in range(2)]
        out = [torch.zeros((2 * h, 2 * w, 4), device="cuda") for _ in range(2)]
        sg.sg_unet_forward(net, xin, w * 4, h, w, out, 2 * w * 4)
        torch.cuda.synchronize()
        sg.sg_unet_check(net)
        gpu = np.stack([o.cpu().numpy() for o in out]).astype(np.float64)
        q = p.astype(np.float64).copy()
        for ws, _ in ou.layer_slices():
            q[ws] = torch.from_numpy(p[ws]).to(torch.bfloat16).to(torch.float64).numpy()
        # (image, crop origin y, x, valid rows / columns of the crop in input pixels)
        crops = [(0, 352, 312, (R, C - R), (R, C - R)), (1, 100, 600, (R, C - R), (R, C - R)),
                 (1, 704, 204, (R, C - R), (R, C - R)), (0, 0, 0, (0, C - R), (0, C - R))]
        worst = dict(max_abs_err=0.0, max_sigma_ratio=0.0, n=0)
        for n, y0, x0, (ya, yb), (xa, xb) in crops:
            xc = x[n:n + 1, y0:y0 + C, x0:x0 + C].astype(np.float64)
            ref, sig = ou.bf16_forward(q, xc)
            sl = (slice(2 * ya, 2 * yb), slice(2 * xa, 2 * xb))
            g = gpu[n, 2 * y0:2 * y0 + 2 * C, 2 * x0:2 * x0 + 2 * C][sl]
            err = np.abs(g - ref[0][sl])
            ratio = err / sig[0][sl]
            assert (ratio <= 8.0).all(), ((n, y0, x0), int((ratio > 8.0).sum()), ratio.max())
            worst = dict(max_abs_err=max(worst["max_abs_err"], err.max()),
                         max_sigma_ratio=max(worst["max_sigma_ratio"], ratio.max()), n=worst["n"] + err.size)
        record_error("output (4 crops of 2 x 720 x 800)", **worst)
    finally:
        sg.sg_unet_destroy(net)
