"""The bench's full-size stereo workload against the FP64 oracle on sampled
outputs: 1024^3 u16 filaments (200 tubes, seed 1002), 64^3 bricks, 4
levels, table seed 2002 over the window [300, 60000], head poses of seed
3002 at 2 x 1440 x 1600, step 0.5, tau 1 px, rendered in the launch shape
the autotuner picks (as bench.py times it). The selection is compared bit
for bit over the whole octree; the image on every 97th pixel of both eyes
(about 47 500 rays); the sample counts on the same pixels of the render
without empty-space skipping, which must equal the skipping one bit for
bit."""
import numpy as np
import pytest

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
def test_full_size_stereo_frame_on_sampled_pixels(bench_case, pose_index):
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


def test_full_size_batched_4d_on_sampled_pixels():
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
                    compare_image(img[pix], oref)
    finally:
        sg.sg_volume_destroy(vol)
