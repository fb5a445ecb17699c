"""Batched rendering: several poses with uneven image sizes in one launch
(one CTA per tile or a persistent tile queue, every supported tile shape),
the project's autotuner, and capture of select + render in a CUDA graph. The
batched images must equal the per-pose renders bit for bit (same per-ray
arithmetic), and the per-pose renders are pinned to the oracle elsewhere."""
import numpy as np
import pytest

import synth
from parity_util import GpuCase, compare_image, compare_selection

pytestmark = pytest.mark.gpu

SIZES = [(144, 160), (108, 120), (72, 80)]


def _case():
    a = synth.blobs_u16((96, 96, 48), seed=1003, channel=0, t=0, nblobs=12)
    b = synth.blobs_u16((96, 96, 48), seed=1003, channel=1, t=0, nblobs=12)
    case = GpuCase([a, b], 16, 3, model=synth.volume_model(96, 0.5))
    case.set_tfs([synth.tf_piecewise(2003, zero_alpha_points=2, colour=(0.1, 0.9, 0.2)),
                  synth.tf_piecewise(2004, zero_alpha_points=2, colour=(0.9, 0.1, 0.8))],
                 [(200.0, 40000.0), (200.0, 40000.0)])
    return case


def _poses(case):
    sg = case.sg
    out = []
    for i, (W, H) in enumerate(SIZES):
        (views, projs), = synth.head_poses(1, seed=3400 + i, extent_m=0.5, width=W, height=H)
        out.append((sg.make_pose(views, projs, W, H, pixel_error=0.5, slot=i), views, projs))
    return out


def _singles(case, poses):
    torch, sg = case.torch, case.sg
    ref = []
    for p, _, _ in poses:
        sg.sg_select_lod(case.vol, p)
        o = [torch.empty((p.height, p.width, 4), device="cuda") for _ in range(2)]
        sg.sg_render(case.vol, p, sg.render_params(), o)
        ref += o
    torch.cuda.synchronize()
    return [r.cpu().numpy() for r in ref]


def test_batch_equals_single_renders_for_every_config():
    case = _case()
    try:
        torch, sg = case.torch, case.sg
        poses = _poses(case)
        ref = _singles(case, poses)
        # the per-pose renders themselves match the oracle
        p, views, projs = poses[0]
        _, _, gsel, oref = case.select(views, projs, p.width, p.height, tau=0.5, slot=7)
        compare_selection(gsel, oref)
        compare_image(ref[0].reshape(-1, 4),
                      case.oracle_render(oref["leaf"], views[0], projs[0], p.width, p.height))
        sg.sg_select_lod_batch(case.vol, [q for q, _, _ in poses])
        shapes = [(16, 8, 1), (8, 16, 1), (32, 4, 1), (8, 8, 1), (16, 16, 2), (32, 8, 2)]
        for persistent in (0, 1):
            for tw, th, rpt in shapes:
                sg.sg_set_render_config(case.vol, persistent, tw, th, rpt)
                outs = [torch.full((q.height, q.width, 4), -1.0, device="cuda") for q, _, _ in poses for _ in range(2)]
                sg.sg_render_batch(case.vol, [q for q, _, _ in poses], sg.render_params(), outs)
                torch.cuda.synchronize()
                for o, r in zip(outs, ref):
                    assert np.array_equal(o.cpu().numpy(), r), (persistent, tw, th, rpt)
        sg.sg_set_render_config(case.vol)  # back to the default kernel
        with pytest.raises(sg.SGError):
            sg.sg_set_render_config(case.vol, 1, 24, 8, 1)
    finally:
        case.close()


def test_autotuner_keeps_the_fastest_config_and_output():
    case = _case()
    try:
        torch, sg = case.torch, case.sg
        poses = _poses(case)
        ref = _singles(case, poses)
        sg.sg_select_lod_batch(case.vol, [q for q, _, _ in poses])
        outs = [torch.empty((q.height, q.width, 4), device="cuda") for q, _, _ in poses for _ in range(2)]
        best, ms = sg.sg_autotune_render(case.vol, [q for q, _, _ in poses], sg.render_params(), outs, reps=2)
        assert ms > 0 and best["tile_w"] > 0 and sg.sg_get_render_config(case.vol) == best
        sg.sg_render_batch(case.vol, [q for q, _, _ in poses], sg.render_params(), outs)
        torch.cuda.synchronize()
        for o, r in zip(outs, ref):
            assert np.array_equal(o.cpu().numpy(), r)
    finally:
        case.close()


def test_select_and_batched_render_replay_in_a_cuda_graph():
    case = _case()
    try:
        torch, sg = case.torch, case.sg
        poses = _poses(case)
        ref = _singles(case, poses)
        sg.sg_set_render_config(case.vol, 1, 16, 8, 1)
        plist = [q for q, _, _ in poses]
        outs = [torch.zeros((q.height, q.width, 4), device="cuda") for q in plist for _ in range(2)]
        prm = sg.render_params()
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):  # warm-up outside the capture (tables built once)
            sg.sg_select_lod_batch(case.vol, plist, stream=s)
            sg.sg_render_batch(case.vol, plist, prm, outs, stream=s)
        torch.cuda.synchronize()
        for o in outs:
            o.zero_()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            sg.sg_select_lod_batch(case.vol, plist, stream=s)
            sg.sg_render_batch(case.vol, plist, prm, outs, stream=s)
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        for o, r in zip(outs, ref):
            assert np.array_equal(o.cpu().numpy(), r)
    finally:
        case.close()


def test_time_points_are_independent_volumes():
    """3D movies: pose.t picks the time point; each matches the oracle of its own data."""
    import torch
    import oracle
    from paper_1804_08197_b300 import sg
    dims = (80, 64, 48)
    model = synth.volume_model(80, 0.5)
    vol = sg.sg_volume_create(dims, sg.SG_U16, 16, 3, timepoints=3, model=model)
    try:
        data = [synth.blobs_u16(dims, seed=1003, channel=0, t=t, nblobs=10) for t in range(3)]
        for t, a in enumerate(data):
            d = torch.from_numpy(a.view(np.int16)).cuda()
            sg.sg_upload_volume_device(vol, t, 0, d.data_ptr())
        table = synth.tf_piecewise(2003, zero_alpha_points=2)
        sg.sg_set_transfer_function(vol, 0, table, 200.0, 40000.0)
        W, H = 120, 128
        (views, projs), = synth.head_poses(1, seed=3700, extent_m=0.5, width=W, height=H)
        poses = [sg.make_pose(views, projs, W, H, pixel_error=0.5, t=t, slot=t) for t in range(3)]
        sg.sg_select_lod_batch(vol, poses)
        outs = [torch.empty((H, W, 4), device="cuda") for _ in range(6)]
        sg.sg_render_batch(vol, poses, sg.render_params(), outs)
        torch.cuda.synchronize()
        otf = oracle.make_tf(table, 200.0, 40000.0)
        for t in (0, 2):
            ov = oracle.Volume([oracle.pyramid(data[t], 3)], 16, model=model)
            ref = ov.select([otf], views, projs, H, tau=0.5)
            cells, _, _ = sg.sg_read_selection(vol, t, len(ref["leaf"]), ov.node_count)
            assert np.array_equal(cells, ref["leaf"])
            compare_image(outs[2 * t].cpu().numpy().reshape(-1, 4),
                          ov.render([otf], ref["leaf"], views[0], projs[0], W, H))
        assert not np.array_equal(outs[0].cpu().numpy(), outs[4].cpu().numpy())
    finally:
        sg.sg_volume_destroy(vol)
