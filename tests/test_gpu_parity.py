"""GPU parity through the C ABI against the FP64 oracle on seeded inputs:
bit-exact bricks and selections, images within 1e-3, sample counts, empty
skipping that changes nothing, ragged and degenerate sizes."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import GpuCase, compare_image, compare_selection

pytestmark = pytest.mark.gpu


def _c1_case():
    v = synth.gaussians_u8(128, seed=1001)
    case = GpuCase([v], 128, 1)
    case.set_tfs([synth.tf_piecewise(2001)], [(0.0, 255.0)])
    return case


def test_plain_ray_cast_single_view_matches_oracle(record_error):
    """128^3 uint8 Gaussians, one 256x256 view, step 0.5 (the plain single-view case)."""
    case = _c1_case()
    try:
        view, proj = synth.orbit_camera(128, seed=3001, width=256, height=256)
        pose, stats, gsel, ref = case.select([view, view], [proj, proj], 256, 256)
        compare_selection(gsel, ref)
        imgs, cnts = case.render(pose, empty_skip=0)
        oref = case.oracle_render(ref["leaf"], view, proj, 256, 256)
        st = compare_image(imgs[0], oref, cnts[0])
        record_error("image 256 x 256", **st)
        assert np.array_equal(imgs[0], imgs[1])  # both eyes share the view
        assert oref["late"][:, 3].max() > 0.5
        skip, _ = case.render(pose, empty_skip=1)
        assert np.array_equal(skip[0], imgs[0])
    finally:
        case.close()


def _filament_case(dims=(256, 256, 256), brick=32, levels=4, seed=1002, ntubes=40):
    v = synth.filaments_u16(dims, seed=seed, ntubes=ntubes)
    model = synth.volume_model(max(dims), 0.5)
    case = GpuCase([v], brick, levels, model=model)
    case.set_tfs([synth.tf_piecewise(2002, zero_alpha_points=2)], [(300.0, 60000.0)])
    return case


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_multilod_stereo_pair_matches_oracle(seed, record_error):
    case = _filament_case()
    try:
        W, H = 360, 400
        (views, projs), = synth.head_poses(1, seed=3100 + seed, extent_m=0.5, width=W, height=H)
        # tau scaled so that a 360x400 image selects as a 1440x1600 one would
        pose, stats, gsel, ref = case.select(views, projs, W, H, tau=0.25)
        compare_selection(gsel, ref)
        levels = {case.ovol.node_coords(i)[0] for i in np.flatnonzero(ref["state"] == oracle.ST_SELECTED)}
        assert stats["selected"] == ref["selected"]
        imgs, cnts = case.render(pose, empty_skip=0)
        for e in range(2):
            oref = case.oracle_render(ref["leaf"], views[e], projs[e], W, H)
            st = compare_image(imgs[e], oref, cnts[e])
            record_error(f"eye {e} image", **st)
        skip, _ = case.render(pose, empty_skip=1)
        assert np.array_equal(skip[0], imgs[0]) and np.array_equal(skip[1], imgs[1])
        assert len(levels) >= 1
    finally:
        case.close()


def test_ragged_volume_and_image_sizes():
    case = _filament_case(dims=(200, 150, 97), brick=16, levels=3, ntubes=15)
    try:
        W, H = 211, 97
        (views, projs), = synth.head_poses(1, seed=3200, extent_m=0.5, width=W, height=H)
        pose, _, gsel, ref = case.select(views, projs, W, H, tau=0.5)
        compare_selection(gsel, ref)
        imgs, cnts = case.render(pose, empty_skip=1)
        for e in range(2):
            oref = case.oracle_render(ref["leaf"], views[e], projs[e], W, H)
            compare_image(imgs[e], oref)
    finally:
        case.close()


def test_bricks_hold_the_box_filtered_pyramid_with_aprons():
    rng = np.random.default_rng(5)
    a = rng.integers(0, 60000, (37, 45, 70)).astype(np.uint16)  # z, y, x: ragged on every axis
    case = GpuCase([a], 16, 3)
    try:
        B = 16
        R = B + 2
        for L in range(3):
            g = case.ovol.channels[0][L]
            nbx, nby, nbz = case.ovol.blocks_per_axis(L)
            for bz in range(nbz):
                for by in range(nby):
                    for bx in range(nbx):
                        out = np.empty((R, R, R), np.uint16)
                        case.sg.sg_read_brick(case.vol, 0, 0, L, bx, by, bz, out)
                        iz = np.clip(np.arange(R) + bz * B - 1, 0, g.shape[0] - 1)
                        iy = np.clip(np.arange(R) + by * B - 1, 0, g.shape[1] - 1)
                        ix = np.clip(np.arange(R) + bx * B - 1, 0, g.shape[2] - 1)
                        assert np.array_equal(out, g[np.ix_(iz, iy, ix)]), (L, bx, by, bz)
    finally:
        case.close()


def test_tiny_and_empty_volumes():
    # 5x3x2 voxels, one brick per level, 1x1 and 3x2 images
    a = (np.arange(30, dtype=np.uint8).reshape(2, 3, 5) * 8)
    case = GpuCase([a], 8, 2)
    try:
        case.set_tfs([synth.tf_piecewise(7)], [(0.0, 255.0)])
        for W, H in ((1, 1), (3, 2)):
            view, proj = synth.orbit_camera(5, seed=9, width=W, height=H, radius_widths=3.0)
            pose, _, gsel, ref = case.select([view, view], [proj, proj], W, H)
            compare_selection(gsel, ref)
            imgs, cnts = case.render(pose, empty_skip=0)
            compare_image(imgs[0], case.oracle_render(ref["leaf"], view, proj, W, H), cnts[0])
    finally:
        case.close()
    z = np.zeros((16, 16, 16), np.uint8)
    case = GpuCase([z], 8, 2)
    try:
        # alpha 0 over the first table entries: value 0 is transparent under the
        # conservative (one-entry margin) emptiness test, so every block drops
        case.set_tfs([synth.tf_piecewise(8, zero_alpha_points=2)], [(0.0, 255.0)])
        view, proj = synth.orbit_camera(16, seed=4, width=32, height=32)
        pose, stats, gsel, ref = case.select([view, view], [proj, proj], 32, 32)
        compare_selection(gsel, ref)
        assert stats["selected"] == 0
        imgs, cnts = case.render(pose)
        assert not imgs[0].any() and not cnts[0].any()
    finally:
        case.close()


def test_two_channels_blend_additively():
    a = synth.blobs_u16((96, 80, 64), seed=1003, channel=0, nblobs=10)
    b = synth.blobs_u16((96, 80, 64), seed=1003, channel=1, nblobs=10)
    case = GpuCase([a, b], 16, 3, model=synth.volume_model(96, 0.5))
    try:
        case.set_tfs([synth.tf_piecewise(2003, zero_alpha_points=2, colour=(0.1, 0.9, 0.2)),
                      synth.tf_piecewise(2004, zero_alpha_points=2, colour=(0.9, 0.1, 0.8))],
                     [(200.0, 40000.0), (200.0, 40000.0)])
        W, H = 160, 176
        (views, projs), = synth.head_poses(1, seed=3300, extent_m=0.5, width=W, height=H)
        pose, _, gsel, ref = case.select(views, projs, W, H, tau=0.5)
        compare_selection(gsel, ref)
        imgs, cnts = case.render(pose, empty_skip=1)
        for e in range(2):
            compare_image(imgs[e], case.oracle_render(ref["leaf"], views[e], projs[e], W, H))
    finally:
        case.close()


def test_call_order_errors():
    from paper_1804_08197_b300 import sg
    case = _c1_case()
    try:
        view, proj = synth.orbit_camera(128, seed=3001, width=64, height=64)
        pose = sg.make_pose([view, view], [proj, proj], 64, 64, slot=3)
        import torch
        outs = [torch.empty((64, 64, 4), device="cuda") for _ in range(2)]
        with pytest.raises(sg.SGError) as ei:
            sg.sg_render(case.vol, pose, sg.render_params(), outs)
        assert ei.value.status == sg.SG_ERR_STATE
        sg.sg_select_lod(case.vol, pose)
        sg.sg_render(case.vol, pose, sg.render_params(), outs)
        # a new transfer function makes the selection stale
        sg.sg_set_transfer_function(case.vol, 0, synth.tf_piecewise(5), 0.0, 255.0)
        with pytest.raises(sg.SGError) as ei:
            sg.sg_render(case.vol, pose, sg.render_params(), outs)
        assert ei.value.status == sg.SG_ERR_STATE
        with pytest.raises(sg.SGError) as ei:
            sg.sg_render(case.vol, pose, sg.render_params(step=-1.0), outs)
        assert ei.value.status == sg.SG_ERR_INVALID_ARG
    finally:
        case.close()


def test_render_host_matches_device_render():
    from paper_1804_08197_b300 import sg
    case = _c1_case()
    try:
        view, proj = synth.orbit_camera(128, seed=3001, width=96, height=80)
        pose, _, _, _ = case.select([view, view], [proj, proj], 96, 80)
        dev, _ = case.render(pose, counts=False)
        host = [np.empty((80, 96, 4), np.float32) for _ in range(2)]
        sg.sg_render_host(case.vol, pose, sg.render_params(), host)
        assert np.array_equal(host[0].reshape(-1, 4), dev[0])
    finally:
        case.close()


def test_pipelined_host_render_matches_device_render():
    """sg_render_host_async keeps up to three frames in flight (each frame's
    copy to host overlaps the next two renders); every frame's host images
    equal the device render of its pose, across staging growth (a larger
    image size midway) and the reuse of every staging pair. A caller that
    waits one frame behind (two in flight) gets the same images."""
    import torch
    from paper_1804_08197_b300 import sg
    case = _c1_case()
    try:
        sizes = [(96, 80)] * 3 + [(128, 112)] * 3
        frames = []
        for i, (w, h) in enumerate(sizes):
            view, proj = synth.orbit_camera(128, seed=3100 + i, width=w, height=h)
            frames.append(([view, view], [proj, proj], w, h))
        refs = []
        for views, projs, w, h in frames:
            pose, _, _, _ = case.select(views, projs, w, h)
            dev, _ = case.render(pose, counts=False)
            refs.append(dev)
        hosts = [[torch.empty((h, w, 4), dtype=torch.float32, pin_memory=True) for _ in range(2)]
                 for _, _, w, h in frames]

        def check(i):
            for e in range(2):
                assert np.array_equal(hosts[i][e].numpy().reshape(-1, 4), refs[i][e]), (i, e)

        for lag in (2, 1):
            for hst in hosts:
                for t in hst:
                    t.fill_(-1.0)
            for i, (views, projs, w, h) in enumerate(frames):
                pose, _, _, _ = case.select(views, projs, w, h)
                sg.sg_render_host_async(case.vol, pose, sg.render_params(), hosts[i])
                if i >= lag:
                    sg.sg_render_host_wait(case.vol, all=False)  # the oldest frame in flight is complete
                    check(i - lag)
            sg.sg_render_host_wait(case.vol, all=True)
            for i in range(len(frames) - lag, len(frames)):
                check(i)
    finally:
        case.close()


@pytest.mark.parametrize("brick,levels,kind", [(64, 3, "u16"), (128, 2, "u8")])
def test_specialised_brick_edges_match_oracle_in_every_launch_shape(brick, levels, kind):
    """Brick edges 32, 64 and 128 run kernels specialised on the edge (the
    other edges run the generic one, covered above): the bench's 64^3 u16
    bricks and 128^3 u8 cell bodies, against the oracle and bit for bit across
    every launch shape."""
    if kind == "u16":
        case = _filament_case(dims=(256, 256, 256), brick=brick, levels=levels)
    else:
        cells = synth.cells_u8_box(256, 0, 0, 0, 256, 256, 256, seed=1004, cell=64)
        case = GpuCase([cells], brick, levels, model=synth.volume_model(256, 0.5))
        case.set_tfs([synth.tf_piecewise(2004, zero_alpha_points=2, zero_span=(60, 80))], [(0.0, 255.0)])
    try:
        sg, torch = case.sg, case.torch
        W, H = 288, 320
        (views, projs), = synth.head_poses(1, seed=3150 + brick, extent_m=0.5, width=W, height=H)
        pose, _, gsel, ref = case.select(views, projs, W, H, tau=0.25)
        compare_selection(gsel, ref)
        imgs, cnts = case.render(pose, empty_skip=0)
        for e in range(2):
            compare_image(imgs[e], case.oracle_render(ref["leaf"], views[e], projs[e], W, H), cnts[e])
        assert max(float(i[:, 3].max()) for i in imgs) > 0.2
        skip, _ = case.render(pose, empty_skip=1)
        assert np.array_equal(skip[0], imgs[0]) and np.array_equal(skip[1], imgs[1])
        for persistent in (0, 1):
            for tw, th, rpt in [(16, 8, 1), (8, 16, 1), (32, 4, 1), (8, 8, 1), (16, 16, 2), (32, 8, 2)]:
                sg.sg_set_render_config(case.vol, persistent, tw, th, rpt)
                got, _ = case.render(pose, empty_skip=1, counts=False)
                assert np.array_equal(got[0], imgs[0]) and np.array_equal(got[1], imgs[1]), (persistent, tw, th, rpt)
        sg.sg_set_render_config(case.vol)
    finally:
        case.close()


@pytest.mark.parametrize("nch", [2, 3])
def test_multichannel_builds_match_oracle_in_every_launch_shape(nch, record_error):
    """Two channels run the emission-absorption kernels built for two
    channels, three the build for any channel count; both skip a channel's
    sample below its table's zero-alpha run. u16 filaments on the bench's
    64^3 bricks: the image against the oracle (additive blend of the
    channels), equal bit for bit with empty skipping off, and across every
    launch shape."""
    chans = [synth.filaments_u16((192, 176, 160), seed=1300 + c, ntubes=30) for c in range(nch)]
    case = GpuCase(chans, 64, 3, model=synth.volume_model(192, 0.5))
    try:
        sg = case.sg
        tables = [synth.tf_piecewise(2300 + c, zero_alpha_points=2, zero_span=(20, 40), alpha_max=0.3)
                  for c in range(nch)]
        case.set_tfs(tables, [(300.0, 60000.0)] * nch)
        W, H = 224, 256
        (views, projs), = synth.head_poses(1, seed=3300 + nch, extent_m=0.5, width=W, height=H)
        pose, _, gsel, ref = case.select(views, projs, W, H, tau=0.5)
        compare_selection(gsel, ref)
        # sample counts compare with the oracle's without empty skipping
        imgs, cnts = case.render(pose, empty_skip=0)
        for e in range(2):
            st = compare_image(imgs[e], case.oracle_render(ref["leaf"], views[e], projs[e], W, H), cnts[e])
            record_error(f"{nch} channels eye {e}", **st)
        assert max(float(i[:, 3].max()) for i in imgs) > 0.2
        skip, _ = case.render(pose, empty_skip=1, counts=False)
        assert np.array_equal(skip[0], imgs[0]) and np.array_equal(skip[1], imgs[1])
        for persistent in (0, 1):
            for tw, th, rpt in [(16, 8, 1), (8, 16, 1), (32, 4, 1), (8, 8, 1), (16, 16, 2), (32, 8, 2)]:
                sg.sg_set_render_config(case.vol, persistent, tw, th, rpt)
                got, _ = case.render(pose, empty_skip=1, counts=False)
                assert np.array_equal(got[0], imgs[0]) and np.array_equal(got[1], imgs[1]), (persistent, tw, th, rpt)
        sg.sg_set_render_config(case.vol)
    finally:
        case.close()


def test_touched_bricks_are_leaves_of_the_selection():
    """The diagnostic render (a flag per brick a sample came from) draws the
    same image as the timed kernel, and every flagged brick is a leaf of the
    selection ("Octree Representation": rays sample only the selected cut)."""
    case = _filament_case()
    try:
        W, H = 360, 400
        (views, projs), = synth.head_poses(1, seed=3105, extent_m=0.5, width=W, height=H)
        pose, _, gsel, ref = case.select(views, projs, W, H, tau=0.25)
        compare_selection(gsel, ref)
        imgs, cnts = case.render(pose, empty_skip=1)
        torch, sg = case.torch, case.sg
        touched = torch.zeros(case.ovol.node_count, dtype=torch.uint8, device="cuda")
        outs = [torch.empty((H, W, 4), dtype=torch.float32, device="cuda") for _ in range(2)]
        sg.sg_render(case.vol, pose, sg.render_params(step=0.5, term_alpha=0.99, empty_skip=1, touched=touched), outs)
        torch.cuda.synchronize()
        for e in range(2):
            assert np.array_equal(outs[e].cpu().numpy().reshape(-1, 4), imgs[e])
        t = np.flatnonzero(touched.cpu().numpy())
        leaves = set(np.unique(ref["leaf"][ref["leaf"] >= 0]).tolist())
        assert len(t) > 0 and (cnts[0].sum() + cnts[1].sum()) > 0
        assert set(t.tolist()) <= leaves
        assert np.all(ref["state"][t] == oracle.ST_SELECTED)
        # the flags are a diagnostic of the default kernel only
        two = sg.render_params(step=0.5, term_alpha=0.99, empty_skip=1, touched=touched,
                               mode=sg.SG_MODE_MIP)
        with pytest.raises(sg.SGError):
            sg.sg_render(case.vol, pose, two, outs)
    finally:
        case.close()


@pytest.mark.parametrize("skip_block", [2, 4, 8, 16])
def test_every_skip_block_size_leaves_the_image_unchanged(skip_block):
    """Empty-space skipping at any cell size is exact: the image equals the
    render without skipping bit for bit, which in turn matches the oracle."""
    from paper_1804_08197_b300 import sg
    import torch
    v = synth.filaments_u16((192, 160, 128), seed=1005, ntubes=20)
    model = synth.volume_model(192, 0.5)
    vol = sg.sg_volume_create((192, 160, 128), sg.SG_U16, 32, 3, model=model, skip_block=skip_block)
    try:
        d = torch.from_numpy(v.view(np.int16)).cuda()
        sg.sg_upload_volume_device(vol, 0, 0, d.data_ptr())
        sg.sg_set_transfer_function(vol, 0, synth.tf_piecewise(2002, zero_alpha_points=2), 300.0, 60000.0)
        W, H = 224, 256
        (views, projs), = synth.head_poses(1, seed=3500 + skip_block, extent_m=0.5, width=W, height=H)
        pose = sg.make_pose(views, projs, W, H, pixel_error=0.3)
        sg.sg_select_lod(vol, pose)
        imgs = {}
        for skip in (0, 1):
            outs = [torch.empty((H, W, 4), device="cuda") for _ in range(2)]
            sg.sg_render(vol, pose, sg.render_params(empty_skip=skip), outs)
            torch.cuda.synchronize()
            imgs[skip] = [o.cpu().numpy() for o in outs]
        assert np.array_equal(imgs[0][0], imgs[1][0]) and np.array_equal(imgs[0][1], imgs[1][1])
        assert imgs[1][0][..., 3].max() > 0.2
        # and the skipping render matches the oracle, both eyes
        ovol = oracle.Volume([oracle.pyramid(v, 3)], 32, model=model)
        otf = oracle.make_tf(synth.tf_piecewise(2002, zero_alpha_points=2), 300.0, 60000.0)
        ref = ovol.select([otf], views, projs, H, tau=0.3)
        cells, _, _ = sg.sg_read_selection(vol, 0, len(ref["leaf"]), ovol.node_count)
        assert np.array_equal(cells, ref["leaf"])
        for e in range(2):
            compare_image(imgs[1][e].reshape(-1, 4), ovol.render([otf], ref["leaf"], views[e], projs[e], W, H))
    finally:
        sg.sg_volume_destroy(vol)
