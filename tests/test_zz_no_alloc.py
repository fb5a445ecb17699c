"""The allocation-free selection entry point, for callers that cannot call
cudaMalloc while they render (a thread under a hard frame budget, or one
recording a CUDA graph). It must give exactly what sg_select_lod gives,
call after call, while using only caller buffers and the library's fixed
scratch array. Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

LEAF_NONE = 1 << 31


def _check_leaf(leaf, cell_node, node_level, slot_of):
    """leaf entries: bit 31 + level where nothing renders (cell_node -1),
    else slot << 5 | own-empty << 4 | level of the rendering node."""
    leaf = leaf.astype(np.uint32)
    none = (leaf & LEAF_NONE) != 0
    assert np.array_equal(none, cell_node < 0)
    r = ~none
    nodes = cell_node[r]
    assert np.array_equal(leaf[r] & 15, node_level[nodes])
    assert np.array_equal((leaf[r] & ~np.uint32(LEAF_NONE)) >> 5, slot_of[nodes].astype(np.uint32))


def _run_noalloc(sg, torch, vol, pose, ncell, nodes):
    leaf = torch.empty(ncell, dtype=torch.int32, device="cuda")
    cell_node = torch.empty(ncell, dtype=torch.int32, device="cuda")
    node_state = torch.empty(nodes, dtype=torch.uint8, device="cuda")
    req = torch.empty(nodes, dtype=torch.int32, device="cuda")
    counters = torch.empty(8, dtype=torch.int32, device="cuda")
    sg.sg_select_lod_noalloc(vol, pose, leaf, cell_node, node_state, req, counters)
    torch.cuda.synchronize()
    c = counters.cpu().numpy()
    return (leaf.cpu().numpy().view(np.uint32), cell_node.cpu().numpy(), node_state.cpu().numpy(),
            np.sort(req.cpu().numpy()[: c[0]]), c)


def _stats_list(stats):
    return [stats["requested"], stats["selected"], stats["culled"], stats["empty"], stats["fallback"],
            stats["nonempty"]]


def test_noalloc_selection_equals_sg_select_lod_on_two_calls_in_a_row():
    import torch
    from paper_1804_08197_b300 import sg

    a = synth.filaments_u16((160, 128, 96), seed=21, ntubes=14)
    vol = sg.sg_volume_create((160, 128, 96), sg.SG_U16, 16, 4, model=synth.volume_model(160, 0.5))
    try:
        d = torch.from_numpy(a.view(np.int16)).cuda()
        sg.sg_upload_volume_device(vol, 0, 0, d.data_ptr())
        sg.sg_set_transfer_function(vol, 0, synth.tf_piecewise(2002, zero_alpha_points=2), 300.0, 60000.0)
        ovol = oracle.Volume([oracle.pyramid(a, 4)], 16)
        ncell = 10 * 8 * 6
        nodes = ovol.node_count
        level = np.array([ovol.node_coords(i)[0] for i in range(nodes)])
        W, H = 200, 220
        expected = []
        for i in range(2):
            (views, projs), = synth.head_poses(1, seed=3500 + i, extent_m=0.5, width=W, height=H)
            pose = sg.make_pose(views, projs, W, H, pixel_error=0.25, slot=i)
            stats = sg.sg_select_lod(vol, pose, stats=True)
            cells, state, req = sg.sg_read_selection(vol, i, ncell, nodes)
            expected.append((pose, stats, cells, state, np.sort(req)))
        slot_of = sg.sg_read_residency(vol, 0, nodes)
        for pose, stats, cells, state, req_ref in expected:  # two calls in a row, different poses
            leaf, cell_node, node_state, req, c = _run_noalloc(sg, torch, vol, pose, ncell, nodes)
            assert np.array_equal(cell_node, cells)
            assert np.array_equal(node_state, state)
            assert np.array_equal(req, req_ref)
            assert [c[0], c[1], c[2], c[3], c[4], c[5]] == _stats_list(stats)
            _check_leaf(leaf, cell_node, level, slot_of)
            assert stats["selected"] > 0
    finally:
        sg.sg_volume_destroy(vol)


def test_noalloc_selection_with_missing_bricks_requests_and_falls_back():
    """A cache volume holding only its two coarsest levels: both entry
    points request the missing children and render their parents, with the
    same requests, counters, states and leaf entries (slots of the cache)."""
    import torch
    from paper_1804_08197_b300 import sg

    dims, B, LV = (128, 128, 128), 16, 4
    a = synth.filaments_u16(dims, seed=31, ntubes=18)
    ovol = oracle.Volume([oracle.pyramid(a, LV)], B)
    nodes = ovol.node_count
    ncell = 8 * 8 * 8
    level = np.array([ovol.node_coords(i)[0] for i in range(nodes)])
    brick_bytes = ((B + 2) ** 3 * 2 + 255) // 256 * 256
    vol = sg.sg_volume_create(dims, sg.SG_U16, B, LV, device_pool_bytes=80 * brick_bytes,
                              model=synth.volume_model(128, 0.5))
    try:
        sg.sg_set_transfer_function(vol, 0, synth.tf_piecewise(2002, zero_alpha_points=2), 300.0, 60000.0)
        R = B + 2
        for L in (3, 2):
            g = ovol.channels[0][L]
            nbx, nby, nbz = ovol.blocks_per_axis(L)
            xyz = np.array([(x, y, z) for z in range(nbz) for y in range(nby) for x in range(nbx)])
            host = np.stack([np.ascontiguousarray(g[np.ix_(np.clip(np.arange(R) + z * B - 1, 0, g.shape[0] - 1),
                                                           np.clip(np.arange(R) + y * B - 1, 0, g.shape[1] - 1),
                                                           np.clip(np.arange(R) + x * B - 1, 0, g.shape[2] - 1))])
                             for x, y, z in xyz])
            sg.sg_upload_bricks(vol, 0, 0, L, xyz, host)
        slot_of = sg.sg_read_residency(vol, 0, nodes)
        W, H = 192, 208
        for i in range(2):
            (views, projs), = synth.head_poses(1, seed=3600 + i, extent_m=0.5, width=W, height=H)
            pose = sg.make_pose(views, projs, W, H, pixel_error=0.3)
            stats = sg.sg_select_lod(vol, pose, stats=True)
            cells, state, req_ref = sg.sg_read_selection(vol, 0, ncell, nodes)
            leaf, cell_node, node_state, req, c = _run_noalloc(sg, torch, vol, pose, ncell, nodes)
            assert stats["requested"] > 0 and stats["fallback"] > 0
            assert np.array_equal(cell_node, cells) and np.array_equal(node_state, state)
            assert np.array_equal(req, np.sort(req_ref))
            assert [c[0], c[1], c[2], c[3], c[4], c[5]] == _stats_list(stats)
            _check_leaf(leaf, cell_node, level, slot_of)
    finally:
        sg.sg_volume_destroy(vol)


def test_noalloc_selection_rejects_levels_beyond_its_fixed_scratch():
    """The fixed scratch holds 65536 blocks per level: a volume of
    64 x 64 x 32 = 131072 level-0 blocks is refused with INVALID_ARG before
    anything is launched."""
    import torch
    from paper_1804_08197_b300 import sg

    # the cache must hold the coarsest level: 32 x 32 x 16 bricks of 10^3 bytes (1 KiB slots)
    vol = sg.sg_volume_create((512, 512, 256), sg.SG_U8, 8, 2, device_pool_bytes=20 << 20)
    try:
        (views, projs), = synth.head_poses(1, seed=3700, extent_m=0.5, width=64, height=64)
        pose = sg.make_pose(views, projs, 64, 64)
        buf = torch.zeros(16, dtype=torch.int32, device="cuda")
        with pytest.raises(sg.SGError) as ei:
            sg.sg_select_lod_noalloc(vol, pose, buf, buf, buf, buf, buf)
        assert ei.value.status == sg.SG_ERR_INVALID_ARG and "65536" in str(ei.value)
    finally:
        sg.sg_volume_destroy(vol)
