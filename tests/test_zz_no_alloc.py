"""The allocation-free selection entry point, for callers that cannot call
cudaMalloc while they render (a thread under a hard frame budget, or one
recording a CUDA graph). It must give exactly what sg_select_lod gives,
call after call, while using only caller buffers and the library's fixed
scratch array. Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_selection_equals_sg_select_lod_on_two_calls_in_a_row():
    import torch
    from paper_1804_08197_b300 import sg

    a = synth.filaments_u16((160, 128, 96), seed=21, ntubes=14)
    vol = sg.sg_volume_create((160, 128, 96), sg.SG_U16, 16, 4, model=synth.volume_model(160, 0.5))
    try:
        d = torch.from_numpy(a.view(np.int16)).cuda()
        sg.sg_upload_volume_device(vol, 0, 0, d.data_ptr())
        sg.sg_set_transfer_function(vol, 0, synth.tf_piecewise(2002, zero_alpha_points=2), 300.0, 60000.0)
        ncell = 10 * 8 * 6
        nodes = 10 * 8 * 6 + 5 * 4 * 3 + 3 * 2 * 2 + 2 * 1 * 1
        W, H = 200, 220
        expected = []
        for i in range(2):
            (views, projs), = synth.head_poses(1, seed=3500 + i, extent_m=0.5, width=W, height=H)
            pose = sg.make_pose(views, projs, W, H, pixel_error=0.25, slot=i)
            stats = sg.sg_select_lod(vol, pose, stats=True)
            cells, state, req = sg.sg_read_selection(vol, i, ncell, nodes)
            expected.append((pose, stats, cells, state, np.sort(req)))
        leaf = torch.empty(ncell, dtype=torch.int32, device="cuda")
        cell_node = torch.empty(ncell, dtype=torch.int32, device="cuda")
        node_state = torch.empty(nodes, dtype=torch.uint8, device="cuda")
        req = torch.empty(nodes, dtype=torch.int32, device="cuda")
        counters = torch.empty(8, dtype=torch.int32, device="cuda")
        for pose, stats, cells, state, req_ref in expected:  # two calls in a row, different poses
            sg.sg_select_lod_noalloc(vol, pose, leaf, cell_node, node_state, req, counters)
            torch.cuda.synchronize()
            c = counters.cpu().numpy()
            assert np.array_equal(cell_node.cpu().numpy(), cells)
            assert np.array_equal(node_state.cpu().numpy(), state)
            assert np.array_equal(np.sort(req.cpu().numpy()[: c[0]]), req_ref)
            assert [c[1], c[2], c[3], c[0], c[4], c[5]] == [stats["selected"], stats["culled"], stats["empty"],
                                                              stats["requested"], stats["fallback"], stats["nonempty"]]
            assert stats["selected"] > 0
    finally:
        sg.sg_volume_destroy(vol)
