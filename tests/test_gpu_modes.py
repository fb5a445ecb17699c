"""Optical models and depth-buffer termination ("DVR Techniques"; "Volumetric
and Mesh Data Compositing") against the oracle: emission-only, maximum
intensity projection and emission-absorption with a per-pixel opaque surface.
Empty-space skipping must leave every image unchanged bit for bit."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import GpuCase, compare_image, compare_selection

pytestmark = pytest.mark.gpu


def _case(dims=(256, 256, 256), brick=32, levels=4, seed=1002, ntubes=40, tf_seed=2002, table=None):
    v = synth.filaments_u16(dims, seed=seed, ntubes=ntubes)
    case = GpuCase([v], brick, levels, model=synth.volume_model(max(dims), 0.5))
    case.set_tfs([synth.tf_piecewise(tf_seed, zero_alpha_points=2) if table is None else table], [(300.0, 60000.0)])
    return case


def _pose(case, W=240, H=272, seed=3600, tau=0.25):
    (views, projs), = synth.head_poses(1, seed=seed, extent_m=0.5, width=W, height=H)
    pose, _, gsel, ref = case.select(views, projs, W, H, tau=tau)
    compare_selection(gsel, ref)
    return pose, views, projs, ref


@pytest.mark.parametrize("mode", [oracle.MODE_EMISSION, oracle.MODE_MIP])
def test_emission_only_and_mip_match_the_oracle(mode):
    case = _case()
    try:
        pose, views, projs, ref = _pose(case)
        W, H = pose.width, pose.height
        imgs, cnts = case.render(pose, empty_skip=0, mode=mode)
        for e in range(2):
            oref = case.oracle_render(ref["leaf"], views[e], projs[e], W, H, mode=mode)
            compare_image(imgs[e], oref, cnts[e])
            if mode == oracle.MODE_EMISSION:
                assert not imgs[e][:, 3].any()  # emission-only leaves alpha 0
        assert max(float(i[:, :3].max()) for i in imgs) > 0.05
        skip, _ = case.render(pose, empty_skip=1, mode=mode)
        assert np.array_equal(skip[0], imgs[0]) and np.array_equal(skip[1], imgs[1])
    finally:
        case.close()


def test_mip_with_a_table_transparent_in_the_middle():
    """A table whose alpha is 0 on a middle band: a transparent block's values
    may exceed every visible sample, so MIP must not skip inside rendered
    blocks; the image still matches the oracle and equals the unskipped one."""
    table = synth.tf_piecewise(2007, points=7, zero_alpha_points=1)
    table[100:140, 3] = 0.0
    case = _case(table=table, seed=1003, ntubes=30)
    try:
        pose, views, projs, ref = _pose(case, seed=3610)
        W, H = pose.width, pose.height
        imgs, cnts = case.render(pose, empty_skip=1, mode=oracle.MODE_MIP)
        for e in range(2):
            compare_image(imgs[e], case.oracle_render(ref["leaf"], views[e], projs[e], W, H, mode=oracle.MODE_MIP),
                          cnts[e])
        noskip, _ = case.render(pose, empty_skip=0, mode=oracle.MODE_MIP)
        assert np.array_equal(noskip[0], imgs[0]) and np.array_equal(noskip[1], imgs[1])
    finally:
        case.close()


@pytest.mark.parametrize("mode", [oracle.MODE_EA, oracle.MODE_EMISSION])
def test_depth_buffer_ends_rays_like_the_oracle(mode):
    """A scene surface per pixel (a tilted plane through the volume, with
    some pixels uncovered): rays take no sample at or beyond it."""
    case = _case()
    try:
        pose, views, projs, ref = _pose(case, seed=3620)
        W, H = pose.width, pose.height
        depth = []
        rng = np.random.default_rng(5)
        for e in range(2):
            head = np.linalg.inv(np.asarray(views[e], np.float64).reshape(4, 4).T)[:3, 3]  # eye in world
            dist = np.linalg.norm(head)
            jj, ii = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
            d = (dist - 0.1 + 0.25 * (ii / W) + 0.1 * (jj / H)).astype(np.float32)
            d[rng.random((H, W)) < 0.1] = np.inf
            depth.append(d)
        imgs, cnts = case.render(pose, empty_skip=0, mode=mode, depth=depth)
        full, _ = case.render(pose, empty_skip=0, mode=mode)
        for e in range(2):
            oref = case.oracle_render(ref["leaf"], views[e], projs[e], W, H, mode=mode, depth=depth[e])
            compare_image(imgs[e], oref, cnts[e])
        assert not np.array_equal(imgs[0], full[0])  # the surface cut some rays short
        skip, _ = case.render(pose, empty_skip=1, mode=mode, depth=depth)
        assert np.array_equal(skip[0], imgs[0]) and np.array_equal(skip[1], imgs[1])
    finally:
        case.close()


def test_depth_buffers_are_rejected_by_the_batch_entry_point():
    from paper_1804_08197_b300 import sg
    import torch
    case = _case(dims=(64, 64, 64), brick=16, levels=2, ntubes=4)
    try:
        pose, views, projs, ref = _pose(case, W=32, H=32)
        d = [torch.full((32, 32), float("inf"), device="cuda") for _ in range(2)]
        outs = [torch.empty((32, 32, 4), device="cuda") for _ in range(2)]
        with pytest.raises(sg.SGError):
            sg.sg_render_batch(case.vol, [pose], sg.render_params(depth=d), outs)
        with pytest.raises(sg.SGError):
            sg.sg_render(case.vol, pose, sg.render_params(mode=7), outs)
    finally:
        case.close()


@pytest.mark.parametrize("mode", [oracle.MODE_EMISSION, oracle.MODE_MIP])
def test_two_channel_u8_models_match_the_oracle(mode):
    """Two u8 channels blended additively, ragged volume and image sizes."""
    a = synth.gaussians_u8(80, seed=41, count=6)
    b = synth.gaussians_u8(80, seed=42, count=5)
    a, b = np.ascontiguousarray(a[:72, :80, :76]), np.ascontiguousarray(b[:72, :80, :76])
    case = GpuCase([a, b], 16, 3, model=synth.volume_model(80, 0.5))
    try:
        case.set_tfs([synth.tf_piecewise(2011, zero_alpha_points=2, colour=(0.1, 0.9, 0.2)),
                      synth.tf_piecewise(2012, zero_alpha_points=2, colour=(0.9, 0.1, 0.8))],
                     [(0.0, 255.0), (0.0, 255.0)])
        W, H = 131, 97
        (views, projs), = synth.head_poses(1, seed=3630, extent_m=0.5, width=W, height=H)
        pose, _, gsel, ref = case.select(views, projs, W, H, tau=0.5)
        compare_selection(gsel, ref)
        imgs, cnts = case.render(pose, empty_skip=0, mode=mode)
        for e in range(2):
            compare_image(imgs[e], case.oracle_render(ref["leaf"], views[e], projs[e], W, H, mode=mode), cnts[e])
        skip, _ = case.render(pose, empty_skip=1, mode=mode)
        assert np.array_equal(skip[0], imgs[0]) and np.array_equal(skip[1], imgs[1])
    finally:
        case.close()


def test_degenerate_depth_values():
    """Depth 0, negative, NaN and +inf: no surface in front of the eye means
    an empty pixel (0, negative), NaN is ignored like +inf (no surface)."""
    case = _case(dims=(96, 96, 96), brick=16, levels=3, ntubes=10)
    try:
        pose, views, projs, ref = _pose(case, W=64, H=48, seed=3640, tau=0.5)
        full, _ = case.render(pose, empty_skip=0, counts=False)
        for value, expect_full in [(0.0, False), (-1.0, False), (np.nan, True), (np.inf, True)]:
            depth = [np.full((48, 64), value, np.float32)] * 2
            imgs, _ = case.render(pose, empty_skip=0, counts=False, depth=depth)
            if expect_full:
                assert np.array_equal(imgs[0], full[0]) and np.array_equal(imgs[1], full[1]), value
            else:
                assert not imgs[0].any() and not imgs[1].any(), value
    finally:
        case.close()
