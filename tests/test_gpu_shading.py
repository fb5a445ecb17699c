"""Gradient-magnitude tables and depth palettes ("Visualization
Enhancements") against the oracle, in every optical model, with selection
(gradient transparency) bit-exact and empty-space skipping exact."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import GpuCase, compare_image, compare_selection

pytestmark = pytest.mark.gpu

PALETTE = np.array([[1.0, 0.2, 0.0], [0.9, 0.9, 0.1], [0.1, 0.8, 0.9], [0.3, 0.0, 1.0]], np.float32)


def _case(gradient, palette, seed=1002):
    v = synth.filaments_u16((256, 256, 256), seed=seed, ntubes=40)
    case = GpuCase([v], 32, 4, model=synth.volume_model(256, 0.5))
    table = synth.tf_piecewise(2002, zero_alpha_points=2)
    window = (50.0, 20000.0) if gradient else (300.0, 60000.0)
    case.set_tfs([table], [window])
    near, far = 0.4, 1.1
    case.sg.sg_set_channel_shading(case.vol, 0, gradient=gradient, palette=palette, near=near, far=far)
    case.otfs = [oracle.make_tf(table, *window, gradient=gradient, palette=palette, near=near, far=far)]
    return case


@pytest.mark.parametrize("gradient,palette,mode", [
    (True, None, oracle.MODE_EA),
    (False, PALETTE, oracle.MODE_EA),
    (True, PALETTE, oracle.MODE_EMISSION),
    (True, PALETTE, oracle.MODE_MIP),
])
def test_gradient_tables_and_depth_palettes_match_the_oracle(gradient, palette, mode):
    case = _case(gradient, palette)
    try:
        W, H = 224, 240
        (views, projs), = synth.head_poses(1, seed=3800, extent_m=0.5, width=W, height=H)
        pose, _, gsel, ref = case.select(views, projs, W, H, tau=0.25)
        compare_selection(gsel, ref)
        imgs, cnts = case.render(pose, empty_skip=0, mode=mode)
        for e in range(2):
            oref = case.oracle_render(ref["leaf"], views[e], projs[e], W, H, mode=mode)
            compare_image(imgs[e], oref, cnts[e])
        assert max(float(i[:, :3].max()) for i in imgs) > 0.05
        skip, _ = case.render(pose, empty_skip=1, mode=mode)
        assert np.array_equal(skip[0], imgs[0]) and np.array_equal(skip[1], imgs[1])
    finally:
        case.close()


def test_shading_arguments_are_checked():
    from paper_1804_08197_b300 import sg
    case = _case(False, None)
    try:
        with pytest.raises(sg.SGError):
            sg.sg_set_channel_shading(case.vol, 0, palette=PALETTE, near=1.0, far=1.0)
        with pytest.raises(sg.SGError):
            sg.sg_set_channel_shading(case.vol, 1)
        with pytest.raises(sg.SGError):
            sg.sg_set_channel_shading(case.vol, 0, palette=PALETTE * 2.0, near=0.0, far=1.0)
    finally:
        case.close()


def test_single_entry_palette_and_u8_gradient():
    """A one-entry palette paints every sample one colour; gradient input on
    u8 data (two levels), both against the oracle."""
    a = synth.gaussians_u8(96, seed=51, count=7)
    case = GpuCase([a], 32, 2, model=synth.volume_model(96, 0.5))
    try:
        table = synth.tf_piecewise(2013, zero_alpha_points=2)
        case.set_tfs([table], [(2.0, 40.0)])
        pal = np.array([[0.2, 0.6, 1.0]], np.float32)
        case.sg.sg_set_channel_shading(case.vol, 0, gradient=True, palette=pal, near=0.1, far=2.0)
        case.otfs = [oracle.make_tf(table, 2.0, 40.0, gradient=True, palette=pal, near=0.1, far=2.0)]
        W, H = 112, 120
        (views, projs), = synth.head_poses(1, seed=3810, extent_m=0.5, width=W, height=H)
        pose, _, gsel, ref = case.select(views, projs, W, H, tau=0.5)
        compare_selection(gsel, ref)
        imgs, cnts = case.render(pose, empty_skip=0)
        for e in range(2):
            compare_image(imgs[e], case.oracle_render(ref["leaf"], views[e], projs[e], W, H), cnts[e])
        img = imgs[0][imgs[0][:, 3] > 0.05]
        assert len(img) and np.allclose(img[:, :3] / img[:, 3:4], pal[0], atol=1e-5)
    finally:
        case.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_transparent_samples_skipped_by_the_plain_kernel_change_nothing(mode):
    """The plain emission-absorption and emission-only kernels skip the
    table lookup and the blend of a channel's sample whose table input falls
    below the table's run of leading zero-alpha entries (it would add
    exactly 0). The shading kernels never skip. With a constant table
    colour, a one-entry palette of that colour makes the shading kernel
    compute the same arithmetic, so the two images must be equal bit for
    bit: one channel (the one-channel build), then two (the second with a
    table of alpha 0 everywhere, read as a gradient in the shading
    kernel)."""
    from paper_1804_08197_b300 import sg
    colour = (0.75, 0.5, 0.25)
    a = synth.filaments_u16((112, 96, 104), seed=1201, ntubes=14)
    tf = synth.tf_piecewise(2201, zero_alpha_points=2, zero_span=(40, 60), alpha_max=0.4, colour=colour)
    assert tf[0, 3] == 0 and tf[30, 3] == 0 and tf[-1, 3] > 0
    views, projs = synth.orbit_camera(112, seed=3201, width=96, height=88)
    for nch in (1, 2):
        chans = [a] if nch == 1 else [a, synth.filaments_u16((112, 96, 104), seed=1202, ntubes=10)]
        case = GpuCase(chans, 16, 3)
        try:
            tables = [tf] if nch == 1 else [tf, np.zeros_like(tf)]
            case.set_tfs(tables, [(300.0, 60000.0)] * nch)
            pose, _, _, _ = case.select([views, views], [projs, projs], 96, 88)
            plain, _ = case.render(pose, counts=False, mode=mode)
            if nch == 1:
                sg.sg_set_channel_shading(case.vol, 0, palette=np.array([colour], np.float32))
            else:
                sg.sg_set_channel_shading(case.vol, 1, gradient=True)
            pose, _, _, _ = case.select([views, views], [projs, projs], 96, 88)
            shaded, _ = case.render(pose, counts=False, mode=mode)
            assert plain[0][:, :3].max() > 0.05  # the channel shows
            for e in range(2):
                assert np.array_equal(plain[e], shaded[e]), (nch, mode, e)
        finally:
            case.close()
