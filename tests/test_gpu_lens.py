"""Rendering in the lens-warped space and unwarping ("DVR for HMD") against
the oracle: one ray per warped pixel through the radial lens map, then the
preimage + bilinear resample to the undistorted image."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import GpuCase, compare_image, compare_selection

pytestmark = pytest.mark.gpu

K1, K2 = 0.22, 0.24
CENTRES = ((0.05, 0.0), (-0.05, 0.0))


def _case():
    v = synth.filaments_u16((256, 256, 256), seed=1002, ntubes=40)
    case = GpuCase([v], 32, 4, model=synth.volume_model(256, 0.5))
    case.set_tfs([synth.tf_piecewise(2002, zero_alpha_points=2)], [(300.0, 60000.0)])
    return case


def _poses(case, W, H, Ww, Hw, seed=3700):
    sg = case.sg
    (views, projs), = synth.head_poses(1, seed=seed, extent_m=0.5, width=W, height=H)
    pose, _, gsel, ref = case.select(views, projs, W, H, tau=0.25)
    compare_selection(gsel, ref)
    # the warped image renders from the same selection slot at its own size
    wpose = sg.make_pose(views, projs, Ww, Hw, pixel_error=0.25)
    return pose, wpose, views, projs, ref


def test_identity_lens_is_the_plain_render():
    case = _case()
    try:
        sg = case.sg
        pose, _, views, projs, ref = _poses(case, 160, 176, 160, 176)
        plain, _ = case.render(pose, counts=False)
        ident = sg.make_lens(0.0, 0.0, 1.0)
        torch = case.torch
        outs = [torch.empty((176, 160, 4), device="cuda") for _ in range(2)]
        sg.sg_render(case.vol, pose, sg.render_params(lens=ident), outs)
        torch.cuda.synchronize()
        for e in range(2):
            assert np.array_equal(outs[e].cpu().numpy().reshape(-1, 4), plain[e])
    finally:
        case.close()


def test_warped_render_and_unwarp_match_the_oracle():
    case = _case()
    try:
        sg, torch = case.sg, case.torch
        W, H = 240, 272
        scale = 1.0 / (1.0 + K1 + K2)
        Ww, Hw = int(round(W * scale)), int(round(H * scale))
        pose, wpose, views, projs, ref = _poses(case, W, H, Ww, Hw)
        ln = sg.make_lens(K1, K2, 0.0, W / H, CENTRES)
        warped = [torch.empty((Hw, Ww, 4), device="cuda") for _ in range(2)]
        sg.sg_render(case.vol, wpose, sg.render_params(lens=ln), warped)
        out = [torch.empty((H, W, 4), device="cuda") for _ in range(2)]
        sg.sg_unwarp(ln, warped, Ww, Hw, out, W, H)
        torch.cuda.synchronize()
        for e in range(2):
            oln = oracle.lens(K1, K2, scale, W / H, *CENTRES[e])
            got = warped[e].cpu().numpy()
            oref = case.ovol.render(case.otfs, ref["leaf"], views[e], projs[e], Ww, Hw, lens=oln)
            compare_image(got.reshape(-1, 4), oref)
            assert got[..., 3].max() > 0.2
            # unwarp of the same warped image, GPU vs FP64
            uref = oracle.unwarp(oln, got, W, H)
            err = np.abs(out[e].cpu().numpy() - uref).max()
            assert err < 1e-4, err
    finally:
        case.close()


def test_lens_arguments_are_checked():
    case = _case()
    try:
        sg, torch = case.sg, case.torch
        pose, _, _, _, _ = _poses(case, 32, 32, 32, 32)
        outs = [torch.empty((32, 32, 4), device="cuda") for _ in range(2)]
        with pytest.raises(sg.SGError):
            sg.sg_render(case.vol, pose, sg.render_params(lens=sg.make_lens(-0.1, 0.0)), outs)
        with pytest.raises(sg.SGError):
            sg.sg_render_batch(case.vol, [pose], sg.render_params(lens=sg.make_lens(0.1, 0.0)), outs)
        with pytest.raises(sg.SGError):
            sg.sg_unwarp(sg.make_lens(0.1, 0.0), outs, 0, 32, outs, 32, 32)
    finally:
        case.close()


def test_odd_sizes_and_off_centre_lens():
    """Ragged warped and output sizes, an off-centre lens with its own scale
    and aspect: warped render and unwarp against the oracle."""
    case = _case()
    try:
        sg, torch = case.sg, case.torch
        W, H, Ww, Hw = 173, 151, 119, 107
        pose, wpose, views, projs, ref = _poses(case, W, H, Ww, Hw, seed=3710)
        centres = ((0.11, -0.07), (-0.09, 0.05))
        ln = sg.make_lens(0.3, 0.1, 0.7, 1.2, centres)
        warped = [torch.empty((Hw, Ww, 4), device="cuda") for _ in range(2)]
        sg.sg_render(case.vol, wpose, sg.render_params(lens=ln), warped)
        out = [torch.empty((H, W, 4), device="cuda") for _ in range(2)]
        sg.sg_unwarp(ln, warped, Ww, Hw, out, W, H)
        torch.cuda.synchronize()
        for e in range(2):
            oln = oracle.lens(0.3, 0.1, 0.7, 1.2, *centres[e])
            got = warped[e].cpu().numpy()
            compare_image(got.reshape(-1, 4),
                          case.ovol.render(case.otfs, ref["leaf"], views[e], projs[e], Ww, Hw, lens=oln))
            assert np.abs(out[e].cpu().numpy() - oracle.unwarp(oln, got, W, H)).max() < 1e-4
    finally:
        case.close()
