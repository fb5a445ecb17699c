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
