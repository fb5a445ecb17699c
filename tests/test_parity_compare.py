"""The image comparison of the GPU parity tests, pinned on the CPU: the
oracle's own image passes; a pixel whose ray has an ambiguous lattice point
passes with any enumerated assignment and fails with a value that matches
none; an unambiguous pixel off by more than the tolerance fails."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import compare_image


@pytest.fixture(scope="module")
def case():
    v = synth.filaments_u16((96, 96, 96), seed=1002, ntubes=20)
    model = synth.volume_model(96, 0.5)
    ovol = oracle.Volume([oracle.pyramid(v, 3)], 16, model=model)
    tf = oracle.make_tf(synth.tf_piecewise(2002, zero_alpha_points=2), 300.0, 60000.0)
    W, H = 120, 128
    (views, projs), = synth.head_poses(1, seed=3101, extent_m=0.5, width=W, height=H)
    sel = ovol.select([tf], views, projs, H, tau=0.25)
    r = ovol.render([tf], sel["leaf"], views[0], projs[0], W, H)
    return r


def _ambiguous_pixel_with_distinct_variants(r):
    for g in r["var_groups"]:
        for i, n in enumerate(g["n"]):
            if n > 1:
                vals = g["late"][i, :n]
                if np.abs(vals - vals[0]).max() > 5e-3:
                    return g, i
    raise AssertionError("no ambiguous pixel with distinct variants")


def test_the_oracle_image_passes(case):
    r = case
    st = compare_image(r["late"].astype(np.float32), r, r["count_late"].astype(np.int64))
    assert st["ambiguous"] > 0 and st["unresolved"] == 0


def test_any_enumerated_assignment_passes_and_others_fail(case):
    r = case
    g, i = _ambiguous_pixel_with_distinct_variants(r)
    pix = g["idx"][i]
    n = g["n"][i]
    img = r["late"].astype(np.float32).copy()
    cnt = r["count_late"].astype(np.int64).copy()
    for v in range(n):
        img[pix] = g["late"][i, v]
        cnt[pix] = g["count_late"][i, v]
        compare_image(img, r, cnt)
    # a value between two assignments that matches neither
    vals = g["late"][i, :n]
    far = int(np.argmax(np.abs(vals - vals[0]).max(axis=1)))
    img[pix] = 0.5 * (vals[0] + vals[far]) + 2e-3 * np.sign(vals[far] - vals[0])
    img[pix] = np.where(np.abs(vals[far] - vals[0]) > 5e-3, img[pix], vals[0] + 5e-3)
    with pytest.raises(AssertionError, match="match none"):
        compare_image(img, r)
    # a right value with a count no assignment has
    img[pix] = vals[0]
    cnt[pix] = g["count_late"][i, :n].max() + 1
    with pytest.raises(AssertionError, match="match none"):
        compare_image(img, r, cnt)


def test_an_unambiguous_pixel_off_by_more_than_the_tolerance_fails(case):
    r = case
    amb = np.zeros(len(r["late"]), bool)
    amb[r["var_idx"]] = True
    j = int(np.flatnonzero(~amb & (r["late"][:, 3] > 0.1))[0])
    img = r["late"].astype(np.float32).copy()
    img[j, 3] += 1.5e-3
    with pytest.raises(AssertionError, match="outside tolerance"):
        compare_image(img, r)
