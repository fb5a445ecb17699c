"""Pins of the oracle's octree traversal (the paper's 'Octree Representation'
section: top-down LOD choice by angular voxel resolution, frustum culling,
fallback to the parent while children are not cached). CPU only."""
import numpy as np
import pytest

import oracle
import synth


def _const_volume(n=256, B=32, levels=4, value=100):
    a = np.full((n, n, n), value, np.uint8)
    return oracle.Volume([oracle.pyramid(a, levels)], B)


def _tf_opaque():
    return oracle.make_tf(np.tile(np.array([0.5, 0.5, 0.5, 0.1], np.float32), (256, 1)), 0.0, 255.0)


def _cam(eye, target, fovy=90.0, H=1024, W=1024, up=(0, 1, 0)):
    v = synth.colmajor(synth.look_at(eye, target, up))
    p = synth.colmajor(synth.perspective(fovy, W / H, 0.1, 1e5))
    return v, p


def _selected_levels(vol, sel):
    return {int(i): vol.node_coords(i)[0] for i in np.flatnonzero(np.isin(sel["state"], [oracle.ST_SELECTED,
                                                                                          oracle.ST_FALLBACK]))}


def test_accept_boundary_is_inclusive_and_scaled_by_pixel_angle():
    # fovy 90 deg -> P11 = 1, H = 1024 -> pixel angle theta = 2^-9 exactly, tau = 1:
    # a level-L voxel (2^L voxels) is accepted iff d >= 512 * 2^L voxels.
    # The root (L=3) is accepted iff the nearer eye is >= 4096 voxels from its box.
    vol = _const_volume()
    tf = _tf_opaque()
    v, p = _cam([128, 128, 256 + 4096], [128, 128, 0])
    sel = vol.select([tf], [v, v], [p, p], 1024)
    eyes, _, K = vol.select_inputs([v, v], [p, p], 1024)
    assert K == 1 << 22 and eyes[0, 2] == (256 + 4096) * 64
    assert _selected_levels(vol, sel) == {int(vol.level_offsets[3]): 3}
    v2, _ = _cam([128, 128, 256 + 4096 - 1 / 64], [128, 128, 0])
    sel2 = vol.select([tf], [v2, v2], [p, p], 1024)
    lv = _selected_levels(vol, sel2)
    assert len(lv) == 8 and set(lv.values()) == {2}


def test_tau_limits_select_roots_or_finest_level():
    vol = _const_volume(n=128, B=16, levels=4)
    tf = _tf_opaque()
    v, p = _cam([64, 64, 400], [64, 64, 64], fovy=60.0)
    coarse = vol.select([tf], [v, v], [p, p], 1024, tau=1e9)
    assert set(_selected_levels(vol, coarse).values()) == {3}
    fine = vol.select([tf], [v, v], [p, p], 1024, tau=1e-9)
    lv = _selected_levels(vol, fine)
    assert set(lv.values()) == {0} and len(lv) == 8 ** 3  # whole volume visible, all level-0 blocks


def _check_structure(vol, sel):
    """Every selected node's ancestors were refined, cells are covered by
    exactly the selected nodes, and no two selected nodes overlap."""
    st = sel["state"]
    leaf = sel["leaf"]
    nb0 = vol.blocks_per_axis(0)
    cover = np.full(leaf.shape, -1, np.int64)
    for i in np.flatnonzero(np.isin(st, [oracle.ST_SELECTED, oracle.ST_FALLBACK])):
        L, (bx, by, bz) = vol.node_coords(i)
        # ancestors refined
        for up in range(L + 1, vol.levels):
            s = 1 << (up - L)
            a_nb = vol.blocks_per_axis(up)
            aid = vol.level_offsets[up] + ((bz // s) * a_nb[1] + by // s) * a_nb[0] + bx // s
            assert st[aid] == oracle.ST_REFINED
        n = 1 << L
        for z in range(bz * n, min((bz + 1) * n, nb0[2])):
            for y in range(by * n, min((by + 1) * n, nb0[1])):
                for x in range(bx * n, min((bx + 1) * n, nb0[0])):
                    c = (z * nb0[1] + y) * nb0[0] + x
                    assert cover[c] == -1
                    cover[c] = i
    assert np.array_equal(cover, leaf.astype(np.int64))


def test_traversal_structure_on_filaments():
    a = synth.filaments_u16((128, 128, 128), seed=5, ntubes=12)
    vol = oracle.Volume([oracle.pyramid(a, 4)], 16)
    tf = oracle.make_tf(synth.tf_piecewise(2002, zero_alpha_points=2), 300.0, 60000.0)
    for seed in range(4):
        (views, projs), = synth.head_poses(1, seed=seed, extent_m=0.5, width=256, height=288)
        views = [vv for vv in views]
        model = synth.volume_model(128, 0.5)
        vol2 = oracle.Volume(vol.channels, 16, model=model)
        sel = vol2.select([tf], views, projs, 288, tau=0.25)
        _check_structure(vol2, sel)
        assert (sel["state"] == oracle.ST_EMPTY).any()  # transparent background is dropped


def test_selection_is_monotone_in_distance():
    vol = _const_volume(n=128, B=16, levels=4)
    tf = _tf_opaque()
    prev = None
    for dist in (150, 300, 600, 1200, 2400, 8000):  # theta = 2 tan(30 deg)/1024: L3 needs d >= 8/theta = 7093
        v, p = _cam([64, 64, 128 + dist], [64, 64, 64], fovy=60.0)
        sel = vol.select([tf], [v, v], [p, p], 1024)
        lev = np.array([vol.node_coords(i)[0] if i >= 0 else -1 for i in sel["leaf"]])
        if prev is not None:
            both = (lev >= 0) & (prev >= 0)
            assert (lev[both] >= prev[both]).all()
        prev = lev
    assert (prev[prev >= 0] == 3).all()


def test_missing_children_fall_back_to_the_parent_and_are_requested():
    vol = _const_volume(n=128, B=16, levels=4)
    tf = _tf_opaque()
    v, p = _cam([64, 64, 128 + 150], [64, 64, 64], fovy=60.0)
    full = vol.select([tf], [v, v], [p, p], 1024)
    # pick a refined level-1 node and make one of its children non-resident
    refined = [i for i in np.flatnonzero(full["state"] == oracle.ST_REFINED) if vol.node_coords(i)[0] == 1]
    parent = refined[0]
    L, (bx, by, bz) = vol.node_coords(parent)
    nb = vol.blocks_per_axis(0)
    child = vol.level_offsets[0] + ((2 * bz) * nb[1] + 2 * by) * nb[0] + 2 * bx
    resident = np.ones(vol.node_count, np.uint8)
    resident[child] = 0
    sel = vol.select([tf], [v, v], [p, p], 1024, resident=resident)
    assert sel["state"][parent] == oracle.ST_FALLBACK
    assert list(sel["requests"]) == [child]
    _check_structure(vol, sel)
    # everything else is unchanged
    others = full["state"] != sel["state"]
    changed = set(np.flatnonzero(others))
    assert parent in changed and all(vol.node_coords(i)[0] <= 1 for i in changed)


def _corners(vol, i):
    L, b = vol.node_coords(i)
    span = vol.brick << L
    n0 = vol.channels[0][0].shape[::-1]
    lo = [b[a] * span for a in range(3)]
    hi = [min((b[a] + 1) * span, n0[a]) for a in range(3)]
    return np.array([[x, y, z, 1.0] for x in (lo[0], hi[0]) for y in (lo[1], hi[1]) for z in (lo[2], hi[2])])


def test_culling_is_conservative_against_clip_space_geometry():
    vol = _const_volume(n=128, B=16, levels=4)
    tf = _tf_opaque()
    # a narrow stereo view of one corner region: many blocks are off screen
    views, projs = [], []
    for dx in (-3.0, 3.0):
        v, p = _cam([40 + dx, 30, 300], [40 + dx, 30, 0], fovy=20.0, H=512, W=640)
        views.append(v)
        projs.append(p)
    sel = vol.select([tf], views, projs, 512, tau=1e-9)
    st = sel["state"]
    assert (st == oracle.ST_CULLED).any() and (st == oracle.ST_SELECTED).any()
    clips = [np.asarray(p, np.float64).reshape(4, 4).T @ np.asarray(v, np.float64).reshape(4, 4).T
             for v, p in zip(views, projs)]
    for i in np.flatnonzero(st > 0):
        cs = [(_corners(vol, i) @ M.T) for M in clips]
        # outside one side plane (w+x<0, w-x<0, w+y<0, w-y<0) for every corner
        outs = [[(c[:, 3] + c[:, 0] < 0).all(), (c[:, 3] - c[:, 0] < 0).all(),
                 (c[:, 3] + c[:, 1] < 0).all(), (c[:, 3] - c[:, 1] < 0).all()] for c in cs]
        if st[i] == oracle.ST_CULLED:
            assert all(any(o) for o in outs)
        elif all(any(o) for o in outs):
            # outside both frusta in clip space: only the one-voxel outward push may keep it,
            # so for some eye every plane it is outside of is within ~1 voxel of a corner
            kept = False
            for e, o in enumerate(outs):
                M = clips[e]
                rows = [M[3] + M[0], M[3] - M[0], M[3] + M[1], M[3] - M[1]]
                ok = True
                for k in range(4):
                    if o[k]:
                        pl = rows[k] / np.linalg.norm(rows[k][:3])
                        ok &= (_corners(vol, i) @ pl).max() > -1.1
                kept |= ok
            assert kept


def test_everything_behind_the_camera_is_culled():
    vol = _const_volume(n=64, B=16, levels=3)
    tf = _tf_opaque()
    v, p = _cam([32, 32, 200], [32, 32, 400])
    sel = vol.select([tf], [v, v], [p, p], 512)
    assert sel["selected"] == 0 and (sel["leaf"] == -1).all()
    top = vol.level_offsets[2]
    assert (sel["state"][top:] == oracle.ST_CULLED).all()


def test_unknown_ranges_are_never_transparent():
    # every voxel 0 and alpha 0 over the low end: every block is transparent...
    a = np.zeros((64, 64, 64), np.uint8)
    vol = oracle.Volume([oracle.pyramid(a, 3)], 16)
    tf = oracle.make_tf(synth.tf_piecewise(8, zero_alpha_points=2), 0.0, 255.0)
    v, p = _cam([32, 32, 300], [32, 32, 32], fovy=60.0)
    r = vol.block_ranges()
    assert vol.select([tf], [v, v], [p, p], 512, ranges=r)["selected"] == 0
    # ...unless its data was never seen (min > max): then it must be rendered
    unk = r.copy()
    unk[: vol.level_offsets[1], 0, 0] = 0xFFFFFFFF
    unk[: vol.level_offsets[1], 0, 1] = 0
    sel = vol.select([tf], [v, v], [p, p], 512, ranges=unk, tau=1e-9)
    assert sel["selected"] == vol.level_offsets[1]  # all level-0 blocks
