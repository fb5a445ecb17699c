"""Pins of the FP64 oracle against closed forms, brute force and hand-derived
values (CPU only). Each test names the property of the paper's method it
fixes; none re-types the oracle's own code."""
import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _axial_camera(eye_z, cx=2.0, cy=2.0, fovy=90.0, size=9):
    view = synth.colmajor(synth.look_at([cx, cy, eye_z], [cx, cy, 0.0], [0.0, 1.0, 0.0]))
    proj = synth.colmajor(synth.perspective(fovy, 1.0, 0.1, 1000.0))
    return view, proj


def _const_tf(rgb, a, n=256, lo=0.0, hi=255.0, ref=0.5):
    tab = np.tile(np.array([*rgb, a], np.float32), (n, 1))
    return oracle.make_tf(tab, lo, hi, ref)


def _render_centre(vol, tfs, view, proj, size=9, step=0.5, brick=None):
    sel = vol.select(tfs, [view, view], [proj, proj], size, tau=1.0)
    c = (size // 2) * size + size // 2
    return vol.render(tfs, sel["leaf"], view, proj, size, size, step=step, pixels=[c])


# ---------------------------------------------------------------- pyramid (Octree Representation)

@pytest.mark.parametrize("shape,dtype", [((7, 13, 10), np.uint16), ((5, 4, 9), np.uint8), ((1, 3, 2), np.uint16)])
def test_pyramid_matches_brute_force_box_filter(shape, dtype):
    rng = np.random.default_rng(7)
    hi = 65535 if dtype == np.uint16 else 255
    a = rng.integers(0, hi + 1, shape).astype(dtype)
    levels = oracle.pyramid(a, 3)
    ref = a.astype(np.int64)
    for L in range(1, 3):
        # brute force: replicate the last plane along odd axes, then average 2x2x2 blocks
        pad = [(0, s % 2) for s in ref.shape]
        e = np.pad(ref, pad, mode="edge")
        z, y, x = (s // 2 for s in e.shape)
        s = e.reshape(z, 2, y, 2, x, 2).sum(axis=(1, 3, 5))
        ref = (s + 4) // 8
        assert levels[L].shape == ref.shape
        assert np.array_equal(levels[L].astype(np.int64), ref)


def test_block_ranges_cover_the_apron():
    rng = np.random.default_rng(3)
    a = rng.integers(0, 60000, (20, 17, 33)).astype(np.uint16)
    B = 8
    vol = oracle.Volume([oracle.pyramid(a, 2)], B)
    r = vol.block_ranges()
    for L in range(2):
        g = vol.channels[0][L]
        nbx, nby, nbz = vol.blocks_per_axis(L)
        for bz in range(nbz):
            for by in range(nby):
                for bx in range(nbx):
                    sl = tuple(slice(max(b * B - 1, 0), min(b * B + B + 1, n))
                               for b, n in zip((bz, by, bx), g.shape))
                    node = vol.level_offsets[L] + (bz * nby + by) * nbx + bx
                    assert r[node, 0, 0] == g[sl].min() and r[node, 0, 1] == g[sl].max()


# ---------------------------------------------------------------- trilinear sampling (DVR Techniques)

def test_trilinear_reproduces_linear_fields_at_two_levels():
    nz, ny, nx = 10, 12, 16
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    lvl0 = (3 * i + 5 * j + 7 * k + 11).astype(np.uint16)
    k1, j1, i1 = np.meshgrid(np.arange(5), np.arange(6), np.arange(8), indexing="ij")
    lvl1 = (13 * i1 + 2 * j1 + 29 * k1 + 100).astype(np.uint16)
    vol = oracle.Volume([[lvl0, lvl1]], 8)
    rng = np.random.default_rng(0)
    for _ in range(200):
        p = rng.uniform(-1.0, [nx + 1.0, ny + 1.0, nz + 1.0])
        u = np.clip(p - 0.5, 0.0, [nx - 1, ny - 1, nz - 1])  # clamp-to-edge beyond the last centres
        assert vol.sample(0, 0, p) == pytest.approx(3 * u[0] + 5 * u[1] + 7 * u[2] + 11, abs=1e-9)
        u1 = np.clip(p / 2.0 - 0.5, 0.0, [7, 5, 4])  # level-1 voxel j is centred at (j+0.5)*2
        assert vol.sample(1, 0, p) == pytest.approx(13 * u1[0] + 2 * u1[1] + 29 * u1[2] + 100, abs=1e-9)


# ---------------------------------------------------------------- transfer function

def test_classification_of_a_linear_ramp_is_the_window_position():
    n = 256
    ramp = np.stack([np.linspace(0, 1, n)] * 4, 1).astype(np.float32)
    tf = oracle.make_tf(ramp, 1000.0, 3000.0)
    tab = oracle.tf_table(tf, 0.5)
    for v, x in [(0.0, 0.0), (1000.0, 0.0), (2000.0, 0.5), (2500.0, 0.75), (3000.0, 1.0), (65535.0, 1.0)]:
        assert oracle.classify(tf, tab, v) == pytest.approx([x] * 4, abs=1e-6)


def test_opacity_correction_composes_like_repeated_samples():
    a = np.linspace(0, 0.9, 256).astype(np.float32)
    tab = np.stack([a, a, a, a], 1)
    tf = oracle.make_tf(tab, 0.0, 255.0, ref_step=0.5)
    t1 = oracle.tf_table(tf, 0.5)
    t4 = oracle.tf_table(tf, 2.0)
    # one sample over 4 reference steps transmits what 4 samples transmit
    assert np.allclose(1.0 - t4[:, 3], (1.0 - t1[:, 3]) ** 4, atol=1e-12)
    assert np.allclose(t1[:, :3], tab[:, :3])


# ---------------------------------------------------------------- compositing: closed forms

def test_constant_volume_is_beer_lambert_with_opacity_correction():
    n = 16
    vol = oracle.Volume([[np.full((n, n, n), 100, np.uint8)]], n)
    a = float(np.float32(0.05))  # the table holds FP32 values
    rgb = tuple(float(np.float32(c)) for c in (0.2, 0.5, 0.8))
    tf = _const_tf(rgb, a)
    view, proj = _axial_camera(40.0, cx=8.0, cy=8.0)
    # step 0.3: samples t0 + 0.3k < t0 + 16 -> k = 0..53 (54 samples), each
    # with alpha' = 1 - (1-a)^(0.3/0.5)
    r = _render_centre(vol, [tf], view, proj, step=0.3)
    A = 1.0 - (1.0 - a) ** (0.6 * 54)
    assert r["count_late"][0] == 54 and r["flags"][0] == 0
    assert r["late"][0] == pytest.approx([rgb[0] * A, rgb[1] * A, rgb[2] * A, A], abs=1e-12)


def test_constant_volume_terminates_at_0_99():
    n = 16
    vol = oracle.Volume([[np.full((n, n, n), 100, np.uint8)]], n)
    tf = _const_tf((1.0, 1.0, 1.0), 0.2)
    view, proj = _axial_camera(40.0, cx=8.0, cy=8.0)
    r = _render_centre(vol, [tf], view, proj, step=0.5)
    # 1 - 0.8^20 = 0.98847 < 0.99 <= 1 - 0.8^21 = 0.99078
    a = float(np.float32(0.2))
    assert r["count_late"][0] == 21
    assert r["late"][0][3] == pytest.approx(1.0 - (1.0 - a) ** 21, abs=1e-12)


def test_step_refinement_with_correction_keeps_opacity():
    n = 16
    vol = oracle.Volume([[np.full((n, n, n), 100, np.uint8)]], n)
    tf = _const_tf((0.3, 0.3, 0.3), 0.03)
    view, proj = _axial_camera(40.3, cx=8.0, cy=8.0)  # entry at t0 = 24.3, exit 40.3 (no lattice point on it)
    r1 = _render_centre(vol, [tf], view, proj, step=0.4)   # 40 samples
    r2 = _render_centre(vol, [tf], view, proj, step=0.2)   # 80 samples
    assert r1["count_late"][0] * 2 == r2["count_late"][0] == 80
    assert r1["late"][0] == pytest.approx(r2["late"][0], abs=1e-12)


def test_empty_volume_and_transparent_tf_give_background():
    n = 16
    vol = oracle.Volume([[np.zeros((n, n, n), np.uint8)]], 8)
    tf = _const_tf((1, 1, 1), 0.0)
    view, proj = synth.orbit_camera(n=n, seed=5, width=17, height=17)
    sel = vol.select([tf], [view, view], [proj, proj], 17)
    assert (sel["leaf"] == -1).all() and sel["selected"] == 0
    r = vol.render([tf], sel["leaf"], view, proj, 17, 17)
    assert not r["late"].any() and not r["count_late"].any()


@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLDEN, "hand_4cubed.json")))["cases"],
                         ids=lambda c: c["name"])
def test_hand_computed_4cubed_cases(case):
    chans = []
    tfs = []
    for planes, e1 in zip(case["planes"], case["tf_entry1"]):
        v = np.zeros((4, 4, 4), np.uint8)
        for k in planes:
            v[k] = 255
        chans.append([v])
        tfs.append(oracle.make_tf(np.array([[0, 0, 0, 0], e1], np.float32), 0.0, 255.0))
    vol = oracle.Volume(chans, 4)
    view, proj = _axial_camera(10.0)
    r = _render_centre(vol, tfs, view, proj)
    assert r["count_late"][0] == case["samples"]
    # the hand values use exact decimals; the table stores them as FP32 (relative error <= 6e-8)
    assert r["late"][0] == pytest.approx(case["rgba"], abs=1e-7)


# ---------------------------------------------------------------- symmetry

def test_stereo_mirror_symmetry():
    n = 32
    rng = np.random.default_rng(11)
    half = rng.integers(0, 255, (n, n, n // 2)).astype(np.uint8)
    v = np.concatenate([half, half[:, :, ::-1]], axis=2)  # v[z,y,x] = v[z,y,n-1-x]
    vol = oracle.Volume([oracle.pyramid(v, 2)], 8)
    tf = oracle.make_tf(synth.tf_piecewise(4), 0.0, 255.0)
    W = H = 24
    proj = synth.colmajor(synth.perspective(60.0, 1.0, 0.1, 500.0))
    views = [synth.colmajor(synth.look_at([n / 2 + s * 6.0, n / 2 + 3.0, 70.0], [n / 2 + s * 6.0, n / 2 + 3.0, 0.0],
                                          [0, 1, 0])) for s in (-1.0, 1.0)]
    sel = vol.select([tf], views, [proj, proj], H, tau=8.0)
    assert sel["selected"] > 1
    left = vol.render([tf], sel["leaf"], views[0], proj, W, H)
    right = vol.render([tf], sel["leaf"], views[1], proj, W, H)
    L = left["late"].reshape(H, W, 4)
    R = right["late"].reshape(H, W, 4)[:, ::-1]
    assert np.abs(L - R).max() < 1e-9
    assert np.array_equal(left["count_late"].reshape(H, W), right["count_late"].reshape(H, W)[:, ::-1])


# ---------------------------------------------------------------- optical models and depth termination

def test_emission_only_is_the_rectangle_rule_of_the_emission_integral():
    """Emission-only ("DVR Techniques"): I = integral of the emitted intensity
    along the ray, no absorption, alpha 0. In a constant medium emitting
    alpha * rgb per reference step, n samples of width step give
    n * step / ref * alpha * rgb, whatever the step."""
    n = 16
    vol = oracle.Volume([[np.full((n, n, n), 100, np.uint8)]], n)
    a = float(np.float32(0.05))
    rgb = tuple(float(np.float32(c)) for c in (0.2, 0.5, 0.8))
    tf = _const_tf(rgb, a)
    view, proj = _axial_camera(40.0, cx=8.0, cy=8.0)
    sel = vol.select([tf], [view, view], [proj, proj], 9, tau=1.0)
    c = 4 * 9 + 4
    # (at steps 0.5 and 0.25 a lattice point falls on the exit, which the
    # oracle flags as a possible one-sample difference; the count is exact)
    for step, count in [(0.3, 54), (0.5, 32), (0.25, 64)]:
        r = vol.render([tf], sel["leaf"], view, proj, 9, 9, step=step, pixels=[c], mode=oracle.MODE_EMISSION)
        assert r["count_late"][0] == count and (r["flags"][0] == 0) == (step == 0.3)
        w = count * step / 0.5 * a
        assert r["late"][0] == pytest.approx([w * rgb[0], w * rgb[1], w * rgb[2], 0.0], abs=1e-12)
        assert np.array_equal(r["early"], r["late"])  # no termination


def test_mip_classifies_the_largest_sample():
    """Maximum intensity projection: the transfer function of the largest
    sampled value along the ray, premultiplied. A ray along z through the
    voxel centres of column (8, 8) samples voxel centres exactly at t0 + 0.5
    + k (step 0.5), so the maximum is the largest voxel of the column."""
    n = 16
    a = np.full((n, n, n), 10, np.uint8)
    a[5, 8, 8] = 180      # z = 5
    a[11, 8, 8] = 140     # z = 11: smaller, nearer the eye
    a[3, 2, 2] = 250      # off the ray
    vol = oracle.Volume([[a]], n)
    ramp = np.zeros((256, 4), np.float32)
    ramp[:, 0] = np.linspace(0, 1, 256)
    ramp[:, 1] = 0.5
    ramp[:, 2] = np.linspace(1, 0, 256)
    ramp[:, 3] = np.linspace(0, 1, 256) ** 2
    tf = oracle.make_tf(ramp, 0.0, 255.0)
    view, proj = _axial_camera(40.0, cx=8.5, cy=8.5)
    sel = vol.select([tf], [view, view], [proj, proj], 9, tau=1.0)
    r = vol.render([tf], sel["leaf"], view, proj, 9, 9, pixels=[4 * 9 + 4], mode=oracle.MODE_MIP)
    e = ramp[180].astype(np.float64)  # q = 180 exactly: entry 180
    assert r["late"][0] == pytest.approx([e[3] * e[0], e[3] * e[1], e[3] * e[2], e[3]], abs=1e-12)
    assert r["count_late"][0] == 32


def test_depth_buffer_ends_the_ray_like_an_opaque_surface():
    """Depth-buffer termination: lattice points at or beyond the surface
    distance are not sampled. Constant medium, step 0.5 = reference step:
    a surface at t0 + 4.25 leaves k = 0..8 (9 samples), A = 1 - (1-a)^9; a
    surface before the entry leaves nothing; inf leaves the full ray."""
    n = 16
    vol = oracle.Volume([[np.full((n, n, n), 100, np.uint8)]], n)
    a = float(np.float32(0.05))
    tf = _const_tf((1.0, 1.0, 1.0), a)
    view, proj = _axial_camera(40.0, cx=8.0, cy=8.0)  # entry t0 = 24 along the centre ray
    sel = vol.select([tf], [view, view], [proj, proj], 9, tau=1.0)
    c = 4 * 9 + 4
    for surf, count in [(24.0 + 4.25, 9), (10.0, 0), (np.inf, 32)]:
        depth = np.full((9, 9), np.inf)
        depth.reshape(-1)[c] = surf
        r = vol.render([tf], sel["leaf"], view, proj, 9, 9, pixels=[c], depth=depth)
        assert r["count_late"][0] == count
        assert r["late"][0][3] == pytest.approx(1.0 - (1.0 - a) ** count, abs=1e-12)
    # with a model that scales voxels to metres, depth is in metres
    model = synth.colmajor(synth.scale_translate(0.01, np.zeros(3)))
    volm = oracle.Volume([[np.full((n, n, n), 100, np.uint8)]], n, model=model)
    viewm = synth.colmajor(synth.look_at([0.08, 0.08, 0.40], [0.08, 0.08, 0.0], [0.0, 1.0, 0.0]))
    projm = synth.colmajor(synth.perspective(90.0, 1.0, 0.001, 10.0))
    selm = volm.select([tf], [viewm, viewm], [projm, projm], 9, tau=1.0)
    depth = np.full((9, 9), np.inf)
    depth.reshape(-1)[c] = 0.2825  # 28.25 voxels of 0.01 m
    r = volm.render([tf], selm["leaf"], viewm, projm, 9, 9, pixels=[c], depth=depth)
    assert r["count_late"][0] == 9


# ---------------------------------------------------------------- warped-space rays (DVR for HMD)

def test_identity_lens_casts_the_plain_rays():
    """k1 = k2 = 0, scale 1: every warped pixel looks through its own centre,
    so the warped render equals the plain one exactly."""
    a = synth.gaussians_u8(32, seed=11, count=3)
    vol = oracle.Volume([oracle.pyramid(a, 2)], 16)
    tf = oracle.make_tf(synth.tf_piecewise(2001), 0.0, 255.0)
    view, proj = synth.orbit_camera(32, seed=12, width=24, height=20)
    sel = vol.select([tf], [view, view], [proj, proj], 20)
    plain = vol.render([tf], sel["leaf"], view, proj, 24, 20)
    warped = vol.render([tf], sel["leaf"], view, proj, 24, 20, lens=oracle.lens(0.0, 0.0, 1.0, 24 / 20))
    assert np.array_equal(plain["late"], warped["late"]) and plain["late"][:, 3].max() > 0.05


def test_lens_inverse_solves_the_radial_polynomial():
    """The unwarp point is the preimage: warping it back gives u again, for a
    barrel model with an off-centre lens (brute force round trip)."""
    ln = oracle.lens(0.22, 0.24, 1.0 / 1.46, 0.9, cx=0.08, cy=-0.03)
    rng = np.random.default_rng(4)
    for ux, uy in rng.uniform(-1, 1, (200, 2)):
        wx, wy = oracle.unwarp_point(ln, ux, uy)
        dx, dy = wx - 0.08, wy + 0.03
        r2 = (dx * 0.9) ** 2 + dy ** 2
        f = (1 + 0.22 * r2 + 0.24 * r2 * r2) / 1.46
        assert 0.08 + dx * f == pytest.approx(ux, abs=1e-13) and -0.03 + dy * f == pytest.approx(uy, abs=1e-13)


def test_unwarp_reproduces_a_linear_warped_image():
    """Bilinear taps reproduce an affine image exactly, so unwarping the
    warped image g(w) = a w_x + b w_y + c gives g at the preimage of every
    output pixel (inside the warped image, away from its edge pixels)."""
    ln = oracle.lens(0.2, 0.1, 1.0 / 1.3, 1.0)
    Ww, Hw, W, H = 40, 40, 56, 56
    jj, ii = np.meshgrid(np.arange(Hw), np.arange(Ww), indexing="ij")
    wx, wy = 2 * (ii + 0.5) / Ww - 1, 1 - 2 * (jj + 0.5) / Hw
    g = np.zeros((Hw, Ww, 4), np.float32)
    g[..., 0] = 0.3 * wx + 0.5
    g[..., 1] = -0.2 * wy + 0.5
    g[..., 3] = 1.0
    out = oracle.unwarp(ln, g, W, H)
    checked = 0
    for j in range(H):
        for i in range(W):
            ux, uy = 2 * (i + 0.5) / W - 1, 1 - 2 * (j + 0.5) / H
            px, py = oracle.unwarp_point(ln, ux, uy)
            if abs(px) > 1 - 2.0 / Ww or abs(py) > 1 - 2.0 / Hw:
                continue
            assert out[j, i, 0] == pytest.approx(0.3 * px + 0.5, abs=2e-7)
            assert out[j, i, 1] == pytest.approx(-0.2 * py + 0.5, abs=2e-7)
            assert out[j, i, 3] == pytest.approx(1.0, abs=1e-12)
            checked += 1
    assert checked > W * H // 3


# ---------------------------------------------------------------- gradient and depth-palette tables (Visualization Enhancements)

def _ramp_table(n=256):
    t = np.zeros((n, 4), np.float32)
    t[:, 0] = np.linspace(0, 1, n)
    t[:, 1] = np.linspace(1, 0, n)
    t[:, 2] = 0.25
    t[:, 3] = np.linspace(0, 0.5, n)
    return t


def test_gradient_input_of_a_linear_field_is_its_slope():
    """Central differences of a trilinear linear field are exact: away from
    the clamped border every sample's gradient magnitude is |(3, 5, 7)| =
    sqrt(83) per voxel, so MIP of the gradient input classifies sqrt(83)."""
    n = 16
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    a = (3 * i + 5 * j + 7 * k + 11).astype(np.uint16)
    vol = oracle.Volume([[a]], n)
    tab = _ramp_table()
    tf = oracle.make_tf(tab, 0.0, 20.0, gradient=True)
    view, proj = _axial_camera(40.0, cx=8.3, cy=7.6)
    sel = vol.select([tf], [view, view], [proj, proj], 9, tau=1.0)
    r = vol.render([tf], sel["leaf"], view, proj, 9, 9, pixels=[4 * 9 + 4], mode=oracle.MODE_MIP)
    q = np.sqrt(83.0) / 20.0 * 255.0
    f = q - np.floor(q)
    e = tab[int(q)].astype(np.float64) * (1 - f) + tab[int(q) + 1].astype(np.float64) * f
    assert r["late"][0] == pytest.approx([e[3] * e[0], e[3] * e[1], e[3] * e[2], e[3]], abs=1e-12)


def test_gradient_input_drops_blocks_of_constant_value():
    """With a table that is transparent at gradient 0, a block whose values
    are all equal (gradient bound sqrt(3) (max - min) = 0) is transparent and
    dropped; a block with varying values is not, even where a value table
    would call it transparent."""
    n = 32
    a = np.full((n, n, n), 40, np.uint16)
    rng = np.random.default_rng(9)
    a[:, :, 18:] = rng.integers(30, 50, (n, n, 14))  # block x = 0 and its apron (x <= 16) stay constant
    vol = oracle.Volume([[a]], 16)
    tab = _ramp_table()
    tab[:3, 3] = 0.0
    view, proj = synth.orbit_camera(n, seed=21, width=32, height=32)
    grad = vol.select([oracle.make_tf(tab, 0.0, 200.0, gradient=True)], [view, view], [proj, proj], 32)
    value = vol.select([oracle.make_tf(tab, 1000.0, 2000.0)], [view, view], [proj, proj], 32)
    assert value["selected"] == 0  # every value sits below the value window
    lvl0 = [vol.node_coords(i)[1] for i in np.flatnonzero(grad["state"] == oracle.ST_SELECTED)]
    assert lvl0 and all(b[0] == 1 for b in lvl0)  # only the varying half (x >= 16) survives


def test_depth_palette_colours_by_distance():
    """Constant medium, palette red at the entry distance to blue at the exit
    distance: colour weights follow the arithmetico-geometric series of the
    sample distances (t_k - t0) / 16 under opacity a' per sample."""
    n = 16
    vol = oracle.Volume([[np.full((n, n, n), 100, np.uint8)]], n)
    a = float(np.float32(0.05))
    tf = oracle.make_tf(np.tile(np.array([0.3, 0.3, 0.3, a], np.float32), (256, 1)), 0.0, 255.0,
                        palette=[[1, 0, 0], [0, 0, 1]], near=24.0, far=40.0)
    view, proj = _axial_camera(40.0, cx=8.0, cy=8.0)
    sel = vol.select([tf], [view, view], [proj, proj], 9, tau=1.0)
    r = vol.render([tf], sel["leaf"], view, proj, 9, 9, step=0.3, pixels=[4 * 9 + 4])
    ap = 1.0 - (1.0 - a) ** 0.6
    q, m = 1.0 - ap, 54
    s0 = (1 - q ** m) / (1 - q)
    s1 = q * (1 - m * q ** (m - 1) + (m - 1) * q ** m) / (1 - q) ** 2
    d = 0.3 / 16.0
    assert r["late"][0] == pytest.approx([ap * (s0 - d * s1), 0.0, ap * d * s1, 1 - q ** m], abs=1e-12)


# ---------------------------------------------------------------- the multi-level sample lattice (Octree Representation)

def _x_ray(eye_x, nx, levels, brick=8, a=0.01):
    """Constant volume nx x 8 x 8 (value 100 at every level), a constant
    table of opacity a per reference step 0.5, and a camera on the axis
    y = z = 4 looking along +x (the centre pixel of a 9 x 9 image)."""
    lv = [np.full((8, 8, nx), 100, np.uint8)]
    for _ in range(1, levels):
        s = lv[-1].shape
        lv.append(np.full(((s[0] + 1) // 2, (s[1] + 1) // 2, (s[2] + 1) // 2), 100, np.uint8))
    vol = oracle.Volume([lv], brick)
    tf = _const_tf((0.25, 0.5, 1.0), float(np.float32(a)))
    view = synth.colmajor(synth.look_at([eye_x, 4.0, 4.0], [eye_x + 1.0, 4.0, 4.0], [0.0, 0.0, 1.0]))
    proj = synth.colmajor(synth.perspective(90.0, 1.0, 0.1, 1000.0))
    return vol, tf, view, proj


def _leaf_of_levels(vol, cell_levels):
    """Leaf map of a row of level-0 cells along x: cell i is rendered by the
    block of level cell_levels[i] that contains it."""
    leaf = []
    for i, L in enumerate(cell_levels):
        nbx = vol.blocks_per_axis(L)[0]
        bx = i >> L
        assert bx < nbx
        leaf.append(int(vol.level_offsets[L]) + bx)
    return np.array(leaf, np.int32)


def _lattice_count(x0, step, lo, hi, stride):
    """Brute force with exact rationals: lattice indices k >= 0 with
    x0 + k step in [lo, hi) and k a multiple of stride."""
    from fractions import Fraction as F
    x0, step = F(x0), F(step)
    n = 0
    k = 0
    while x0 + k * step < hi:
        if x0 + k * step >= lo and k % stride == 0:
            n += 1
        k += 1
    return n


@pytest.mark.parametrize("eye_x,levels_of_cells,nlev,step", [
    (-10.0, [1, 1, 0, 0], 2, "0.3"),    # entry at x = 0; a level-1 block, then two level-0 blocks
    (-10.0, [0, 0, 1, 1], 2, "0.3"),    # the reverse
    ("1.15", [1, 1, 0, 0], 2, "0.3"),   # eye inside the volume: the lattice starts at the eye
    ("-7.3", [2, 2, 2, 2, 0, 0, 1, 1], 3, "0.35"),
    ("2.9", [0, 0, 2, 2, 2, 2, 1, 1], 3, "0.35"),
])
def test_each_level_takes_every_2L_th_point_of_one_global_lattice(eye_x, levels_of_cells, nlev, step):
    """A3: samples lie on one lattice t0 + k step anchored at the volume
    entry; a block of level L takes the points k = 0 mod 2^L inside it and
    corrects opacity for the spacing step 2^L. Along an axial ray through a
    constant medium the count per block is the brute-force count of such
    points, and A = 1 - (1 - a)^(sum over samples of step 2^L / 0.5). A
    lattice anchored at each block's entry instead gives other counts on
    these layouts."""
    from fractions import Fraction as F
    nx = 8 * len(levels_of_cells)
    vol, tf, view, proj = _x_ray(float(eye_x), nx, nlev)
    leaf = _leaf_of_levels(vol, levels_of_cells)
    r = vol.render([tf], leaf, view, proj, 9, 9, step=float(step), pixels=[40])
    x0 = max(F(eye_x), F(0))
    count, expo = 0, F(0)
    i = 0
    while i < len(levels_of_cells):
        L = levels_of_cells[i]
        j = i
        while j < len(levels_of_cells) and levels_of_cells[j] == L and (j >> L) == (i >> L):
            j += 1
        n = _lattice_count(x0, F(step), 8 * i, 8 * j, 2 ** L)
        count += n
        expo += n * F(step) * 2 ** L / F("0.5")
        i = j
    a = float(np.float32(0.01))
    A = 1.0 - (1.0 - a) ** float(expo)
    assert r["flags"][0] == 0
    assert r["count_late"][0] == count
    assert r["late"][0] == pytest.approx([0.25 * A, 0.5 * A, 1.0 * A, A], abs=1e-12)
    # the block-entry anchoring this pins against
    if eye_x == -10.0 and levels_of_cells[0] == 1:
        entry_anchor = _lattice_count(0, F(step), 0, 16, 2) + _lattice_count(16, F(step), 16, 32, 1)
        assert entry_anchor != count


def test_a_point_on_a_face_between_levels_has_both_assignments():
    """A16: with step 0.5 the lattice point k = 32 lies exactly on the face
    x = 16 between two level-0 blocks and a level-1 block. Assigned to the
    level-1 block (the exact cell), it is one of that block's samples at
    spacing 1.0; assigned to the level-0 block before the face, it is a
    level-0 sample at spacing 0.5 and the level-1 block starts at k = 34.
    The oracle flags the pixel and enumerates exactly these two results:
    exponents (32 + 16 * 2) and (33 + 15 * 2) reference steps."""
    vol, tf, view, proj = _x_ray(-10.0, 32, 2)
    leaf = _leaf_of_levels(vol, [0, 0, 1, 1])
    r = vol.render([tf], leaf, view, proj, 9, 9, step=0.5, pixels=[40])
    assert r["flags"][0] & oracle.FL_FACE and r["flags"][0] & oracle.FL_TEDGE
    a = float(np.float32(0.01))
    g = r["var_groups"][0]
    n = g["n"][0]
    got = sorted((int(g["count_late"][0][i]), g["late"][0][i][3]) for i in range(n))
    # k = 64 lies on the exit face x = 32 as well: a ray that ends there takes
    # no sample, one that ends a rounding later takes a last level-1 sample
    # (two more reference steps); both are legitimate
    want = sorted((c + extra, 1.0 - (1.0 - a) ** (e + 2 * extra))
                  for c, e in [(32 + 16, 64), (33 + 15, 63)] for extra in (0, 1))
    assert [c for c, _ in got] == [c for c, _ in want]
    for (c, A), (_, Aw) in zip(got, want):
        assert A == pytest.approx(Aw, abs=1e-12)
    # the exact result (the face point in the level-1 block, the exit point
    # not taken) is one of them
    assert int(r["count_late"][0]) == 48
    assert r["late"][0][3] == pytest.approx(1.0 - (1.0 - a) ** 64, abs=1e-12)


def test_a_ray_grazing_a_face_has_one_crossing_per_variant():
    """A ray nearly parallel to the face x = 16 between a level-0 and a
    level-1 block keeps many lattice points within eps of it. A
    floating-point ray crosses that face once, so the legitimate results are
    the m + 1 crossing positions among the m points whose assignment
    matters, not 2^m: the enumeration stays small and every variant's sample
    count lies between the all-before and all-after assignments."""
    vol, tf, view, proj = _x_ray(-10.0, 32, 2)
    leaf = _leaf_of_levels(vol, [0, 0, 1, 1])
    # the centre ray runs along +y, rising 1e-5 voxel in x per voxel of y,
    # from x = 15.99994 where it enters at y = 0; step 0.3: points
    # y_k = 0.3 k, k = 0..26 (the exit y = 8 is not a lattice point), all
    # within 1e-3 of x = 16 (the ray crosses it near k = 20)
    eye = np.array([15.9999, -6.0, 4.0])
    view = synth.colmajor(synth.look_at(eye, eye + np.array([1e-5, 1.0, 0.0]), [0.0, 0.0, 1.0]))
    r = vol.render([tf], leaf, view, proj, 9, 9, step=0.3, pixels=[40])
    assert r["flags"][0] & oracle.FL_FACE and not r["flags"][0] & (oracle.FL_MANY | oracle.FL_TEDGE)
    g = r["var_groups"][-1]
    n = int(g["n"][0])
    # every point's assignment matters (level 0 samples it; level 1 samples
    # even k at level 1 and skips odd k): 27 + 1 crossing positions
    assert n == 28
    cl = np.sort(g["count_late"][0][:n])
    # all before the face: 27 level-0 samples; all after: the 14 even k
    assert cl[0] == 14 and cl[-1] == 27
    assert int(r["count_late"][0]) in cl
