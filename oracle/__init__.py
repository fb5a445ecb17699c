"""FP64 CPU oracle of the DVR hot path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg
may import this package. It wraps ``oracle.c`` (plain C, FP64, OpenMP over
pixels) with ctypes and numpy and shares no code with the CUDA path.

Public functions:
  pyramid(level0, levels)           -> list of global level arrays
  Volume(levels_per_channel, brick, model)
  Volume.block_ranges()             -> uint32 [node, channel, 2]
  Volume.select(tfs, views, projs, height, tau, resident=None)
  Volume.render(tfs, leaf, view, proj, W, H, step, ...)
  Volume.sample(level, channel, p)  -> trilinear value
  tf_table(tf, spacing), classify(tf, table, value)
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

MAX_LEVELS = 16
MAX_CH = 4

ST_UNSEEN, ST_CULLED, ST_EMPTY, ST_SELECTED, ST_FALLBACK, ST_REFINED = range(6)
# pixel flags of Volume.render: FL_FACE / FL_TEDGE mark pixels with lattice
# points within eps of a face between differently sampled cells / of the
# ray's end (resolved: every legitimate assignment is enumerated), FL_TERM a
# termination decision within term_tol, FL_ENTRY an eye within eps of a
# volume face and FL_MANY more assignments than the cap (both unresolved)
FL_FACE, FL_TEDGE, FL_TERM, FL_ENTRY, FL_MANY = 1, 2, 4, 8, 16
MODE_EA, MODE_EMISSION, MODE_MIP = 0, 1, 2


def build(force=False):
    """Compile the oracle with gcc: FP64, no fused multiply-add contraction."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", _SRC, "-o", _LIB, "-lm"])
    return _LIB


class _Vol(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("levels", ctypes.c_int32), ("brick", ctypes.c_int32),
                ("nch", ctypes.c_int32), ("dims", (ctypes.c_int64 * 3) * MAX_LEVELS),
                ("data", (ctypes.c_void_p * MAX_CH) * MAX_LEVELS), ("model", ctypes.c_double * 16)]


class _TF(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("lo", ctypes.c_float), ("hi", ctypes.c_float),
                ("ref_step", ctypes.c_float), ("rgba", ctypes.c_void_p), ("input", ctypes.c_int32),
                ("m", ctypes.c_int32), ("pnear", ctypes.c_float), ("pfar", ctypes.c_float),
                ("palette", ctypes.c_void_p)]


def _load():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        L.or_pyramid_level.argtypes = [vp, i32, vp, vp]
        L.or_node_count.argtypes = [vp, vp]
        L.or_node_count.restype = i64
        L.or_block_ranges.argtypes = [vp, vp]
        L.or_select.argtypes = [vp, vp, vp, vp, vp, i32, dbl, vp, vp, vp, vp, i32, vp, vp]
        L.or_cache_place.argtypes = [vp, i64, ctypes.c_uint64, vp, vp, vp, i32, vp, vp]
        L.or_cache_place.restype = i32
        L.or_select.restype = i32
        L.or_select_inputs.argtypes = [vp, vp, vp, i32, dbl, vp, vp, vp]
        L.or_sample.argtypes = [vp, i32, i32, vp]
        L.or_sample.restype = dbl
        L.or_tf_table.argtypes = [vp, dbl, vp]
        L.or_classify.argtypes = [vp, vp, dbl, vp]
        L.or_render.argtypes = [vp, vp, vp, vp, vp, i32, i32, dbl, dbl, dbl, dbl, vp, i64,
                                vp, vp, vp, vp, vp, i32, i32, vp, vp]
        L.or_render_variants.argtypes = [vp, vp, vp, vp, vp, i32, i32, dbl, dbl, dbl, dbl, vp, i64, i32,
                                         vp, vp, vp, vp, vp, i32, i32, vp, vp]
        L.or_render_variants.restype = i32
        L.or_lens_unwarp_point.argtypes = [vp, dbl, dbl, vp, vp]
        L.or_unwarp.argtypes = [vp, vp, i32, i32, vp, i32, i32]
        L.or_render.restype = i32
        L.or_max_threads.restype = i32
        _lib = L
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def max_threads():
    return _load().or_max_threads()


def level_dims(dims0, levels):
    """(nx, ny, nz) of every level: N_{L+1} = ceil(N_L / 2)."""
    out = [tuple(int(d) for d in dims0)]
    for _ in range(1, levels):
        out.append(tuple((d + 1) // 2 for d in out[-1]))
    return out


def pyramid(level0, levels):
    """Global arrays of every level from a (z, y, x) level-0 array."""
    lib = _load()
    out = [np.ascontiguousarray(level0)]
    dt = 1 if level0.dtype == np.uint8 else 2
    for _ in range(1, levels):
        src = out[-1]
        sd = np.array([src.shape[2], src.shape[1], src.shape[0]], np.int64)
        dst = np.empty(((src.shape[0] + 1) // 2, (src.shape[1] + 1) // 2, (src.shape[2] + 1) // 2), src.dtype)
        lib.or_pyramid_level(_p(src), dt, _p(sd), _p(dst))
        out.append(dst)
    return out


class Lens(ctypes.Structure):
    """Radial lens model of one eye ("DVR for HMD"): warped NDC w looks
    through undistorted NDC u = c + (w - c) (1 + k1 r^2 + k2 r^4) scale,
    r^2 = ((w - c)_x aspect)^2 + (w - c)_y^2."""
    _fields_ = [("k1", ctypes.c_double), ("k2", ctypes.c_double), ("scale", ctypes.c_double),
                ("aspect", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double)]


def lens(k1, k2, scale, aspect, cx=0.0, cy=0.0):
    return Lens(float(k1), float(k2), float(scale), float(aspect), float(cx), float(cy))


def unwarp_point(ln, ux, uy):
    wx, wy = ctypes.c_double(), ctypes.c_double()
    _load().or_lens_unwarp_point(ctypes.byref(ln), float(ux), float(uy), ctypes.byref(wx), ctypes.byref(wy))
    return wx.value, wy.value


def unwarp(ln, warped, W, H):
    """warped: (Hw, Ww, 4) float32 RGBA -> (H, W, 4) FP64 in the undistorted space."""
    w = np.ascontiguousarray(warped, np.float32)
    out = np.zeros((H, W, 4))
    _load().or_unwarp(ctypes.byref(ln), _p(w), w.shape[1], w.shape[0], _p(out), W, H)
    return out


INPUT_VALUE, INPUT_GRADIENT = 0, 1


def make_tf(table, lo, hi, ref_step=0.5, gradient=False, palette=None, near=0.0, far=1.0):
    """Transfer function of one channel; keeps the numpy arrays alive
    alongside the ctypes struct. gradient: the table reads the gradient
    magnitude (value units per level-0 voxel) instead of the value; palette:
    (m, 3) RGB replacing the table's colour, indexed by the sample's world
    distance from the eye over [near, far]."""
    t = np.ascontiguousarray(table, np.float32)
    s = _TF(t.shape[0], lo, hi, ref_step, t.ctypes.data)
    s.input = INPUT_GRADIENT if gradient else INPUT_VALUE
    s._keep = [t]
    if palette is not None:
        pal = np.ascontiguousarray(palette, np.float32).reshape(-1, 3)
        s.m, s.pnear, s.pfar, s.palette = pal.shape[0], near, far, pal.ctypes.data
        s._keep.append(pal)
    return s


def _tf_array(tfs):
    arr = (_TF * len(tfs))()
    for i, t in enumerate(tfs):
        arr[i] = t
    return arr


class Volume:
    """Global multi-resolution volume as the oracle sees it.

    channels: list (per channel) of lists (per level) of (z, y, x) arrays.
    brick: block edge B; model: column-major voxel -> world matrix."""

    def __init__(self, channels, brick, model=None):
        self.channels = [[np.ascontiguousarray(a) for a in ch] for ch in channels]
        self.levels = len(self.channels[0])
        self.brick = int(brick)
        self.nch = len(self.channels)
        s = _Vol()
        s.dtype = 1 if self.channels[0][0].dtype == np.uint8 else 2
        s.levels, s.brick, s.nch = self.levels, self.brick, self.nch
        self.level_dims = []
        for L in range(self.levels):
            a = self.channels[0][L]
            s.dims[L][0], s.dims[L][1], s.dims[L][2] = a.shape[2], a.shape[1], a.shape[0]
            self.level_dims.append((a.shape[2], a.shape[1], a.shape[0]))
            for c in range(self.nch):
                s.data[L][c] = self.channels[c][L].ctypes.data
        self._finish(s, model)

    @classmethod
    def layout(cls, dims, brick, levels, model=None, dtype=np.uint8, nch=1):
        """A volume of the given layout (level-0 dims (x, y, z); each level
        halves every axis, rounding up, as pyramid() does) with no voxel
        data: for the selection only, which reads the geometry, the block
        ranges (pass them to select) and the residency, never a voxel."""
        self = cls.__new__(cls)
        self.channels = None
        self.levels, self.brick, self.nch = int(levels), int(brick), int(nch)
        s = _Vol()
        s.dtype = 1 if np.dtype(dtype) == np.uint8 else 2
        s.levels, s.brick, s.nch = self.levels, self.brick, self.nch
        self.level_dims = []
        d = [int(x) for x in dims]
        for L in range(self.levels):
            s.dims[L][0], s.dims[L][1], s.dims[L][2] = d
            self.level_dims.append(tuple(d))
            d = [(x + 1) // 2 for x in d]
        self._finish(s, model)
        return self

    def _finish(self, s, model):
        m = np.eye(4).T.reshape(16) if model is None else np.asarray(model, np.float64)
        self.model = np.asarray(m, np.float64).reshape(16).copy()
        for i in range(16):
            s.model[i] = float(m[i])
        self._s = s
        offs = np.zeros(MAX_LEVELS + 1, np.int64)
        self.node_count = _load().or_node_count(ctypes.byref(s), _p(offs))
        self.level_offsets = offs[: self.levels + 1].copy()

    def blocks_per_axis(self, L):
        return tuple((d + self.brick - 1) // self.brick for d in self.level_dims[L])

    def node_coords(self, node_id):
        L = int(np.searchsorted(self.level_offsets, node_id, side="right") - 1)
        nbx, nby, _ = self.blocks_per_axis(L)
        r = int(node_id - self.level_offsets[L])
        return L, (r % nbx, (r // nbx) % nby, r // (nbx * nby))

    def block_ranges(self):
        out = np.zeros((self.node_count, self.nch, 2), np.uint32)
        _load().or_block_ranges(ctypes.byref(self._s), _p(out))
        return out

    def select(self, tfs, views, projs, height, tau=1.0, resident=None, ranges=None, req_cap=1 << 20):
        """LOD + residency selection for a stereo pose (pass the same view
        twice for a single view). Returns dict(leaf, state, requests,
        selected, used); used marks the blocks whose cache stamps this
        traversal renews."""
        if ranges is None and self.channels is None:
            raise ValueError("a layout-only volume needs the block ranges")
        if ranges is None:
            ranges = self.block_ranges()
        nb0 = self.blocks_per_axis(0)
        leaf = np.empty(nb0[2] * nb0[1] * nb0[0], np.int32)
        state = np.zeros(self.node_count, np.uint8)
        used = np.zeros(self.node_count, np.uint8)
        req = np.zeros(req_cap, np.int32)
        nreq = ctypes.c_int(0)
        v = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float64).reshape(16) for x in views]))
        p = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float64).reshape(16) for x in projs]))
        res = None if resident is None else np.ascontiguousarray(resident, np.uint8)
        nsel = _load().or_select(ctypes.byref(self._s), _tf_array(tfs), _p(np.ascontiguousarray(ranges)),
                                 _p(v), _p(p), int(height), float(tau), _p(res), _p(leaf), _p(state),
                                 _p(req), req_cap, ctypes.byref(nreq), _p(used))
        return dict(leaf=leaf, state=state, requests=req[: nreq.value].copy(), selected=nsel, used=used.astype(bool))

    def select_inputs(self, views, projs, height, tau=1.0):
        eyes = np.zeros(6, np.int64)
        planes = np.zeros(32, np.int64)
        K = ctypes.c_uint64(0)
        v = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float64).reshape(16) for x in views]))
        p = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float64).reshape(16) for x in projs]))
        _load().or_select_inputs(ctypes.byref(self._s), _p(v), _p(p), int(height), float(tau), _p(eyes),
                                 _p(planes), ctypes.byref(K))
        return eyes.reshape(2, 3), planes.reshape(2, 4, 4), K.value

    def sample(self, L, c, p):
        pp = np.ascontiguousarray(p, np.float64)
        return _load().or_sample(ctypes.byref(self._s), int(L), int(c), _p(pp))

    def render(self, tfs, leaf, view, proj, W, H, step=0.5, term=0.99, term_tol=1e-4, eps=1e-3,
               pixels=None, nthreads=0, mode=MODE_EA, depth=None, lens=None, variants=True, var_cap=1024):
        """Cast rays for `pixels` (flat ids j*W+i; None = all). Returns dict
        with early/late RGBA (n,4) FP64, sample counts and flags, all for the
        exact assignment of lattice points to cells.

        mode: MODE_EA (emission-absorption), MODE_EMISSION (emission only),
        MODE_MIP (maximum intensity projection). depth: optional (H, W)
        distances in world units from the eye along each pixel's ray to an
        opaque surface that ends the ray (inf = none); converted to level-0
        voxels with the model's uniform scale. lens: a Lens for rays through
        the warped image (W x H is then the warped image's size).

        variants: for every pixel flagged FL_FACE or FL_TEDGE, also every
        legitimate result (one per assignment of its ambiguous lattice
        points, at most var_cap): var_idx (positions of those pixels in this
        result) and var_groups, a list of dicts with idx (positions), n
        (results per pixel: 0 = more than the group's cap, -1 = in a later
        group), early / late (m, k, 4) and count_early / count_late (m, k)."""
        pix = None if pixels is None else np.ascontiguousarray(pixels, np.int64)
        tmax = self._tmax(depth)
        n = W * H if pix is None else len(pix)
        e = np.zeros((n, 4)); l = np.zeros((n, 4))
        ce = np.zeros(n, np.uint32); cl = np.zeros(n, np.uint32); fl = np.zeros(n, np.uint8)
        v = np.ascontiguousarray(np.asarray(view, np.float64).reshape(16))
        p = np.ascontiguousarray(np.asarray(proj, np.float64).reshape(16))
        lf = np.ascontiguousarray(leaf, np.int32)
        tfa = _tf_array(tfs)
        ok = _load().or_render(ctypes.byref(self._s), tfa, _p(lf), _p(v), _p(p), W, H, step, term, term_tol, eps,
                               _p(pix), n, _p(e), _p(l), _p(ce), _p(cl), _p(fl), int(nthreads), int(mode), _p(tmax),
                               ctypes.byref(lens) if lens is not None else None)
        if not ok:
            raise ValueError("singular view/projection/model matrix")
        out = dict(early=e, late=l, count_early=ce, count_late=cl, flags=fl)
        if variants:
            idx = np.flatnonzero(fl & (FL_FACE | FL_TEDGE))
            ids = np.ascontiguousarray(idx if pix is None else pix[idx], np.int64)
            args = (tfa, lf, v, p, W, H, step, term, term_tol, eps, nthreads, mode, tmax, lens)
            groups = []
            first = self._variants(args, ids, 32)
            over = first["n"] == 0
            first["idx"] = idx
            groups.append(first)
            if over.any():
                # the few pixels with many assignments, with a larger cap
                second = self._variants(args, ids[over], var_cap)
                second["idx"] = idx[over]
                first["n"][over] = -1  # handled by the second group
                groups.append(second)
            out["var_groups"] = groups
            out["var_idx"] = idx
        return out

    def _variants(self, args, ids, cap):
        tfa, lf, v, p, W, H, step, term, term_tol, eps, nthreads, mode, tmax, lens = args
        m = len(ids)
        ve = np.zeros((m, cap, 4)); vl = np.zeros((m, cap, 4))
        vce = np.zeros((m, cap), np.uint32); vcl = np.zeros((m, cap), np.uint32)
        vn = np.zeros(m, np.int32)
        if m:
            _load().or_render_variants(ctypes.byref(self._s), tfa, _p(lf), _p(v), _p(p), W, H, step, term, term_tol,
                                       eps, _p(np.ascontiguousarray(ids, np.int64)), m, int(cap), _p(ve), _p(vl),
                                       _p(vce), _p(vcl), _p(vn), int(nthreads), int(mode), _p(tmax),
                                       ctypes.byref(lens) if lens is not None else None)
        k = max(int(vn.max()) if m else 1, 1)
        return dict(n=vn, early=ve[:, :k].copy(), late=vl[:, :k].copy(), count_early=vce[:, :k].copy(),
                    count_late=vcl[:, :k].copy())

    def _tmax(self, depth):
        if depth is None:
            return None
        m = np.asarray(self.model, np.float64).reshape(4, 4).T  # column-major -> row-major
        voxel = np.linalg.norm(m[:3, 0])
        return np.ascontiguousarray(np.asarray(depth, np.float64).reshape(-1) / voxel)


class Cache:
    """The GPU brick cache as the oracle sees it ("Volumetric Data Cashing"):
    at most `slots` resident blocks, each with the frame of its last use.
    Mirror every selection with select(...) (frames count selections, as the
    library's do) and every placement with place(...)."""

    def __init__(self, volume, slots):
        self.vol = volume
        self.slots = int(slots)
        self.resident = np.zeros(volume.node_count, np.uint8)
        self.stamp = np.zeros(volume.node_count, np.uint64)
        self.frame = 0

    def select(self, tfs, views, projs, height, tau=1.0, ranges=None):
        self.frame += 1
        ref = self.vol.select(tfs, views, projs, height, tau=tau, resident=self.resident, ranges=ranges)
        self.stamp[ref["used"] & (self.resident != 0)] = self.frame
        return ref

    def place(self, req):
        """Places req in order; returns (requests processed, evicted ids)."""
        r = np.ascontiguousarray(req, np.int32)
        ev = np.zeros(max(len(r), 1), np.int32)
        nev = ctypes.c_int(0)
        m = _load().or_cache_place(ctypes.byref(self.vol._s), self.slots, ctypes.c_uint64(self.frame),
                                   _p(self.resident), _p(self.stamp), _p(r), len(r), _p(ev), ctypes.byref(nev))
        return m, ev[: nev.value].copy()


def tf_table(tf, spacing):
    out = np.zeros((tf.n, 4))
    _load().or_tf_table(ctypes.byref(tf), float(spacing), _p(out))
    return out


def classify(tf, table, value):
    out = np.zeros(4)
    t = np.ascontiguousarray(table, np.float64)
    _load().or_classify(ctypes.byref(tf), _p(t), float(value), _p(out))
    return out
