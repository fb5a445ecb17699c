"""Seeded synthetic inputs shaped like the paper's microscopy workloads.

Volumes come from the C generators in ``synth.c`` (counter-based randomness,
so any sub-box can be regenerated alone); transfer functions, cameras and head
poses are built here with numpy's seeded PCG64. Nothing in this module
performs any step of the rendering method: it only produces inputs, which the
CUDA path and the CPU oracle both consume.

Conventions: volume arrays are numpy (z, y, x), x fastest; matrices are 4x4
column-major float32 in OpenGL conventions (clip z in [-1, 1]); voxel space is
[0, N]^3 with voxel centres at integer + 0.5.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_GPU_SRC = os.path.join(_HERE, "synth_gpu.cu")
_GPU_LIB = os.path.join(_HERE, "libsynth_gpu.so")
_lib = None
_gpu_lib = None


def build(force=False):
    """Compile the generator library with gcc (OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", _LIB, "-lm"])
    return _LIB


def build_gpu(force=False):
    """Compile the GPU twin of the cell-body generator with nvcc (sm_103a)."""
    if force or not os.path.exists(_GPU_LIB) or os.path.getmtime(_GPU_LIB) < os.path.getmtime(_GPU_SRC):
        nvcc = "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared",
                               "-Xcompiler", "-fPIC", _GPU_SRC, "-o", _GPU_LIB + ".tmp"])
        os.replace(_GPU_LIB + ".tmp", _GPU_LIB)
    return _GPU_LIB


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        u64, i32, dbl, vp = ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        _lib.sy_gaussians_u8.argtypes = [vp, i32, i32, i32, u64, i32, dbl]
        _lib.sy_filaments_u16.argtypes = [vp, i32, i32, i32, u64, i32, dbl, dbl, dbl, dbl, dbl]
        _lib.sy_filaments_u16.restype = i32
        _lib.sy_blobs_u16.argtypes = [vp, i32, i32, i32, u64, i32, i32, i32, dbl]
        _lib.sy_cells_u8_box.argtypes = [vp, ctypes.c_long, u64, ctypes.c_long, ctypes.c_long,
                                         ctypes.c_long, i32, i32, i32, i32]
        _lib.sy_cell_table.argtypes = [vp, ctypes.c_long, u64, i32]
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


# --------------------------------------------------------------------------- volumes

def gaussians_u8(n=128, seed=1001, count=8, noise=16.0):
    """Sum of `count` isotropic Gaussians (centres U[0.2,0.8] N, sigma U[6,20],
    amplitude U[80,255]) plus U[0,noise] noise, rounded and clamped, uint8."""
    out = np.empty((n, n, n), np.uint8)
    _load().sy_gaussians_u8(_ptr(out), n, n, n, seed, count, noise)
    return out


def filaments_u16(dims=(1024, 1024, 1024), seed=1002, ntubes=200, lam=300.0,
                  radius=(2.0, 6.0), intensity=(2000.0, 60000.0)):
    """Catmull-Rom tubes (4-6 control points, radius U[2,6], intensity
    U[2000,60000] with a 1-voxel linear falloff) max-combined over a
    Poisson(lam) background, uint16. dims = (nx, ny, nz)."""
    nx, ny, nz = dims
    out = np.empty((nz, ny, nx), np.uint16)
    _load().sy_filaments_u16(_ptr(out), nx, ny, nz, seed, ntubes, lam, radius[0], radius[1],
                             intensity[0], intensity[1])
    return out


def blobs_u16(dims=(512, 512, 256), seed=1003, channel=0, t=0, nblobs=40, noise=100.0):
    """Gaussian blobs drifting 1-3 voxels per time point and growing 1-2 %
    per time point, plus U[0,noise] noise, uint16, for channel `channel`."""
    nx, ny, nz = dims
    out = np.empty((nz, ny, nx), np.uint16)
    _load().sy_blobs_u16(_ptr(out), nx, ny, nz, seed, channel, t, nblobs, noise)
    return out


def cells_u8_box(N, x0, y0, z0, sx, sy, sz, seed=1004, cell=64):
    """Box [x0,x0+sx) x [y0,y0+sy) x [z0,z0+sz) of the procedural cell-body
    volume of edge N (jittered `cell`-voxel grid, a sphere per cell with p=0.6,
    radius U[cell/8, 5 cell/8], interior U[120,160], 2-voxel membrane 230,
    background 20, + N(0,8) noise). Coordinates outside [0,N) are clamped,
    which replicates the edge."""
    out = np.empty((sz, sy, sx), np.uint8)
    _load().sy_cells_u8_box(_ptr(out), N, seed, x0, y0, z0, sx, sy, sz, cell)
    return out


def cells_u8_device(N, dev_ptr, seed=1004, cell=64, z0=0, nz=None):
    """Slices [z0, z0 + nz) of the same cell-body volume as cells_u8_box,
    generated on the current GPU into device memory at dev_ptr (nz * N * N
    bytes, x fastest). The cell parameters come from the CPU code; distances
    and noise are FP32, so a small fraction of voxels (sphere boundaries,
    rounding of the noisy value) may differ from cells_u8_box."""
    global _gpu_lib
    nz = N - z0 if nz is None else nz
    if _gpu_lib is None:
        build_gpu()
        _gpu_lib = ctypes.CDLL(_GPU_LIB)
        _gpu_lib.sy_cells_u8_gpu.argtypes = [ctypes.c_void_p, ctypes.c_long, ctypes.c_uint64, ctypes.c_long,
                                             ctypes.c_long, ctypes.c_int, ctypes.c_void_p, ctypes.c_long]
    ng = (N + cell - 1) // cell
    table = np.empty(ng * ng * ng * 8, np.float32)
    _load().sy_cell_table(_ptr(table), N, seed, cell)
    err = _gpu_lib.sy_cells_u8_gpu(ctypes.c_void_p(dev_ptr), N, seed, z0, nz, cell, _ptr(table), ng)
    if err != 0:
        raise RuntimeError(f"sy_cells_u8_gpu failed with CUDA error {err}")


# --------------------------------------------------------------------------- transfer functions

def tf_piecewise(seed=2001, n=256, points=6, alpha_max=0.2, zero_alpha_points=1, zero_span=(4, 20),
                 colour=None):
    """Seeded piecewise-linear RGBA table of `n` entries from `points` control
    points at 0, sorted U(1, n-2) positions, and n-1. RGB U[0,1] (or the fixed
    `colour`), alpha U[0, alpha_max]; the first `zero_alpha_points` points have
    alpha 0 (with two, the second sits at U(zero_span) so the low end of the
    window is fully transparent). Returns float32 (n, 4)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    inner = np.sort(rng.uniform(1, n - 2, points - 2))
    if zero_alpha_points >= 2:
        inner[0] = rng.uniform(*zero_span)
        inner = np.sort(np.concatenate([inner[:1], np.maximum(inner[1:], inner[0] + 1)]))
    pos = np.concatenate([[0.0], inner, [n - 1.0]])
    rgb = rng.uniform(0, 1, (points, 3)) if colour is None else np.tile(np.asarray(colour, float), (points, 1))
    a = rng.uniform(0, alpha_max, points)
    a[:zero_alpha_points] = 0.0
    xs = np.arange(n, dtype=np.float64)
    tab = np.stack([np.interp(xs, pos, rgb[:, 0]), np.interp(xs, pos, rgb[:, 1]),
                    np.interp(xs, pos, rgb[:, 2]), np.interp(xs, pos, a)], axis=1)
    return tab.astype(np.float32)


# --------------------------------------------------------------------------- cameras

def perspective(fovy_deg, aspect, near=0.01, far=100.0):
    f = 1.0 / np.tan(np.radians(fovy_deg) / 2.0)
    m = np.zeros((4, 4))
    m[0, 0] = f / aspect
    m[1, 1] = f
    m[2, 2] = (far + near) / (near - far)
    m[2, 3] = 2.0 * far * near / (near - far)
    m[3, 2] = -1.0
    return m


def look_at(eye, target, up):
    eye, target, up = (np.asarray(v, np.float64) for v in (eye, target, up))
    f = target - eye
    f /= np.linalg.norm(f)
    s = np.cross(f, up)
    s /= np.linalg.norm(s)
    u = np.cross(s, f)
    m = np.eye(4)
    m[0, :3], m[1, :3], m[2, :3] = s, u, -f
    m[:3, 3] = -m[:3, :3] @ eye
    return m


def colmajor(m):
    """4x4 row-major numpy -> flat column-major float32[16]."""
    return np.asarray(m, np.float64).T.reshape(16).astype(np.float32)


def scale_translate(s, t):
    m = np.eye(4)
    m[0, 0] = m[1, 1] = m[2, 2] = s
    m[:3, 3] = t
    return m


def _unit(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def orbit_camera(n=128, seed=3001, fovy=45.0, width=256, height=256, radius_widths=2.0):
    """One perspective view from a seeded point on a sphere of radius
    radius_widths * n voxels around the volume centre, looking at the centre.
    Model = identity (world = voxel units). Returns (view, proj) column-major."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = np.full(3, n / 2.0)
    eye = c + radius_widths * n * _unit(rng)
    up = np.array([0.0, 0.0, 1.0]) if abs(eye[2] - c[2]) < 0.9 * radius_widths * n else np.array([0.0, 1.0, 0.0])
    return colmajor(look_at(eye, c, up)), colmajor(perspective(fovy, width / height, 0.1, 10.0 * n))


def head_poses(count=64, seed=3002, extent_m=0.5, dist=(0.3, 1.0), gaze_half=0.125, roll_deg=10.0,
               ipd=0.064, fovy=100.0, width=1440, height=1600):
    """Seeded stereo head poses around a volume of world extent `extent_m`
    centred at the origin: head at U[dist] from the centre in a uniform
    direction, gazing at a uniform point of the central half, rolled U[-10,10]
    degrees; eyes at head -/+ ipd/2 along the head's x axis with parallel
    axes. Returns a list of (views[2], projs[2]) column-major float32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    proj = colmajor(perspective(fovy, width / height, 0.01, 10.0))
    poses = []
    for _ in range(count):
        head = _unit(rng) * rng.uniform(*dist)
        target = rng.uniform(-gaze_half, gaze_half, 3) * (extent_m / 0.5)
        f = target - head
        f /= np.linalg.norm(f)
        up0 = np.array([0.0, 0.0, 1.0]) if abs(f[2]) < 0.95 else np.array([0.0, 1.0, 0.0])
        s = np.cross(f, up0); s /= np.linalg.norm(s)
        u = np.cross(s, f)
        roll = np.radians(rng.uniform(-roll_deg, roll_deg))
        up = np.cos(roll) * u + np.sin(roll) * s
        s = np.cross(f, up); s /= np.linalg.norm(s)
        views = []
        for sign in (-1.0, 1.0):
            e = head + sign * 0.5 * ipd * s
            views.append(colmajor(look_at(e, e + f, up)))
        poses.append((views, [proj, proj]))
    return poses


def volume_model(n_vox, extent_m):
    """Model matrix mapping voxel space [0, n_vox]^3 onto a cube of side
    extent_m centred at the origin (uniform scale)."""
    s = extent_m / float(n_vox)
    return colmajor(scale_translate(s, np.full(3, -extent_m / 2.0)))


def flythrough_poses(count=256, seed=3004, extent_m=1.0, ipd=0.064, fovy=100.0, width=1440, height=1600):
    """Seeded Catmull-Rom fly-through that starts outside a volume of world
    extent `extent_m` (centred at the origin) and wanders through its central
    part; each pose looks a little ahead along the path. Returns a list of
    (views[2], projs[2]) column-major float32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    e = extent_m
    start = _unit(rng) * 1.2 * e
    pts = [start * 1.3, start] + [rng.uniform(-0.3 * e, 0.3 * e, 3) for _ in range(5)] + [rng.uniform(-0.3 * e, 0.3 * e, 3)]

    def cr(p0, p1, p2, p3, t):
        return 0.5 * (2 * p1 + (-p0 + p2) * t + (2 * p0 - 5 * p1 + 4 * p2 - p3) * t * t +
                      (-p0 + 3 * p1 - 3 * p2 + p3) * t ** 3)

    nseg = len(pts) - 3
    path = []
    for i in range(count + 1):
        u = i / count * nseg
        k = min(int(u), nseg - 1)
        path.append(cr(pts[k], pts[k + 1], pts[k + 2], pts[k + 3], u - k))
    proj = colmajor(perspective(fovy, width / height, 0.005, 10.0))
    poses = []
    for i in range(count):
        head, ahead = path[i], path[i + 1]
        f = ahead - head
        if np.linalg.norm(f) < 1e-9:
            f = -head
        f = f / np.linalg.norm(f)
        up = np.array([0.0, 0.0, 1.0]) if abs(f[2]) < 0.95 else np.array([0.0, 1.0, 0.0])
        s = np.cross(f, up)
        s /= np.linalg.norm(s)
        views = [colmajor(look_at(head + k * 0.5 * ipd * s, head + k * 0.5 * ipd * s + f, up)) for k in (-1.0, 1.0)]
        poses.append((views, [proj, proj]))
    return poses
