"""ctypes binding of libsg.so (include/sg.h). Argument marshalling only.

Every function here forwards to the C entry point of the same name; device
buffers are passed as raw pointers (e.g. torch tensors' data_ptr()) and
streams as cudaStream_t handles (torch.cuda.Stream.cuda_stream). There is no
fallback: if libsg.so is missing or fails to load, importing this module
raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# SG_LIBRARY may point at another build of the same library (e.g. a tuning variant)
LIB_PATH = os.environ.get("SG_LIBRARY") or os.path.join(HERE, "libsg.so")

SG_OK, SG_ERR_INVALID_ARG, SG_ERR_OOM, SG_ERR_CUDA, SG_ERR_NOT_RESIDENT, SG_ERR_TIMEOUT, SG_ERR_STATE, SG_ERR_IO = range(8)
SG_U8, SG_U16 = 1, 2
SG_MODE_EMISSION_ABSORPTION, SG_MODE_EMISSION, SG_MODE_MIP = 0, 1, 2
SG_INPUT_VALUE, SG_INPUT_GRADIENT = 0, 1
STATUS_NAMES = {0: "SG_OK", 1: "SG_ERR_INVALID_ARG", 2: "SG_ERR_OOM", 3: "SG_ERR_CUDA", 4: "SG_ERR_NOT_RESIDENT",
                5: "SG_ERR_TIMEOUT", 6: "SG_ERR_STATE", 7: "SG_ERR_IO"}

EXPORTS = ["sg_volume_create", "sg_volume_destroy", "sg_upload_volume_device", "sg_upload_bricks",
           "sg_set_transfer_function", "sg_select_lod", "sg_select_lod_batch", "sg_read_selection", "sg_read_brick",
           "sg_render", "sg_render_host", "sg_render_host_async", "sg_render_host_wait", "sg_render_batch", "sg_set_render_config", "sg_get_render_config",
           "sg_autotune_render", "sg_render_config_store", "sg_render_config_lookup", "sg_select_lod_noalloc", "sg_read_residency", "sg_set_brick_ranges", "sg_unet_create", "sg_unet_destroy",
           "sg_unet_param_count", "sg_unet_get_params", "sg_unet_set_params", "sg_unet_forward", "sg_unet_backward",
           "sg_unet_adam_step", "sg_unet_set_tensor_path", "sg_unet_check", "sg_unet_wait_selftest", "sg_unet_save", "sg_unet_load", "sg_render_learned", "sg_psnr", "sg_read_ranges", "sg_upload_brick_list", "sg_unwarp", "sg_set_channel_shading",
           "sg_container_create", "sg_container_open", "sg_container_append", "sg_container_finish",
           "sg_container_get_info", "sg_container_read", "sg_container_close", "sg_host_cache_create",
           "sg_host_cache_destroy", "sg_host_cache_fetch", "sg_host_cache_clear_failures", "sg_stream_requests",
           "sg_stream_requests_async", "sg_host_cache_prefetch", "sg_host_cache_wait", "sg_upload_brick_list_async",
           "sg_last_error",
           "sg_version"]


class SGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class sg_volume_desc(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 3), ("dtype", ctypes.c_int32), ("channels", ctypes.c_int32),
                ("timepoints", ctypes.c_int32), ("brick_size", ctypes.c_int32), ("apron", ctypes.c_int32),
                ("lod_levels", ctypes.c_int32), ("skip_block", ctypes.c_int32), ("device_pool_bytes", ctypes.c_uint64),
                ("model", ctypes.c_float * 16)]


class sg_pose(ctypes.Structure):
    _fields_ = [("view", (ctypes.c_float * 16) * 2), ("proj", (ctypes.c_float * 16) * 2), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("pixel_error", ctypes.c_float), ("t", ctypes.c_int32),
                ("slot", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class sg_select_stats(ctypes.Structure):
    _fields_ = [("selected", ctypes.c_uint32), ("culled", ctypes.c_uint32), ("empty", ctypes.c_uint32),
                ("requested", ctypes.c_uint32), ("fallback", ctypes.c_uint32), ("nonempty", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32 * 2)]


class sg_container_info(ctypes.Structure):
    _fields_ = [("desc", sg_volume_desc), ("chunks", ctypes.c_int64), ("nodes", ctypes.c_int64),
                ("raw_bytes", ctypes.c_uint64), ("compressed_bytes", ctypes.c_uint64), ("complete", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class sg_stream_stats(ctypes.Structure):
    _fields_ = [("requested", ctypes.c_int32), ("served", ctypes.c_int32), ("host_hits", ctypes.c_int32),
                ("disk_reads", ctypes.c_int32), ("missing", ctypes.c_int32), ("failed", ctypes.c_int32),
                ("disk_bytes", ctypes.c_uint64), ("upload_bytes", ctypes.c_uint64), ("queued", ctypes.c_int32),
                ("in_flight", ctypes.c_int32)]


class sg_lens(ctypes.Structure):
    _fields_ = [("k1", ctypes.c_float), ("k2", ctypes.c_float), ("scale", ctypes.c_float), ("aspect", ctypes.c_float),
                ("centre", (ctypes.c_float * 2) * 2)]


def make_lens(k1, k2, scale=0.0, aspect=0.0, centres=((0.0, 0.0), (0.0, 0.0))):
    ln = sg_lens()
    ln.k1, ln.k2, ln.scale, ln.aspect = k1, k2, scale, aspect
    for e in range(2):
        ln.centre[e][0], ln.centre[e][1] = centres[e]
    return ln


class sg_render_params(ctypes.Structure):
    _fields_ = [("step", ctypes.c_float), ("term_alpha", ctypes.c_float), ("mode", ctypes.c_int32),
                ("empty_skip", ctypes.c_int32), ("sample_count", ctypes.c_void_p * 2),
                ("sample_total", ctypes.c_void_p), ("depth", ctypes.c_void_p * 2),
                ("lens", ctypes.POINTER(sg_lens)), ("touched", ctypes.c_void_p)]


class sg_render_config(ctypes.Structure):
    _fields_ = [("persistent", ctypes.c_int32), ("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32),
                ("rays_per_thread", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]

    def as_dict(self):
        return dict(persistent=self.persistent, tile_w=self.tile_w, tile_h=self.tile_h,
                    rays_per_thread=self.rays_per_thread)


class sg_learned_params(ctypes.Structure):
    _fields_ = [("step", ctypes.c_float), ("term_alpha", ctypes.c_float), ("pixel_error_half", ctypes.c_float),
                ("threshold_db", ctypes.c_float), ("judge", ctypes.c_int32), ("half_slot", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2), ("half_config", sg_render_config),
                ("full_config", sg_render_config)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libsg.so not built at {LIB_PATH}: run python -m paper_1804_08197_b300.build")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float
    P = ctypes.POINTER
    sig = {
        "sg_volume_create": [P(sg_volume_desc), P(vp)],
        "sg_volume_destroy": [vp],
        "sg_upload_volume_device": [vp, i32, i32, vp, vp],
        "sg_upload_bricks": [vp, i32, i32, i32, i32, vp, vp, vp],
        "sg_upload_brick_list": [vp, i32, i32, i32, vp, vp, P(ctypes.c_int32), vp],
        "sg_upload_brick_list_async": [vp, i32, i32, i32, vp, vp, P(ctypes.c_int32), vp],
        "sg_unwarp": [P(sg_lens), P(vp), i32, i32, P(vp), i32, i32, vp],
        "sg_set_channel_shading": [vp, i32, i32, vp, i32, f32, f32, vp],
        "sg_container_create": [ctypes.c_char_p, P(sg_volume_desc), P(vp)],
        "sg_container_open": [ctypes.c_char_p, P(vp)],
        "sg_container_append": [vp, i32, i32, i32, i32, i32, i32, vp, ctypes.c_uint32, ctypes.c_uint32],
        "sg_container_finish": [vp],
        "sg_container_get_info": [vp, P(sg_container_info)],
        "sg_container_read": [vp, i32, i32, i64, vp, vp],
        "sg_container_close": [vp],
        "sg_host_cache_create": [vp, ctypes.c_uint64, i32, i32, P(vp)],
        "sg_host_cache_destroy": [vp],
        "sg_host_cache_fetch": [vp, i32, i32, i64, P(vp), P(ctypes.c_int)],
        "sg_host_cache_clear_failures": [vp],
        "sg_stream_requests": [vp, i32, vp, ctypes.c_uint64, P(sg_stream_stats), vp],
        "sg_stream_requests_async": [vp, i32, vp, ctypes.c_uint64, P(sg_stream_stats), vp],
        "sg_host_cache_prefetch": [vp, i32, i32, P(ctypes.c_int64), i32, P(i32)],
        "sg_host_cache_wait": [vp, P(i32)],
        "sg_set_transfer_function": [vp, i32, vp, i32, f32, f32, f32, vp],
        "sg_select_lod": [vp, P(sg_pose), P(sg_select_stats), vp],
        "sg_select_lod_batch": [vp, P(sg_pose), i32, vp],
        "sg_read_selection": [vp, i32, vp, i64, vp, i64, vp, i32, vp, vp],
        "sg_read_brick": [vp, i32, i32, i32, i32, i32, i32, vp, vp],
        "sg_read_residency": [vp, i32, vp, i64],
        "sg_read_ranges": [vp, i32, vp, i64],
        "sg_set_brick_ranges": [vp, i32, i32, i32, i32, vp, vp, vp],
        "sg_unet_create": [i32, i32, i32, ctypes.c_uint64, P(vp)],
        "sg_unet_destroy": [vp],
        "sg_unet_param_count": [vp, P(i64)],
        "sg_unet_get_params": [vp, vp, i64, i32],
        "sg_unet_set_params": [vp, vp, i64],
        "sg_unet_forward": [vp, vp, i64, i32, i32, i32, vp, i64, vp],
        "sg_unet_backward": [vp, vp, i64, vp, i64, vp, vp],
        "sg_unet_adam_step": [vp, f32, f32, f32, f32, vp],
        "sg_psnr": [vp, vp, i64, vp, vp],
        "sg_unet_set_tensor_path": [vp, i32],
        "sg_unet_check": [vp],
        "sg_unet_wait_selftest": [vp, ctypes.c_uint32, vp],
        "sg_unet_save": [vp, ctypes.c_char_p],
        "sg_unet_load": [vp, ctypes.c_char_p],
        "sg_render_learned": [vp, vp, P(sg_pose), P(sg_learned_params), P(vp), vp, vp, vp],
        "sg_render": [vp, P(sg_pose), P(sg_render_params), P(vp), vp],
        "sg_render_host": [vp, P(sg_pose), P(sg_render_params), P(vp), vp],
        "sg_render_host_async": [vp, P(sg_pose), P(sg_render_params), P(vp), vp],
        "sg_render_host_wait": [vp, i32],
        "sg_render_batch": [vp, P(sg_pose), i32, P(sg_render_params), P(vp), vp],
        "sg_select_lod_noalloc": [vp, P(sg_pose), vp, vp, vp, vp, vp, vp],
        "sg_set_render_config": [vp, P(sg_render_config)],
        "sg_get_render_config": [vp, P(sg_render_config)],
        "sg_render_config_store": [ctypes.c_char_p, ctypes.c_char_p, P(sg_render_config)],
        "sg_render_config_lookup": [ctypes.c_char_p, ctypes.c_char_p, P(sg_render_config), P(ctypes.c_int)],
        "sg_autotune_render": [vp, P(sg_pose), i32, P(sg_render_params), P(vp), i32, P(sg_render_config),
                               P(ctypes.c_float), vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.sg_last_error.restype = ctypes.c_char_p
    L.sg_last_error.argtypes = []
    L.sg_version.restype = ctypes.c_char_p
    L.sg_version.argtypes = []
    return L


lib = _load()


def _check(status):
    if status != SG_OK:
        raise SGError(status, lib.sg_last_error().decode())


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(x.ctypes.data)  # numpy


# --------------------------------------------------------------------------- entry points

def sg_version():
    return lib.sg_version().decode()


def sg_volume_create(dims, dtype, brick_size, lod_levels, channels=1, timepoints=1, apron=1,
                     device_pool_bytes=0, model=None, skip_block=0):
    d = sg_volume_desc()
    d.dims[:] = [int(x) for x in dims]
    d.dtype = dtype
    d.channels = channels
    d.timepoints = timepoints
    d.brick_size = brick_size
    d.apron = apron
    d.lod_levels = lod_levels
    d.device_pool_bytes = device_pool_bytes
    d.skip_block = skip_block
    m = [1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1] if model is None else [float(x) for x in model]
    d.model[:] = m
    h = ctypes.c_void_p()
    _check(lib.sg_volume_create(ctypes.byref(d), ctypes.byref(h)))
    return h


def sg_volume_destroy(vol):
    _check(lib.sg_volume_destroy(vol))


def sg_upload_volume_device(vol, t, c, dev_level0, stream=None):
    _check(lib.sg_upload_volume_device(vol, t, c, _ptr(dev_level0), _stream(stream)))


def sg_upload_bricks(vol, t, c, level, brick_xyz, host, stream=None):
    import numpy as np
    xyz = np.ascontiguousarray(brick_xyz, np.int32).reshape(-1, 3)
    _check(lib.sg_upload_bricks(vol, t, c, level, len(xyz), _ptr(xyz), _ptr(host), _stream(stream)))


def sg_upload_brick_list(vol, t, c, nodes, host_ptrs, stream=None, asynchronous=False):
    """Uploads bricks by node id from per-brick host pointers (ints, numpy
    arrays or tensors); returns how many (a prefix of the list) were cached.
    asynchronous=True: sg_upload_brick_list_async (copies queued; keep the
    host bricks unchanged until the stream has passed them)."""
    import numpy as np
    ids = np.ascontiguousarray(nodes, np.int32).reshape(-1)
    ptrs = _ptr_array(host_ptrs) if len(ids) else None
    done = ctypes.c_int32(0)
    fn = lib.sg_upload_brick_list_async if asynchronous else lib.sg_upload_brick_list
    _check(fn(vol, t, c, len(ids), _ptr(ids), ptrs, ctypes.byref(done), _stream(stream)))
    return done.value


def sg_set_transfer_function(vol, c, rgba, lo, hi, ref_step=0.5, stream=None):
    import numpy as np
    tab = np.ascontiguousarray(rgba, np.float32).reshape(-1, 4)
    _check(lib.sg_set_transfer_function(vol, c, _ptr(tab), len(tab), lo, hi, ref_step, _stream(stream)))


def volume_desc(dims, dtype, brick_size, lod_levels, channels=1, timepoints=1, model=None):
    d = sg_volume_desc()
    d.dims[:] = [int(x) for x in dims]
    d.dtype, d.channels, d.timepoints, d.brick_size, d.apron, d.lod_levels = dtype, channels, timepoints, brick_size, 1, lod_levels
    m = [1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1] if model is None else [float(x) for x in model]
    d.model[:] = m
    return d


def sg_container_create(path, desc):
    h = ctypes.c_void_p()
    _check(lib.sg_container_create(str(path).encode(), ctypes.byref(desc), ctypes.byref(h)))
    return h


def sg_container_open(path):
    h = ctypes.c_void_p()
    _check(lib.sg_container_open(str(path).encode(), ctypes.byref(h)))
    return h


def sg_container_append(k, t, c, level, bx, by, bz, brick, vmin, vmax):
    _check(lib.sg_container_append(k, t, c, level, bx, by, bz, _ptr(brick), int(vmin), int(vmax)))


def sg_container_finish(k):
    _check(lib.sg_container_finish(k))


def sg_container_get_info(k):
    info = sg_container_info()
    _check(lib.sg_container_get_info(k, ctypes.byref(info)))
    return dict(chunks=info.chunks, nodes=info.nodes, raw_bytes=info.raw_bytes,
                compressed_bytes=info.compressed_bytes, complete=bool(info.complete))


def sg_container_read(k, t, c, node, out):
    mm = (ctypes.c_uint32 * 2)()
    _check(lib.sg_container_read(k, t, c, node, _ptr(out), mm))
    return int(mm[0]), int(mm[1])


def sg_container_close(k):
    _check(lib.sg_container_close(k))


def sg_host_cache_create(k, nbytes, pinned=False, threads=8):
    h = ctypes.c_void_p()
    _check(lib.sg_host_cache_create(k, int(nbytes), int(bool(pinned)), int(threads), ctypes.byref(h)))
    return h


def sg_host_cache_destroy(hc):
    _check(lib.sg_host_cache_destroy(hc))


def sg_host_cache_fetch(hc, t, c, node):
    """(address of the cached brick, hit)"""
    p, hit = ctypes.c_void_p(), ctypes.c_int(0)
    _check(lib.sg_host_cache_fetch(hc, t, c, node, ctypes.byref(p), ctypes.byref(hit)))
    return p.value, bool(hit.value)


def sg_stream_requests(vol, slot, hc, max_bytes, stream=None, asynchronous=False):
    """Serves a selection's requests; returns the stats as a dict. A call in
    which some chunks failed (SG_ERR_IO) still served the others: it returns
    the stats (failed > 0) instead of raising. asynchronous=True: the
    non-blocking form (sg_stream_requests_async)."""
    st = sg_stream_stats()
    fn = lib.sg_stream_requests_async if asynchronous else lib.sg_stream_requests
    status = fn(vol, slot, hc, int(max_bytes), ctypes.byref(st), _stream(stream))
    if status != SG_ERR_IO:
        _check(status)
    out = {f[0]: getattr(st, f[0]) for f in sg_stream_stats._fields_}
    if status == SG_ERR_IO and out["failed"] == 0:
        _check(status)  # an I/O error that left no stats
    return out


def sg_host_cache_clear_failures(hc):
    _check(lib.sg_host_cache_clear_failures(hc))


def sg_host_cache_prefetch(hc, t, c, nodes):
    """Queues background loads of the listed bricks; returns how many were queued."""
    import numpy as np
    arr = np.ascontiguousarray(nodes, np.int64)
    q = ctypes.c_int32(0)
    _check(lib.sg_host_cache_prefetch(hc, t, c, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(arr),
                                      ctypes.byref(q)))
    return q.value


def sg_host_cache_wait(hc):
    """Waits for the background loads; returns how many failed."""
    f = ctypes.c_int32(0)
    _check(lib.sg_host_cache_wait(hc, ctypes.byref(f)))
    return f.value


def sg_set_channel_shading(vol, c, gradient=False, palette=None, near=0.0, far=1.0, stream=None):
    """Channel c's table reads the gradient magnitude (gradient=True) or the
    value; palette: optional (m, 3) RGB in [0, 1] indexed by world distance
    from the eye over [near, far]."""
    import numpy as np
    pal = None if palette is None else np.ascontiguousarray(palette, np.float32).reshape(-1, 3)
    _check(lib.sg_set_channel_shading(vol, c, SG_INPUT_GRADIENT if gradient else SG_INPUT_VALUE, _ptr(pal),
                                      0 if pal is None else len(pal), near, far, _stream(stream)))


def make_pose(views, projs, width, height, pixel_error=1.0, t=0, slot=0):
    p = sg_pose()
    for e in range(2):
        p.view[e][:] = [float(x) for x in views[e]]
        p.proj[e][:] = [float(x) for x in projs[e]]
    p.width, p.height = int(width), int(height)
    p.pixel_error = pixel_error
    p.t, p.slot = t, slot
    return p


def sg_select_lod(vol, pose, stats=False, stream=None):
    st = sg_select_stats() if stats else None
    _check(lib.sg_select_lod(vol, ctypes.byref(pose), ctypes.byref(st) if st is not None else None, _stream(stream)))
    if st is not None:
        return dict(selected=st.selected, culled=st.culled, empty=st.empty, requested=st.requested,
                    fallback=st.fallback, nonempty=st.nonempty)
    return None


def sg_select_lod_batch(vol, poses, stream=None):
    arr = (sg_pose * len(poses))(*poses)
    _check(lib.sg_select_lod_batch(vol, arr, len(poses), _stream(stream)))


def sg_read_selection(vol, slot, ncell, nnode, req_cap=1 << 16, stream=None):
    import numpy as np
    cells = np.empty(ncell, np.int32)
    state = np.empty(nnode, np.uint8)
    req = np.empty(req_cap, np.int32)
    nreq = ctypes.c_int32(0)
    _check(lib.sg_read_selection(vol, slot, _ptr(cells), ncell, _ptr(state), nnode, _ptr(req), req_cap,
                                 ctypes.byref(nreq), _stream(stream)))
    return cells, state, req[: min(nreq.value, req_cap)].copy()


def sg_read_brick(vol, t, c, level, bx, by, bz, host_out, stream=None):
    _check(lib.sg_read_brick(vol, t, c, level, bx, by, bz, _ptr(host_out), _stream(stream)))


def render_params(step=0.5, term_alpha=0.99, empty_skip=1, sample_count=None, sample_total=None,
                  mode=SG_MODE_EMISSION_ABSORPTION, depth=None, lens=None, touched=None):
    """depth: optional pair of device float buffers (H, W) per eye, the world
    distance along each pixel's ray to an opaque surface (inf = none).
    lens: optional sg_lens (make_lens) for rays through the warped image; the
    structure must stay alive while the parameters are used. touched:
    optional device uint8 buffer, one byte per cache slot, set for every
    brick a sample was taken from (a diagnostic render)."""
    r = sg_render_params()
    if touched is not None:
        r.touched = _ptr(touched).value
    if lens is not None:
        r.lens = ctypes.pointer(lens)
    if sample_total is not None:
        r.sample_total = _ptr(sample_total).value
    r.step, r.term_alpha, r.mode, r.empty_skip = step, term_alpha, mode, empty_skip
    if sample_count is not None:
        r.sample_count[0] = _ptr(sample_count[0]).value
        r.sample_count[1] = _ptr(sample_count[1]).value
    if depth is not None:
        r.depth[0] = _ptr(depth[0]).value
        r.depth[1] = _ptr(depth[1]).value
    return r


def sg_unwarp(lens, warped, Ww, Hw, outs, W, H, stream=None):
    """Unwarps both eyes: warped/outs are pairs of device RGBA float buffers."""
    wa = (ctypes.c_void_p * 2)(_ptr(warped[0]).value, _ptr(warped[1]).value)
    oa = (ctypes.c_void_p * 2)(_ptr(outs[0]).value, _ptr(outs[1]).value)
    _check(lib.sg_unwarp(ctypes.byref(lens), wa, Ww, Hw, oa, W, H, _stream(stream)))


def sg_render(vol, pose, params, outs, stream=None):
    arr = (ctypes.c_void_p * 2)(_ptr(outs[0]).value, _ptr(outs[1]).value)
    _check(lib.sg_render(vol, ctypes.byref(pose), ctypes.byref(params), arr, _stream(stream)))


def sg_render_host(vol, pose, params, host_outs, stream=None):
    arr = (ctypes.c_void_p * 2)(_ptr(host_outs[0]).value, _ptr(host_outs[1]).value)
    _check(lib.sg_render_host(vol, ctypes.byref(pose), ctypes.byref(params), arr, _stream(stream)))


def sg_render_host_async(vol, pose, params, host_outs, stream=None):
    """Pipelined host render (see include/sg.h): returns before the images land."""
    arr = (ctypes.c_void_p * 2)(_ptr(host_outs[0]).value, _ptr(host_outs[1]).value)
    _check(lib.sg_render_host_async(vol, ctypes.byref(pose), ctypes.byref(params), arr, _stream(stream)))


def sg_render_host_wait(vol, all=True):
    _check(lib.sg_render_host_wait(vol, 1 if all else 0))


def sg_render_batch(vol, poses, params, outs, stream=None):
    parr = (sg_pose * len(poses))(*poses)
    oarr = (ctypes.c_void_p * len(outs))(*[_ptr(o).value for o in outs])
    _check(lib.sg_render_batch(vol, parr, len(poses), ctypes.byref(params), oarr, _stream(stream)))


def sg_set_render_config(vol, persistent=0, tile_w=0, tile_h=0, rays_per_thread=1):
    c = sg_render_config()
    c.persistent, c.tile_w, c.tile_h, c.rays_per_thread = persistent, tile_w, tile_h, rays_per_thread
    _check(lib.sg_set_render_config(vol, ctypes.byref(c)))


def sg_get_render_config(vol):
    c = sg_render_config()
    _check(lib.sg_get_render_config(vol, ctypes.byref(c)))
    return c.as_dict()


def sg_autotune_render(vol, poses, params, outs, reps=3, stream=None):
    """Returns (best config dict, mean ms per launch); the volume keeps the best."""
    parr = (sg_pose * len(poses))(*poses)
    oarr = (ctypes.c_void_p * len(outs))(*[_ptr(o).value for o in outs])
    best = sg_render_config()
    ms = ctypes.c_float(0.0)
    _check(lib.sg_autotune_render(vol, parr, len(poses), ctypes.byref(params), oarr, reps, ctypes.byref(best),
                                  ctypes.byref(ms), _stream(stream)))
    return best.as_dict(), ms.value


def sg_select_lod_noalloc(vol, pose, leaf, cell_node, node_state, req, counters, stream=None):
    """Allocation-free selection into caller-owned device buffers (see include/sg.h)."""
    _check(lib.sg_select_lod_noalloc(vol, ctypes.byref(pose), _ptr(leaf), _ptr(cell_node), _ptr(node_state),
                                     _ptr(req), _ptr(counters), _stream(stream)))


def sg_read_residency(vol, t, nnode):
    import numpy as np
    out = np.empty(nnode, np.int32)
    _check(lib.sg_read_residency(vol, t, _ptr(out), nnode))
    return out


def sg_set_brick_ranges(vol, t, c, level, brick_xyz, minmax, stream=None):
    import numpy as np
    xyz = np.ascontiguousarray(brick_xyz, np.int32).reshape(-1, 3)
    mm = np.ascontiguousarray(minmax, np.uint32).reshape(-1, 2)
    _check(lib.sg_set_brick_ranges(vol, t, c, level, len(xyz), _ptr(xyz), _ptr(mm), _stream(stream)))


# --------------------------------------------------------------------------- learned reconstruction

def _ptr_array(xs):
    return (ctypes.c_void_p * len(xs))(*[_ptr(x).value for x in xs])


def sg_unet_create(max_batch, max_h, max_w, seed=1):
    h = ctypes.c_void_p()
    _check(lib.sg_unet_create(max_batch, max_h, max_w, seed, ctypes.byref(h)))
    return h


def sg_unet_destroy(net):
    _check(lib.sg_unet_destroy(net))


def sg_unet_param_count(net):
    n = ctypes.c_int64(0)
    _check(lib.sg_unet_param_count(net, ctypes.byref(n)))
    return n.value


def sg_unet_get_params(net, which=0):
    import numpy as np
    n = sg_unet_param_count(net)
    out = np.empty(n, np.float32)
    _check(lib.sg_unet_get_params(net, _ptr(out), n, which))
    return out


def sg_unet_set_params(net, params):
    import numpy as np
    p = np.ascontiguousarray(params, np.float32)
    _check(lib.sg_unet_set_params(net, _ptr(p), len(p)))


def sg_unet_forward(net, ins, in_pitch, h, w, outs, out_pitch, stream=None):
    """ins/outs: lists of device buffers (or int pointers); pitches in floats."""
    _check(lib.sg_unet_forward(net, _ptr_array(ins), in_pitch, len(ins), h, w, _ptr_array(outs), out_pitch,
                               _stream(stream)))


def sg_unet_backward(net, targets, target_pitch, outs, out_pitch, loss=None, stream=None):
    _check(lib.sg_unet_backward(net, _ptr_array(targets), target_pitch, _ptr_array(outs), out_pitch, _ptr(loss),
                                _stream(stream)))


def sg_unet_adam_step(net, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib.sg_unet_adam_step(net, lr, beta1, beta2, eps, _stream(stream)))


def sg_psnr(a, b, count, out_db, stream=None):
    _check(lib.sg_psnr(_ptr(a), _ptr(b), count, _ptr(out_db), _stream(stream)))


def sg_unet_set_tensor_path(net, tcgen05=1):
    _check(lib.sg_unet_set_tensor_path(net, tcgen05))


def sg_unet_check(net):
    _check(lib.sg_unet_check(net))


def sg_unet_save(net, path):
    _check(lib.sg_unet_save(net, os.fsencode(str(path))))


def sg_unet_load(net, path):
    _check(lib.sg_unet_load(net, os.fsencode(str(path))))


def learned_params(step=0.5, term_alpha=0.99, pixel_error_half=0.0, threshold_db=40.0, judge=False, half_slot=201,
                   half_config=None, full_config=None):
    p = sg_learned_params()
    p.step, p.term_alpha, p.pixel_error_half, p.threshold_db = step, term_alpha, pixel_error_half, threshold_db
    p.judge, p.half_slot = int(bool(judge)), half_slot
    for name, cfg in (("half_config", half_config), ("full_config", full_config)):
        if cfg:
            c = getattr(p, name)
            c.persistent, c.tile_w, c.tile_h, c.rays_per_thread = (cfg["persistent"], cfg["tile_w"], cfg["tile_h"],
                                                                   cfg["rays_per_thread"])
    return p


def sg_render_learned(vol, net, pose, params, outs, psnr_db=None, fell_back=None, stream=None):
    """A learned stereo frame into outs (two device buffers); psnr_db (3
    floats) and fell_back (one int32) are device buffers, needed when judging."""
    _check(lib.sg_render_learned(vol, net, ctypes.byref(pose), ctypes.byref(params), _ptr_array(outs), _ptr(psnr_db),
                                 _ptr(fell_back), _stream(stream)))


def sg_unet_wait_selftest(net, polls, stream=None):
    """Failure-detection self-test: a bounded wait that nothing satisfies
    gives up after `polls` polls and raises the network's error word."""
    _check(lib.sg_unet_wait_selftest(net, int(polls), _stream(stream)))


def sg_read_ranges(vol, t, nnode, channels=1):
    import numpy as np
    out = np.empty((nnode, channels, 2), np.uint32)
    _check(lib.sg_read_ranges(vol, t, _ptr(out), nnode))
    return out


def sg_read_requests(vol, slot, cap=1 << 16, stream=None):
    """Requested node ids of a selection (ascending), without the other outputs."""
    import numpy as np
    req = np.empty(cap, np.int32)
    nreq = ctypes.c_int32(0)
    _check(lib.sg_read_selection(vol, slot, None, 0, None, 0, _ptr(req), cap, ctypes.byref(nreq), _stream(stream)))
    return req[: min(nreq.value, cap)].copy()


def sg_render_config_store(path, key, cfg):
    """Appends the autotuner's pick (a dict as sg_autotune_render returns) for key."""
    c = sg_render_config()
    c.persistent, c.tile_w, c.tile_h, c.rays_per_thread = (cfg["persistent"], cfg["tile_w"], cfg["tile_h"],
                                                           cfg["rays_per_thread"])
    _check(lib.sg_render_config_store(os.fsencode(str(path)), key.encode(), ctypes.byref(c)))


def sg_render_config_lookup(path, key):
    """The stored pick for key as a dict, or None."""
    c = sg_render_config()
    found = ctypes.c_int(0)
    _check(lib.sg_render_config_lookup(os.fsencode(str(path)), key.encode(), ctypes.byref(c), ctypes.byref(found)))
    return c.as_dict() if found.value else None
