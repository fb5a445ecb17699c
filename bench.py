"""Stereo DVR throughput of the B300 library on the bricked multi-LOD workload.

Workload (one "step" = one stereo frame: LOD/residency selection + ray casting
of both eyes for one head pose): a 1024^3 uint16 volume of 200 seeded
Catmull-Rom filaments (radius 2-6, intensity 2000-60000) over a Poisson(300)
background, 64^3 bricks with a one-voxel apron, 4 pyramid levels; 64 seeded
head poses (0.3-1.0 m from a 0.5 m volume, 64 mm IPD, 100 deg fovy), two
1440x1600 eyes, step 0.5 voxel, tau 1 pixel, early termination at 0.99.
Synthetic data; the brick pool (2.7 GB) is far larger than L2, and every step
renders a different pose.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). Under torchrun each rank renders its own poses
(replicas, weak scaling); timing is the max over ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "stereo fps @2x1440x1600 + Gsamples/s; learned vs plain fps at >=40 dB PSNR"
W_EYE, H_EYE = 1440, 1600
N_VOX, BRICK, LEVELS, NPOSES = 1024, 64, 4, 64
SEEDS = dict(volume=1002, tf=2002, poses=3002)
WINDOW = (300.0, 60000.0)
STEP, TAU, TERM = 0.5, 1.0, 0.99
WORKLOAD = ("bricked multi-LOD stereo: 1024^3 u16 filaments, 64^3 bricks + apron, 4 levels, "
            "64 head poses, 2x1440x1600, step 0.5, tau 1 px")


def workload_config(extra=None):
    c = {"workload": WORKLOAD, "volume": [N_VOX] * 3, "dtype_voxels": "u16", "brick": BRICK, "apron": 1,
         "lod_levels": LEVELS, "poses": NPOSES, "eye": [W_EYE, H_EYE], "step_voxels": STEP, "tau_px": TAU,
         "term_alpha": TERM, "l2": "inputs larger than L2 (2.7 GB brick pool, a different pose every step)"}
    if extra:
        c.update(extra)
    return c


def rank_poses(seq, rank, world):
    """This rank's pose order for weak scaling: rank r takes r, r + world,
    r + 2 world, ... (cyclically), so the first k steps of all ranks render
    k * world different poses while there are enough."""
    return [seq[(rank + world * i) % len(seq)] for i in range(len(seq))]


def max_over_ranks(ms, world, device):
    """The job's time: the slowest rank's (all-reduce MAX; a no-op on one rank)."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def make_inputs(n_vox=N_VOX):
    import synth
    vol = synth.filaments_u16((n_vox,) * 3, seed=SEEDS["volume"], ntubes=max(1, 200 * n_vox // N_VOX))
    tf = synth.tf_piecewise(SEEDS["tf"], zero_alpha_points=2)
    poses = synth.head_poses(NPOSES, seed=SEEDS["poses"], width=W_EYE, height=H_EYE)
    model = synth.volume_model(n_vox, 0.5)
    return vol, tf, poses, model


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self, window=None):
        """Median SM clock and the throttle reasons of the samples taken within
        window (host perf_counter seconds: the timed region), or of all
        samples if none fell within it."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        inside = [ln for t, ln in self.lines if window and window[0] <= t <= window[1]]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in inside or [ln for _, ln in self.lines]:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "samples_in_timed_region": len(inside),
                "interval_ms": 50}


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def measured_peak_bf16():
    """Dense BF16 tensor peak (TFLOP/s): the burst figure, for kernels timed in
    sub-millisecond bursts like the U-Net forward."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured (burst)"
    except Exception:
        return 1800.0, "fallback"


def tensor_roofline(tflops):
    peak, kind = measured_peak_bf16()
    return {"bound": "tensor", "achieved": round(tflops, 1), "peak": peak, "unit": "TFLOP/s",
            "frac": round(tflops / peak, 4), "peak_source": kind,
            "scope": "3x3 convolution FLOPs over the whole forward, elementwise kernels included"}


def profiled_traffic(alg_bytes):
    """DRAM bytes per render launch from the committed ncu summary, scaled to
    this run's algorithmic bytes; None if the kernel changed since."""
    import hashlib
    try:
        rec = {}
        for line in open(os.path.join(ROOT, "profiles", "render_traffic.txt")):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                rec[k.strip()] = v.strip()
        sha = hashlib.sha256(open(os.path.join(ROOT, "paper_1804_08197_b300", "csrc", "render.cu"), "rb").read())
        if sha.hexdigest()[:16] != rec["render_cu_sha256_16"]:
            return None
        return int(float(rec["traffic_bytes_per_launch"]) * alg_bytes / float(rec["algorithmic_bytes_per_launch"]))
    except (OSError, KeyError, ValueError):
        return None


def cpu_baseline(vol, tf_table, poses, model, pose_ids, stride=32, npose_1core=4, stride_1core=512):
    """The FP64 oracle, as it stands, on bounded pixel samples of the bench poses.

    Block value ranges are an ingest quantity: computed once, untimed. A
    frame is one selection plus every pixel of both eyes; the sample times
    each pose's selection and every `stride`-th pixel, extrapolates only the
    per-pixel work, and reports frames / total time over the poses pose_ids:
    the GPU arm's timed poses, which the reference arm run with the same
    --steps / --warmup steps through too (the cost varies a lot from pose to
    pose). Also timed: the same on one core and the full 256 x 256 view of
    the plain 128^3 u8 ray-cast workload."""
    import oracle
    import synth
    t_setup = time.perf_counter()
    ovol = oracle.Volume([oracle.pyramid(vol, LEVELS)], BRICK, model=model)
    otf = oracle.make_tf(tf_table, *WINDOW)
    ranges = ovol.block_ranges()
    setup_s = time.perf_counter() - t_setup
    npix = W_EYE * H_EYE

    def frames(ids, stride, nthreads):
        total_s, samples, busy = 0.0, 0, 0.0
        for i in ids:
            views, projs = poses[i % len(poses)]
            t0 = time.perf_counter()
            sel = ovol.select([otf], views, projs, H_EYE, tau=TAU, ranges=ranges)
            t_sel = time.perf_counter() - t0
            t_pix = 0.0
            for e in range(2):
                pix = np.arange((i * 13 + e * 7) % stride, npix, stride)
                t1 = time.perf_counter()
                r = ovol.render([otf], sel["leaf"], views[e], projs[e], W_EYE, H_EYE, step=STEP, pixels=pix,
                                nthreads=nthreads, variants=False)
                t_pix += time.perf_counter() - t1
                samples += int(r["count_late"].sum()) * stride
            total_s += t_sel + t_pix * stride  # the whole frame: selection + every pixel
            busy += t_sel + t_pix
        return total_s, samples, busy

    cores = oracle.max_threads()
    npose = len(pose_ids)
    frame_s, samples, busy = frames(pose_ids, stride, 0)
    frame1_s, samples1, busy1 = frames(pose_ids[:npose_1core], stride_1core, 1)
    npose_1core = min(npose_1core, npose)
    # the plain single-view workload: 128^3 u8 Gaussians, one 256 x 256 view
    a = synth.gaussians_u8(128, seed=1001)
    v1 = oracle.Volume([[a]], 128)
    tf1 = oracle.make_tf(synth.tf_piecewise(2001), 0.0, 255.0)
    view1, proj1 = synth.orbit_camera(128, seed=3001, width=256, height=256)
    t0 = time.perf_counter()
    sel1 = v1.select([tf1], [view1, view1], [proj1, proj1], 256)
    r1 = v1.render([tf1], sel1["leaf"], view1, proj1, 256, 256, step=0.5, variants=False)
    c1_s = time.perf_counter() - t0
    return {"value": round(npose / frame_s, 6), "unit": "stereo frames/s", "cores": cores, "kind": "oracle",
            "sample": f"{npose} poses (ids {pose_ids[0]}..{pose_ids[-1]} mod {len(poses)}: the GPU arm's timed poses), "
                      f"each with its selection and every {stride}th pixel of both eyes "
                      f"({busy:.1f} s timed), per-pixel time extrapolated to full 2 x {W_EYE} x {H_EYE} frames "
                      f"({frame_s:.1f} s for {npose}); block ranges computed once at ingest (untimed)",
            "msamples_per_s": round(samples / frame_s / 1e6, 3), "setup_s": round(setup_s, 2),
            "one_core": {"value": round(npose_1core / frame1_s, 6), "unit": "stereo frames/s", "cores": 1,
                         "msamples_per_s": round(samples1 / frame1_s / 1e6, 3),
                         "sample": f"the first {min(npose_1core, npose)} of those poses, every {stride_1core}th pixel, "
                                   f"{busy1:.1f} s"},
            "plain_256": {"value": round(1.0 / c1_s, 4), "unit": "images/s", "cores": cores,
                          "msamples_per_s": round(int(r1["count_late"].sum()) / c1_s / 1e6, 3),
                          "sample": "the full 256 x 256 view of 128^3 u8 Gaussians with its selection"}}


BATCH_DIMS, BATCH_T, BATCH_RES = (512, 512, 256), 16, [(1440, 1600), (1080, 1200), (720, 800)]


def batched_4d(sg, torch, dev, reps=10):
    """Batched 4D multichannel render: 16 time points of a 512x512x256 u16
    volume with 2 channels (drifting, growing blobs; green/magenta tables,
    additive blend), 3 stereo viewers at 1440x1600, 1080x1200 and 720x800:
    96 images of uneven sizes per persistent launch, select + render captured
    in one CUDA graph and replayed. Configuration chosen by the autotuner."""
    import synth
    stream = torch.cuda.Stream(device=dev)  # graphs are captured on a side stream
    model = synth.volume_model(max(BATCH_DIMS), 0.5)
    vol = sg.sg_volume_create(BATCH_DIMS, sg.SG_U16, BRICK, LEVELS, channels=2, timepoints=BATCH_T, model=model)
    t0 = time.perf_counter()
    for t in range(BATCH_T):
        for c in range(2):
            a = synth.blobs_u16(BATCH_DIMS, seed=1003, channel=c, t=t, nblobs=40)
            d = torch.from_numpy(a.view(np.int16)).to(dev)
            torch.cuda.synchronize()
            sg.sg_upload_volume_device(vol, t, c, d.data_ptr(), stream=stream)
            torch.cuda.synchronize()
    ingest_s = time.perf_counter() - t0
    sg.sg_set_transfer_function(vol, 0, synth.tf_piecewise(2003, zero_alpha_points=2, colour=(0.1, 0.9, 0.2)),
                                200.0, 40000.0)
    sg.sg_set_transfer_function(vol, 1, synth.tf_piecewise(2004, zero_alpha_points=2, colour=(0.9, 0.1, 0.8)),
                                200.0, 40000.0)
    viewers = [synth.head_poses(1, seed=3003 + i, width=w, height=h)[0] for i, (w, h) in enumerate(BATCH_RES)]
    poses, outs = [], []
    for t in range(BATCH_T):
        for i, (w, h) in enumerate(BATCH_RES):
            views, projs = viewers[i]
            poses.append(sg.make_pose(views, projs, w, h, pixel_error=TAU, t=t, slot=t * 3 + i))
            outs += [torch.empty((h, w, 4), dtype=torch.float32, device=dev) for _ in range(2)]
    total = torch.zeros(1, dtype=torch.int64, device=dev)
    prm = sg.render_params(step=STEP, term_alpha=TERM, empty_skip=1, sample_total=total)
    sg.sg_select_lod_batch(vol, poses, stream=stream)
    tuned, _ = sg.sg_autotune_render(vol, poses, prm, outs, reps=2, stream=stream)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        sg.sg_select_lod_batch(vol, poses, stream=stream)
        sg.sg_render_batch(vol, poses, prm, outs, stream=stream)
    with torch.cuda.stream(stream):
        for _ in range(2):
            g.replay()
        torch.cuda.synchronize()
        total.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            g.replay()
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    px = sum(2 * w * h for w, h in BATCH_RES) * BATCH_T
    res = {"workload": "batched 4D multichannel: 16 t x 512x512x256 u16 x 2 ch, 3 stereo viewers "
                       "(1440x1600, 1080x1200, 720x800) = 96 images per launch, CUDA graph",
           "ms_per_launch": round(ms, 3), "images_per_s": round(96 / (ms / 1e3), 1),
           "mpixels_per_s": round(px / (ms / 1e3) / 1e6, 1),
           "gsamples_per_s": round(total.item() / reps / (ms / 1e3) / 1e9, 3), "render_config": tuned,
           "ingest_s": round(ingest_s, 2), "launches_per_replay": 2}
    sg.sg_volume_destroy(vol)
    return res


def host_mem_available():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def streaming_flythrough(sg, torch, dev, full=None, count=256, budget_bytes=256 << 20):
    """Large volume under a memory budget: cell bodies with membranes (u8,
    seed 1004, 4096 voxels over 1 m) served from a pinned host brick store
    (every brick with its apron, in node order, plus the index of brick value
    ranges) through a device brick cache. Per frame: select (missing children
    are requested, the parent renders), upload the requests coarse-first under
    a per-frame byte budget in one call that queues the copies without
    waiting for them, render both eyes. Reports frame time p50/p99 (wall
    clock, synchronised per frame on the render), the cache hit rate, the
    host time of the upload call (it waits only while the previous frame's
    copies still hold its staging) and the copies' bandwidth (device time on
    the copy stream).

    full: 4096^3 in 128^3 bricks, 6 levels, 40 GB cache (level 0 generated on
    the GPU, 82 GB pinned host store); else the 1024^3 stand-in (64^3 bricks,
    4 levels, cache of a quarter of the bricks). None picks full when the
    device and the host have room for it."""
    import synth
    free_dev, _ = torch.cuda.mem_get_info(dev)
    if full is None:
        full = free_dev > 190e9 and host_mem_available() > 130e9
    if full:
        n_vox, brick, levels, cache_bytes = 4096, 128, 6, 40_000_000_000
    else:
        n_vox, brick, levels, cache_bytes = 1024, 64, 4, None
    extent = n_vox / 4096.0
    model = synth.volume_model(n_vox, extent)
    # the container: built once by the library's own ingest into a resident
    # volume, then read back brick by brick into pinned host memory
    t0 = time.perf_counter()
    d = torch.empty((n_vox, n_vox, n_vox), dtype=torch.uint8, device=dev)
    if full:
        synth.cells_u8_device(n_vox, d.data_ptr(), seed=1004, cell=64)
    else:
        d.copy_(torch.from_numpy(synth.cells_u8_box(n_vox, 0, 0, 0, n_vox, n_vox, n_vox, seed=1004, cell=64)))
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    src = sg.sg_volume_create((n_vox,) * 3, sg.SG_U8, brick, levels, model=model)
    sg.sg_upload_volume_device(src, 0, 0, d.data_ptr())
    torch.cuda.synchronize()
    del d
    torch.cuda.empty_cache()
    geo = []  # (level, bx, by, bz) by node id
    for L in range(levels):
        nb = -(-(-(-n_vox // (1 << L))) // brick)
        geo += [(L, x, y, z) for z in range(nb) for y in range(nb) for x in range(nb)]
    nodes = len(geo)
    R3 = (brick + 2) ** 3
    # page-locked in place (exactly the bytes needed; a caching pinned
    # allocator may round an 82 GB request up to the next power of two)
    host = np.empty(nodes * R3, np.uint8)
    cudart = torch.cuda.cudart()
    rc = cudart.cudaHostRegister(host.ctypes.data, host.nbytes, 0)
    if int(rc) != 0:
        raise RuntimeError(f"cudaHostRegister of the brick store failed: {rc}")
    for i, (L, x, y, z) in enumerate(geo):
        sg.sg_read_brick(src, 0, 0, L, x, y, z, host[i * R3:(i + 1) * R3])
    ranges = sg.sg_read_ranges(src, 0, nodes)
    sg.sg_volume_destroy(src)
    ingest_s = time.perf_counter() - t0
    slot_bytes = (R3 + 255) // 256 * 256
    cache_bricks = cache_bytes // slot_bytes if cache_bytes else nodes // 4
    vol = sg.sg_volume_create((n_vox,) * 3, sg.SG_U8, brick, levels, model=model,
                              device_pool_bytes=cache_bricks * slot_bytes)
    tf = synth.tf_piecewise(2004, zero_alpha_points=2, zero_span=(60, 80))
    sg.sg_set_transfer_function(vol, 0, tf, 0.0, 255.0)
    off = 0
    for L in range(levels):
        nl = sum(1 for g in geo if g[0] == L)
        sg.sg_set_brick_ranges(vol, 0, 0, L, np.array([g[1:] for g in geo[off:off + nl]]), ranges[off:off + nl, 0, :])
        off += nl
    base = host.ctypes.data
    top = [i for i, g in enumerate(geo) if g[0] == levels - 1]
    sg.sg_upload_brick_list(vol, 0, 0, top, [base + i * R3 for i in top])
    poses = synth.flythrough_poses(count, seed=3004, extent_m=extent, width=W_EYE, height=H_EYE)
    outs = [torch.empty((H_EYE, W_EYE, 4), dtype=torch.float32, device=dev) for _ in range(2)]
    prm = sg.render_params(step=STEP, term_alpha=TERM)
    per_frame = budget_bytes // R3
    frame_ms, up_ms, hits, up_bricks = [], [], [], 0
    up_events = []  # (start, end) on the copy stream around each frame's upload: the copies' device time
    # pipelined frames: select and render on the compute stream; the bricks
    # this frame requested upload on a copy stream while its render runs
    # (sg_upload_brick_list_async: the call returns once the copies are
    # queued), and are in the cache for the next selection
    comp, copy = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    torch.cuda.synchronize()
    for views, projs in poses:
        t0 = time.perf_counter()
        pose = sg.make_pose(views, projs, W_EYE, H_EYE, pixel_error=TAU)
        st = sg.sg_select_lod(vol, pose, stats=True, stream=comp)
        # blocks drawn at the wanted detail / blocks wanted (drawn + missing)
        drawn = st["selected"] - st["fallback"]
        hits.append(drawn / (drawn + st["requested"]) if drawn + st["requested"] else 1.0)
        req = []
        if st["requested"]:
            req = sorted((int(n) for n in sg.sg_read_requests(vol, 0, stream=comp)),
                         key=lambda n: (-geo[n][0], n))[:per_frame]
        sg.sg_render(vol, pose, prm, outs, stream=comp)
        tu = time.perf_counter()
        if req:
            # queued on the copy stream, not waited for: the next selection
            # waits for it on the device (the store never changes)
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ea.record(copy)
            up_bricks += sg.sg_upload_brick_list(vol, 0, 0, req, [base + n * R3 for n in req], stream=copy,
                                                 asynchronous=True)
            eb.record(copy)
            up_events.append((ea, eb))
        up_ms.append((time.perf_counter() - tu) * 1e3)
        comp.synchronize()
        frame_ms.append((time.perf_counter() - t0) * 1e3)
    torch.cuda.synchronize()
    up_dev_s = sum(a.elapsed_time(b) for a, b in up_events) / 1e3
    sg.sg_volume_destroy(vol)
    cudart.cudaHostUnregister(host.ctypes.data)
    del host
    fm, um = np.array(frame_ms), np.array(up_ms)
    kind = "full size" if full else "scaled stand-in"
    return {"workload": f"large volume under a memory budget ({kind}): {n_vox}^3 u8 cell bodies + membranes "
                        f"(4096 voxels per m), {brick}^3 bricks, {levels} levels, device cache "
                        f"{cache_bricks} of {nodes} bricks ({cache_bricks * slot_bytes / 1e9:.1f} GB), pinned host "
                        f"brick store ({nodes * R3 / 1e9:.1f} GB), {count}-pose fly-through, 2x{W_EYE}x{H_EYE}, "
                        f"<= {budget_bytes >> 20} MiB uploaded per frame",
            "frame_ms_p50": round(float(np.percentile(fm, 50)), 3),
            "frame_ms_p99": round(float(np.percentile(fm, 99)), 3),
            "upload_ms_p99": round(float(np.percentile(um, 99)), 3),
            "cache_hit_rate": round(float(np.mean(hits)), 4),
            "h2d_gbs": round(up_bricks * R3 / up_dev_s / 1e9, 2) if up_bricks and up_dev_s > 0 else None,
            "uploaded_bricks": int(up_bricks), "generate_s": round(gen_s, 1), "ingest_and_store_s": round(ingest_s, 1)}


def container_streaming(sg, torch, dev, n_vox=1024, brick=64, levels=4, count=128, budget_bytes=128 << 20, hz=90.0):
    """The storage path end to end ("Volumetric Data Storage" + "Cashing"):
    the cell-body volume converted into an LZ4 brick container on local disk,
    then a fly-through served from a host cache of half the bricks (misses
    read + decompressed on 16 host threads) into a GPU cache of a quarter of
    them; renders pipelined on a compute stream, frames presented at hz (a
    head-mounted display's refresh). The fly-through runs twice
    from cold caches: with sg_stream_requests (each frame waits for its
    reads) and with sg_stream_requests_async (reads in the background,
    frames render resident ancestors meanwhile). Reports conversion
    throughput, compression ratio, frame time p50/p99 (the frame's own work,
    not the wait for its slot), missed deadlines and where the bricks came
    from, per mode."""
    import shutil
    import tempfile
    import synth
    extent = n_vox / 4096.0
    model = synth.volume_model(n_vox, extent)
    d = torch.empty((n_vox,) * 3, dtype=torch.uint8, device=dev)
    synth.cells_u8_device(n_vox, d.data_ptr(), seed=1004, cell=64)
    src = sg.sg_volume_create((n_vox,) * 3, sg.SG_U8, brick, levels, model=model)
    sg.sg_upload_volume_device(src, 0, 0, d.data_ptr())
    torch.cuda.synchronize()
    del d
    geo = []
    for L in range(levels):
        nb = -(-(-(-n_vox // (1 << L))) // brick)
        geo += [(L, x, y, z) for z in range(nb) for y in range(nb) for x in range(nb)]
    nodes = len(geo)
    R3 = (brick + 2) ** 3
    ranges = sg.sg_read_ranges(src, 0, nodes)
    tmp = tempfile.mkdtemp(prefix="sgc_")
    path = os.path.join(tmp, "cells.sgc")
    t0 = time.perf_counter()
    k = sg.sg_container_create(path, sg.volume_desc((n_vox,) * 3, sg.SG_U8, brick, levels, model=model))
    # conversion on 16 host threads (the library calls release the GIL)
    from concurrent.futures import ThreadPoolExecutor

    def convert(part):
        buf = np.empty(R3, np.uint8)
        for i in part:
            L, x, y, z = geo[i]
            sg.sg_read_brick(src, 0, 0, L, x, y, z, buf)
            sg.sg_container_append(k, 0, 0, L, x, y, z, buf, *ranges[i, 0])

    with ThreadPoolExecutor(16) as ex:
        list(ex.map(convert, [range(j, nodes, 16) for j in range(16)]))
    sg.sg_container_finish(k)
    convert_s = time.perf_counter() - t0
    info = sg.sg_container_get_info(k)
    sg.sg_container_close(k)
    sg.sg_volume_destroy(src)
    k = sg.sg_container_open(path)
    slot_bytes = (R3 + 255) // 256 * 256
    poses = synth.flythrough_poses(count, seed=3004, extent_m=extent, width=W_EYE, height=H_EYE)
    top = [i for i, g in enumerate(geo) if g[0] == levels - 1]

    period = 1.0 / hz

    def flythrough(asynchronous):
        """One fly-through from cold caches (a fresh GPU cache and host cache),
        frames presented at hz: a frame that finishes early waits for its slot."""
        vol = sg.sg_volume_create((n_vox,) * 3, sg.SG_U8, brick, levels, model=model,
                                  device_pool_bytes=(nodes // 4) * slot_bytes)
        hc = sg.sg_host_cache_create(k, (nodes // 2) * R3, pinned=True, threads=16)
        try:
            sg.sg_set_transfer_function(vol, 0, synth.tf_piecewise(2004, zero_alpha_points=2, zero_span=(60, 80)),
                                        0.0, 255.0)
            off = 0
            for L in range(levels):
                nl = sum(1 for g in geo if g[0] == L)
                sg.sg_set_brick_ranges(vol, 0, 0, L, np.array([g[1:] for g in geo[off:off + nl]]),
                                       ranges[off:off + nl, 0, :])
                off += nl
            ptrs = [sg.sg_host_cache_fetch(hc, 0, 0, n)[0] for n in top]
            sg.sg_upload_brick_list(vol, 0, 0, top, ptrs)
            outs = [torch.empty((H_EYE, W_EYE, 4), dtype=torch.float32, device=dev) for _ in range(2)]
            prm = sg.render_params(step=STEP, term_alpha=TERM)
            comp, copy = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
            frame_ms, stream_ms, pending = [], [], []
            tot = dict(served=0, host_hits=0, disk_reads=0, disk_bytes=0, upload_bytes=0)
            torch.cuda.synchronize()
            for views, projs in poses:
                t0 = time.perf_counter()
                pose = sg.make_pose(views, projs, W_EYE, H_EYE, pixel_error=TAU)
                st = sg.sg_select_lod(vol, pose, stats=True, stream=comp)
                sg.sg_render(vol, pose, prm, outs, stream=comp)
                pending.append(st["requested"])
                ts = time.perf_counter()
                if st["requested"]:
                    s = sg.sg_stream_requests(vol, 0, hc, budget_bytes, stream=copy, asynchronous=asynchronous)
                    for key in tot:
                        tot[key] += s[key]
                stream_ms.append((time.perf_counter() - ts) * 1e3)
                comp.synchronize()
                frame_ms.append((time.perf_counter() - t0) * 1e3)
                rest = period - (time.perf_counter() - t0)
                if rest > 0:
                    time.sleep(rest)
        finally:
            sg.sg_host_cache_destroy(hc)
            sg.sg_volume_destroy(vol)
        fm, sm = np.array(frame_ms), np.array(stream_ms)
        return {"frame_ms_p50": round(float(np.percentile(fm, 50)), 3),
                "frame_ms_p99": round(float(np.percentile(fm, 99)), 3),
                "stream_ms_p99": round(float(np.percentile(sm, 99)), 3),
                "bricks_served": int(tot["served"]), "host_hits": int(tot["host_hits"]),
                "disk_reads": int(tot["disk_reads"]),
                "missed_deadlines": int((fm > period * 1e3).sum()),
                "missed_frames": [int(i) for i in np.flatnonzero(fm > period * 1e3)][:16],
                "frame_ms_max": round(float(fm.max()), 3),
                "frames_with_requests": int(sum(1 for p in pending if p)),
                "requests_per_frame_mean": round(float(np.mean(pending)), 1),
                "disk_read_gbs": round(tot["disk_bytes"] / max(sm.sum() / 1e3, 1e-9) / 1e9, 3)}

    try:
        blocking = flythrough(False)
        nonblocking = flythrough(True)
    finally:
        sg.sg_container_close(k)
        shutil.rmtree(tmp, ignore_errors=True)
    out = {"workload": f"brick container + host cache: {n_vox}^3 u8 cell bodies, {brick}^3 bricks, {levels} levels, "
                       f"{nodes} LZ4 chunks on local disk; host cache {nodes // 2} bricks (pinned, 16 decode "
                       f"threads), GPU cache {nodes // 4} bricks; {count}-pose fly-through, 2x{W_EYE}x{H_EYE}, "
                       f"<= {budget_bytes >> 20} MiB per frame, frames presented at {hz:g} Hz; each mode from cold "
                       f"caches",
           "convert_s": round(convert_s, 2), "convert_gbs": round(info["raw_bytes"] / convert_s / 1e9, 3),
           "compression_ratio": round(info["raw_bytes"] / max(info["compressed_bytes"], 1), 3)}
    out.update(blocking)
    out["async"] = dict(nonblocking, mode="sg_stream_requests_async: misses loaded in the background, "
                                          "frames render resident ancestors meanwhile")
    return out


def learned_recon(sg, torch, dev, vol, tf_table, model, pairs=20000, steps_per_pair=4, eval_poses=16, tau_half=None,
                  threshold_db=40.0, frame_log=None):
    """Learned reconstruction vs the plain path on the same GPU: training on
    `pairs` seeded (pose, full-rate render, half-res render) pairs of the
    bench volume, evaluation on a held-out volume seed and held-out poses.
    Learned frame = select + render both eyes at 720x800, step 1.0, + the
    U-Net to 2x1440x1600; a frame under the PSNR threshold falls back to (and
    also pays for) the plain full-rate render."""
    import synth
    from paper_1804_08197_b300.learned import Learned
    stream = torch.cuda.current_stream()
    rec = Learned(vol, W_EYE, H_EYE, step=STEP, tau=TAU, max_batch=16, crop=64, seed=7, tau_half=tau_half)
    # held-out volume (different seed) and poses
    ev = synth.filaments_u16((N_VOX,) * 3, seed=9001)
    vol2 = sg.sg_volume_create((N_VOX,) * 3, sg.SG_U16, BRICK, LEVELS, model=model)
    d = torch.from_numpy(ev.view(np.int16)).to(dev)
    sg.sg_upload_volume_device(vol2, 0, 0, d.data_ptr())
    torch.cuda.synchronize()
    del d, ev
    sg.sg_set_transfer_function(vol2, 0, tf_table, *WINDOW)
    held = synth.head_poses(eval_poses, seed=9300, width=W_EYE, height=H_EYE)
    # the untrained network is exactly the bilinear upsampling: the method without it
    rec.vol = vol2
    bilinear = np.array([rec.evaluate(v, p) for v, p in held])
    rec.vol = vol
    t0 = time.perf_counter()
    train = synth.head_poses(512, seed=9100, width=W_EYE, height=H_EYE)
    for i in range(pairs):
        v, p = train[i % len(train)]
        lr = 8e-4 * (0.05 + 0.95 * 0.5 * (1.0 + np.cos(np.pi * i / pairs)))  # cosine decay
        rec.train_on_pair(v, p, steps=steps_per_pair, batch=16, lr=lr)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    sg.sg_unet_check(rec.net)
    rec.vol = vol2
    # launch shapes of both render rates tuned on a pose outside the evaluation set
    rec.tune(*synth.head_poses(1, seed=9400, width=W_EYE, height=H_EYE)[0], stream=stream)
    for v, p in held[:2]:  # warm-up
        rec.evaluate(v, p)
    ev_ = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    t_learned, t_plain, t_net, marks = [], [], [], []
    for i, (v, p) in enumerate(held):
        # a learned frame as served: sg_render_learned without judging
        a, b = ev_()
        a.record(stream)
        rec.frame(v, p, stream=stream)
        b.record(stream)
        # its parts, for the breakdown: the reduced render, then the network
        c, dd = ev_()
        rec.render_half(v, p, stream=stream)
        c.record(stream)
        rec.reconstruct(stream=stream)
        dd.record(stream)
        # the plain path
        e, f = ev_()
        e.record(stream)
        rec.render_full(v, p, stream=stream)
        f.record(stream)
        # the judge (full-rate render, stereo PSNR, fallback on the device)
        rec.frame(v, p, judge=True, threshold_db=threshold_db, index=i, stream=stream)
        marks.append((a, b, c, dd, e, f))
    torch.cuda.synchronize()
    for a, b, c, dd, e, f in marks:
        t_learned.append(a.elapsed_time(b))
        t_net.append(c.elapsed_time(dd))
        t_plain.append(e.elapsed_time(f))
    psnrs = rec.psnr_frames[:len(held), 2].cpu().numpy().astype(np.float64)
    fell = rec.fell_back[:len(held)].cpu().numpy().astype(bool)
    if frame_log:
        # per held-out frame, appended to the render leg's lines
        with open(frame_log, "a") as f:
            for i in range(len(held)):
                f.write(json.dumps({"leg": "learned", "frame": i, "psnr_db": round(float(psnrs[i]), 3),
                                    "fell_back": bool(fell[i]), "learned_ms": round(t_learned[i], 4),
                                    "net_ms": round(t_net[i], 4), "half_render_ms": round(t_learned[i] - t_net[i], 4),
                                    "plain_ms": round(t_plain[i], 4)}) + "\n")
    # the same frames with two in flight: the half-rate render of frame i + 1
    # overlaps the network on frame i (a second stream); a frame that falls
    # back still adds its plain render
    rs, ns = torch.cuda.Stream(), torch.cuda.Stream()
    rec.run_pipelined(held, rs, ns)  # warm-up
    pipe_ms = min(rec.run_pipelined(held, rs, ns) for _ in range(3)) / len(held)
    # the plain path gets the same treatment: each selection overlapping the
    # render before it (as in the device-timed loop)
    rec.run_plain_pipelined(held, rs, ns)  # warm-up
    plain_pipe_ms = min(rec.run_plain_pipelined(held, rs, ns) for _ in range(3)) / len(held)
    sg.sg_volume_destroy(vol2)
    rec.close()
    fall = fell
    assert np.array_equal(fall, psnrs < threshold_db)
    serial_ms = float(np.mean(np.array(t_learned) + np.where(fall, t_plain, 0.0)))
    pipelined_ms = pipe_ms + float(np.mean(np.where(fall, t_plain, 0.0)))
    # the headline takes the faster of the two schedules (both reported)
    learned_ms = min(serial_ms, pipelined_ms)
    plain_serial_ms = float(np.mean(t_plain))
    plain_ms = min(plain_serial_ms, plain_pipe_ms)
    net_flop = 2 * 268.0e9 / 2  # ~134 GFLOP per eye (3x3 convs), both eyes
    return {"workload": "learned reconstruction: 2x720x800 at step 1.0 -> U-Net (32/64/128, BF16) -> 2x1440x1600; "
                        f"trained on {pairs} seeded pairs of the bench volume, evaluated on a held-out volume "
                        f"seed and {eval_poses} held-out poses",
            "learned_fps": round(1e3 / learned_ms, 2), "plain_fps": round(1e3 / plain_ms, 2),
            "learned_over_plain": round(plain_ms / learned_ms, 3),
            "learned_mode": "two frames in flight" if pipelined_ms < serial_ms else "one frame at a time",
            "learned_fps_serial": round(1e3 / serial_ms, 2),
            "learned_fps_two_in_flight": round(1e3 / pipelined_ms, 2),
            "plain_fps_serial": round(1e3 / plain_serial_ms, 2),
            "plain_fps_selection_overlapped": round(1e3 / plain_pipe_ms, 2),
            "psnr_db": {"mean": round(float(psnrs.mean()), 2), "min": round(float(psnrs.min()), 2),
                        "median": round(float(np.median(psnrs)), 2)},
            "bilinear_psnr_db": {"mean": round(float(bilinear.mean()), 2), "min": round(float(bilinear.min()), 2)},
            "fallback_rate": round(float(fall.mean()), 3), "threshold_db": threshold_db,
            "net_ms": round(float(np.mean(t_net)), 3),
            "net_tflops": round(net_flop / (float(np.mean(t_net)) / 1e3) / 1e12, 1),
            "net_roofline": tensor_roofline(net_flop / (float(np.mean(t_net)) / 1e3) / 1e12),
            "half_render_ms": round(float(np.mean(np.array(t_learned) - np.array(t_net))), 3),
            "learned_frame": "sg_render_learned (reduced render + network, one C-ABI call); judged frames: "
                             "full-rate render, stereo PSNR and fallback on the device",
            "render_config": {"full": rec.cfg_full, "half": rec.cfg_half}, "half_tau_px": rec.tau_half,
            "train_s": round(train_s, 1), "train_pairs": pairs, "steps_per_pair": steps_per_pair}


def run_net_only(args):
    """U-Net forwards on both eyes at 720x800 (random input), for profiling."""
    import torch
    from paper_1804_08197_b300 import sg
    torch.cuda.set_device(0)
    net = sg.sg_unet_create(2, H_EYE // 2, W_EYE // 2, seed=1)
    if args.tensor_path >= 0:
        sg.sg_unet_set_tensor_path(net, args.tensor_path)
    x = [torch.rand((H_EYE // 2, W_EYE // 2, 4), device="cuda") for _ in range(2)]
    o = [torch.empty((H_EYE, W_EYE, 4), device="cuda") for _ in range(2)]
    for _ in range(args.warmup):
        sg.sg_unet_forward(net, x, W_EYE // 2 * 4, H_EYE // 2, W_EYE // 2, o, W_EYE * 4)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        sg.sg_unet_forward(net, x, W_EYE // 2 * 4, H_EYE // 2, W_EYE // 2, o, W_EYE * 4)
    b.record()
    torch.cuda.synchronize()
    sg.sg_unet_check(net)
    ms = a.elapsed_time(b) / args.steps
    tf = 268e9 / (ms / 1e3) / 1e12
    print(json.dumps({"net_forward_ms": round(ms, 4), "tflops": round(tf, 1), "roofline": tensor_roofline(tf)}),
          flush=True)
    sg.sg_unet_destroy(net)


def run_learned_only(args):
    """The learned-reconstruction measurement alone (training + held-out
    evaluation), on the bench volume with its autotuned launch shape."""
    import torch
    from paper_1804_08197_b300 import sg
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    vol_host, tf_table, poses, model = make_inputs(args.volume)
    vol = sg.sg_volume_create((args.volume,) * 3, sg.SG_U16, BRICK, LEVELS, model=model)
    d0 = torch.from_numpy(vol_host.view(np.int16)).to(dev)
    sg.sg_upload_volume_device(vol, 0, 0, d0.data_ptr())
    torch.cuda.synchronize()
    del d0
    sg.sg_set_transfer_function(vol, 0, tf_table, *WINDOW)
    stream = torch.cuda.current_stream()
    outs = [torch.empty((H_EYE, W_EYE, 4), dtype=torch.float32, device=dev) for _ in range(2)]
    p0 = sg.make_pose(*poses[0], W_EYE, H_EYE, pixel_error=TAU, slot=0)
    sg.sg_select_lod(vol, p0, stream=stream)
    sg.sg_autotune_render(vol, [p0], sg.render_params(step=STEP), outs, reps=3, stream=stream)
    print(json.dumps(learned_recon(sg, torch, dev, vol, tf_table, model, pairs=args.learned_pairs,
                                   tau_half=args.learned_half_tau)), flush=True)
    sg.sg_volume_destroy(vol)


def run_train_only(args):
    """Training steps alone (16 random 64x64 crops of one rendered pair:
    forward, loss, backward, Adam), timed with CUDA events after warm-up."""
    import torch
    from paper_1804_08197_b300 import sg
    from paper_1804_08197_b300.learned import Learned
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    vol_host, tf_table, poses, model = make_inputs(args.volume)
    vol = sg.sg_volume_create((args.volume,) * 3, sg.SG_U16, BRICK, LEVELS, model=model)
    d0 = torch.from_numpy(vol_host.view(np.int16)).to(dev)
    sg.sg_upload_volume_device(vol, 0, 0, d0.data_ptr())
    torch.cuda.synchronize()
    del d0
    sg.sg_set_transfer_function(vol, 0, tf_table, *WINDOW)
    rec = Learned(vol, W_EYE, H_EYE, step=STEP, tau=TAU, max_batch=16, crop=64, seed=7)
    rec.train_on_pair(*poses[0], steps=args.warmup)  # renders the pair, then the warm-up steps
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c = rec.crop
    outs = [rec.crop_out[i].data_ptr() for i in range(16)]
    a.record()
    for _ in range(args.steps):
        ins, tgts = rec._crops(16)
        sg.sg_unet_forward(rec.net, ins, rec.w * 4, c, c, outs, 2 * c * 4)
        sg.sg_unet_backward(rec.net, tgts, rec.W * 4, outs, 2 * c * 4, loss=rec.loss)
        sg.sg_unet_adam_step(rec.net, 1e-4)
    b.record()
    torch.cuda.synchronize()
    sg.sg_unet_check(rec.net)
    ms = a.elapsed_time(b) / args.steps
    flop = 3 * 268e9 * (16 * 64 * 64) / (2 * (H_EYE // 2) * (W_EYE // 2))  # forward, input and weight gradients
    print(json.dumps({"train_step_ms": round(ms, 4), "crops": "16 x 64 x 64 (half-rate) -> 128 x 128",
                      "tflops": round(flop / (ms / 1e3) / 1e12, 1)}), flush=True)
    rec.close()
    sg.sg_volume_destroy(vol)


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle on the host cores, bounded sample per
    step. Block ranges are computed once at ingest (untimed); a step is the
    pose's selection plus every 32nd pixel of both eyes (the sample
    cpu_baseline takes of the same poses), and a frame's time extrapolates
    only the per-pixel part."""
    if rank != 0:
        return
    import oracle
    vol, tf_table, poses, model = make_inputs(args.volume)
    ovol = oracle.Volume([oracle.pyramid(vol, LEVELS)], BRICK, model=model)
    otf = oracle.make_tf(tf_table, *WINDOW)
    ranges = ovol.block_ranges()
    stride = 32
    npix = W_EYE * H_EYE

    def step(i):
        views, projs = poses[i % NPOSES]
        t0 = time.perf_counter()
        sel = ovol.select([otf], views, projs, H_EYE, tau=TAU, ranges=ranges)
        t_sel = time.perf_counter() - t0
        s, t_pix = 0, 0.0
        for e in range(2):
            t1 = time.perf_counter()
            r = ovol.render([otf], sel["leaf"], views[e], projs[e], W_EYE, H_EYE, step=STEP,
                            pixels=np.arange((i * 13 + e * 7) % stride, npix, stride), variants=False)
            t_pix += time.perf_counter() - t1
            s += int(r["count_late"].sum())
        return s * stride, t_sel + t_pix * stride, t_sel + t_pix

    for i in range(args.warmup):
        step(i)
    frames_s, samples, busy = 0.0, 0, 0.0
    for i in range(args.steps):
        n, f, b = step(args.warmup + i)
        samples += n
        frames_s += f
        busy += b
    fps = args.steps / frames_s
    line = {"metric": METRIC, "value": round(fps, 6), "unit": "stereo frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(frames_s / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": workload_config(dict(
                {"sample": f"selection + every {stride}th pixel of both eyes per step", "volume": [args.volume] * 3},
                **({} if args.volume == N_VOX else {
                    "workload": WORKLOAD.replace(f"{N_VOX}^3", f"{args.volume}^3") + " (a smaller volume)"}))),
            "gsamples_per_s": round(samples / frames_s / 1e9, 6),
            "cpu_baseline": {"value": round(fps, 6), "unit": "stereo frames/s", "cores": oracle.max_threads(),
                             "kind": "oracle",
                             "sample": f"each step: pose i with its selection, every {stride}th pixel of both eyes "
                                       f"({busy:.1f} s timed in all); per-pixel time extrapolated to full frames; "
                                       "block ranges computed once at ingest (untimed)"},
            "e2e": {"value": round(fps, 6), "unit": "stereo frames/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1804_08197_b300 import sg
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    n_vox = args.volume
    vol_host, tf_table, poses, model = make_inputs(n_vox)
    vol = sg.sg_volume_create((n_vox,) * 3, sg.SG_U16, BRICK, LEVELS, model=model, skip_block=args.skip_block)
    d0 = torch.from_numpy(vol_host.view(np.int16)).to(dev)
    sg.sg_upload_volume_device(vol, 0, 0, d0.data_ptr())
    torch.cuda.synchronize()
    del d0
    sg.sg_set_transfer_function(vol, 0, tf_table, *WINDOW)
    # a transfer-function edit: tables, node flags, sub-block flags and the
    # directional distance maps of every brick, until the GPU is done
    tf_ms = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sg.sg_set_transfer_function(vol, 0, tf_table, *WINDOW)
        torch.cuda.synchronize()
        tf_ms.append((time.perf_counter() - t0) * 1e3)
    stream = torch.cuda.current_stream()
    outs = [torch.empty((H_EYE, W_EYE, 4), dtype=torch.float32, device=dev) for _ in range(2)]
    total = torch.zeros(1, dtype=torch.int64, device=dev)
    pose_objs = [sg.make_pose(v, p, W_EYE, H_EYE, pixel_error=TAU, slot=0) for v, p in poses]
    mine = rank_poses(pose_objs, rank, world)
    prm = sg.render_params(step=STEP, term_alpha=TERM, empty_skip=1, sample_total=total)
    # the project's autotuner picks tile shape / persistence on the first pose
    # (untimed setup); with --tune-cache the pick is kept across runs
    sg.sg_select_lod(vol, mine[0], stream=stream)
    tune_key = f"{torch.cuda.get_device_name(dev)} {n_vox}^3 u16 {W_EYE}x{H_EYE} skip{args.skip_block}"
    tuned = sg.sg_render_config_lookup(args.tune_cache, tune_key) if args.tune_cache else None
    if tuned is not None:
        sg.sg_set_render_config(vol, **tuned)
        tuned_ms = None
    else:
        tuned, tuned_ms = sg.sg_autotune_render(vol, [mine[0]], prm, outs, reps=3, stream=stream)
        if args.tune_cache and rank == 0:
            sg.sg_render_config_store(args.tune_cache, tune_key, tuned)

    # selection of pose i + 1 (its own slot, a second stream) overlaps the
    # render of pose i; a slot is selected again only after the render that
    # read it (two slots, alternating)
    sel_stream = torch.cuda.Stream(dev)
    mine2 = [[p, sg.make_pose(*pv, W_EYE, H_EYE, pixel_error=TAU, slot=1)]
             for p, pv in zip(mine, rank_poses(poses, rank, world))]
    selected = [torch.cuda.Event(), torch.cuda.Event()]
    rendered = [None, None]

    def step(i, ev=None):
        k = i % 2
        p = mine2[i % NPOSES][k]
        if rendered[k] is not None:
            sel_stream.wait_event(rendered[k])
        if ev is not None:
            ev[2].record(sel_stream)
        sg.sg_select_lod(vol, p, stream=sel_stream)
        selected[k].record(sel_stream)
        stream.wait_event(selected[k])
        if ev is not None:
            ev[0].record(stream)
        sg.sg_render(vol, p, prm, outs, stream=stream)
        if ev is not None:
            ev[1].record(stream)
        rendered[k] = torch.cuda.Event()
        rendered[k].record(stream)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    total.zero_()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    rev = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(args.steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    e0.record(stream)
    sel_stream.wait_event(e0)
    for i in range(args.steps):
        step(args.warmup + i, rev[i])
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop(window=(w0, time.perf_counter()))
    ms = e0.elapsed_time(e1)
    render_ms = [a.elapsed_time(b) for a, b, _ in rev]
    # frame period: from the previous frame's render end (the loop start for
    # the first) to this one's; a pose's selection overlaps the render before
    ends = [e0] + [b for _, b, _ in rev]
    frame_ms = np.array([ends[i].elapsed_time(ends[i + 1]) for i in range(args.steps)])
    samples = int(total.item())
    ms_max = max_over_ranks(ms, world, dev)

    # algorithmic bytes of the render launches (outside the timed region):
    # the distinct bricks a sample was taken from (a diagnostic render of
    # each timed pose marks them) + the two output images
    brick_bytes = (BRICK + 2) ** 3 * 2
    out_bytes = 2 * W_EYE * H_EYE * 16
    nodes = sum(-(-(-(-n_vox // 2 ** L)) // BRICK) ** 3 for L in range(LEVELS))
    touched = torch.zeros(nodes, dtype=torch.uint8, device=dev)
    frame_samples = torch.zeros(1, dtype=torch.int64, device=dev)
    prm_touch = sg.render_params(step=STEP, term_alpha=TERM, empty_skip=1, touched=touched,
                                 sample_total=frame_samples)
    saved_cfg = sg.sg_get_render_config(vol)
    sg.sg_set_render_config(vol)
    alg, alg_selected, frame_records = [], [], []
    for i in range(args.steps):
        p = mine[(args.warmup + i) % NPOSES]
        st = sg.sg_select_lod(vol, p, stats=True, stream=stream)
        touched.zero_()
        frame_samples.zero_()
        sg.sg_render(vol, p, prm_touch, outs, stream=stream)
        nt = int(touched.sum().item())
        alg.append(nt * brick_bytes + out_bytes)
        alg_selected.append(st["nonempty"] * brick_bytes + out_bytes)
        if args.frame_log:
            ns = int(frame_samples.item())
            frame_records.append({"leg": "render", "frame": i, "pose": (args.warmup + i) % NPOSES, "rank": rank,
                                  "frame_ms": round(float(frame_ms[i]), 4), "render_ms": round(render_ms[i], 4),
                                  "fps": round(1e3 / float(frame_ms[i]), 2), "samples": ns,
                                  "gsamples_per_s": round(ns / render_ms[i] / 1e6, 3),
                                  "bricks_selected": st["selected"], "bricks_nonempty": st["nonempty"],
                                  "bricks_touched": nt, "requested": st["requested"], "fallback": st["fallback"],
                                  "culled": st["culled"], "empty": st["empty"]})
    sg.sg_set_render_config(vol, **saved_cfg)
    sel_stats = st
    if args.frame_log:
        # one JSON object per timed frame (rank r writes PATH.r on multi-GPU runs)
        path = args.frame_log if world == 1 else f"{args.frame_log}.{rank}"
        with open(path, "w") as f:
            for r in frame_records:
                f.write(json.dumps(r) + "\n")
    peak, peak_kind = measured_peak_hbm()
    avg_render_s = sum(render_ms) / len(render_ms) / 1e3
    achieved = (sum(alg) / len(alg)) / avg_render_s / 1e9

    # the other optical models on the same poses (select + render per step)
    modes = {}
    for name, mode in (("emission_only", sg.SG_MODE_EMISSION), ("mip", sg.SG_MODE_MIP)):
        prm_m = sg.render_params(step=STEP, term_alpha=TERM, empty_skip=1, mode=mode)
        for i in range(3):
            sg.sg_select_lod(vol, mine[i], stream=stream)
            sg.sg_render(vol, mine[i], prm_m, outs, stream=stream)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nm = min(args.steps, 32)
        torch.cuda.synchronize()
        a0.record(stream)
        for i in range(nm):
            p = mine[(args.warmup + i) % NPOSES]
            sg.sg_select_lod(vol, p, stream=stream)
            sg.sg_render(vol, p, prm_m, outs, stream=stream)
        a1.record(stream)
        torch.cuda.synchronize()
        modes[name] = {"fps": round(nm / (a0.elapsed_time(a1) / 1e3), 2), "steps": nm}

    # lens-warped stereo ("DVR for HMD"): one ray per pixel of the warped
    # image at the undistorted image's density at the lens centre, then the
    # unwarp to 2x1440x1600; quality = PSNR against the plain render over the
    # pixels the warped image covers
    lens_k1, lens_k2 = 0.22, 0.24
    lscale = 1.0 / (1.0 + lens_k1 + lens_k2)
    Ww, Hw = int(round(W_EYE * lscale)), int(round(H_EYE * lscale))
    ln = sg.make_lens(lens_k1, lens_k2, 0.0, W_EYE / H_EYE, ((0.05, 0.0), (-0.05, 0.0)))
    warped = [torch.empty((Hw, Ww, 4), dtype=torch.float32, device=dev) for _ in range(2)]
    unwarped = [torch.empty((H_EYE, W_EYE, 4), dtype=torch.float32, device=dev) for _ in range(2)]
    prm_w = sg.render_params(step=STEP, term_alpha=TERM, empty_skip=1, lens=ln)
    wposes = [sg.make_pose(v, p, Ww, Hw, pixel_error=TAU, slot=0) for v, p in poses]
    wmine = rank_poses(wposes, rank, world)

    def warped_step(i):
        sg.sg_select_lod(vol, mine[i % NPOSES], stream=stream)
        sg.sg_render(vol, wmine[i % NPOSES], prm_w, warped, stream=stream)
        sg.sg_unwarp(ln, warped, Ww, Hw, unwarped, W_EYE, H_EYE, stream=stream)

    for i in range(3):
        warped_step(i)
    nw = min(args.steps, 32)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a0.record(stream)
    for i in range(nw):
        warped_step(args.warmup + i)
    a1.record(stream)
    torch.cuda.synchronize()
    warped_fps = nw / (a0.elapsed_time(a1) / 1e3)
    ones = [torch.ones((Hw, Ww, 4), dtype=torch.float32, device=dev) for _ in range(2)]
    cover = [torch.empty((H_EYE, W_EYE, 4), dtype=torch.float32, device=dev) for _ in range(2)]
    sg.sg_unwarp(ln, ones, Ww, Hw, cover, W_EYE, H_EYE, stream=stream)
    psnr = []
    for i in range(4):
        p = mine[(args.warmup + i) % NPOSES]
        warped_step(args.warmup + i)
        sg.sg_render(vol, p, prm, outs, stream=stream)
        torch.cuda.synchronize()
        for e in range(2):
            m = cover[e][..., 3] > 0.999
            mse = float(((unwarped[e] - outs[e])[m] ** 2).mean())
            psnr.append(10 * np.log10(1.0 / mse) if mse > 0 else 1000.0)
    warped_line = {"fps": round(warped_fps, 2), "steps": nw, "warped_eye": [Ww, Hw],
                   "rays_fraction": round(Ww * Hw / (W_EYE * H_EYE), 4), "lens": {"k1": lens_k1, "k2": lens_k2},
                   "psnr_db_vs_plain": {"mean": round(float(np.mean(psnr)), 2), "min": round(float(np.min(psnr)), 2)},
                   "covered_fraction": round(float((cover[0][..., 3] > 0.999).float().mean()), 4)}
    del ones, cover

    # end to end through the public C ABI with host buffers: pose in, both
    # images out. Up to three frames in flight (sg_render_host_async): the
    # copy of frame i to host overlaps the renders of frames i + 1 and i + 2
    # (a render can be shorter than a copy), and the selection of each pose
    # (its own slot, on the selection stream) overlaps the render before it,
    # as in the device-timed loop; every frame's copy lands inside the
    # timed region. The serial sg_render_host loop is reported beside it.
    host = [[torch.empty((H_EYE, W_EYE, 4), dtype=torch.float32, pin_memory=True) for _ in range(2)]
            for _ in range(3)]
    e2e_steps = max(4, args.steps)  # the poses of the device-timed loop: steady state, not pipeline fill

    def e2e_pipelined(n, first):
        read = [None, None]  # the last render that read each selection slot
        for i in range(n):
            k = i % 2
            p = mine2[(first + i) % NPOSES][k]
            if read[k] is not None:
                sel_stream.wait_event(read[k])
            sg.sg_select_lod(vol, p, stream=sel_stream)
            selected[k].record(sel_stream)
            stream.wait_event(selected[k])
            sg.sg_render_host_async(vol, p, prm, host[i % 3], stream=stream)
            read[k] = torch.cuda.Event()
            read[k].record(stream)
            if i >= 2:
                sg.sg_render_host_wait(vol, all=False)  # frame i - 2's images are on the host
        sg.sg_render_host_wait(vol, all=True)

    e2e_pipelined(2, 0)  # untimed: copy stream, events and staging set up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_pipelined(e2e_steps, 0)
    e2e_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        p = mine[i % NPOSES]
        sg.sg_select_lod(vol, p, stream=stream)
        sg.sg_render_host(vol, p, prm, host[0], stream=stream)
    e2e_serial_s = time.perf_counter() - t0

    batched = learned = streaming = container = None
    # the single-GPU measurements run on one-GPU runs only, so a multi-GPU
    # run does not hold every GPU while one rank works alone
    if rank == 0 and world == 1 and not args.no_extra and n_vox == N_VOX:
        batched = batched_4d(sg, torch, dev)
        streaming = streaming_flythrough(sg, torch, dev)
        container = container_streaming(sg, torch, dev)
        learned = learned_recon(sg, torch, dev, vol, tf_table, model, pairs=args.learned_pairs,
                                frame_log=args.frame_log)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and n_vox == N_VOX:
        # the GPU arm's timed poses (at most 32, so the sample stays within ~15 s)
        ids = [(args.warmup + i) % NPOSES for i in range(min(args.steps, 32))]
        cpu = cpu_baseline(vol_host, tf_table, poses, model, ids)

    if rank == 0:
        fps = args.steps * world / (ms_max / 1e3)
        line = {"metric": METRIC, "value": round(fps, 3), "unit": "stereo frames/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 4),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": workload_config(dict(
                    {"parallelism": f"replicas x{world}", "volume": [n_vox] * 3, "render_config": tuned},
                    **({} if n_vox == N_VOX else {
                        "workload": WORKLOAD.replace(f"{N_VOX}^3", f"{n_vox}^3") + " (a smaller volume, for profiling)",
                        "l2": "a different pose every step"}))),
                "gsamples_per_s": round(samples * world / (ms_max / 1e3) / 1e9, 3),
                "samples_per_step": samples // args.steps,
                "render_ms_mean": round(sum(render_ms) / len(render_ms), 4),
                "frame_ms": {"mean": round(float(frame_ms.mean()), 4),
                             "p50": round(float(np.percentile(frame_ms, 50)), 4),
                             "p99": round(float(np.percentile(frame_ms, 99)), 4)},
                "gpu_launches": 2 * args.steps,
                "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                             "frac": round(achieved / peak, 5), "traffic": profiled_traffic(sum(alg) / len(alg)),
                             "kernel": "k_render", "peak_source": peak_kind,
                             "algorithmic_bytes_per_launch": int(sum(alg) / len(alg)),
                             "algorithmic_bytes": "distinct bricks a sample was taken from x (64+2)^3 x 2 B "
                                                  "+ both FP32 outputs",
                             "selected_nonempty_bytes_per_launch": int(sum(alg_selected) / len(alg_selected))},
                "clocks": clk,
                "e2e": {"value": round(e2e_s and e2e_steps / e2e_s, 3), "unit": "stereo frames/s",
                        "h2d_bytes_per_step": int(np.dtype(np.uint8).itemsize * len(bytes(mine[0]))),
                        "d2h_bytes_per_step": out_bytes, "frames": e2e_steps,
                        "mode": "sg_render_host_async, up to three frames in flight",
                        "serial_value": round(e2e_serial_s and e2e_steps / e2e_serial_s, 3)},
                "select_stats_last": sel_stats,
                "tf_edit_ms": round(min(tf_ms), 3),
                "optical_models": modes,
                "lens_warped": warped_line}
        if cpu:
            line["cpu_baseline"] = cpu
        if batched:
            line["batched_4d"] = batched
        if learned:
            line["learned"] = learned
        if streaming:
            line["streaming"] = streaming
        if container:
            line["container_streaming"] = container
        print(json.dumps(line), flush=True)
    sg.sg_volume_destroy(vol)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=64)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the batched 4D and learned measurements")
    ap.add_argument("--learned-half-tau", type=float, default=None,
                    help="pixel error bound of the reduced render (default: half of tau, the full image's LOD)")
    ap.add_argument("--frame-log", default=None, metavar="PATH",
                    help="write per-frame metrics of the timed frames as JSON lines (untimed replay of each pose: "
                         "samples, bricks selected / touched / requested, fallback; times from the timed region)")
    ap.add_argument("--learned-pairs", type=int, default=20000,
                    help="training pairs for the learned path (the configuration's 20000, about 3 min)")
    ap.add_argument("--tensor-path", type=int, default=-1,
                    help="U-Net convolution path (0 mma.sync, 1 tcgen05, 2 halo, 3 halo + TMA; -1 the default)")
    ap.add_argument("--skip-block", type=int, default=0,
                    help="empty-space skipping cell edge in voxels (0 = the library's default)")
    ap.add_argument("--streaming-size", choices=["auto", "full", "scaled"], default="auto",
                    help="large-volume fly-through at 4096^3 (full), at 1024^3 (scaled), or full when it fits")
    ap.add_argument("--only", choices=["net", "learned", "train", "streaming", "container", "batched"], default=None,
                    help="net: only U-Net forwards at 2x720x800 (a small case for profiling the convolutions); "
                         "streaming: only the large-volume fly-through")
    ap.add_argument("--volume", type=int, default=N_VOX, help="volume edge (default 1024; smaller for profiling)")
    ap.add_argument("--tune-cache", default=None,
                    help="file keeping the autotuner's pick across runs (default: tune every run)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.warmup < 3:
        args.warmup = 3
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local_rank)
        dist.init_process_group(backend)
    if args.only == "net":
        run_net_only(args)
    elif args.only == "learned":
        run_learned_only(args)
    elif args.only == "train":
        run_train_only(args)
    elif args.only == "streaming":
        import torch
        from paper_1804_08197_b300 import sg
        torch.cuda.set_device(local_rank)
        full = {"auto": None, "full": True, "scaled": False}[args.streaming_size]
        print(json.dumps(streaming_flythrough(sg, torch, torch.device("cuda"), full=full)), flush=True)
    elif args.only == "container":
        import torch
        from paper_1804_08197_b300 import sg
        torch.cuda.set_device(local_rank)
        print(json.dumps(container_streaming(sg, torch, torch.device("cuda"))), flush=True)
    elif args.only == "batched":
        import torch
        from paper_1804_08197_b300 import sg
        torch.cuda.set_device(local_rank)
        print(json.dumps(batched_4d(sg, torch, torch.device("cuda"))), flush=True)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
