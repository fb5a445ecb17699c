"""Streaming through the brick cache ("Volumetric Data Cashing"): a pooled
volume starts with only its coarsest level; each frame selects (falling back
one level and requesting missing children, "Octree Representation"), then
uploads the requested bricks, evicting the least recently used ones when the
cache is full. The oracle runs its own cache beside the GPU's (oracle.Cache:
its own stamps from its own selections, its own evictions): the resident set
must be the same after every upload, every frame's selection must equal the
oracle's bit for bit, and the rendered frames must match the oracle."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import compare_image, compare_selection

pytestmark = pytest.mark.gpu

B, LEVELS, DIMS = 16, 4, (128, 128, 128)


def _brick(ovol, L, bx, by, bz):
    g = ovol.channels[0][L]
    R = B + 2
    iz = np.clip(np.arange(R) + bz * B - 1, 0, g.shape[0] - 1)
    iy = np.clip(np.arange(R) + by * B - 1, 0, g.shape[1] - 1)
    ix = np.clip(np.arange(R) + bx * B - 1, 0, g.shape[2] - 1)
    return np.ascontiguousarray(g[np.ix_(iz, iy, ix)])


def _stereo(head, target, W, H, fovy=40.0, ipd=0.064):
    """Two eyes -/+ ipd/2 along the head's x axis, parallel, looking at target."""
    head, target = np.asarray(head, float), np.asarray(target, float)
    f = (target - head) / np.linalg.norm(target - head)
    s = np.cross(f, [0.0, 0.0, 1.0])
    s /= np.linalg.norm(s)
    proj = synth.colmajor(synth.perspective(fovy, W / H, 0.01, 10.0))
    views = [synth.colmajor(synth.look_at(head + k * ipd / 2 * s, head + k * ipd / 2 * s + f, [0, 0, 1]))
             for k in (-1.0, 1.0)]
    return views, [proj, proj]


@pytest.mark.parametrize("mode", ["bricks", "list", "pipelined", "list_async"])
def test_streaming_frames_match_the_oracle_and_evict_lru(mode, index_ranges=True):
    import torch
    from paper_1804_08197_b300 import sg
    a = synth.filaments_u16(DIMS, seed=31, ntubes=18)
    model = synth.volume_model(128, 0.5)
    ovol = oracle.Volume([oracle.pyramid(a, LEVELS)], B, model=model)
    full = ovol.block_ranges()
    table = synth.tf_piecewise(2002, zero_alpha_points=2)
    otf = oracle.make_tf(table, 300.0, 60000.0)
    W, H, tau = 192, 208, 0.3
    poses = [_stereo((-0.32, 0.05, 0.22), (-0.14, 0.0, 0.0), W, H), _stereo((0.32, -0.05, 0.22), (0.14, 0.0, 0.0), W, H)]
    # working sets of the converged (fully resident) selections size the cache
    need = []
    for views, projs in poses:
        st = ovol.select([otf], views, projs, H, tau=tau)["state"]
        need.append(set(np.flatnonzero(np.isin(st, [oracle.ST_SELECTED, oracle.ST_FALLBACK, oracle.ST_REFINED]))))
    cap = max(len(n) for n in need) + 8
    assert len(need[0] | need[1]) > cap, "the two views must not fit the cache together"
    brick_bytes = ((B + 2) ** 3 * 2 + 255) // 256 * 256
    vol = sg.sg_volume_create(DIMS, sg.SG_U16, B, LEVELS, device_pool_bytes=cap * brick_bytes, model=model)
    try:
        sg.sg_set_transfer_function(vol, 0, table, 300.0, 60000.0)
        known = np.zeros(ovol.node_count, bool)
        if index_ranges:
            # the container's index table gives every brick's range up front
            for L in range(LEVELS):
                nbx, nby, nbz = ovol.blocks_per_axis(L)
                xyz = np.array([(x, y, z) for z in range(nbz) for y in range(nby) for x in range(nbx)])
                lo, hi = ovol.level_offsets[L], ovol.level_offsets[L + 1]
                sg.sg_set_brick_ranges(vol, 0, 0, L, xyz, full[lo:hi, 0, :])
            known[:] = True

        comp = torch.cuda.Stream() if mode == "pipelined" else None
        copy = torch.cuda.Stream() if mode in ("pipelined", "list_async") else None
        keep = []  # page-locked bricks of queued uploads stay alive until the end
        cache = oracle.Cache(ovol, cap)
        nevicted = 0

        def same_residency():
            res = sg.sg_read_residency(vol, 0, ovol.node_count) >= 0
            assert np.array_equal(res, cache.resident != 0), (
                f"GPU-only {np.flatnonzero(res & (cache.resident == 0))}, "
                f"oracle-only {np.flatnonzero(~res & (cache.resident != 0))}")
            return res

        def upload(ids):
            nonlocal nevicted
            if mode in ("list", "pipelined", "list_async"):
                # one call per frame, by node id, coarse levels first
                ids = sorted((int(i) for i in ids), key=lambda n: (-ovol.node_coords(n)[0], n))
                host = []
                for n in ids:
                    L, b = ovol.node_coords(n)
                    host.append(_brick(ovol, L, *b))
                if mode == "list_async":
                    # queued on a copy stream, never waited for here: the next
                    # selection (another stream) waits for it on the device
                    host = [torch.from_numpy(h.view(np.int16)).pin_memory() for h in host]
                    keep.extend(host)
                done = sg.sg_upload_brick_list(vol, 0, 0, ids, host, stream=copy, asynchronous=mode == "list_async")
                m, ev = cache.place(ids)
                assert 0 < done <= len(ids) and done == m
                nevicted += len(ev)
                same_residency()
                known[np.array(ids[:done], dtype=np.int64)] = True
                return
            by_level = {}
            for i in ids:
                L, b = ovol.node_coords(int(i))
                by_level.setdefault(L, []).append((int(i), b))
            for L, nb in by_level.items():
                host = np.stack([_brick(ovol, L, *b) for _, b in nb])
                sg.sg_upload_bricks(vol, 0, 0, L, np.array([b for _, b in nb]), host)
                m, ev = cache.place([n for n, _ in nb])
                assert m == len(nb)
                nevicted += len(ev)
            same_residency()
            known[np.array(list(ids), dtype=np.int64)] = True

        upload([ovol.level_offsets[LEVELS - 1]])  # the root
        for views, projs in poses:
            pose = sg.make_pose(views, projs, W, H, pixel_error=tau)
            for frame in range(24):  # overlap bricks evicted early come back a few frames later
                stats = sg.sg_select_lod(vol, pose, stats=True)
                gsel = sg.sg_read_selection(vol, 0, len(ovol.select([otf], views, projs, H)["leaf"]), ovol.node_count)
                same_residency()
                ranges = full.copy()
                ranges[~known, 0, 0] = 0xFFFFFFFF
                ranges[~known, 0, 1] = 0
                ref = cache.select([otf], views, projs, H, tau=tau, ranges=ranges)
                compare_selection(gsel, ref)
                if stats["requested"] == 0:
                    break
                if mode == "pipelined" and frame < 3:
                    # this frame renders on one stream while its requests
                    # upload on another (evicting only bricks it does not use)
                    outs = [torch.empty((H, W, 4), device="cuda") for _ in range(2)]
                    sg.sg_render(vol, pose, sg.render_params(), outs, stream=comp)
                    upload(gsel[2])
                    comp.synchronize()
                    # early frames mix levels (fallbacks next to refined
                    # blocks): more pixels have points near a face between
                    # levels, each resolved by the oracle's assignments
                    compare_image(outs[0].cpu().numpy().reshape(-1, 4),
                                  ovol.render([otf], ref["leaf"], views[0], projs[0], W, H))
                    continue
                upload(gsel[2])
            assert stats["requested"] == 0 and stats["fallback"] == 0
        assert nevicted > 0, "the second view should have evicted bricks of the first"
        # the converged second view renders like the oracle
        views, projs = poses[1]
        pose = sg.make_pose(views, projs, W, H, pixel_error=tau)
        sg.sg_select_lod(vol, pose)
        outs = [torch.empty((H, W, 4), device="cuda") for _ in range(2)]
        sg.sg_render(vol, pose, sg.render_params(), outs)
        torch.cuda.synchronize()
        ref = ovol.select([otf], views, projs, H, tau=tau)
        for e in range(2):
            compare_image(outs[e].cpu().numpy().reshape(-1, 4),
                          ovol.render([otf], ref["leaf"], views[e], projs[e], W, H))
    finally:
        sg.sg_volume_destroy(vol)


def test_upload_list_cut_short_leaves_a_consistent_cache():
    """A request list longer than the cache: placement stops at the first
    brick that finds every slot used by the current frame, the placed prefix
    is resident and consistent (page table, ranges, flags), and the next
    selection and render match the oracle for exactly that residency."""
    import torch
    from paper_1804_08197_b300 import sg
    a = synth.filaments_u16(DIMS, seed=32, ntubes=24)
    model = synth.volume_model(128, 0.5)
    ovol = oracle.Volume([oracle.pyramid(a, LEVELS)], B, model=model)
    full = ovol.block_ranges()
    table = synth.tf_piecewise(2002, zero_alpha_points=2)
    otf = oracle.make_tf(table, 300.0, 60000.0)
    W, H, tau = 160, 176, 0.3
    views, projs = _stereo((-0.3, 0.06, 0.2), (0.0, 0.0, 0.0), W, H)
    cap = 14
    brick_bytes = ((B + 2) ** 3 * 2 + 255) // 256 * 256
    vol = sg.sg_volume_create(DIMS, sg.SG_U16, B, LEVELS, device_pool_bytes=cap * brick_bytes, model=model)
    try:
        sg.sg_set_transfer_function(vol, 0, table, 300.0, 60000.0)
        for L in range(LEVELS):
            nbx, nby, nbz = ovol.blocks_per_axis(L)
            xyz = np.array([(x, y, z) for z in range(nbz) for y in range(nby) for x in range(nbx)])
            lo, hi = ovol.level_offsets[L], ovol.level_offsets[L + 1]
            sg.sg_set_brick_ranges(vol, 0, 0, L, xyz, full[lo:hi, 0, :])

        def bricks(ids):
            out = []
            for n in ids:
                L, b = ovol.node_coords(int(n))
                out.append(_brick(ovol, L, *b))
            return out

        cache = oracle.Cache(ovol, cap)
        root = [int(ovol.level_offsets[LEVELS - 1])]
        assert sg.sg_upload_brick_list(vol, 0, 0, root, bricks(root)) == 1
        cache.place(root)
        pose = sg.make_pose(views, projs, W, H, pixel_error=tau)
        cut = False
        for frame in range(6):
            sg.sg_select_lod(vol, pose)
            cache.select([otf], views, projs, H, tau=tau, ranges=full)
            req = sg.sg_read_requests(vol, 0)
            if len(req) == 0:
                break
            ids = sorted((int(n) for n in req), key=lambda n: (-ovol.node_coords(n)[0], n))
            host = bricks(ids)
            done = sg.sg_upload_brick_list(vol, 0, 0, ids, host)
            m, _ = cache.place(ids)
            assert done == m
            cut |= done < len(ids)
            res = sg.sg_read_residency(vol, 0, ovol.node_count)
            assert np.array_equal(res >= 0, cache.resident != 0)
            assert len(set(res[res >= 0].tolist())) == np.count_nonzero(res >= 0) <= cap
            # every resident brick holds its own data
            for n in np.flatnonzero(res >= 0)[:6]:
                L, b = ovol.node_coords(int(n))
                got = np.empty((B + 2) ** 3, np.uint16)
                sg.sg_read_brick(vol, 0, 0, L, *b, got)
                assert np.array_equal(got, _brick(ovol, L, *b).reshape(-1))
            # selection and image for exactly this residency
            sg.sg_select_lod(vol, pose)
            ref = cache.select([otf], views, projs, H, tau=tau, ranges=full)
            gsel = sg.sg_read_selection(vol, 0, len(ref["leaf"]), ovol.node_count)
            compare_selection(gsel, ref)
            outs = [torch.empty((H, W, 4), device="cuda") for _ in range(2)]
            sg.sg_render(vol, pose, sg.render_params(), outs)
            torch.cuda.synchronize()
            compare_image(outs[0].cpu().numpy().reshape(-1, 4), ovol.render([otf], ref["leaf"], views[0], projs[0], W, H))
        assert cut, "the cache should have been too small for one frame's requests"
    finally:
        sg.sg_volume_destroy(vol)


def test_streaming_from_a_container_through_the_host_cache(tmp_path):
    """The full storage path: every brick LZ4-compressed in a container,
    a host cache smaller than the volume, sg_stream_requests per frame
    (coarse first, misses decompressed on host threads, one list upload).
    The GPU cache's residency equals the oracle cache's after every frame,
    every frame's selection equals the oracle's, and the converged frame
    renders like the oracle."""
    import torch
    from paper_1804_08197_b300 import sg
    a = synth.filaments_u16(DIMS, seed=33, ntubes=18)
    model = synth.volume_model(128, 0.5)
    ovol = oracle.Volume([oracle.pyramid(a, LEVELS)], B, model=model)
    full = ovol.block_ranges()
    table = synth.tf_piecewise(2002, zero_alpha_points=2)
    otf = oracle.make_tf(table, 300.0, 60000.0)
    path = tmp_path / "vol.sgc"
    desc = sg.volume_desc(DIMS, sg.SG_U16, B, LEVELS, model=model)
    k = sg.sg_container_create(path, desc)
    for n in range(ovol.node_count):
        L, b = ovol.node_coords(n)
        sg.sg_container_append(k, 0, 0, L, *b, _brick(ovol, L, *b), *full[n, 0])
    sg.sg_container_finish(k)
    sg.sg_container_close(k)
    k = sg.sg_container_open(path)
    brick_bytes = ((B + 2) ** 3 * 2 + 255) // 256 * 256
    W, H, tau = 192, 208, 0.3
    views, projs = _stereo((-0.3, 0.05, 0.2), (-0.1, 0.0, 0.0), W, H)
    st_full = ovol.select([otf], views, projs, H, tau=tau)["state"]
    need = int(np.isin(st_full, [oracle.ST_SELECTED, oracle.ST_FALLBACK, oracle.ST_REFINED]).sum())
    # the GPU cache holds the working set; the host cache only half of it
    vol = sg.sg_volume_create(DIMS, sg.SG_U16, B, LEVELS, device_pool_bytes=(need + 8) * brick_bytes, model=model)
    hc = sg.sg_host_cache_create(k, max(need // 2, 48) * (B + 2) ** 3 * 2, pinned=True, threads=4)
    try:
        sg.sg_set_transfer_function(vol, 0, table, 300.0, 60000.0)
        for L in range(LEVELS):
            nbx, nby, nbz = ovol.blocks_per_axis(L)
            xyz = np.array([(x, y, z) for z in range(nbz) for y in range(nby) for x in range(nbx)])
            lo, hi = ovol.level_offsets[L], ovol.level_offsets[L + 1]
            sg.sg_set_brick_ranges(vol, 0, 0, L, xyz, full[lo:hi, 0, :])
        root = int(ovol.level_offsets[LEVELS - 1])
        ptr, _ = sg.sg_host_cache_fetch(hc, 0, 0, root)
        assert sg.sg_upload_brick_list(vol, 0, 0, [root], [ptr]) == 1
        cache = oracle.Cache(ovol, need + 8)
        cache.place([root])
        pose = sg.make_pose(views, projs, W, H, pixel_error=tau)
        total = dict(disk_reads=0, host_hits=0, served=0)
        for frame in range(40):
            stats = sg.sg_select_lod(vol, pose, stats=True)
            res = sg.sg_read_residency(vol, 0, ovol.node_count) >= 0
            assert np.array_equal(res, cache.resident != 0)
            ref = cache.select([otf], views, projs, H, tau=tau, ranges=full)
            compare_selection(sg.sg_read_selection(vol, 0, len(ref["leaf"]), ovol.node_count), ref)
            if stats["requested"] == 0:
                break
            st = sg.sg_stream_requests(vol, 0, hc, 24 * (B + 2) ** 3 * 2)
            assert st["requested"] == stats["requested"] and 0 < st["served"] <= 24 and st["missing"] == 0, (
                frame, st, stats, sg.lib.sg_last_error().decode())
            # served coarse levels first, then by node id, 24 bricks at most
            order = sorted((int(n) for n in ref["requests"]), key=lambda n: (-ovol.node_coords(n)[0], n))
            m, _ = cache.place(order[:24])
            assert m == st["served"]
            for key in total:
                total[key] += st[key]
        assert stats["requested"] == 0 and stats["fallback"] == 0
        assert total["disk_reads"] > 0 and total["served"] > 0
        outs = [torch.empty((H, W, 4), device="cuda") for _ in range(2)]
        sg.sg_render(vol, pose, sg.render_params(), outs)
        torch.cuda.synchronize()
        ref = ovol.select([otf], views, projs, H, tau=tau)
        for e in range(2):
            compare_image(outs[e].cpu().numpy().reshape(-1, 4), ovol.render([otf], ref["leaf"], views[e], projs[e], W, H))
    finally:
        sg.sg_host_cache_destroy(hc)
        sg.sg_volume_destroy(vol)
        sg.sg_container_close(k)


def _corrupt_chunk(path, node, nbytes=16):
    """Overwrites part of the payload of node's chunk (time point 0, channel
    0) in a finished container: footer -> index -> chunk header (48 bytes) ->
    payload. The chunk's checksum no longer matches."""
    import struct
    data = bytearray(open(path, "rb").read())
    magic, version, index_off, chunks = struct.unpack_from("<IIQQ", data, len(data) - 24)
    for i in range(chunks):
        key, off = struct.unpack_from("<qQ", data, index_off + 16 * i)
        if key == node:
            p = off + 48 + 8
            data[p:p + nbytes] = bytes((b ^ 0x5A) for b in data[p:p + nbytes])
            open(path, "wb").write(bytes(data))
            return
    raise AssertionError(f"no chunk for node {node}")


def test_streaming_survives_unreadable_chunks(tmp_path):
    """Failure injected on the host: two level-0 chunks of the container are
    overwritten on disk after conversion. sg_stream_requests serves every
    other request, reports the two (SG_ERR_IO with stats, `failed`), and
    skips them in later frames without spending budget, so streaming keeps
    making progress. Their parents keep rendering in their place ("Octree
    Representation"): frame by frame the GPU cache equals the oracle's and
    the selection equals the oracle's for that residency, the view converges
    with only the two bricks still requested, and the image matches the
    oracle's."""
    import torch
    from paper_1804_08197_b300 import sg
    a = synth.filaments_u16(DIMS, seed=33, ntubes=18)
    model = synth.volume_model(128, 0.5)
    ovol = oracle.Volume([oracle.pyramid(a, LEVELS)], B, model=model)
    full = ovol.block_ranges()
    table = synth.tf_piecewise(2002, zero_alpha_points=2)
    otf = oracle.make_tf(table, 300.0, 60000.0)
    path = tmp_path / "vol.sgc"
    desc = sg.volume_desc(DIMS, sg.SG_U16, B, LEVELS, model=model)
    k = sg.sg_container_create(path, desc)
    for n in range(ovol.node_count):
        L, b = ovol.node_coords(n)
        sg.sg_container_append(k, 0, 0, L, *b, _brick(ovol, L, *b), *full[n, 0])
    sg.sg_container_finish(k)
    sg.sg_container_close(k)
    W, H, tau = 192, 208, 0.3
    views, projs = _stereo((-0.3, 0.05, 0.2), (-0.1, 0.0, 0.0), W, H)
    st_full = ovol.select([otf], views, projs, H, tau=tau)["state"]
    lvl0 = [n for n in np.flatnonzero(st_full == oracle.ST_SELECTED) if ovol.node_coords(int(n))[0] == 0]
    bad = {int(lvl0[len(lvl0) // 3]), int(lvl0[2 * len(lvl0) // 3])}
    for n in bad:
        _corrupt_chunk(path, n)
    k = sg.sg_container_open(path)
    need = int(np.isin(st_full, [oracle.ST_SELECTED, oracle.ST_FALLBACK, oracle.ST_REFINED]).sum())
    brick_bytes = ((B + 2) ** 3 * 2 + 255) // 256 * 256
    vol = sg.sg_volume_create(DIMS, sg.SG_U16, B, LEVELS, device_pool_bytes=(need + 8) * brick_bytes, model=model)
    hc = sg.sg_host_cache_create(k, (need + 8) * (B + 2) ** 3 * 2, pinned=True, threads=4)
    try:
        sg.sg_set_transfer_function(vol, 0, table, 300.0, 60000.0)
        for L in range(LEVELS):
            nbx, nby, nbz = ovol.blocks_per_axis(L)
            xyz = np.array([(x, y, z) for z in range(nbz) for y in range(nby) for x in range(nbx)])
            lo, hi = ovol.level_offsets[L], ovol.level_offsets[L + 1]
            sg.sg_set_brick_ranges(vol, 0, 0, L, xyz, full[lo:hi, 0, :])
        root = int(ovol.level_offsets[LEVELS - 1])
        ptr, _ = sg.sg_host_cache_fetch(hc, 0, 0, root)
        assert sg.sg_upload_brick_list(vol, 0, 0, [root], [ptr]) == 1
        cache = oracle.Cache(ovol, need + 8)
        cache.place([root])
        pose = sg.make_pose(views, projs, W, H, pixel_error=tau)
        failed, known_bad = 0, set()
        for frame in range(40):
            stats = sg.sg_select_lod(vol, pose, stats=True)
            res = sg.sg_read_residency(vol, 0, ovol.node_count) >= 0
            assert np.array_equal(res, cache.resident != 0)
            ref = cache.select([otf], views, projs, H, tau=tau, ranges=full)
            compare_selection(sg.sg_read_selection(vol, 0, len(ref["leaf"]), ovol.node_count), ref)
            if set(int(n) for n in ref["requests"]) <= bad:
                break
            st = sg.sg_stream_requests(vol, 0, hc, 24 * (B + 2) ** 3 * 2)
            failed += st["failed"]
            # a bad brick met for the first time is read (and fails) within
            # the budget; once known it is skipped without spending any
            order = sorted((int(n) for n in ref["requests"]), key=lambda n: (-ovol.node_coords(n)[0], n))
            taken = [n for n in order if n not in known_bad][:24]
            assert st["failed"] == len(known_bad & set(order)) + len(bad & set(taken))
            known_bad |= bad & set(taken)
            m, _ = cache.place([n for n in taken if n not in bad])
            assert m == st["served"] and st["missing"] == 0
        else:
            raise AssertionError("streaming made no progress past the unreadable chunks")
        # both bad bricks were requested, reported, never placed; their
        # parents render as fallbacks
        assert known_bad == bad and failed >= len(bad)
        assert not res[list(bad)].any() and stats["fallback"] > 0
        assert set(int(n) for n in ref["requests"]) == bad
        outs = [torch.empty((H, W, 4), device="cuda") for _ in range(2)]
        sg.sg_render(vol, pose, sg.render_params(), outs)
        torch.cuda.synchronize()
        for e in range(2):
            compare_image(outs[e].cpu().numpy().reshape(-1, 4),
                          ovol.render([otf], ref["leaf"], views[e], projs[e], W, H))
        # after clearing the failures the chunks are tried (and fail) again
        sg.sg_host_cache_clear_failures(hc)
        sg.sg_select_lod(vol, pose)
        cache.select([otf], views, projs, H, tau=tau, ranges=full)
        st = sg.sg_stream_requests(vol, 0, hc, 24 * (B + 2) ** 3 * 2)
        assert st["failed"] == len(bad) and st["served"] == 0
    finally:
        sg.sg_host_cache_destroy(hc)
        sg.sg_volume_destroy(vol)
        sg.sg_container_close(k)


def test_async_streaming_never_waits_and_converges(tmp_path):
    """sg_stream_requests_async: misses go to the host cache's loader
    threads and the call returns at once (the first, cold call serves
    nothing and queues the budget), later calls place what has arrived. The
    residency then depends on timing, so each frame is checked against the
    oracle's selection for the GPU's actual residency. One chunk made
    unreadable on disk is reported by the call that learns of it and
    skipped afterwards; the view converges with only that brick requested
    (its parent renders in its place), and the image matches the oracle."""
    import time
    import torch
    from paper_1804_08197_b300 import sg
    a = synth.filaments_u16(DIMS, seed=33, ntubes=18)
    model = synth.volume_model(128, 0.5)
    ovol = oracle.Volume([oracle.pyramid(a, LEVELS)], B, model=model)
    full = ovol.block_ranges()
    table = synth.tf_piecewise(2002, zero_alpha_points=2)
    otf = oracle.make_tf(table, 300.0, 60000.0)
    path = tmp_path / "vol.sgc"
    desc = sg.volume_desc(DIMS, sg.SG_U16, B, LEVELS, model=model)
    k = sg.sg_container_create(path, desc)
    for n in range(ovol.node_count):
        L, b = ovol.node_coords(n)
        sg.sg_container_append(k, 0, 0, L, *b, _brick(ovol, L, *b), *full[n, 0])
    sg.sg_container_finish(k)
    sg.sg_container_close(k)
    W, H, tau = 192, 208, 0.3
    views, projs = _stereo((-0.3, 0.05, 0.2), (-0.1, 0.0, 0.0), W, H)
    st_full = ovol.select([otf], views, projs, H, tau=tau)["state"]
    lvl0 = [n for n in np.flatnonzero(st_full == oracle.ST_SELECTED) if ovol.node_coords(int(n))[0] == 0]
    bad = int(lvl0[len(lvl0) // 2])
    _corrupt_chunk(path, bad)
    k = sg.sg_container_open(path)
    need = int(np.isin(st_full, [oracle.ST_SELECTED, oracle.ST_FALLBACK, oracle.ST_REFINED]).sum())
    brick_bytes = ((B + 2) ** 3 * 2 + 255) // 256 * 256
    vol = sg.sg_volume_create(DIMS, sg.SG_U16, B, LEVELS, device_pool_bytes=(need + 8) * brick_bytes, model=model)
    hc = sg.sg_host_cache_create(k, (need + 8) * (B + 2) ** 3 * 2, pinned=True, threads=4)
    budget = 24 * (B + 2) ** 3 * 2
    try:
        sg.sg_set_transfer_function(vol, 0, table, 300.0, 60000.0)
        for L in range(LEVELS):
            nbx, nby, nbz = ovol.blocks_per_axis(L)
            xyz = np.array([(x, y, z) for z in range(nbz) for y in range(nby) for x in range(nbx)])
            lo, hi = ovol.level_offsets[L], ovol.level_offsets[L + 1]
            sg.sg_set_brick_ranges(vol, 0, 0, L, xyz, full[lo:hi, 0, :])
        root = int(ovol.level_offsets[LEVELS - 1])
        ptr, _ = sg.sg_host_cache_fetch(hc, 0, 0, root)
        assert sg.sg_upload_brick_list(vol, 0, 0, [root], [ptr]) == 1
        pose = sg.make_pose(views, projs, W, H, pixel_error=tau)
        failed, served, reads = 0, 0, 0
        for frame in range(2000):
            stats = sg.sg_select_lod(vol, pose, stats=True)
            res = sg.sg_read_residency(vol, 0, ovol.node_count) >= 0
            ref = ovol.select([otf], views, projs, H, tau=tau, resident=res.astype(np.uint8), ranges=full)
            compare_selection(sg.sg_read_selection(vol, 0, len(ref["leaf"]), ovol.node_count), ref)
            reqs = set(int(n) for n in ref["requests"])
            if reqs <= {bad} and failed:
                break
            st = sg.sg_stream_requests(vol, 0, hc, budget, asynchronous=True)
            assert st["missing"] == 0 and st["served"] <= 24 and st["requested"] == stats["requested"]
            if frame == 0:
                # a cold host cache: nothing to place yet, a full budget of loads queued
                assert st["served"] == 0 and st["queued"] == min(24, len(reqs))
                assert 0 <= st["in_flight"] <= st["queued"]  # the loaders may already have finished some
            failed += st["failed"]
            served += st["served"]
            reads += st["disk_reads"]
            if st["served"] == 0:
                time.sleep(0.002)  # nothing arrived yet: let the loaders work
        else:
            raise AssertionError("asynchronous streaming did not converge")
        assert failed >= 1 and served > 0 and reads >= served
        assert not res[bad] and stats["fallback"] > 0
        outs = [torch.empty((H, W, 4), device="cuda") for _ in range(2)]
        sg.sg_render(vol, pose, sg.render_params(), outs)
        torch.cuda.synchronize()
        for e in range(2):
            compare_image(outs[e].cpu().numpy().reshape(-1, 4),
                          ovol.render([otf], ref["leaf"], views[e], projs[e], W, H))
        # the blocking call on the same cache waits for nothing and places nothing new
        st = sg.sg_stream_requests(vol, 0, hc, budget)
        assert st["served"] == 0 and st["failed"] == 1
    finally:
        sg.sg_host_cache_destroy(hc)
        sg.sg_volume_destroy(vol)
        sg.sg_container_close(k)


def test_full_size_large_volume_selection_and_cache_match_the_oracle():
    """The large-volume configuration's layout at full size: 4096^3 u8 over
    1 m, 128^3 bricks, 6 levels (37 449 blocks), along a 48-pose seeded
    fly-through (seed 3004) at 2 x 1440 x 1600, tau 1 px, a 2000-brick device
    cache and 64 bricks uploaded per frame (coarse first). The transfer
    function has non-zero alpha everywhere, so no block is transparent
    whatever its values and the selection depends only on the geometry and
    the residency: uploads can be zero bricks, and the oracle needs no voxel
    data (a layout-only volume with every range [0, 255]). Every frame the
    GPU cache's residency equals the oracle cache's and the selection (leaf
    map, node states, requests) equals the oracle's bit for bit."""
    import torch
    from paper_1804_08197_b300 import sg
    N, BB, LV, slots, per_frame = 4096, 128, 6, 2000, 64
    model = synth.volume_model(N, 1.0)
    ovol = oracle.Volume.layout((N, N, N), BB, LV, model=model, dtype=np.uint8)
    assert ovol.node_count == 37449
    ranges = np.zeros((ovol.node_count, 1, 2), np.uint32)
    ranges[:, 0, 1] = 255
    table = synth.tf_piecewise(2004).copy()
    table[:, 3] = np.maximum(table[:, 3], 0.05)  # opaque enough everywhere: nothing is transparent
    otf = oracle.make_tf(table, 0.0, 255.0)
    R = BB + 2
    brick_bytes = (R ** 3 + 255) // 256 * 256
    vol = sg.sg_volume_create((N, N, N), sg.SG_U8, BB, LV, model=model, device_pool_bytes=slots * brick_bytes)
    zero = torch.zeros(R ** 3, dtype=torch.uint8).pin_memory()
    try:
        sg.sg_set_transfer_function(vol, 0, table, 0.0, 255.0)
        for L in range(LV):
            nbx, nby, nbz = ovol.blocks_per_axis(L)
            xyz = np.array([(x, y, z) for z in range(nbz) for y in range(nby) for x in range(nbx)])
            lo, hi = ovol.level_offsets[L], ovol.level_offsets[L + 1]
            sg.sg_set_brick_ranges(vol, 0, 0, L, xyz, ranges[lo:hi, 0, :])
        root = int(ovol.level_offsets[LV - 1])
        assert sg.sg_upload_brick_list(vol, 0, 0, [root], [zero.data_ptr()]) == 1
        cache = oracle.Cache(ovol, slots)
        cache.place([root])
        W, H = 1440, 1600
        poses = synth.flythrough_poses(48, seed=3004, extent_m=1.0, width=W, height=H)
        nb0 = ovol.blocks_per_axis(0)
        ncell = nb0[0] * nb0[1] * nb0[2]
        evicted, requested, fallback = 0, 0, 0
        for views, projs in poses:
            pose = sg.make_pose(views, projs, W, H, pixel_error=1.0)
            stats = sg.sg_select_lod(vol, pose, stats=True)
            res = sg.sg_read_residency(vol, 0, ovol.node_count) >= 0
            assert np.array_equal(res, cache.resident != 0)
            ref = cache.select([otf], views, projs, H, tau=1.0, ranges=ranges)
            compare_selection(sg.sg_read_selection(vol, 0, ncell, ovol.node_count), ref)
            assert stats["selected"] == ref["selected"] and stats["empty"] == 0
            requested += stats["requested"]
            fallback += stats["fallback"]
            order = sorted((int(n) for n in ref["requests"]), key=lambda n: (-ovol.node_coords(n)[0], n))[:per_frame]
            if order:
                done = sg.sg_upload_brick_list(vol, 0, 0, order, [zero.data_ptr()] * len(order))
                m, ev = cache.place(order)
                assert m == done
                evicted += len(ev)
        assert requested > 0 and fallback > 0 and evicted > 0
    finally:
        sg.sg_volume_destroy(vol)


def test_two_channel_container_streams_both_channels_together(tmp_path):
    """A 2-channel container (blob channels 0 and 1, their own tables,
    additive blend): a brick is placed only once both of its channels are in
    the host cache, so the GPU never holds one channel of a brick. Streamed
    asynchronously until the view converges; every frame's selection equals
    the oracle's for the GPU's residency, and the converged image matches
    the oracle's two-channel rendering."""
    import time
    import torch
    from paper_1804_08197_b300 import sg
    dims = (96, 80, 64)
    chans = [synth.blobs_u16(dims, seed=1003, channel=c, nblobs=10) for c in range(2)]
    model = synth.volume_model(96, 0.5)
    ovol = oracle.Volume([oracle.pyramid(a, 3) for a in chans], 16, model=model)
    full = ovol.block_ranges()
    tables = [synth.tf_piecewise(2003, zero_alpha_points=2, colour=(0.1, 0.9, 0.2)),
              synth.tf_piecewise(2004, zero_alpha_points=2, colour=(0.9, 0.1, 0.8))]
    otfs = [oracle.make_tf(t, 200.0, 40000.0) for t in tables]
    path = tmp_path / "two.sgc"
    k = sg.sg_container_create(path, sg.volume_desc(dims, sg.SG_U16, 16, 3, channels=2, model=model))
    for n in range(ovol.node_count):
        L, b = ovol.node_coords(n)
        for c in range(2):
            g = ovol.channels[c][L]
            R = 18
            iz = np.clip(np.arange(R) + b[2] * 16 - 1, 0, g.shape[0] - 1)
            iy = np.clip(np.arange(R) + b[1] * 16 - 1, 0, g.shape[1] - 1)
            ix = np.clip(np.arange(R) + b[0] * 16 - 1, 0, g.shape[2] - 1)
            sg.sg_container_append(k, 0, c, L, *b, np.ascontiguousarray(g[np.ix_(iz, iy, ix)]), *full[n, c])
    sg.sg_container_finish(k)
    sg.sg_container_close(k)
    k = sg.sg_container_open(path)
    brick_bytes = (18 ** 3 * 2 + 255) // 256 * 256
    vol = sg.sg_volume_create(dims, sg.SG_U16, 16, 3, channels=2, model=model,
                              device_pool_bytes=ovol.node_count * brick_bytes * 2)
    hc = sg.sg_host_cache_create(k, 2 * ovol.node_count * 18 ** 3 * 2, pinned=True, threads=4)
    try:
        for c in range(2):
            sg.sg_set_transfer_function(vol, c, tables[c], 200.0, 40000.0)
            for L in range(3):
                nbx, nby, nbz = ovol.blocks_per_axis(L)
                xyz = np.array([(x, y, z) for z in range(nbz) for y in range(nby) for x in range(nbx)])
                lo, hi = ovol.level_offsets[L], ovol.level_offsets[L + 1]
                sg.sg_set_brick_ranges(vol, 0, c, L, xyz, full[lo:hi, c, :])
        top = list(range(int(ovol.level_offsets[2]), int(ovol.level_offsets[3])))  # the coarsest level (pinned)
        for c in range(2):
            ptrs = [sg.sg_host_cache_fetch(hc, 0, c, n)[0] for n in top]
            assert sg.sg_upload_brick_list(vol, 0, c, top, ptrs) == len(top)
        W, H, tau = 160, 176, 0.5
        views, projs = _stereo((-0.3, 0.05, 0.2), (-0.05, 0.0, 0.0), W, H)
        pose = sg.make_pose(views, projs, W, H, pixel_error=tau)
        for frame in range(2000):
            stats = sg.sg_select_lod(vol, pose, stats=True)
            res = sg.sg_read_residency(vol, 0, ovol.node_count) >= 0
            ref = ovol.select(otfs, views, projs, H, tau=tau, resident=res.astype(np.uint8), ranges=full)
            nb0 = ovol.blocks_per_axis(0)
            compare_selection(sg.sg_read_selection(vol, 0, nb0[0] * nb0[1] * nb0[2], ovol.node_count), ref)
            if stats["requested"] == 0:
                break
            st = sg.sg_stream_requests(vol, 0, hc, 16 * 18 ** 3 * 2 * 2, asynchronous=True)
            assert st["failed"] == 0 and st["missing"] == 0
            if st["served"] == 0:
                time.sleep(0.002)
        else:
            raise AssertionError("two-channel streaming did not converge")
        assert stats["fallback"] == 0
        outs = [torch.empty((H, W, 4), device="cuda") for _ in range(2)]
        sg.sg_render(vol, pose, sg.render_params(), outs)
        torch.cuda.synchronize()
        for e in range(2):
            compare_image(outs[e].cpu().numpy().reshape(-1, 4), ovol.render(otfs, ref["leaf"], views[e], projs[e], W, H))
    finally:
        sg.sg_host_cache_destroy(hc)
        sg.sg_volume_destroy(vol)
        sg.sg_container_close(k)


def test_async_streaming_through_a_small_host_cache_keeps_bricks_intact(tmp_path):
    """sg_stream_requests_async with a host cache of 40 bricks, far fewer
    than the views need: nearly every call evicts entries that the previous
    call's queued copies read, on one stream or alternating between two. An
    entry reused while a copy still reads it would leave a wrong brick on
    the GPU, so after an eight-pose fly-through every resident brick is read
    back and compared voxel for voxel with the oracle's pyramid, and the
    last frame's selection and image match the oracle."""
    import time
    import torch
    from paper_1804_08197_b300 import sg
    a = synth.filaments_u16(DIMS, seed=35, ntubes=24)
    model = synth.volume_model(128, 0.5)
    ovol = oracle.Volume([oracle.pyramid(a, LEVELS)], B, model=model)
    full = ovol.block_ranges()
    table = synth.tf_piecewise(2004, zero_alpha_points=2)
    otf = oracle.make_tf(table, 300.0, 60000.0)
    path = tmp_path / "vol.sgc"
    k = sg.sg_container_create(path, sg.volume_desc(DIMS, sg.SG_U16, B, LEVELS, model=model))
    for n in range(ovol.node_count):
        L, b = ovol.node_coords(n)
        sg.sg_container_append(k, 0, 0, L, *b, _brick(ovol, L, *b), *full[n, 0])
    sg.sg_container_finish(k)
    sg.sg_container_close(k)
    k = sg.sg_container_open(path)
    R = B + 2
    brick_bytes = (R ** 3 * 2 + 255) // 256 * 256
    vol = sg.sg_volume_create(DIMS, sg.SG_U16, B, LEVELS, device_pool_bytes=ovol.node_count * brick_bytes, model=model)
    hc = sg.sg_host_cache_create(k, 40 * R ** 3 * 2, pinned=True, threads=4)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    W, H, tau = 160, 176, 0.3
    try:
        sg.sg_set_transfer_function(vol, 0, table, 300.0, 60000.0)
        for L in range(LEVELS):
            nbx, nby, nbz = ovol.blocks_per_axis(L)
            xyz = np.array([(x, y, z) for z in range(nbz) for y in range(nby) for x in range(nbx)])
            lo, hi = ovol.level_offsets[L], ovol.level_offsets[L + 1]
            sg.sg_set_brick_ranges(vol, 0, 0, L, xyz, full[lo:hi, 0, :])
        root = int(ovol.level_offsets[LEVELS - 1])
        ptr, _ = sg.sg_host_cache_fetch(hc, 0, 0, root)
        assert sg.sg_upload_brick_list(vol, 0, 0, [root], [ptr]) == 1
        reads, calls = 0, 0
        for i in range(8):
            ang = 2 * np.pi * i / 8
            head = (0.45 * np.cos(ang), 0.45 * np.sin(ang), 0.05)
            views, projs = _stereo(head, (0.0, 0.0, 0.0), W, H)
            pose = sg.make_pose(views, projs, W, H, pixel_error=tau)
            for frame in range(400):
                stats = sg.sg_select_lod(vol, pose, stats=True)
                if stats["requested"] == 0:
                    break
                s = streams[(calls // 3) % 2] if i % 2 else streams[0]
                st = sg.sg_stream_requests(vol, 0, hc, 24 * R ** 3 * 2, stream=s, asynchronous=True)
                assert st["failed"] == 0 and st["missing"] == 0
                reads += st["disk_reads"]
                calls += 1
                if st["served"] == 0:
                    time.sleep(0.002)
            else:
                raise AssertionError(f"pose {i}: streaming did not converge")
        torch.cuda.synchronize()
        assert reads > 3 * 40  # the host cache turned over several times
        res = sg.sg_read_residency(vol, 0, ovol.node_count)
        got = np.empty((R, R, R), np.uint16)
        checked = 0
        for n in np.flatnonzero(res >= 0):
            L, b = ovol.node_coords(int(n))
            sg.sg_read_brick(vol, 0, 0, L, *b, got)
            assert np.array_equal(got, _brick(ovol, L, *b)), (int(n), L, b)
            checked += 1
        assert checked > 40
        ref = ovol.select([otf], views, projs, H, tau=tau, resident=(res >= 0).astype(np.uint8), ranges=full)
        compare_selection(sg.sg_read_selection(vol, 0, len(ref["leaf"]), ovol.node_count), ref)
        assert len(ref["requests"]) == 0
        outs = [torch.empty((H, W, 4), device="cuda") for _ in range(2)]
        sg.sg_render(vol, pose, sg.render_params(), outs)
        torch.cuda.synchronize()
        for e in range(2):
            compare_image(outs[e].cpu().numpy().reshape(-1, 4), ovol.render([otf], ref["leaf"], views[e], projs[e], W, H))
    finally:
        sg.sg_host_cache_destroy(hc)
        sg.sg_volume_destroy(vol)
        sg.sg_container_close(k)
