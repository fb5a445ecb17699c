"""Brick container and host cache ("Volumetric Data Storage", "Volumetric
Data Cashing"), host only: the chunk codec against the LZ4 block format
(a hand-built block decoded by the library; the library's blocks decoded by
an independent decoder written here from the format definition), resumed
conversions, the index, and the host cache's least-recently-used order."""
import ctypes
import os
import struct

import numpy as np
import pytest

import synth

B = 8
R3 = (B + 2) ** 3


def _sg():
    from paper_1804_08197_b300 import sg
    return sg


def lz4_decode(block, n):
    """LZ4 block format: token (literals << 4 | match - 4), extension bytes
    of 255 continue a length, literals, 2-byte little-endian offset."""
    out = bytearray()
    i = 0
    while i < len(block):
        tok = block[i]
        i += 1
        lit = tok >> 4
        if lit == 15:
            while True:
                b = block[i]
                i += 1
                lit += b
                if b != 255:
                    break
        out += block[i:i + lit]
        i += lit
        if i == len(block):
            break
        off = block[i] | (block[i + 1] << 8)
        i += 2
        ml = tok & 15
        if ml == 15:
            while True:
                b = block[i]
                i += 1
                ml += b
                if b != 255:
                    break
        ml += 4
        for _ in range(ml):
            out.append(out[-off])
    assert len(out) == n
    return bytes(out)


def fnv1a(data):
    h = 2166136261
    for b in data:
        h = ((h ^ b) * 16777619) & 0xFFFFFFFF
    return h


def _desc(dims=(16, 16, 8), levels=2, dtype=None):
    sg = _sg()
    return sg.volume_desc(dims, sg.SG_U8 if dtype is None else dtype, B, levels)


def _chunks(path, desc_size):
    """(header fields, payload) of every chunk, read from the documented layout."""
    data = open(path, "rb").read()
    off = 8 + desc_size
    out = []
    while off + 48 <= len(data) and data[off:off + 4] == b"CHNK":
        fields = struct.unpack_from("<4s6i5I", data, off)
        comp = fields[8]
        out.append((fields, data[off + 48:off + 48 + comp]))
        off += 48 + comp
    return out


def test_library_decodes_a_hand_built_lz4_block(tmp_path):
    sg = _sg()
    desc = _desc()
    pattern = bytes(b"abcd"[i % 4] for i in range(R3))
    # literals "abcd"; match offset 4, length 991 (987 = 15 + 255*3 + 207);
    # last literals "dabcd"
    block = bytes([0x4F]) + b"abcd" + bytes([4, 0, 255, 255, 255, 207, 0x50]) + b"dabcd"
    assert lz4_decode(block, R3) == pattern  # the test's own decoder agrees
    path = tmp_path / "hand.sgc"
    head = struct.pack("<II", 0x31434753, 1) + bytes(desc)
    chunk = struct.pack("<4s6i5I", b"CHNK", 0, 0, 0, 1, 1, 0, R3, len(block), 97, 100, fnv1a(block)) + block
    path.write_bytes(head + chunk)
    k = sg.sg_container_open(path)
    try:
        info = sg.sg_container_get_info(k)
        assert info["chunks"] == 1 and not info["complete"]
        out = np.zeros(R3, np.uint8)
        node = 0 * 0 + (0 * 1 + 1) * 2 + 1  # level 0, blocks (2, 2, 1): node = (bz*2 + by)*2 + bx
        assert sg.sg_container_read(k, 0, 0, node, out) == (97, 100)
        assert out.tobytes() == pattern
    finally:
        sg.sg_container_close(k)


def _bricks(levels=2):
    a = synth.cells_u8_box(16, 0, 0, 0, 16, 16, 8, seed=1004, cell=8)
    rng = np.random.default_rng(1)
    out = {}
    for L in range(levels):
        nb = (2, 2, 1) if L == 0 else (1, 1, 1)
        for bz in range(nb[2]):
            for by in range(nb[1]):
                for bx in range(nb[0]):
                    b = np.roll(a, L * 3 + bx, axis=2)[:10, :10, :10].copy() if bz == 0 else None
                    b = np.pad(b, ((0, 10 - b.shape[0]), (0, 0), (0, 0)), mode="edge")
                    if (L + bx + by) % 2:
                        b = rng.integers(0, 256, (10, 10, 10)).astype(np.uint8)  # incompressible
                    out[(L, bx, by, bz)] = np.ascontiguousarray(b)
    return out


def _node(L, bx, by, bz):
    return (0 if L == 0 else 4) + (bz * (2 if L == 0 else 1) + by) * (2 if L == 0 else 1) + bx


def test_round_trip_index_and_format(tmp_path):
    sg = _sg()
    desc = _desc()
    path = tmp_path / "v.sgc"
    bricks = _bricks()
    k = sg.sg_container_create(path, desc)
    for (L, bx, by, bz), b in bricks.items():
        sg.sg_container_append(k, 0, 0, L, bx, by, bz, b, int(b.min()), int(b.max()))
    sg.sg_container_finish(k)
    with pytest.raises(sg.SGError):
        sg.sg_container_append(k, 0, 0, 0, 0, 0, 0, bricks[(0, 0, 0, 0)], 0, 0)
    sg.sg_container_close(k)
    # every payload is a valid LZ4 block of the brick (independent decoder)
    chunks = _chunks(path, ctypes.sizeof(desc))
    assert len(chunks) == len(bricks)
    for fields, payload in chunks:
        _, t, c, L, bx, by, bz, raw, comp, vmin, vmax, cs = fields
        assert raw == R3 and fnv1a(payload) == cs
        assert lz4_decode(payload, R3) == bricks[(L, bx, by, bz)].tobytes()
    k = sg.sg_container_open(path)
    try:
        info = sg.sg_container_get_info(k)
        assert info["complete"] and info["chunks"] == len(bricks) and info["raw_bytes"] == R3 * len(bricks)
        assert info["compressed_bytes"] < info["raw_bytes"]  # the structured bricks compress
        out = np.zeros(R3, np.uint8)
        for (L, bx, by, bz), b in bricks.items():
            assert sg.sg_container_read(k, 0, 0, _node(L, bx, by, bz), out) == (b.min(), b.max())
            assert np.array_equal(out, b.reshape(-1))
    finally:
        sg.sg_container_close(k)


def test_interrupted_conversion_resumes_after_the_last_complete_chunk(tmp_path):
    sg = _sg()
    desc = _desc()
    path = tmp_path / "v.sgc"
    bricks = list(_bricks().items())
    k = sg.sg_container_create(path, desc)
    for (L, bx, by, bz), b in bricks[:3]:
        sg.sg_container_append(k, 0, 0, L, bx, by, bz, b, int(b.min()), int(b.max()))
    sg.sg_container_close(k)  # no index: the conversion "stopped"
    size = os.path.getsize(path)
    with open(path, "r+b") as f:  # tear the third chunk
        f.truncate(size - 7)
    k = sg.sg_container_open(path)
    info = sg.sg_container_get_info(k)
    assert info["chunks"] == 2 and not info["complete"]
    for (L, bx, by, bz), b in bricks[2:]:
        sg.sg_container_append(k, 0, 0, L, bx, by, bz, b, int(b.min()), int(b.max()))
    sg.sg_container_finish(k)
    sg.sg_container_close(k)
    k = sg.sg_container_open(path)
    try:
        info = sg.sg_container_get_info(k)
        assert info["complete"] and info["chunks"] == len(bricks)
        out = np.zeros(R3, np.uint8)
        for (L, bx, by, bz), b in bricks:
            sg.sg_container_read(k, 0, 0, _node(L, bx, by, bz), out)
            assert np.array_equal(out, b.reshape(-1))
    finally:
        sg.sg_container_close(k)


def test_host_cache_keeps_the_most_recently_used_bricks(tmp_path):
    sg = _sg()
    desc = _desc()
    path = tmp_path / "v.sgc"
    bricks = _bricks()
    k = sg.sg_container_create(path, desc)
    for (L, bx, by, bz), b in bricks.items():
        sg.sg_container_append(k, 0, 0, L, bx, by, bz, b, 0, 255)
    sg.sg_container_finish(k)
    hc = sg.sg_host_cache_create(k, 3 * R3 + 10, pinned=False, threads=2)
    try:
        # three entries: 0, 1, 2 fill it; 0 hits; 3 evicts 1 (least recently
        # used); 1 evicts 2; 0 hits; 4 evicts 3 (last used before 1 and 0);
        # so 3 misses again
        seq = [0, 1, 2, 0, 3, 1, 0, 4, 3]
        expect_hit = [False, False, False, True, False, False, True, False, False]
        for n, hit in zip(seq, expect_hit):
            ptr, h = sg.sg_host_cache_fetch(hc, 0, 0, n)
            assert h == hit, (n, h)
            key = [kk for kk in bricks if _node(*kk) == n][0]
            got = np.ctypeslib.as_array((ctypes.c_uint8 * R3).from_address(ptr))
            assert np.array_equal(got, bricks[key].reshape(-1))
        with pytest.raises(sg.SGError):
            sg.sg_host_cache_fetch(hc, 0, 0, 99)
    finally:
        sg.sg_host_cache_destroy(hc)
        sg.sg_container_close(k)


def test_container_arguments_are_checked(tmp_path):
    sg = _sg()
    with pytest.raises(sg.SGError):
        sg.sg_container_open(tmp_path / "missing.sgc")
    (tmp_path / "junk.sgc").write_bytes(b"not a container at all, no header here")
    with pytest.raises(sg.SGError):
        sg.sg_container_open(tmp_path / "junk.sgc")
    k = sg.sg_container_create(tmp_path / "v.sgc", _desc())
    try:
        with pytest.raises(sg.SGError):
            sg.sg_container_append(k, 0, 0, 0, 5, 0, 0, np.zeros(R3, np.uint8), 0, 0)
        with pytest.raises(sg.SGError):
            sg.sg_container_read(k, 0, 0, 0, np.zeros(R3, np.uint8))
    finally:
        sg.sg_container_close(k)


def _chunk_offsets(path, desc_size):
    """file offset of each chunk's payload, by (level, bx, by, bz)."""
    data = open(path, "rb").read()
    off = 8 + desc_size
    out = {}
    while off + 48 <= len(data) and data[off:off + 4] == b"CHNK":
        fields = struct.unpack_from("<4s6i5I", data, off)
        out[tuple(fields[3:7])] = off + 48
        off += 48 + fields[8]
    return out


def test_background_loads_land_in_the_host_cache(tmp_path):
    """sg_host_cache_prefetch hands misses to loader threads; after
    sg_host_cache_wait every good brick is a hit holding its data, and a
    chunk made unreadable on disk is reported, remembered and skipped until
    the failures are cleared ("Volumetric Data Cashing")."""
    sg = _sg()
    desc = _desc()
    path = tmp_path / "v.sgc"
    bricks = _bricks()
    k = sg.sg_container_create(path, desc)
    for (L, bx, by, bz), b in bricks.items():
        sg.sg_container_append(k, 0, 0, L, bx, by, bz, b, 0, 255)
    sg.sg_container_finish(k)
    sg.sg_container_close(k)
    bad = (0, 0, 1, 0)  # level 0, brick (0, 1, 0): node 2
    off = _chunk_offsets(path, ctypes.sizeof(desc))[bad]
    with open(path, "r+b") as f:
        f.seek(off)
        f.write(b"\xff" * 8)
    k = sg.sg_container_open(path)
    hc = sg.sg_host_cache_create(k, 5 * R3 + 10, pinned=False, threads=3)
    try:
        nodes = [_node(*kk) for kk in bricks]
        assert sg.sg_host_cache_prefetch(hc, 0, 0, nodes) == len(nodes)
        assert sg.sg_host_cache_wait(hc) == 1
        for kk, b in bricks.items():
            if kk == bad:
                continue
            ptr, hit = sg.sg_host_cache_fetch(hc, 0, 0, _node(*kk))
            assert hit
            got = np.ctypeslib.as_array((ctypes.c_uint8 * R3).from_address(ptr))
            assert np.array_equal(got, b.reshape(-1))
        # the bad chunk is skipped, read again once the failures are cleared
        assert sg.sg_host_cache_prefetch(hc, 0, 0, [_node(*bad)]) == 0
        sg.sg_host_cache_clear_failures(hc)
        assert sg.sg_host_cache_prefetch(hc, 0, 0, [_node(*bad)]) == 1
        assert sg.sg_host_cache_wait(hc) == 1
        with pytest.raises(sg.SGError):
            sg.sg_host_cache_fetch(hc, 0, 0, _node(*bad))
        with pytest.raises(sg.SGError):
            sg.sg_host_cache_prefetch(hc, 0, 0, [99])
    finally:
        sg.sg_host_cache_destroy(hc)
    # a cache of two entries: the third load of one call finds none free
    hc = sg.sg_host_cache_create(k, 2 * R3 + 10, pinned=False, threads=2)
    try:
        with pytest.raises(sg.SGError):
            sg.sg_host_cache_prefetch(hc, 0, 0, [0, 1, 3])
        assert sg.sg_host_cache_wait(hc) == 0
        assert sg.sg_host_cache_fetch(hc, 0, 0, 1)[1]
    finally:
        sg.sg_host_cache_destroy(hc)
    # destroyed with loads still queued: the loaders stop and are joined
    hc = sg.sg_host_cache_create(k, 5 * R3 + 10, pinned=False, threads=1)
    sg.sg_host_cache_prefetch(hc, 0, 0, [0, 1, 3, 4])
    sg.sg_host_cache_destroy(hc)
    sg.sg_container_close(k)


def test_loads_in_flight_are_never_evicted(tmp_path):
    """A host cache of 8 entries fed faster than its 4 loader threads
    finish: calls that find every entry either loading or used this frame
    place nothing (SG_ERR_OOM) instead of evicting an entry a loader is
    still writing. After every wait each cached brick holds its own chunk's
    data, and the cache never holds more bricks than entries."""
    sg = _sg()
    desc = sg.volume_desc((64, 64, 64), sg.SG_U8, B, 3)
    nodes = 8 ** 3 + 4 ** 3 + 2 ** 3
    rng = np.random.default_rng(7)
    bricks = {}
    path = tmp_path / "v.sgc"
    k = sg.sg_container_create(path, desc)
    for n in range(nodes):
        L = 0 if n < 512 else (1 if n < 576 else 2)
        nb = 8 >> L
        i = n - (0 if L == 0 else (512 if L == 1 else 576))
        bx, by, bz = i % nb, (i // nb) % nb, i // (nb * nb)
        b = rng.integers(0, 256, (B + 2,) * 3).astype(np.uint8)
        b[0, 0, :2] = (n & 255, n >> 8)  # the brick's own id in its first voxels
        bricks[n] = b
        sg.sg_container_append(k, 0, 0, L, bx, by, bz, b, 0, 255)
    sg.sg_container_finish(k)
    sg.sg_container_close(k)
    k = sg.sg_container_open(path)
    hc = sg.sg_host_cache_create(k, 8 * R3, pinned=False, threads=4)
    try:
        full = 0
        for rnd in range(300):
            want = [int(x) for x in rng.choice(nodes, 8, replace=False)]
            try:
                sg.sg_host_cache_prefetch(hc, 0, 0, want)
            except sg.SGError:
                full += 1
            if rnd % 10 == 9:
                assert sg.sg_host_cache_wait(hc) == 0
                for n in want:
                    ptr, hit = sg.sg_host_cache_fetch(hc, 0, 0, n)
                    got = np.ctypeslib.as_array((ctypes.c_uint8 * R3).from_address(ptr))
                    assert np.array_equal(got, bricks[n].reshape(-1)), (rnd, n, hit)
        assert full > 0  # the loaders were outpaced at least once
    finally:
        sg.sg_host_cache_destroy(hc)
        sg.sg_container_close(k)
