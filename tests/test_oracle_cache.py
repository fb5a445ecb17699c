"""Pins of the oracle's brick cache ("Volumetric Data Cashing": chunks carry
time stamps; when the GPU cache is full the oldest is dropped). Reading:
evict the smallest stamp older than the current frame, ties to the coarser
block and then to the lower node id; blocks of the coarsest level are
pinned; requests are placed in the order given and placement stops at the
first one that finds every unpinned block in use this frame."""
import numpy as np

import oracle


def _vol():
    # 32 x 16 x 16 voxels, blocks of 8: level 0 has 4 x 2 x 2 = 16 blocks
    # (ids 0..15), level 1 has 2 (ids 16, 17), level 2 one root (id 18)
    lv = [np.zeros((16, 16, 32), np.uint8), np.zeros((8, 8, 16), np.uint8), np.zeros((4, 4, 8), np.uint8)]
    vol = oracle.Volume([lv], 8)
    assert vol.node_count == 19 and list(vol.level_offsets) == [0, 16, 18, 19]
    return vol


def _cache(vol, slots, stamps, frame):
    c = oracle.Cache(vol, slots)
    for i, st in stamps.items():
        c.resident[i] = 1
        c.stamp[i] = st
    c.frame = frame
    return c


def test_hand_worked_evictions():
    """Five slots hold the root 18 (pinned) and 16 (stamp 3), 17 (5), 0 (3),
    1 (4); frame 6 requests 2, 3, 4.
      2: smallest stamp 3 is shared by 16 (level 1) and 0 (level 0): the
         coarser 16 goes.
      3: stamps left 17:5, 0:3, 1:4: 0 goes.
      4: 17:5, 1:4: 1 goes.
    A second list in the same frame, 5 then 6: 5 evicts 17 (the only block
    older than frame 6); 6 finds 2, 3, 4, 5 all stamped 6 and stops the list
    after one request."""
    vol = _vol()
    c = _cache(vol, 5, {18: 0, 16: 3, 17: 5, 0: 3, 1: 4}, 6)
    m, ev = c.place([2, 3, 4])
    assert m == 3 and list(ev) == [16, 0, 1]
    assert set(np.flatnonzero(c.resident)) == {18, 17, 2, 3, 4}
    assert all(c.stamp[i] == 6 for i in (2, 3, 4))
    m, ev = c.place([5, 6])
    assert m == 1 and list(ev) == [17]
    assert set(np.flatnonzero(c.resident)) == {18, 2, 3, 4, 5}
    # a resident request is left as it is
    m, ev = c.place([3])
    assert m == 1 and len(ev) == 0


def test_equal_stamps_on_one_level_evict_the_lower_id_first():
    vol = _vol()
    c = _cache(vol, 5, {18: 0, 0: 2, 5: 2, 9: 2, 12: 2}, 3)
    m, ev = c.place([1, 7])
    assert m == 2 and list(ev) == [0, 5]


def test_free_slots_are_used_before_any_eviction():
    vol = _vol()
    c = _cache(vol, 8, {18: 0, 0: 1}, 4)
    m, ev = c.place([1, 2, 3, 4, 5, 6])
    assert m == 6 and len(ev) == 0 and c.resident.sum() == 8
    m, ev = c.place([7])
    assert m == 1 and list(ev) == [0]


def test_invariants_over_random_histories():
    """Whatever the history: never more than `slots` resident, the root is
    never evicted, no block stamped with the current frame is evicted, a
    list is processed as a prefix, and every eviction takes a block whose
    (stamp, -level, id) is the smallest among the unpinned blocks older than
    the frame at that moment."""
    vol = _vol()
    rng = np.random.default_rng(5)
    level = np.array([0] * 16 + [1, 1, 2])
    for trial in range(200):
        slots = int(rng.integers(2, 10))
        c = oracle.Cache(vol, slots)
        c.place([18])
        for frame in range(1, 8):
            c.frame = frame
            # blocks "used" this frame get its stamp
            used = rng.random(19) < 0.3
            c.stamp[used & (c.resident != 0)] = frame
            req = rng.choice(18, size=int(rng.integers(0, 6)), replace=False)
            before_res = c.resident.copy()
            before_st = c.stamp.copy()
            m, ev = c.place(req)
            assert c.resident.sum() <= slots and c.resident[18]
            assert 0 <= m <= len(req)
            if m < len(req):
                # the list stopped: no evictable block was left
                cand = (c.resident != 0) & (np.arange(19) < 18) & (c.stamp < frame)
                assert not cand.any() and c.resident.sum() == slots
            # replay the evictions against the key order
            res = before_res.copy()
            st = before_st.copy()
            evs = list(ev)
            for r in req[:m]:
                if res[r]:
                    continue
                if res.sum() >= slots:
                    cand = [j for j in range(18) if res[j] and st[j] < frame]
                    best = min(cand, key=lambda j: (st[j], -level[j], j))
                    assert evs and evs.pop(0) == best
                    res[best] = 0
                res[r] = 1
                st[r] = frame
            assert not evs
            assert np.array_equal(res, c.resident)


def test_layout_only_volume_selects_like_the_volume_with_data():
    """Volume.layout (geometry without voxels) gives the same level offsets,
    blocks and selection as the volume built from data, given the same block
    ranges and residency; it refuses to select without ranges."""
    import pytest
    import synth
    a = synth.filaments_u16((77, 50, 39), seed=11, ntubes=6)  # ragged on every axis
    model = synth.volume_model(77, 0.5)
    full = oracle.Volume([oracle.pyramid(a, 4)], 8, model=model)
    bare = oracle.Volume.layout((77, 50, 39), 8, 4, model=model, dtype=np.uint16)
    assert bare.node_count == full.node_count and list(bare.level_offsets) == list(full.level_offsets)
    for L in range(4):
        assert bare.blocks_per_axis(L) == full.blocks_per_axis(L)
    ranges = full.block_ranges()
    tf = oracle.make_tf(synth.tf_piecewise(2002, zero_alpha_points=2), 300.0, 60000.0)
    rng = np.random.default_rng(3)
    resident = (rng.random(full.node_count) < 0.7).astype(np.uint8)
    resident[full.level_offsets[3]:] = 1
    (views, projs), = synth.head_poses(1, seed=3101, extent_m=0.5, width=96, height=80)
    for res in (None, resident):
        r1 = full.select([tf], views, projs, 80, tau=0.5, resident=res, ranges=ranges)
        r2 = bare.select([tf], views, projs, 80, tau=0.5, resident=res, ranges=ranges)
        for k in ("leaf", "state", "requests", "used"):
            assert np.array_equal(r1[k], r2[k]), k
        assert r1["selected"] == r2["selected"]
    with pytest.raises(ValueError):
        bare.select([tf], views, projs, 80)
