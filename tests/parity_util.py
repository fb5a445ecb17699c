"""Shared helpers of the GPU parity tests: run one case through the C ABI
(libsg.so) and through the FP64 oracle on the same seeded inputs, then compare.

Image bar (tolerance 1e-3 per RGBA channel). For a pixel whose ray has no
ambiguous lattice point, the GPU value must lie within [min(early, late) -
1e-3, max(early, late) + 1e-3] per channel, where early/late are the
oracle's results with the termination threshold moved by -/+1e-4 (equal
unless a sample lands within 1e-4 of the threshold), and its sample count
within [count_early, count_late]. A pixel whose ray has lattice points within
1e-3 voxel of a face between differently sampled cells, or of where the ray
ends, may legitimately take them either way: the oracle enumerates every
such assignment, and the GPU pixel must match one of them on all four
channels and on the count. Pixels the oracle cannot resolve (an eye on a
volume face, more assignments than the enumeration's cap) are counted and
must not occur. Selections must match bit for bit."""
import numpy as np

import oracle

TOL = 1e-3


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


class GpuCase:
    """A volume on the GPU through the C ABI plus its oracle twin."""

    def __init__(self, level0_channels, brick, levels, model=None, timepoints_data=None):
        import torch
        from paper_1804_08197_b300 import sg
        self.sg = sg
        self.torch = torch
        a0 = level0_channels[0]
        self.dtype = sg.SG_U8 if a0.dtype == np.uint8 else sg.SG_U16
        dims = (a0.shape[2], a0.shape[1], a0.shape[0])
        self.dims = dims
        self.brick = brick
        self.levels = levels
        self.model = model
        self.vol = sg.sg_volume_create(dims, self.dtype, brick, levels, channels=len(level0_channels), model=model)
        for c, a in enumerate(level0_channels):
            d = torch.from_numpy(np.ascontiguousarray(a).view(np.int16 if a.dtype == np.uint16 else np.uint8)).cuda()
            sg.sg_upload_volume_device(self.vol, 0, c, d.data_ptr())
            torch.cuda.synchronize()
            del d
        self.ovol = oracle.Volume([oracle.pyramid(a, levels) for a in level0_channels], brick, model=model)
        self.ranges = self.ovol.block_ranges()
        nb0 = self.ovol.blocks_per_axis(0)
        self.ncell = nb0[0] * nb0[1] * nb0[2]

    def set_tfs(self, tables, windows, ref_step=0.5):
        self.tables = tables
        self.windows = windows
        for c, (t, (lo, hi)) in enumerate(zip(tables, windows)):
            self.sg.sg_set_transfer_function(self.vol, c, t, lo, hi, ref_step)
        self.otfs = [oracle.make_tf(t, lo, hi, ref_step) for t, (lo, hi) in zip(tables, windows)]

    def select(self, views, projs, W, H, tau=1.0, slot=0):
        sg = self.sg
        pose = sg.make_pose(views, projs, W, H, pixel_error=tau, slot=slot)
        stats = sg.sg_select_lod(self.vol, pose, stats=True)
        cells, state, req = sg.sg_read_selection(self.vol, slot, self.ncell, self.ovol.node_count)
        ref = self.ovol.select(self.otfs, views, projs, H, tau=tau, ranges=self.ranges)
        return pose, stats, (cells, state, req), ref

    def render(self, pose, step=0.5, empty_skip=1, counts=True, term=0.99, mode=0, depth=None):
        """depth: optional pair of (H, W) float32 numpy arrays (world distances)."""
        torch, sg = self.torch, self.sg
        W, H = pose.width, pose.height
        outs = [torch.empty((H, W, 4), dtype=torch.float32, device="cuda") for _ in range(2)]
        cnt = [torch.zeros((H, W), dtype=torch.int32, device="cuda") for _ in range(2)] if counts else None
        dd = None if depth is None else [torch.from_numpy(np.ascontiguousarray(d, np.float32)).cuda() for d in depth]
        prm = sg.render_params(step=step, term_alpha=term, empty_skip=empty_skip, sample_count=cnt, mode=mode,
                               depth=dd)
        sg.sg_render(self.vol, pose, prm, outs)
        torch.cuda.synchronize()
        imgs = [o.cpu().numpy().reshape(-1, 4) for o in outs]
        cs = [c.cpu().numpy().reshape(-1).astype(np.int64) for c in cnt] if counts else None
        return imgs, cs

    def oracle_render(self, leaf, view, proj, W, H, step=0.5, pixels=None, mode=0, depth=None):
        return self.ovol.render(self.otfs, leaf, view, proj, W, H, step=step, pixels=pixels, mode=mode,
                                depth=depth)

    def close(self):
        self.sg.sg_volume_destroy(self.vol)


def compare_selection(gpu, ref):
    cells, state, req = gpu
    assert np.array_equal(cells, ref["leaf"]), f"leaf map differs in {np.count_nonzero(cells != ref['leaf'])} cells"
    assert np.array_equal(state, ref["state"]), f"node states differ in {np.count_nonzero(state != ref['state'])}"
    assert np.array_equal(np.sort(req), ref["requests"])


def compare_image(img, ref, counts=None, tol=TOL, max_unresolved=0):
    """img: (n,4) GPU pixels matching ref's pixel order (ref from
    oracle.Volume.render). Returns dict(max_err, max_err_ambiguous,
    ambiguous, unresolved, n): the largest |gpu - oracle| over unambiguous
    pixels, the largest distance to the best-matching variant over ambiguous
    ones, the fraction of ambiguous pixels and the count of unresolved ones."""
    fl = ref["flags"]
    n = len(img)
    amb = np.zeros(n, bool)
    amb[ref["var_idx"]] = True
    unres = (fl & (oracle.FL_ENTRY | oracle.FL_MANY)) != 0
    for grp in ref["var_groups"]:
        unres[grp["idx"][grp["n"] == 0]] = True
    strict = ~amb & ~unres
    lo = np.minimum(ref["early"], ref["late"]) - tol
    hi = np.maximum(ref["early"], ref["late"]) + tol
    bad = strict[:, None] & ((img < lo) | (img > hi))
    err = np.where(strict[:, None], np.abs(img - ref["late"]), 0.0)
    worst = np.unravel_index(np.argmax(err), err.shape) if n else (0, 0)
    assert not bad.any(), (f"{np.count_nonzero(bad.any(1))} pixels outside tolerance; worst {err.max():.3g} at "
                           f"{worst}: gpu {img[worst[0]]} oracle {ref['late'][worst[0]]} flags {fl[worst[0]]}")
    if counts is not None:
        ok = (counts >= ref["count_early"]) & (counts <= ref["count_late"])
        assert ok[strict].all(), f"{np.count_nonzero(~ok[strict])} sample-count mismatches"
    # ambiguous pixels: some enumerated assignment matches on every channel
    # (and on the count)
    amb_err = 0.0
    for grp in ref["var_groups"]:
        sel = grp["n"] > 0
        idx = grp["idx"][sel]
        if not len(idx):
            continue
        nv = grp["n"][sel]
        ve, vl = grp["early"][sel], grp["late"][sel]
        live = np.arange(ve.shape[1])[None, :] < nv[:, None]
        g = img[idx][:, None, :]
        vlo, vhi = np.minimum(ve, vl) - tol, np.maximum(ve, vl) + tol
        match = ((g >= vlo) & (g <= vhi)).all(axis=2) & live
        if counts is not None:
            c = counts[idx][:, None]
            match &= (c >= grp["count_early"][sel]) & (c <= grp["count_late"][sel])
        dist = np.where(live, np.abs(g - vl).max(axis=2), np.inf)
        amb_err = max(amb_err, float(dist.min(axis=1).max()))
        miss = ~match.any(axis=1)
        if miss.any():
            i = int(np.flatnonzero(miss)[0])
            j = int(np.argmin(dist[i]))
            raise AssertionError(f"{int(miss.sum())} ambiguous pixels match none of their assignments; pixel "
                                 f"{idx[i]}: gpu {img[idx[i]]} (count {None if counts is None else counts[idx[i]]}) "
                                 f"nearest variant {vl[i, j]} of {nv[i]} flags {fl[idx[i]]}")
    nunres = int(unres.sum())
    assert nunres <= max_unresolved, f"{nunres} pixels the oracle cannot resolve (flags {np.unique(fl[unres])})"
    # achieved errors: |gpu - oracle| where the termination decision is not
    # in question (early == late), else the distance to the [early, late]
    # bracket
    tie = (fl & oracle.FL_TERM) != 0
    plain = strict & ~tie
    e_plain = float(np.abs(img - ref["late"])[plain].max()) if plain.any() else 0.0
    d_br = np.maximum(np.minimum(ref["early"], ref["late"]) - img, img - np.maximum(ref["early"], ref["late"]))
    e_tie = float(np.maximum(d_br, 0.0)[strict & tie].max()) if (strict & tie).any() else 0.0
    return dict(max_err=e_plain, max_err_termination_bracket=e_tie, max_err_ambiguous=amb_err,
                ambiguous=float(amb.mean()) if n else 0.0, termination_ties=int(tie.sum()), unresolved=nunres, n=n)
