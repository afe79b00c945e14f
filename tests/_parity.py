"""Shared helpers of the parity tests: run a workload on the GPU through the
C-ABI binding and on the CPU oracle with the same seeded inputs, and compare
with the tolerances the tests state."""
from __future__ import annotations

import numpy as np

from oracle import oracle as O
from paper_2606_02226_gb300 import workloads as W

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


def gpu_render(wl, jobs=None, stream=None, discards=None, depth_test=None, fast_trig=False,
               fold_linear=False):
    """Renders every job of ``wl`` on the GPU; returns host numpy buffers and
    the per-target discard counts."""
    import torch
    from paper_2606_02226_gb300 import cfs
    tensors = [cfs.alloc_target(t) for t in wl.targets]
    disc = torch.zeros(len(wl.targets), dtype=torch.int64, device="cuda")
    for job in (jobs or wl.jobs):
        sysh = cfs.System(job.system)
        ch = cfs.Chain(wl.chain, job.system.dim, fast_trig=fast_trig, fold_linear=fold_linear)
        cfs.render(sysh, ch, wl.targets, tensors, n_points=job.n_points, iters=wl.iters,
                   burn_in=wl.burn_in, seed=wl.seed, system_id=job.system_id,
                   point_begin=job.point_begin, discards=disc, stream=stream)
    torch.cuda.synchronize()
    return [to_host(t, d) for t, d in zip(tensors, wl.targets)], [int(v) for v in disc.cpu()]


def to_host(t, desc):
    a = t.cpu().numpy()
    if desc.kind == "hist_u32":
        return a.view(np.uint32)
    if desc.kind == "depth_u64":
        return a.view(np.uint64)
    return a


def oracle_render(wl, jobs=None, margin_px=0.0, track=False, band_eps=0.0):
    """The oracle's render of every job of ``wl`` into one set of buffers; with
    ``track`` the near-edge records (margin ``margin_px`` pixels) accumulate
    over the jobs."""
    res = None
    for job in (jobs or wl.jobs):
        res = O.render(job.system, wl.chain, wl.targets, n_points=job.n_points, iters=wl.iters,
                       burn_in=wl.burn_in, seed=wl.seed, system_id=job.system_id,
                       point_begin=job.point_begin, margin_px=margin_px, track=track,
                       prev=res, band_eps=band_eps)
    return res


def fixed_margin(targets, pos_tol):
    """The near-edge margin of the parity bound: the position tolerance in
    pixels of the finest target (the largest pixels-per-unit of any axis).
    A splat may change bins only if its position moves across an edge, and a
    position that meets the tolerance moves by at most pos_tol."""
    scale = max(max(t.W / (t.view[1] - t.view[0]), t.H / (t.view[3] - t.view[2]))
                for t in targets)
    m = pos_tol * scale
    print(f"near-edge margin: {m:.3e} px ({pos_tol:g} in position x {scale:g} px per unit)")
    return m


def depth_of(keys):
    return (keys >> np.uint64(32)).astype(np.uint32).view(np.float32)


def check_hist_close(g, o, amb, total, rel_l1=1e-5):
    """Per bin |gpu - oracle| <= the oracle's near-edge slack of that bin, and
    the summed difference <= rel_l1 of the total."""
    d = np.abs(g.astype(np.int64) - o.astype(np.int64))
    slack = amb if d.ndim == amb.ndim else np.broadcast_to(amb, d.shape)
    bad = d > slack
    assert not bad.any(), f"{bad.sum()} bins differ beyond the near-edge slack"
    assert d.sum() <= rel_l1 * total, (d.sum(), total)


def check_rgba_close(g, o, amb, total, rel_l1=1e-5):
    """Palette components are <= 1, so one moved splat changes a channel by
    at most 1: |gpu - oracle| <= slack per channel; alpha difference summed
    <= rel_l1 of the total."""
    d = np.abs(g.astype(np.float64) - o.astype(np.float64))
    bad = d > amb[..., None]
    assert not bad.any(), f"{bad.sum()} RGBA values differ beyond the near-edge slack"
    print(f"RGBA alpha L1: {d[..., 3].sum():.0f} of {total} splats "
          f"({d[..., 3].sum() / max(total, 1):.2e}; bar {rel_l1:.0e})")
    assert d[..., 3].sum() <= rel_l1 * total, (d[..., 3].sum(), total)


def check_depth_close(g, o, rel=1e-5, min_decided=0.2):
    """Depth layer ``g`` (GPU keys) against the oracle's tracked result ``o``.

    Per pixel the GPU's depth lies between the lowest depth that may land
    there (zlo) and the lowest that surely lands there (zhi), within relative
    ``rel`` (the chain's FP32 differences).  A pixel is decided when its
    lowest candidate is sure (zlo == zhi) and every candidate of another (or
    unsure) colour is deeper by more than the tolerance on both sides
    (zalt (1 - rel) > zhi (1 + rel)): the GPU's winner is then a splat of the
    lowest candidate's colour, so on decided pixels the colours agree
    exactly.  At least ``min_decided`` of the covered pixels must be decided.
    Returns the number of decided pixels."""
    zlo, zhi, klo, zalt = o.zlo, o.zhi, o.klo, o.zalt
    ge = g == EMPTY
    # a GPU-empty pixel must not have a sure splat
    assert not (ge & np.isfinite(zhi)).any(), "GPU left a pixel empty that surely has a splat"
    zg = depth_of(g[~ge]).astype(np.float64)
    lo = zlo[~ge].astype(np.float64)
    hi = zhi[~ge].astype(np.float64)
    assert np.all(np.isfinite(lo)), "GPU splatted where no point can land"
    assert np.all(zg >= lo * (1 - rel)), "GPU depth below every candidate"
    assert np.all(zg <= hi * (1 + rel) + (~np.isfinite(hi)) * 1e30), "GPU depth above a sure splat"
    z_hi = zhi.astype(np.float64)
    decided = (np.isfinite(zhi) & (zlo == zhi) &
               (zalt.astype(np.float64) * (1 - rel) > z_hi * (1 + rel)))
    col = np.uint64(0xFFFFFFFF)
    # the oracle's own layer holds the lowest candidate's colour there
    assert np.array_equal(o.buf[decided] & col, klo[decided] & col)
    bad = decided & ((g & col) != (klo & col))
    assert not bad.any(), f"{int(bad.sum())} decided pixels have another colour"
    n_dec = int(decided.sum())
    covered = int((~ge).sum())
    print(f"depth parity: {n_dec} of {covered} covered pixels decided, colours equal on all")
    assert n_dec >= min_decided * covered, (n_dec, covered)
    return n_dec




def merge_tracked(parts):
    """Combines tracked oracle results of disjoint point ranges (lists of
    TargetResult, one list per part) into the result of the whole range:
    counts and sums add, depth keys and depth bounds take the minimum, and
    the lowest depth of another colour follows from each part's lowest key
    (every candidate of a part is at least as deep as that part's lowest)."""
    out = []
    for j in range(len(parts[0])):
        rs = [p[j] for p in parts]
        r = O.TargetResult(rs[0].buf.copy(), None if rs[0].amb is None else rs[0].amb.copy(),
                           None if rs[0].zlo is None else rs[0].zlo.copy(),
                           None if rs[0].zhi is None else rs[0].zhi.copy(),
                           None if rs[0].klo is None else rs[0].klo.copy(),
                           None if rs[0].zalt is None else rs[0].zalt.copy())
        r.n_splat, r.n_discard, r.n_amb = rs[0].n_splat, rs[0].n_discard, rs[0].n_amb
        for b in rs[1:]:
            if r.buf.dtype == np.uint64:
                np.minimum(r.buf, b.buf, out=r.buf)
            else:
                r.buf += b.buf
            r.n_splat += b.n_splat
            r.n_discard += b.n_discard
            r.n_amb += b.n_amb
            if r.amb is not None:
                r.amb += b.amb
            if r.zlo is not None:
                np.minimum(r.zlo, b.zlo, out=r.zlo)
                np.minimum(r.zhi, b.zhi, out=r.zhi)
                ka, kb = r.klo, b.klo
                col = np.uint64(0xFFFFFFFF)
                same = (ka & col) == (kb & col)
                da = np.where(ka == EMPTY, np.inf, depth_of(ka)).astype(np.float32)
                db = np.where(kb == EMPTY, np.inf, depth_of(kb)).astype(np.float32)
                alt = np.where(same, np.minimum(r.zalt, b.zalt),
                               np.where(ka < kb, np.minimum(r.zalt, db),
                                        np.minimum(b.zalt, da)))
                alt = np.where(kb == EMPTY, r.zalt, np.where(ka == EMPTY, b.zalt, alt))
                r.zalt = alt.astype(np.float32)
                r.klo = np.minimum(ka, kb)
        out.append(r)
    return out


def _oracle_worker(args):
    wl, jobs, margin_px, track, band_eps = args
    res = None
    for job in jobs:
        res = O.render(job.system, wl.chain, wl.targets, n_points=job.n_points, iters=wl.iters,
                       burn_in=wl.burn_in, seed=wl.seed, system_id=job.system_id,
                       point_begin=job.point_begin, margin_px=margin_px, track=track,
                       prev=res, band_eps=band_eps)
    return res


def split_jobs(wl, parts):
    """The workload's jobs cut into `parts` lists of disjoint point ranges."""
    out = [[] for _ in range(parts)]
    for job in wl.jobs:
        per = -(-job.n_points // parts)
        for p in range(parts):
            b = p * per
            n = min(per, job.n_points - b)
            if n > 0:
                out[p].append(W.RenderJob(job.system, job.point_begin + b, n, job.system_id))
    return [o for o in out if o]


def oracle_render_parallel(wl, workers, margin_px=0.0, track=False, band_eps=0.0):
    """The oracle's render of ``wl`` on ``workers`` spawned processes over
    disjoint point ranges, merged (spawn: a forked child of a process that
    holds a GPU context can hang)."""
    import multiprocessing as mp
    chunks = split_jobs(wl, workers)
    with mp.get_context("spawn").Pool(len(chunks)) as pool:
        parts = pool.map(_oracle_worker, [(wl, c, margin_px, track, band_eps) for c in chunks])
    return merge_tracked(parts)


def _points_worker(args):
    xyz, fn, chain, targets, margin_px, track, band_eps = args
    return O.render_points(xyz, fn, chain, targets, margin_px=margin_px, track=track,
                           band_eps=band_eps)


def oracle_render_points_parallel(xyz, fn, chain, targets, workers, margin_px=0.0, track=False,
                                  band_eps=0.0):
    """The oracle's render of stored points (xyz [n][3], fn [n]) on spawned
    processes over disjoint point ranges, merged."""
    import multiprocessing as mp
    n = xyz.shape[0]
    per = -(-n // workers)
    parts = [(xyz[b:b + per], fn[b:b + per], chain, targets, margin_px, track, band_eps)
             for b in range(0, n, per)]
    with mp.get_context("spawn").Pool(len(parts)) as pool:
        res = pool.map(_points_worker, parts)
    return merge_tracked(res)
