"""Pins of the oracle's near-edge bookkeeping, the part of the splat rule that
every parity test of a transcendental chain rests on.

A splat may land in another bin on the GPU only if its position, within the
position tolerance, can cross a bin edge.  The oracle records, per target:
  * amb  -- per bin, how many splats could have landed there or next door
            (the slack of the per-bin histogram comparison);
  * n_amb -- how many splats were near an edge (the slack of the discard count);
  * zlo / zhi -- the lowest depth that may land in a pixel / that surely does;
  * klo / zalt -- the lowest key (depth, colour) that may land in a pixel, and
            the lowest depth of a candidate with another or an unsure colour.
These tests place single points by hand (on an edge, inside and outside the
margin, at a corner, on the closed last edge, just outside the view) and
check each record exactly; a brute-force restatement on random points near
edges checks the same records in bulk; and the parity checker built on them
is shown to reject planted disagreements.
"""
import os
import sys

import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_02226_gb300 import workloads as W

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from _parity import (EMPTY, check_depth_close, check_hist_close, merge_tracked,  # noqa: E402
                     oracle_render, split_jobs, _oracle_worker)

M = 0.01          # margin in pixels
SPLAT = [W.Op("splat", (0,))]


def _hist(W_=8, H_=8, view=(0.0, 8.0, 0.0, 8.0), C=1):
    return W.Target("hist_u32", W_, H_, C, view)


def _depth(W_=8, H_=8, view=(0.0, 8.0, 0.0, 8.0)):
    return W.Target("depth_u64", W_, H_, 1, view,
                    palette8=np.arange(1, 17, dtype=np.uint32) * 0x01010101)


def _one(x, y, z=1.0, k=0, target=None, margin=M, prev=None, chain=SPLAT, band_eps=0.0):
    t = target or _hist()
    xyz = np.array([[x, y, z]], dtype=np.float32)
    fn = np.array([k], dtype=np.uint8)
    return O.render_points(xyz, fn, chain, [t], margin_px=margin, track=True, prev=prev,
                           band_eps=band_eps)


def _amb_pixels(r):
    ys, xs = np.nonzero(r[0].amb)
    return sorted(zip(ys.tolist(), xs.tolist())), r[0].amb[r[0].amb > 0].tolist()


# ---------------------------------------------------------------------------
# single points, histogram target (8 x 8 bins of one unit each)
# ---------------------------------------------------------------------------
def test_centre_of_a_bin_is_not_near_an_edge():
    r = _one(2.5, 3.5)
    assert r[0].n_amb == 0 and r[0].n_splat == 1 and r[0].n_discard == 0
    assert int(r[0].amb.sum()) == 0
    assert r[0].buf[0, 3, 2] == 1 and int(r[0].buf.sum()) == 1


@pytest.mark.parametrize("x", [2.0, 2.0 + 0.5 * M, 2.0 - 0.5 * M])
def test_on_or_within_the_margin_of_an_inner_edge(x):
    # the point can land in column 1 or column 2 of row 3: one unit of slack
    # on each, one near-edge splat, and the oracle's own splat in its bin
    r = _one(x, 3.5)
    pix, val = _amb_pixels(r)
    assert pix == [(3, 1), (3, 2)] and val == [1, 1]
    assert r[0].n_amb == 1 and r[0].n_splat == 1 and r[0].n_discard == 0
    col = 2 if x >= 2.0 else 1
    assert r[0].buf[0, 3, col] == 1


@pytest.mark.parametrize("x", [2.0 + 2 * M, 2.0 - 2 * M])
def test_outside_the_margin_is_not_near_an_edge(x):
    r = _one(x, 3.5)
    assert r[0].n_amb == 0 and int(r[0].amb.sum()) == 0 and r[0].n_splat == 1


def test_corner_gives_slack_to_four_bins():
    r = _one(2.0, 3.0)
    pix, val = _amb_pixels(r)
    assert pix == [(2, 1), (2, 2), (3, 1), (3, 2)] and val == [1, 1, 1, 1]
    assert r[0].n_amb == 1 and r[0].buf[0, 3, 2] == 1


def test_near_an_edge_along_y_only():
    r = _one(4.5, 6.0 - 0.3 * M)
    pix, val = _amb_pixels(r)
    assert pix == [(5, 4), (6, 4)] and val == [1, 1]
    assert r[0].buf[0, 5, 4] == 1


def test_closed_last_edge():
    # x == x1 lands in the last (closed) bin; moved right it would leave the
    # view: slack only on the last bin, and the splat is not discarded
    r = _one(8.0, 0.5)
    pix, val = _amb_pixels(r)
    assert pix == [(0, 7)] and val == [1]
    assert r[0].n_amb == 1 and r[0].n_splat == 1 and r[0].n_discard == 0
    assert r[0].buf[0, 0, 7] == 1


def test_just_outside_the_view_within_the_margin():
    # discarded here, could land in the edge bin elsewhere
    for x, col in ((8.0 + 0.5 * M, 7), (-0.5 * M, 0)):
        r = _one(x, 0.5)
        pix, val = _amb_pixels(r)
        assert pix == [(0, col)] and val == [1]
        assert r[0].n_amb == 1 and r[0].n_splat == 0 and r[0].n_discard == 1
        assert int(r[0].buf.sum()) == 0


def test_outside_the_view_beyond_the_margin_and_nan():
    for x in (8.0 + 2 * M, -2 * M, float("nan")):
        r = _one(x, 0.5)
        assert r[0].n_amb == 0 and r[0].n_discard == 1 and int(r[0].amb.sum()) == 0


def test_no_margin_means_no_bookkeeping():
    r = _one(2.0, 3.0, margin=0.0)
    assert r[0].n_amb == 0 and int(r[0].amb.sum()) == 0 and r[0].n_splat == 1


def test_slack_accumulates_per_splat():
    r = None
    for _ in range(3):
        r = _one(2.0, 3.5, prev=r)
    pix, val = _amb_pixels(r)
    assert pix == [(3, 1), (3, 2)] and val == [3, 3]
    assert r[0].n_amb == 3 and r[0].n_splat == 3


def test_scaled_view_edges_in_pixels():
    # view [-1, 1] over 16 bins: 8 px per unit; x = 0.25 is the edge of bins
    # 9 and 10; 0.25 + 0.4 M / 8 lies 0.4 M px from it
    t = _hist(16, 16, (-1.0, 1.0, -1.0, 1.0))
    r = _one(0.25 + 0.4 * M / 8, 0.03, target=t)
    pix, _ = _amb_pixels(r)
    assert pix == [(8, 9), (8, 10)]
    r = _one(0.25 + 3 * M / 8, 0.03, target=t)
    assert r[0].n_amb == 0


# ---------------------------------------------------------------------------
# depth targets: zlo, zhi, klo, zalt
# ---------------------------------------------------------------------------
def _key(z, col):
    return (int(np.float32(z).view(np.uint32)) << 32) | int(col)


def test_depth_candidates_sure_and_near_edge():
    t = _depth()
    pal = t.palette8
    P = (3, 2)              # row 3, column 2
    # a sure splat at depth 2, colour 0
    r = _one(2.5, 3.5, z=2.0, k=0, target=t)
    assert r[0].zlo[P] == 2.0 and r[0].zhi[P] == 2.0
    assert int(r[0].klo[P]) == _key(2.0, pal[0]) and np.isinf(r[0].zalt[P])
    # a near-edge splat between columns 1 and 2 at depth 1.5, colour 1: it may
    # land in P (lower zlo, zhi unchanged) or in its neighbour; the old lowest
    # (depth 2, colour 0) becomes the lowest depth of another colour
    r = _one(2.0, 3.5, z=1.5, k=1, target=t, prev=r)
    assert r[0].zlo[P] == 1.5 and r[0].zhi[P] == 2.0
    assert int(r[0].klo[P]) == _key(1.5, pal[1]) and r[0].zalt[P] == 2.0
    assert r[0].zlo[3, 1] == 1.5 and np.isinf(r[0].zhi[3, 1])
    # the oracle's own layer: the near-edge splat landed in column 2 (x = 2.0)
    assert int(r[0].buf[P]) == _key(1.5, pal[1])
    # a sure splat at depth 1, colour 1: lowest key again of colour 1, so the
    # lowest depth of another colour stays 2
    r = _one(2.5, 3.5, z=1.0, k=1, target=t, prev=r)
    assert r[0].zlo[P] == 1.0 and r[0].zhi[P] == 1.0
    assert int(r[0].klo[P]) == _key(1.0, pal[1]) and r[0].zalt[P] == 2.0
    # a deeper sure splat of colour 0 lowers zalt, nothing else
    r = _one(2.5, 3.5, z=1.2, k=0, target=t, prev=r)
    assert r[0].zlo[P] == 1.0 and r[0].zhi[P] == 1.0 and r[0].zalt[P] == np.float32(1.2)
    # a deeper splat of the lowest colour changes nothing
    r = _one(2.5, 3.5, z=1.1, k=1, target=t, prev=r)
    assert r[0].zalt[P] == np.float32(1.2) and int(r[0].klo[P]) == _key(1.0, pal[1])
    # equal depth, smaller colour: the key order decides, and the pixel's
    # runner-up of another colour is now at the same depth
    r = _one(2.5, 3.5, z=1.0, k=0, target=t, prev=r)
    assert int(r[0].klo[P]) == _key(1.0, pal[0]) and r[0].zalt[P] == 1.0


def test_depth_near_edge_only_never_sure():
    t = _depth()
    r = _one(4.0, 4.0, z=3.0, k=2, target=t)      # a corner: four pixels
    for P in ((3, 3), (3, 4), (4, 3), (4, 4)):
        assert r[0].zlo[P] == 3.0 and np.isinf(r[0].zhi[P])
        assert int(r[0].klo[P]) == _key(3.0, t.palette8[2])


def test_band_edge_makes_the_colour_unsure():
    # bands on x with frequency 1: x = 2.5 + 1e-6 is 1e-6 from the edge
    # between bands 2 and 3 (phase 0.5); with band_eps 1e-5 the colour is
    # unsure: the lowest candidate counts as a candidate of another colour
    t = _depth(8, 8, (0.0, 8.0, 0.0, 8.0))
    chain = [W.Op("bands", (0.0, 1.0, 0.5, 4.0, 0.0)), W.Op("splat", (0,))]
    r = _one(2.5 + 1e-6, 3.5, z=2.0, target=t, chain=chain, band_eps=1e-5)
    assert r[0].zalt[3, 2] == 2.0 and r[0].zhi[3, 2] == 2.0
    assert r[0].amb[3, 2] == 1 and r[0].n_amb == 0
    r = _one(2.2, 3.5, z=2.0, target=t, chain=chain, band_eps=1e-5)
    assert np.isinf(r[0].zalt[3, 2]) and r[0].amb[3, 2] == 0
    r = _one(2.5 + 1e-6, 3.5, z=2.0, target=t, chain=chain, band_eps=0.0)
    assert np.isinf(r[0].zalt[3, 2])


# ---------------------------------------------------------------------------
# brute force: the same records restated per splat on random points
# ---------------------------------------------------------------------------
def _brute(xyz, fn, t, m):
    """Per-pixel records by the definitions, one splat at a time, in numpy."""
    x0, x1, y0, y1 = (np.float32(v) for v in t.view)
    sx = np.float32(t.W) / (x1 - x0)
    sy = np.float32(t.H) / (y1 - y0)
    amb = np.zeros((t.H, t.W), np.uint32)
    zlo = np.full((t.H, t.W), np.inf, np.float32)
    zhi = np.full((t.H, t.W), np.inf, np.float32)
    cands = [[[] for _ in range(t.W)] for _ in range(t.H)]
    n_amb = 0

    def bin_px(u, n):
        if not (0.0 <= u <= n):
            return -1
        return min(int(np.floor(u)), n - 1)

    for (x, y, z), k in zip(xyz, fn):
        ux = float((np.float32(x) - x0) * sx)
        uy = float((np.float32(y) - y0) * sy)
        bx = {bin_px(ux - m, t.W), bin_px(ux + m, t.W)}
        by = {bin_px(uy - m, t.H), bin_px(uy + m, t.H)}
        near = len(bx) > 1 or len(by) > 1
        n_amb += near
        own = (bin_px(ux, t.W), bin_px(uy, t.H))
        for i in bx:
            for j in by:
                if i < 0 or j < 0:
                    continue
                sure = not near and (i, j) == own
                if near:
                    amb[j, i] += 1
                zlo[j, i] = min(zlo[j, i], z)
                if sure:
                    zhi[j, i] = min(zhi[j, i], z)
                cands[j][i].append((_key(z, t.palette8[k]), z, int(t.palette8[k])))
    klo = np.full((t.H, t.W), EMPTY, np.uint64)
    zalt = np.full((t.H, t.W), np.inf, np.float32)
    for j in range(t.H):
        for i in range(t.W):
            if cands[j][i]:
                best = min(c[0] for c in cands[j][i])
                klo[j, i] = best
                others = [c[1] for c in cands[j][i] if c[2] != (best & 0xFFFFFFFF)]
                if others:
                    zalt[j, i] = min(others)
    return amb, zlo, zhi, klo, zalt, n_amb


def test_records_match_brute_force_on_points_near_edges():
    rng = np.random.default_rng(11)
    t = _depth(12, 10, (-1.0, 2.0, 0.5, 3.0))
    n = 3000
    sx, sy = 12 / 3.0, 10 / 2.5
    # half the points on or near bin edges (and the view's border), half anywhere
    ex = rng.integers(0, 13, n) / sx - 1.0 + rng.normal(0, 0.02 / sx, n)
    ey = rng.integers(0, 11, n) / sy + 0.5 + rng.normal(0, 0.02 / sy, n)
    ax = rng.uniform(-1.1, 2.1, n)
    ay = rng.uniform(0.4, 3.1, n)
    pick = rng.random(n) < 0.5
    xyz = np.stack([np.where(pick, ex, ax), np.where(pick, ey, ay),
                    rng.choice([1.0, 1.5, 2.0, 2.5], n) + rng.integers(0, 2, n) * 1e-3],
                   axis=1).astype(np.float32)
    fn = rng.integers(0, 4, n).astype(np.uint8)
    m = 0.03
    r = O.render_points(xyz, fn, SPLAT, [t], margin_px=m, track=True)[0]
    amb, zlo, zhi, klo, zalt, n_amb = _brute(xyz, fn, t, m)
    assert r.n_amb == n_amb and n_amb > 200
    assert np.array_equal(r.amb, amb)
    assert np.array_equal(r.zlo, zlo) and np.array_equal(r.zhi, zhi)
    assert np.array_equal(r.klo, klo)
    assert np.array_equal(r.zalt, zalt)


# ---------------------------------------------------------------------------
# the checkers built on the records reject planted disagreements
# ---------------------------------------------------------------------------
def _scene_records(seed=5):
    rng = np.random.default_rng(seed)
    t = _depth(16, 16, (0.0, 1.0, 0.0, 1.0))
    n = 4000
    xyz = np.stack([rng.random(n), rng.random(n), rng.uniform(1.0, 3.0, n)],
                   axis=1).astype(np.float32)
    fn = rng.integers(0, 3, n).astype(np.uint8)
    return t, xyz, fn, O.render_points(xyz, fn, SPLAT, [t], margin_px=1e-3, track=True)[0]


def test_depth_checker_accepts_the_oracle_and_rejects_a_wrong_colour():
    t, xyz, fn, r = _scene_records()
    n_dec = check_depth_close(r.buf.copy(), r, min_decided=0.5)
    assert n_dec > 100
    decided = np.isfinite(r.zhi) & (r.zlo == r.zhi) & (r.zalt * (1 - 1e-5) > r.zhi * (1 + 1e-5))
    g = r.buf.copy()
    j = np.flatnonzero(decided.ravel())[7]
    g.ravel()[j] = (g.ravel()[j] & ~np.uint64(0xFFFFFFFF)) | np.uint64(t.palette8[9])
    with pytest.raises(AssertionError):
        check_depth_close(g, r)
    # a depth above the sure splat, and a splat where nothing may land
    g = r.buf.copy()
    g.ravel()[j] = np.uint64(_key(3.5, t.palette8[0]))
    with pytest.raises(AssertionError):
        check_depth_close(g, r)
    g = r.buf.copy()
    empty = np.flatnonzero((r.buf == EMPTY).ravel())
    if empty.size:
        g.ravel()[empty[0]] = np.uint64(_key(1.0, t.palette8[0]))
        with pytest.raises(AssertionError):
            check_depth_close(g, r)


def test_hist_checker_rejects_moves_beyond_the_slack():
    rng = np.random.default_rng(2)
    t = _hist(16, 16, (0.0, 1.0, 0.0, 1.0), C=2)
    n = 5000
    xyz = np.stack([rng.random(n), rng.random(n), np.zeros(n)], axis=1).astype(np.float32)
    fn = rng.integers(0, 2, n).astype(np.uint8)
    r = O.render_points(xyz, fn, SPLAT, [t], margin_px=1e-2, track=True)[0]
    check_hist_close(r.buf, r.buf, r.amb, n)
    g = r.buf.copy()
    free = np.argwhere(r.amb == 0)[0]
    g[0, free[0], free[1]] += 1          # a moved splat where no edge is near
    with pytest.raises(AssertionError):
        check_hist_close(g, r.buf, r.amb, n)


# ---------------------------------------------------------------------------
# records of disjoint point ranges merge into the records of the whole range
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("parts", [2, 3])
def test_merged_records_equal_one_process(parts):
    wl = W.composed_render(n_points=1201, iters=40, W=48)
    m = 0.05
    whole = oracle_render(wl, margin_px=m, track=True)
    merged = merge_tracked([_oracle_worker((wl, c, m, True, 0.0))
                            for c in split_jobs(wl, parts)])
    for a, b in zip(whole, merged):
        assert np.array_equal(a.buf, b.buf)
        assert (a.n_splat, a.n_discard, a.n_amb) == (b.n_splat, b.n_discard, b.n_amb)
        assert np.array_equal(a.amb, b.amb)
        if a.zlo is not None:
            for k in ("zlo", "zhi", "klo", "zalt"):
                assert np.array_equal(getattr(a, k), getattr(b, k)), k
    assert whole[1].n_amb > 0 and np.isfinite(whole[1].zalt).sum() > 100
