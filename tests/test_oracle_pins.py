"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these re-types the oracle's own formulas: each checks a published
known answer, a closed form, an invariant, a special case or a brute-force
count, so that a dropped term, a wrong sign or index, or a transposed operand
in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_02226_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Philox4x32-10: published known answers
# ---------------------------------------------------------------------------
def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    assert list(O.philox(ctr, key)) == expect


def test_philox_words_uniform():
    # 4 * 20000 words: mean and the top-bit frequency within 5 sigma
    words = np.concatenate([O.philox([i, 7, 3, 0], [11, 13]) for i in range(20000)])
    u = words.astype(np.float64) / 2.0**32
    n = u.size
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / n)
    top = (words >> 31).mean()
    assert abs(top - 0.5) < 5 * math.sqrt(0.25 / n)


# ---------------------------------------------------------------------------
# thresholds and map choice
# ---------------------------------------------------------------------------
def test_dyadic_thresholds_are_exact():
    assert list(O.thresholds([0.25] * 4)) == [1 << 30, 1 << 31, 3 << 30]
    assert list(O.thresholds([1, 1])) == [1 << 31]
    assert list(O.thresholds([1, 3])) == [1 << 30]
    assert list(O.thresholds([5])) == []


def test_choice_boundaries():
    T = O.thresholds([0.25] * 4)
    assert O.choose(0, T, 4) == 0
    assert O.choose((1 << 30) - 1, T, 4) == 0
    assert O.choose(1 << 30, T, 4) == 1        # tie goes to the next map
    assert O.choose((3 << 30) - 1, T, 4) == 2
    assert O.choose(0xFFFFFFFF, T, 4) == 3


def test_zero_probability_maps_never_chosen():
    T = O.thresholds([0.5, 0.0, 0.5, 0.0])
    for w in [0, (1 << 31) - 1, 1 << 31, 0xFFFFFFFF, 0xFFFFFFFE]:
        assert O.choose(w, T, 4) in (0, 2)
    assert O.choose(0xFFFFFFFF, T, 4) == 2


def test_invalid_probabilities_rejected():
    for bad in ([0.0, 0.0], [-1.0, 2.0], [float("nan"), 1.0], [float("inf"), 1.0]):
        with pytest.raises(ValueError):
            O.thresholds(bad)


def test_choice_frequencies_match_probabilities():
    probs = np.array([0.1, 0.35, 0.05, 0.2, 0.3])
    sys = W.System(2, [W.Map("affine", (0.5, 0, 0, 0.5, 0, 0))] * 5, list(probs))
    n_pts, steps = 200, 400
    k, _, _ = O.trace(sys, [W.Op("splat", (0,))], np.arange(n_pts), iters=steps)
    counts = np.bincount(k.ravel(), minlength=5)
    n = k.size
    for j in range(5):
        sd = math.sqrt(n * probs[j] * (1 - probs[j]))
        assert abs(counts[j] - n * probs[j]) < 5 * sd


# ---------------------------------------------------------------------------
# square primitive (Section 1): exact total, uniform fill, quadrant colours
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def square_full():
    wl = W.square_render()
    job = wl.jobs[0]
    res = O.render(job.system, wl.chain, wl.targets, n_points=job.n_points, iters=wl.iters,
                   burn_in=wl.burn_in, seed=wl.seed)
    return wl, res[0]


def test_square_total_exact(square_full):
    wl, r = square_full
    assert int(r.buf.sum(dtype=np.uint64)) == (1 << 16) * 180 == 11796480
    assert r.n_discard == 0
    assert r.n_splat == 11796480


def test_square_uniform_within_5_sigma(square_full):
    _, r = square_full
    tot = r.buf.sum(axis=0).astype(np.float64)
    mean = 11796480 / 512**2
    sd = math.sqrt(11796480 * (1 / 512**2) * (1 - 1 / 512**2))
    assert abs(mean - 45.0) < 1e-12
    assert np.all(np.abs(tot - mean) < 5 * sd), (tot.min(), tot.max())


def test_square_channel_quadrants(square_full):
    # map k = 2 [y >= 1/2] + [x >= 1/2] moves the point into quadrant k, so
    # channel k (last map applied) is confined to quadrant k.  The only FP32
    # exception: a coordinate rounded to exactly 1.0 and then halved lands on
    # 0.5, i.e. in column / row 256 of the neighbouring quadrant.
    _, r = square_full
    h = r.buf
    for k in range(4):
        qx, qy = k & 1, k >> 1
        mask = np.ones((512, 512), dtype=bool)
        mask[qy * 256:(qy + 1) * 256, qx * 256:(qx + 1) * 256] = False
        if qx == 0:
            mask[:, 256] = False
        if qy == 0:
            mask[256, :] = False
        assert h[k][mask].sum() == 0
        inside = h[k][qy * 256:(qy + 1) * 256, qx * 256:(qx + 1) * 256]
        assert inside.sum() > 0.24 * 11796480


def test_square_bins_follow_choice_bits():
    # With exact halvings the bin after step n >= 9 is fixed by the last nine
    # choices: ix = sum_j bx(k_{n-j}) 2^(8-j), iy likewise (brute force over
    # the recorded choice sequence).
    sys = W.square_system()
    ids = np.arange(64)
    k, p, _ = O.trace(sys, [W.Op("splat", (0,))], ids, iters=40)
    bx, by = (k & 1), (k >> 1)
    for n in range(9, 40):
        ix = sum(bx[:, n - j] << (8 - j) for j in range(9))
        iy = sum(by[:, n - j] << (8 - j) for j in range(9))
        gx = np.minimum(np.floor(p[:, n, 0] * 512).astype(int), 511)
        gy = np.minimum(np.floor(p[:, n, 1] * 512).astype(int), 511)
        ok = (p[:, n - 9, 0] < 1.0) & (p[:, n - 9, 1] < 1.0)
        assert np.all(gx[ok] == ix[ok]) and np.all(gy[ok] == iy[ok])


# ---------------------------------------------------------------------------
# Sierpinski triangle: box-counting dimension and exact box set
# ---------------------------------------------------------------------------
def _render_hist(sys, n_points, iters, W_=512, burn_in=20, view=(0.0, 1.0, 0.0, 1.0)):
    t = W.Target("hist_u32", W_, W_, 1, view)
    r = O.render(sys, [W.Op("splat", (0,))], [t], n_points=n_points, iters=iters,
                 burn_in=burn_in)
    return r[0].buf[0], r[0]


def test_sierpinski_box_dimension():
    h, _ = _render_hist(W.sierpinski_system(), 1 << 14, 200)
    occ = h > 0
    levels, counts = [], []
    # box sizes 2^-5 .. 2^-9: at coarser sizes the count is dominated by the
    # square grid cutting the triangle's outline (local slopes 1.66, 1.63)
    for lvl in range(5, 10):
        f = 512 >> lvl
        boxes = occ.reshape(1 << lvl, f, 1 << lvl, f).any(axis=(1, 3))
        levels.append(lvl)
        counts.append(boxes.sum())
    slope = np.polyfit(np.array(levels) * math.log(2), np.log(counts), 1)[0]
    assert abs(slope - math.log(3) / math.log(2)) < 0.02, slope


def test_right_angle_sierpinski_occupies_exactly_the_3k_boxes():
    # vertices (0,0), (1,0), (0,1): the attractor is the set of points whose
    # binary digits of x and y are never both 1, i.e. boxes (i, j) with
    # i & j == 0 at every dyadic level; there are 3^k of them.
    h, _ = _render_hist(W.sierpinski_system(right_angle=True), 1 << 14, 200)
    for lvl in range(1, 10):
        f = 512 >> lvl
        occ = (h.reshape(1 << lvl, f, 1 << lvl, f).sum(axis=(1, 3)) > 0)
        jj, ii = np.meshgrid(np.arange(1 << lvl), np.arange(1 << lvl), indexing="ij")
        on = (ii & jj) == 0
        assert on.sum() == 3**lvl
        assert occ[on].all()                       # every attractor box is reached
        assert occ[~on].sum() <= 2 ** (lvl + 1)    # only boundary boxes beyond


# ---------------------------------------------------------------------------
# fixed points of contractions
# ---------------------------------------------------------------------------
def test_affine_fixed_point_closed_form():
    c, s = math.cos(1.1), math.sin(1.1)
    A = 0.6 * np.array([[c, -s], [s, c]])
    b = np.array([0.3, -0.2])
    sys = W.single_affine_system(A[0, 0], A[0, 1], A[1, 0], A[1, 1], b[0], b[1])
    _, p, _ = O.trace(sys, [W.Op("splat", (0,))], np.arange(8), iters=60)
    Af = np.array(sys.maps[0].params[:4], dtype=np.float64).reshape(2, 2)
    bf = np.array(sys.maps[0].params[4:6], dtype=np.float64)
    pstar = np.linalg.solve(np.eye(2) - Af, bf)
    err = np.abs(p[:, -1, :2] - pstar).max()
    assert err < 0.6**60 * 2 + 1e-6
    # and the point is not trivially there after one step
    assert np.abs(p[:, 0, :2] - pstar).max() > 1e-3


@pytest.mark.parametrize("k", range(4))
def test_square_single_map_converges_to_corner(k):
    sys = W.square_system()
    probs = [0.0] * 4
    probs[k] = 1.0
    sys.probs = probs
    kk, p, _ = O.trace(sys, [W.Op("splat", (0,))], np.arange(16), iters=40)
    assert np.all(kk == k)
    corner = np.array([k & 1, k >> 1], dtype=np.float64)
    assert np.abs(p[:, -1, :2] - corner).max() < 1e-6


# ---------------------------------------------------------------------------
# totals: splats + discards = points x (iters - burn_in), every target
# ---------------------------------------------------------------------------
def test_totals_invariant_composed_small():
    wl = W.composed_render(n_points=2048, iters=60, W=128)
    wl.targets[1].view = (-0.4, 0.4, -0.4, 0.4)       # crop the torus: discards
    bufs = [O.alloc_target_buffer(t) for t in wl.targets]
    n_sp = [0, 0]
    n_dc = [0, 0]
    for job in wl.jobs:
        res = O.render(job.system, wl.chain, wl.targets, n_points=job.n_points,
                       point_begin=job.point_begin, iters=wl.iters, burn_in=wl.burn_in,
                       seed=wl.seed, bufs=bufs)
        for j, r in enumerate(res):
            n_sp[j] += r.n_splat
            n_dc[j] += r.n_discard
    expect = 2048 * (60 - 20)
    for j in range(2):
        assert n_sp[j] + n_dc[j] == expect
    # RGBA alpha channel counts the splats exactly (alpha 1 each)
    assert int(bufs[0][..., 3].sum()) == n_sp[0]
    assert n_dc[0] == 0                 # the sinusoidal output lies in [-1, 1]^2
    assert 0 < n_dc[1] < expect         # the cropped view discards part of the torus
    # every depth key holds a depth within the camera's range
    d = bufs[1][bufs[1] != np.uint64(0xFFFFFFFFFFFFFFFF)]
    z = (d >> np.uint64(32)).astype(np.uint32).view(np.float32)
    assert np.all((z > 3.5 - 1.36) & (z < 3.5 + 1.36))


# ---------------------------------------------------------------------------
# transforms: closed-form identities
# ---------------------------------------------------------------------------
_ID = W.single_affine_system(1, 0, 0, 1, 0, 0)


def _apply(chain, pts):
    """q at the first SPLAT op for explicit 2D start points (identity generator)."""
    pts = np.asarray(pts, dtype=np.float32)
    _, _, q = O.trace(_ID, chain + [W.Op("splat", (0,))], np.arange(len(pts)), iters=1,
                      start=pts)
    return q[:, 0, 0, :]


def _apply3(chain, pts):
    sys3 = W.System(3, [W.Map("affine", (1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0))], [1.0])
    pts = np.asarray(pts, dtype=np.float32)
    _, _, q = O.trace(sys3, chain + [W.Op("splat", (0,))], np.arange(len(pts)), iters=1,
                      start=pts)
    return q[:, 0, 0, :]


def test_identity_generator_keeps_points():
    pts = W.uniform_points(50, 2, 1) * 4 - 2
    q = _apply([], pts)
    assert np.array_equal(q[:, :2], pts)


def test_rotation_preserves_norm_and_angle():
    pts = W.uniform_points(200, 2, 2) * 2 - 1
    q = _apply([W.Op("rotate2", (0.7,))], pts)
    assert np.allclose(np.hypot(q[:, 0], q[:, 1]), np.hypot(pts[:, 0], pts[:, 1]), atol=1e-6)
    a0 = np.arctan2(pts[:, 1], pts[:, 0])
    a1 = np.arctan2(q[:, 1], q[:, 0])
    d = np.angle(np.exp(1j * (a1 - a0)))
    assert np.allclose(d, 0.7, atol=1e-5)


def test_rotate3_about_x():
    pts = W.uniform_points(100, 3, 3) * 2 - 1
    q = _apply3([W.Op("rotate3", (1.0, 0.0))], pts)
    assert np.allclose(q[:, 0], pts[:, 0], atol=0)
    c, s = math.cos(1.0), math.sin(1.0)
    assert np.allclose(q[:, 1], c * pts[:, 1] - s * pts[:, 2], atol=1e-6)
    assert np.allclose(q[:, 2], s * pts[:, 1] + c * pts[:, 2], atol=1e-6)


def test_swirl_fixes_origin_and_preserves_radius():
    q = _apply([W.Op("swirl")], [[0.0, 0.0]])
    assert q[0, 0] == 0 and q[0, 1] == 0
    pts = W.uniform_points(200, 2, 4) * 2 - 1
    q = _apply([W.Op("swirl")], pts)
    assert np.allclose(np.hypot(q[:, 0], q[:, 1]), np.hypot(pts[:, 0], pts[:, 1]), atol=1e-6)
    # swirl is a rotation by pi/2 - r^2: with z = x + iy, z' = z exp(i(pi/2 - r^2))
    r2 = (pts.astype(np.float64) ** 2).sum(1)
    d = np.angle(np.exp(1j * (np.arctan2(q[:, 1], q[:, 0]) - np.arctan2(pts[:, 1], pts[:, 0])
                              - (math.pi / 2 - r2))))
    assert np.abs(d).max() < 1e-5


def test_sinusoidal_is_odd_and_bounded():
    pts = (W.uniform_points(100, 2, 5) * 8 - 4)
    q1 = _apply([W.Op("sinusoidal")], pts)
    q2 = _apply([W.Op("sinusoidal")], -pts)
    assert np.array_equal(q1[:, :2], -q2[:, :2])
    assert np.all(np.abs(q1[:, :2]) <= 1.0)
    q = _apply([W.Op("sinusoidal")], [[math.pi / 2, 0.0]])
    assert abs(q[0, 0] - 1.0) < 1e-7 and q[0, 1] == 0.0


def test_stretch_eq2_special_values():
    # Eq. 2: x2 = 2x, y2 = y - cos(x)
    q = _apply([W.Op("stretch")], [[0.0, 0.25], [math.pi / 2, 0.5], [math.pi, 0.0]])
    assert q[0, 0] == 0.0 and abs(q[0, 1] - (-0.75)) < 1e-7
    assert abs(q[1, 0] - math.pi) < 1e-6 and abs(q[1, 1] - 0.5) < 1e-6
    assert abs(q[2, 0] - 2 * math.pi) < 1e-6 and abs(q[2, 1] - 1.0) < 1e-6


def test_torus_implicit_equation():
    uv = W.uniform_points(500, 2, 6)
    q = _apply([W.Op("torus", (1.0, 0.35))], uv)
    rho = np.hypot(q[:, 0], q[:, 1]).astype(np.float64)
    resid = (rho - 1.0) ** 2 + q[:, 2].astype(np.float64) ** 2 - 0.35**2
    assert np.abs(resid).max() < 1e-5
    # u = 0 lies in the x-z plane at x >= R - r
    q0 = _apply([W.Op("torus", (1.0, 0.35))], [[0.0, 0.0], [0.0, 0.5]])
    assert abs(q0[0, 0] - 1.35) < 1e-6 and abs(q0[1, 0] - 0.65) < 1e-6


def test_inversion_is_an_involution():
    pts = W.uniform_points(200, 3, 7) * 4 - 2
    inv = W.Op("inversion", (0.0, 0.0, 6.0, 4.0))
    q = _apply3([inv, inv], pts)
    assert np.abs(q[:, :3] - pts).max() < 1e-5
    # points on the sphere are fixed
    on = np.array([[0.0, 0.0, 2.0], [4.0, 0.0, 6.0]], dtype=np.float32)
    q1 = _apply3([inv], on)
    assert np.abs(q1[:, :3] - on).max() < 1e-6


def test_perspective_and_near_plane():
    pts = np.array([[1.0, -0.5, 2.0], [0.3, 0.2, 0.0], [0.3, 0.2, -1.0]], dtype=np.float32)
    q = _apply3([W.Op("perspective", (2.0, 1e-3))], pts)
    assert abs(q[0, 0] - 1.0) < 1e-7 and abs(q[0, 1] + 0.5) < 1e-7 and q[0, 2] == 2.0
    assert q[0, 3] == 1.0 and q[1, 3] == 0.0 and q[2, 3] == 0.0   # behind camera: discard


def test_twist_and_bend_reduce_to_identity():
    pts = W.uniform_points(50, 3, 8) * 2 - 1
    q = _apply3([W.Op("twist_z", (0.0,))], pts)
    assert np.array_equal(q[:, :3], pts)
    # twist rotates by kappa z in the xy-plane, keeping |xy| and z
    q = _apply3([W.Op("twist_z", (1.3,))], pts)
    assert np.allclose(np.hypot(q[:, 0], q[:, 1]), np.hypot(pts[:, 0], pts[:, 1]), atol=1e-6)
    assert np.array_equal(q[:, 2], pts[:, 2])
    # bend leaves the axis x = z = 0 in place
    ax = np.array([[0.0, 0.3, 0.0], [0.0, -0.7, 0.0]], dtype=np.float32)
    q = _apply3([W.Op("bend", (0.5,))], ax)
    assert np.array_equal(q[:, :3], ax)
    # and turns the point about the axis through (0, *, 1/b) by the angle b x
    b = 0.5
    q = _apply3([W.Op("bend", (b,))], pts)
    ang = np.arctan2(q[:, 0], 1 / b - q[:, 2])
    assert np.allclose(ang, b * pts[:, 0], atol=1e-5)
    # bend keeps the distance to the bend axis: |(x', z' - 1/b)| = |1/b - z|
    b = 0.5
    q = _apply3([W.Op("bend", (b,))], pts)
    lhs = np.hypot(q[:, 0], q[:, 2] - 1 / b)
    assert np.allclose(lhs, np.abs(1 / b - pts[:, 2]), atol=1e-5)


# ---------------------------------------------------------------------------
# composition semantics (Fig. 2): copy keeps the generator trajectory
# ---------------------------------------------------------------------------
def test_copy_semantics_keeps_generator_trajectory():
    sys = W.square_system()
    ids = np.arange(32)
    k1, p1, _ = O.trace(sys, [W.Op("splat", (0,))], ids, iters=50)
    k2, p2, _ = O.trace(sys, [W.Op("stretch"), W.Op("swirl"), W.Op("splat", (0,))], ids, iters=50)
    assert np.array_equal(k1, k2) and np.array_equal(p1, p2)


def test_reuse_semantics_changes_trajectory():
    sys = W.circle_system()
    chain = [W.Op("stretch"), W.Op("splat", (0,))]
    ids = np.arange(16)
    _, pc, _ = O.trace(sys, chain, ids, iters=10)
    _, pr, _ = O.trace(sys, chain, ids, iters=10, reuse=True)
    assert not np.allclose(pc, pr)
    t = W.Target("hist_u32", 64, 64, 2, (-3, 3, -3, 3))
    a = O.render(sys, chain, [t], n_points=256, iters=40, burn_in=20)[0].buf
    b = O.render(sys, chain, [t], n_points=256, iters=40, burn_in=20, reuse=True)[0].buf
    assert not np.array_equal(a, b)


# ---------------------------------------------------------------------------
# circle IFS (Eq. 1): disk containment and halves by f_id
# ---------------------------------------------------------------------------
def test_circle_ifs_disk_and_halves():
    k, p, _ = O.trace(W.circle_system(), [W.Op("splat", (0,))], np.arange(256), iters=60)
    r = np.hypot(p[..., 0], p[..., 1])
    assert r.max() <= 1.0 + 1e-6
    # once the input lies in the disk (every step after the first, since the
    # start is uniform in the unit square), map 0 lands in the upper half and
    # map 1 in the lower half
    up = p[:, 1:, 1][k[:, 1:] == 0]
    lo = p[:, 1:, 1][k[:, 1:] == 1]
    assert up.min() >= -1e-6 and lo.max() <= 1e-6
    # the angle after a step is pi * (|p_prev| + f_id)
    rp = np.hypot(p[:, :-1, 0], p[:, :-1, 1])
    ang = np.mod(np.arctan2(p[:, 1:, 1], p[:, 1:, 0]), 2 * np.pi)
    expect = np.pi * (rp + k[:, 1:])
    good = r[:, 1:] > 1e-3
    d = np.angle(np.exp(1j * (ang - expect)))[good]
    assert np.abs(d).max() < 1e-4


# ---------------------------------------------------------------------------
# splat rule and targets
# ---------------------------------------------------------------------------
def _splat_points(pts, target, fn=None):
    pts = np.asarray(pts, dtype=np.float32)
    if pts.shape[1] == 2:
        pts = np.concatenate([pts, np.zeros((len(pts), 1), np.float32)], 1)
    fn = np.zeros(len(pts), np.uint8) if fn is None else np.asarray(fn, np.uint8)
    return O.render_points(pts, fn, [W.Op("splat", (0,))], [target])[0]


def test_bin_rule_half_open_last_closed():
    t = W.Target("hist_u32", 4, 4, 1, (0.0, 1.0, 0.0, 1.0))
    r = _splat_points([[0.0, 0.0], [0.25, 0.0], [0.2499999, 0.0], [1.0, 1.0],
                       [1.0000001, 0.5], [-1e-9, 0.5], [float("nan"), 0.5]], t)
    h = r.buf[0]
    assert h[0, 0] == 2          # 0.0 and 0.2499999 share bin 0
    assert h[0, 1] == 1          # 0.25 opens bin 1 (half-open bins)
    assert h[3, 3] == 1          # x = x1, y = y1: the last bin is closed
    assert h.sum() == 4
    assert r.n_discard == 3 and r.n_splat == 4   # beyond x1, below x0, NaN


def test_depth_min_keeps_nearest_and_colour():
    t = W.Target("depth_u64", 2, 2, 1, (-1.0, 1.0, -1.0, 1.0),
                 palette8=np.array([0x11, 0x22, 0x33], np.uint32))
    pts = [[0.5, 0.5, 3.0], [0.5, 0.5, 2.0], [0.5, 0.5, 2.5], [-0.5, -0.5, 1.0]]
    r = _splat_points(pts, t, fn=[0, 1, 2, 2])
    d = r.buf
    z = lambda v: np.float32(v).view(np.uint32).astype(np.uint64)
    assert d[1, 1] == (z(2.0) << np.uint64(32)) | np.uint64(0x22)
    assert d[0, 0] == (z(1.0) << np.uint64(32)) | np.uint64(0x33)
    assert d[0, 1] == np.uint64(0xFFFFFFFFFFFFFFFF)


def test_rgba_accumulates_palette():
    t = W.Target("rgba_f32", 2, 1, 4, (0.0, 1.0, 0.0, 1.0), palette=W.palette_rgba(16))
    r = _splat_points([[0.1, 0.5]] * 3 + [[0.9, 0.5]] * 2, t, fn=[0, 1, 1, 6, 6])
    pal = W.palette_rgba(16)
    assert np.array_equal(r.buf[0, 0], pal[0] + 2 * pal[1])
    assert np.array_equal(r.buf[0, 1], 2 * pal[6])


def test_histogram_channel_is_map_index_mod_C():
    t = W.Target("hist_u32", 1, 1, 4, (0.0, 1.0, 0.0, 1.0))
    r = _splat_points([[0.5, 0.5]] * 6, t, fn=[0, 1, 5, 6, 7, 3])
    assert list(r.buf[:, 0, 0]) == [1, 2, 1, 2]


def test_render_matches_trace_histogram():
    # the render's histogram equals the one rebuilt from recorded choices and
    # positions (brute force over the trace)
    sys = W.sierpinski_system()
    n, iters, B = 300, 30, 5
    t = W.Target("hist_u32", 32, 32, 3, (0.0, 1.0, 0.0, 1.0))
    h = O.render(sys, [W.Op("splat", (0,))], [t], n_points=n, iters=iters, burn_in=B)[0].buf
    k, p, _ = O.trace(sys, [W.Op("splat", (0,))], np.arange(n), iters=iters)
    ref = np.zeros_like(h)
    for j in range(n):
        for s in range(B, iters):
            ix = min(int(math.floor(p[j, s, 0] * np.float32(32))), 31)
            iy = min(int(math.floor(p[j, s, 1] * np.float32(32))), 31)
            ref[k[j, s] % 3, iy, ix] += 1
    assert np.array_equal(h, ref)


def test_step_window_and_start_override():
    # steps n in [step_begin, iters) with explicit start points continue a
    # trajectory exactly where a full run stands
    sys = W.square_system()
    ids = np.arange(20)
    k, p, _ = O.trace(sys, [W.Op("splat", (0,))], ids, iters=30)
    k2, p2, _ = O.trace(sys, [W.Op("splat", (0,))], ids, iters=30, step_begin=12,
                        start=p[:, 11, :2])
    assert np.array_equal(k2, k[:, 12:]) and np.array_equal(p2, p[:, 12:])


def test_pointcloud_is_trajectory_endpoint():
    sys = W.cloud_system()
    xyz, fn = O.pointcloud_generate(sys, 64, 32)
    k, p, _ = O.trace(sys, [W.Op("splat", (0,))], np.arange(64), iters=32)
    assert np.array_equal(xyz, p[:, -1, :]) and np.array_equal(fn, k[:, -1])
    # the attractor bound |x| <= |b| / (1 - s_max) for s <= 0.55, |b| <= sqrt(3)
    assert np.linalg.norm(xyz, axis=1).max() <= math.sqrt(3) / 0.45


# ---------------------------------------------------------------------------
# density-estimation display (log density, gamma, 8-bit RGBA)
# ---------------------------------------------------------------------------
def _unpack8(v):
    v = int(v)
    return [(v >> (8 * c)) & 0xFF for c in range(4)]


def _rgba_layer(W_, H_):
    return W.Target("rgba_f32", W_, H_, 1, (0.0, 1.0, 0.0, 1.0)), np.zeros((H_, W_, 4), np.float32)


def test_tonemap_closed_forms():
    t, buf = _rgba_layer(4, 2)
    buf[0, 0] = [8.0, 4.0, 0.0, 8.0]       # 8 splats of (1, 0.5, 0, 1): the maximum
    buf[0, 1] = [2.0, 1.0, 0.0, 2.0]       # ln 3 / ln 9 = 1/2
    buf[0, 2] = [0.0, 0.0, 3.0, 3.0]       # blue, ln 4 / ln 9
    out, _, used = O.tonemap(t, buf, gamma=1.0, background=0x11223344)
    assert used == 8.0
    assert _unpack8(out[0, 0]) == [255, 128, 0, 255]
    assert _unpack8(out[0, 1]) == [128, 64, 0, 128]
    v = math.log(4) / math.log(9)
    assert _unpack8(out[0, 2]) == [0, 0, round(255 * v), round(255 * v)]
    assert all(int(x) == 0x11223344 for x in out[1])           # empty pixels
    out2, _, _ = O.tonemap(t, buf, gamma=2.0)
    s = math.sqrt(0.5)
    assert _unpack8(out2[0, 1]) == [round(255 * s), round(127.5 * s), 0, round(255 * s)]
    # brightness saturates; an explicit maximum replaces the layer's own
    out3, _, _ = O.tonemap(t, buf, gamma=1.0, brightness=2.0)
    assert _unpack8(out3[0, 0]) == [255, 255, 0, 255]
    out4, _, used4 = O.tonemap(t, buf, gamma=1.0, a_max=2.0)
    assert used4 == 2.0 and _unpack8(out4[0, 1]) == [255, 128, 0, 255]


def test_tonemap_alpha_monotone_in_density():
    t, buf = _rgba_layer(64, 1)
    a = np.arange(64, dtype=np.float32) * 17
    buf[0, :, 3] = a
    buf[0, :, 0] = a
    out, _, _ = O.tonemap(t, buf, gamma=2.2)
    alpha = [(int(v) >> 24) & 0xFF for v in out[0]]
    red = [int(v) & 0xFF for v in out[0]]
    assert alpha[0] == 0 and alpha[-1] == 255
    assert all(x <= y for x, y in zip(alpha, alpha[1:]))
    assert red == alpha                    # pure red: the colour equals the density


def test_tonemap_histogram_equals_rgba_sums():
    # a C-channel histogram displays as the RGBA layer of its palette sums
    rng = np.random.default_rng(11)
    pal = W.palette_rgba(4)
    ht = W.Target("hist_u32", 16, 8, 4, (0.0, 1.0, 0.0, 1.0), palette=pal)
    h = rng.integers(0, 50, size=(4, 8, 16)).astype(np.uint32)
    h[:, 0, 0] = 0
    t, rgba = _rgba_layer(16, 8)
    p = np.asarray(pal, np.float64)[:4]
    rgba[:] = np.einsum("chw,ck->hwk", h.astype(np.float64), p).astype(np.float32)
    o1, _, m1 = O.tonemap(ht, h, gamma=2.2, background=7)
    o2, _, m2 = O.tonemap(t, rgba, gamma=2.2, background=7)
    assert m1 == m2 == float(h.sum(axis=0).max())
    assert np.array_equal(o1, o2) and o1[0, 0] == 7


def test_tonemap_depth_resolves_colour():
    t = W.Target("depth_u64", 3, 1, 1, (0.0, 1.0, 0.0, 1.0))
    keys = np.array([[(np.uint64(0x3F800000) << np.uint64(32)) | np.uint64(0xFF00FF00),
                      np.uint64(0xFFFFFFFFFFFFFFFF),
                      (np.uint64(0x40000000) << np.uint64(32)) | np.uint64(0x01020304)]],
                    dtype=np.uint64)
    out, _, _ = O.tonemap(t, keys, background=0xDEADBEEF)
    assert [int(v) for v in out[0]] == [0xFF00FF00, 0xDEADBEEF, 0x01020304]


# ---------------------------------------------------------------------------
# duplication (stars), hemisphere and band recolouring (Section 3.2's scene)
# ---------------------------------------------------------------------------
def _circle_trace(chain, n=64, iters=40, seed=5):
    sysd = W.circle_system()
    k, p, q = O.trace(sysd, chain, np.arange(n, dtype=np.uint32), iters=iters, seed=seed)
    return k, p, q


def test_stars_are_scaled_copies_at_fixed_centres():
    box = (-10.0, 10.0, -6.0, 6.0, 12.0, 20.0)
    s0, s1, n = 0.05, 0.1, 5
    chain = [W.Op("stars", (float(n),) + box + (s0, s1)), W.Op("splat", (0,))]
    k, p, q = _circle_trace(chain, n=400, iters=24)
    pts = q[:, 4:, 0, :3].reshape(-1, 3).astype(np.float64)      # after the first steps
    # 2D input: a star's points share one z, which identifies the star
    zs = np.unique(pts[:, 2])
    assert len(zs) == n                        # every star is hit, no others
    counts = []
    for z in zs:
        g = pts[pts[:, 2] == z]
        counts.append(len(g))
        c = g[:, :2].mean(axis=0)              # the disk attractor's mean is ~0
        r = np.linalg.norm(g[:, :2] - c, axis=1).max()
        assert box[0] <= c[0] <= box[1] and box[2] <= c[1] <= box[3] and box[4] <= z <= box[5]
        assert 0.8 * s0 <= r <= 1.05 * s1      # a disk of radius s in [s0, s1]
    m = len(pts) / n
    assert all(abs(c - m) < 5 * np.sqrt(m) for c in counts)     # uniform star choice


def test_hemisphere_lies_on_the_sphere():
    chain = [W.Op("hemisphere", (2.0,)), W.Op("splat", (0,))]
    k, p, q = _circle_trace(chain)
    pts = q[:, :, 0, :3].reshape(-1, 3).astype(np.float64)
    src = p.reshape(-1, 3).astype(np.float64)
    inside = np.hypot(src[:, 0], src[:, 1]) <= 1.0
    r = np.linalg.norm(pts[inside], axis=1)
    assert np.all(np.abs(r - 2.0) < 2e-5 * 2.0)
    assert np.all(pts[:, 2] <= 0.0)
    assert np.allclose(pts[:, :2], 2.0 * src[:, :2], rtol=0, atol=1e-6)


def test_bands_recolour_by_coordinate_and_reset_restores():
    t = W.Target("hist_u32", 64, 64, 2, (0.0, 1.0, 0.0, 1.0))
    chain = [W.Op("bands", (0.0, 4.0, 0.0, 2.0, 0.0)), W.Op("splat", (0,))]
    res = O.render(W.square_system(), chain, [t], n_points=4096, iters=40, burn_in=8, seed=3)
    h = res[0].buf
    cols = np.arange(64)
    band = (cols * 4) // 64 % 2                # floor(4 x) mod 2 of each column
    for c in range(2):
        assert h[c][:, band != c].sum() == 0 and h[c][:, band == c].sum() > 0
    # a new branch starts from the generator's colour again (k mod 2)
    chain2 = [W.Op("bands", (0.0, 0.0, 0.0, 1.0, 3.0)), W.Op("reset"), W.Op("splat", (0,))]
    t4 = W.Target("hist_u32", 2, 2, 4, (0.0, 1.0, 0.0, 1.0))
    res2 = O.render(W.square_system(), chain2, [t4], n_points=512, iters=30, burn_in=8, seed=3)
    h2 = res2[0].buf
    for c in range(4):                          # channel k holds quadrant k only
        assert h2[c].sum() == h2[c][c // 2, c % 2]
