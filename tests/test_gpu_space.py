"""GPU parity of the many-objects-from-one-primitive scene (stars by
duplication, a banded hemisphere planet and a torus ring from the circle IFS
of Eq. 1) against the CPU oracle, through the C ABI; and the same ops in a
batch (bit-exact with affine generators)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_02226_gb300 import workloads as W

from _parity import EMPTY, check_depth_close, depth_of, fixed_margin, gpu_render, oracle_render

pytestmark = pytest.mark.gpu

POS_TOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _trace_both(torch, sysd, chain, ids, iters, seed=0):
    from paper_2606_02226_gb300 import cfs
    k, p, q = cfs.trace(cfs.System(sysd), cfs.Chain(chain, sysd.dim),
                        torch.from_numpy(np.asarray(ids, np.uint32).view(np.int32)).cuda(),
                        iters=iters, seed=seed)
    ko, po, qo = O.trace(sysd, chain, ids, iters=iters, seed=seed)
    return (k.cpu().numpy(), p.cpu().numpy(), q.cpu().numpy()), (ko, po, qo)


def _worst(g, o):
    (k, p, q), (ko, po, qo) = g, o
    assert np.array_equal(k, ko), "map-index sequences differ"
    assert np.array_equal(q[..., 3], qo[..., 3]), "alive flags differ"
    alive = qo[..., 3] > 0
    d = np.abs(q[..., :3] - qo[..., :3])[alive]
    return float(d.max()) if d.size else 0.0


def _worst_xy(g, o):
    """Largest screen-coordinate (x, y) difference at the splats."""
    (_, _, q), (_, _, qo) = g, o
    alive = qo[..., 3] > 0
    d = np.abs(q[..., :2] - qo[..., :2])[alive]
    return float(d.max()) if d.size else 0.0


def test_space_trace_parity(torch_cuda):
    # a short horizon: Eq. 1's map separates GPU and host trajectories over
    # many steps (see the circle-scene test below)
    wl = W.space_render(n_points=4096, iters=24)
    ids = np.linspace(0, 4095, 64).astype(np.uint32)
    g, o = _trace_both(torch_cuda, wl.jobs[0].system, wl.chain, ids, wl.iters, seed=wl.seed)
    assert _worst(g, o) <= POS_TOL * 20       # positions up to z = 20: relative 1e-5
    # the star branch lands exactly on the oracle's star (same centre, same z)
    assert np.array_equal(g[2][..., 0, 2], o[2][..., 0, 2])


def _disk_square():
    """Four maps x' = x / 2 + (+-1/2, +-1/2): the uniform square [-1, 1]^2 with
    bit-exact generator positions (dyadic arithmetic)."""
    maps = [W.Map("affine", (0.5, 0.0, 0.0, 0.5, bx, by)) for by in (-0.5, 0.5)
            for bx in (-0.5, 0.5)]
    return W.System(2, maps, [0.25] * 4)


@pytest.mark.parametrize("W_,H_,fold", [(320, 180, False), (257, 131, False), (320, 180, True)])
def test_space_render_parity_small(torch_cuda, W_, H_, fold):
    # the scene's chain on an exact generator: every difference comes from
    # the chain's FP32 transcendentals and is covered by the near-edge slack;
    # fold: the planet's and the ring's rotations and translations run as
    # one affine op each
    wl = W.space_render(n_points=3001, iters=40, W=W_, H=H_)
    wl.jobs[0].system = _disk_square()
    sysd = wl.jobs[0].system
    ids = np.linspace(0, 3000, 48).astype(np.uint32)
    g, o = _trace_both(torch_cuda, sysd, wl.chain, ids, wl.iters, seed=wl.seed)
    assert _worst(g, o) <= POS_TOL * 20
    # screen coordinates (after the perspective) within the position bar
    assert _worst_xy(g, o) <= POS_TOL
    gl, disc = gpu_render(wl, fold_linear=fold)
    # band colours: a band op's coordinate (before the perspective) within
    # the position bar of a band edge makes the splat's colour unsure
    ol = oracle_render(wl, margin_px=fixed_margin(wl.targets, POS_TOL), track=True,
                       band_eps=POS_TOL)
    check_depth_close(gl[0], ol[0])
    total = 3001 * (40 - 20) * 3                     # three splats per step
    assert ol[0].n_splat + ol[0].n_discard == total
    assert abs(disc[0] - ol[0].n_discard) <= ol[0].n_amb
    assert (gl[0] != EMPTY).sum() > 0


def test_space_full_size_sampled(torch_cuda):
    """The bench scene (2^20 points x 200 steps, 1920 x 1080) in its launch
    configuration: every key is a colour the scene can produce at a depth its
    object can have; sampled trajectories against the oracle."""
    wl = W.space_render()
    g, disc = gpu_render(wl)
    keys = g[0][g[0] != EMPTY]
    z = depth_of(keys).astype(np.float64)
    col = (keys & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    pal = W.space_palette8()
    star, ring = pal[W.SPACE_STAR_COLOUR], pal[W.SPACE_RING_COLOUR]
    bands = set(pal[W.SPACE_BAND_BASE:W.SPACE_BAND_BASE + 4].tolist())
    assert set(np.unique(col).tolist()) <= {int(star), int(ring)} | bands
    assert np.all((z[col == star] >= 14.0) & (z[col == star] <= 20.0 + 0.04))
    bmask = np.isin(col, list(bands))
    assert bmask.any() and np.all((z[bmask] >= 5.0 - 1e-4) & (z[bmask] <= 6.0 + 1e-4))
    assert np.all(np.abs(z[col == ring] - 6.0) <= 1.84 + 1e-4)
    ids = np.array([0, 99991, (1 << 19) + 7, (1 << 20) - 1], dtype=np.uint32)
    gg, oo = _trace_both(torch_cuda, wl.jobs[0].system, wl.chain, ids, wl.iters, seed=wl.seed)
    assert _worst(gg, oo) <= POS_TOL * 20


def _stars(n):
    return W.Op("stars", (float(n), -4.0, 4.0, -4.0, 4.0, 0.0, 1.0, 0.2, 0.5))


@pytest.mark.parametrize("chain_ops", [
    # the first duplication op reads the per-CTA table of its stars
    [_stars(7), W.Op("bands", (1.0, 2.0, 0.25, 3.0, 0.0)), W.Op("splat", (0,))],
    # more stars than the table holds: the Philox block per step
    [_stars(700), W.Op("bands", (1.0, 2.0, 0.25, 3.0, 0.0)), W.Op("splat", (0,))],
    # a second duplication op in the chain: the table is the first op's only
    [_stars(5), W.Op("splat", (0,)), W.Op("reset"), _stars(9),
     W.Op("bands", (0.0, 1.0, 0.0, 2.0, 1.0)), W.Op("splat", (0,))],
], ids=["table", "over-512", "two-ops"])
def test_stars_in_a_batch_are_bit_exact(torch_cuda, chain_ops):
    from paper_2606_02226_gb300 import cfs
    torch = torch_cuda
    frames = W.animation_frames(n_frames=6, seed=5, min_log2=9, max_log2=11, resolutions=(64,))
    chain = cfs.Chain(chain_ops, 2)
    items, descs, tens = [], [], []
    begin = 0
    for f, fr in enumerate(frames):
        t = W.Target("hist_u32", 64, 64, 4, (-6.0, 6.0, -6.0, 6.0))
        ten = cfs.alloc_target(t)
        items.append((cfs.System(fr.system), fr.n_points, begin, f, [t], [ten]))
        descs.append(t)
        tens.append(ten)
        begin += fr.n_points
    b = cfs.Batch(chain, items, iters=36, burn_in=12, seed=9)
    b.launch(clear=True)
    torch.cuda.synchronize()
    begin = 0
    for f, fr in enumerate(frames):
        res = O.render(fr.system, chain_ops, [descs[f]], n_points=fr.n_points, iters=36,
                       burn_in=12, seed=9, system_id=f, point_begin=begin)
        assert np.array_equal(tens[f].cpu().numpy().view(np.uint32), res[0].buf), f
        begin += fr.n_points


def test_stars_rejected_for_stored_clouds(torch_cuda):
    from paper_2606_02226_gb300 import cfs
    torch = torch_cuda
    xyz = torch.zeros((3, 8), dtype=torch.float32, device="cuda")
    fn = torch.zeros(8, dtype=torch.uint8, device="cuda")
    t = W.Target("hist_u32", 8, 8, 1, (-1.0, 1.0, -1.0, 1.0))
    ch = cfs.Chain([W.Op("stars", (3.0, -1, 1, -1, 1, 0, 1, 0.1, 0.2)), W.Op("splat", (0,))], 3)
    with pytest.raises(cfs.CfsError):
        cfs.render_points(ch, xyz, fn, [t], [cfs.alloc_target(t)])


def test_space_circle_scene_close(torch_cuda):
    """The scene on the circle IFS itself.  Eq. 1's map stretches distances
    (the output angle is pi times the input radius; the output radius
    sqrt(theta / 2 pi) is steep at small angles) and cuts the plane along the
    positive x axis, so a trajectory's ulp-level difference between CUDA's
    and the host's sin/cos/atan2 grows from step to step and now and then
    jumps across the cut.  Trajectories agree over short horizons (the trace
    test); the image is compared pixel by pixel with the exact-generator
    bounds, and all but 1% of the covered pixels must meet them."""
    wl = W.space_render(n_points=20001, iters=40, W=320, H=180)
    ids = np.linspace(0, 4000, 48).astype(np.uint32)
    g, o = _trace_both(torch_cuda, wl.jobs[0].system, wl.chain, ids, wl.iters, seed=wl.seed)
    assert _worst(g, o) <= POS_TOL * 20
    gl, _ = gpu_render(wl)
    ol = oracle_render(wl, margin_px=fixed_margin(wl.targets, POS_TOL), track=True)
    gk, zlo, zhi = gl[0], ol[0].zlo, ol[0].zhi
    ge = gk == EMPTY
    zg = np.where(ge, np.inf, depth_of(gk).astype(np.float64))
    bad = (ge & np.isfinite(zhi)) | (~ge & ~np.isfinite(zlo))
    bad |= ~ge & np.isfinite(zlo) & ((zg < zlo * (1 - 1e-5)) | (zg > np.where(
        np.isfinite(zhi), zhi * (1 + 1e-5), np.inf)))
    covered = int((~ge).sum())
    assert covered > 1000
    assert bad.sum() <= 1e-2 * covered, (int(bad.sum()), covered)
