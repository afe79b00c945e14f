"""GPU checks of the learned warm-start sampler against the fp64 oracle
(oracle/sampler_oracle.py): forward and gradients on the same BF16-rounded
operands, the sliced-Wasserstein loss, Adam; then training reduces the loss
and the trained network starts points closer to the attractor than the
method without it (uniform start) after the same number of cleanup steps."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from oracle import sampler_oracle as SO
from paper_2606_02226_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _flat(params):
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in params]).astype(np.float32)


def _unflat(v):
    out, o = [], 0
    for (n_out, n_in) in SO.LAYERS:
        Wl = v[o:o + n_out * n_in].reshape(n_out, n_in); o += n_out * n_in
        bl = v[o:o + n_out]; o += n_out
        out.append((Wl, bl))
    return out


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _setup(torch, B=1000, seed=1):
    from paper_2606_02226_gb300 import cfs
    params = SO.init_params(seed)
    params = [(Wl, bl + 0.05 * np.sin(np.arange(len(bl))).astype(np.float32)) for Wl, bl in params]
    rng = np.random.default_rng(seed)
    U = rng.normal(size=(B, SO.D_IN)).astype(np.float32)
    U[:, 51:] = 0
    Ub = SO.bf16_round(U)
    s = cfs.Sampler(_flat(params))
    Ut = torch.from_numpy(Ub).cuda().to(torch.bfloat16)
    return cfs, s, params, Ub, Ut


def test_param_count_and_roundtrip(torch_cuda):
    cfs, s, params, _, _ = _setup(torch_cuda, 64)
    assert s.n_params == 41602 == sum(o * i + o for o, i in SO.LAYERS)
    w, m, v, st = s.get_params()
    assert np.array_equal(w, _flat(params)) and not m.any() and not v.any() and st == 0


@pytest.mark.parametrize("B", [37, 129, 1000])
def test_forward_matches_oracle(torch_cuda, B):
    # 37: fewer rows than one tile; 129 and 1000: a ragged last tile
    cfs, s, params, Ub, Ut = _setup(torch_cuda, B)
    Y = s.forward(Ut).cpu().numpy()
    Yo, _ = SO.forward(params, Ub, bf16=True)
    assert _rel(Y, Yo) < 1e-2, _rel(Y, Yo)


@pytest.mark.parametrize("B", [37, 129, 777, 4096])
def test_backward_matches_oracle(torch_cuda, B):
    # 777 rows: a ragged last row tile and a ragged K range in the weight
    # gradients; 4096 rows: the weight gradients split over 16 CTAs
    torch = torch_cuda
    cfs, s, params, Ub, Ut = _setup(torch, B)
    rng = np.random.default_rng(9)
    dY = rng.normal(size=(B, 2)).astype(np.float32)
    g = s.backward(Ut, torch.from_numpy(dY).cuda()).cpu().numpy()
    _, cache = SO.forward(params, Ub, bf16=True)
    go = SO.backward(params, cache, dY, bf16=True)
    gl = _unflat(g)
    for l in range(4):
        assert _rel(gl[l][0], go[l][0]) < 2e-2, (l, "W", _rel(gl[l][0], go[l][0]))
        assert _rel(gl[l][1], go[l][1]) < 2e-2, (l, "b", _rel(gl[l][1], go[l][1]))


def test_sw_loss_matches_oracle(torch_cuda):
    torch = torch_cuda
    from paper_2606_02226_gb300 import cfs
    rng = np.random.default_rng(3)
    X = rng.normal(size=(3, 256, 2)).astype(np.float32)
    T = (rng.normal(size=(3, 256, 2)) * 0.5 + 0.3).astype(np.float32)
    phi = (np.arange(16) * 2 * math.pi / 16 + 0.1).astype(np.float32)
    loss, dX = cfs.sw_loss(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(),
                           torch.from_numpy(phi).cuda())
    Lo, go = SO.sw_loss_grad(X, T, phi.astype(np.float64))
    assert abs(float(loss.item()) - Lo) < 1e-5 * Lo
    assert _rel(dX.cpu().numpy(), go) < 1e-4


@pytest.mark.parametrize("S,N,P", [(1, 32, 1), (2, 64, 5), (3, 128, 16), (2, 512, 7),
                                   (2, 1024, 3), (4, 1024, 64)])
def test_sw_loss_sizes_match_oracle(torch_cuda, S, N, P):
    """Every group size of the register-blocked sort (N / 8 threads), CTAs
    whose last run of projections is short (P not a multiple of the run),
    one projection, and the training shape's 1024 points."""
    torch = torch_cuda
    from paper_2606_02226_gb300 import cfs
    rng = np.random.default_rng(100 + N + P)
    X = rng.normal(size=(S, N, 2)).astype(np.float32)
    T = (rng.standard_t(3, size=(S, N, 2)) * 0.4 - 0.2).astype(np.float32)
    phi = rng.uniform(0.0, 2 * math.pi, size=P).astype(np.float32)
    loss, dX = cfs.sw_loss(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(),
                           torch.from_numpy(phi).cuda())
    Lo, go = SO.sw_loss_grad(X, T, phi.astype(np.float64))
    assert abs(float(loss.item()) - Lo) < 1e-5 * Lo
    assert _rel(dX.cpu().numpy(), go) < 1e-4


def test_sw_loss_sorted_sets_give_zero(torch_cuda):
    """Equal predicted and target sets: every rank matches itself, so the
    loss and the gradient vanish exactly (the sort and the rank search must
    pair each key with its own copy)."""
    torch = torch_cuda
    from paper_2606_02226_gb300 import cfs
    rng = np.random.default_rng(7)
    X = rng.normal(size=(2, 1024, 2)).astype(np.float32)
    T = X[:, rng.permutation(1024), :].copy()
    phi = rng.uniform(0.0, 2 * math.pi, size=9).astype(np.float32)
    loss, dX = cfs.sw_loss(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(),
                           torch.from_numpy(phi).cuda())
    assert float(loss.item()) == 0.0
    assert not dX.abs().max().item()


def test_adam_matches_oracle(torch_cuda):
    torch = torch_cuda
    cfs, s, params, _, _ = _setup(torch, 64)
    w0 = _flat(params)
    rng = np.random.default_rng(4)
    m0 = rng.normal(size=w0.size).astype(np.float32) * 1e-3
    v0 = np.abs(rng.normal(size=w0.size)).astype(np.float32) * 1e-6
    g = rng.normal(size=w0.size).astype(np.float32) * 1e-2
    s.set_params(w0, m0, v0)
    s.adam(torch.from_numpy(g).cuda(), t=5, lr=1e-3)
    w1, m1, v1, _ = s.get_params()
    wo, mo, vo = SO.adam_step(w0, g, m0, v0, 5, lr=1e-3)
    # FP32 arithmetic with FP32 hyper-parameters: 1 - 0.999f = 1.0000467e-3,
    # a 4.7e-5 relative offset of the new-gradient term against the fp64
    # oracle's exact 1e-3
    assert np.allclose(m1, mo, rtol=1e-4, atol=1e-9)
    assert np.allclose(v1, vo, rtol=1e-4, atol=1e-12)
    assert np.abs(w1 - wo).max() < 1e-6


def test_start_points_match_oracle(torch_cuda):
    """The fused inference kernel (noise drawn in the kernel, layer 1 as a
    rank-2 update, layers 2-4 on the tensor cores) against the oracle's
    noise and forward pass."""
    cfs, s, params, _, _ = _setup(torch_cuda, 64)
    fr = W.animation_frames(n_frames=3, seed=4)[2]
    sysh = cfs.System(fr.system)
    n = 1000
    st = s.start_points(sysh, fr.t, n, seed=77).cpu().numpy().T
    Yo = SO.start_points(params, [m.params for m in fr.system.maps], fr.t, n, 77)
    assert _rel(st, Yo) < 2e-2, _rel(st, Yo)
    # ragged sizes and the n = 1 edge
    st1 = s.start_points(sysh, fr.t, 1, seed=77).cpu().numpy().T
    assert _rel(st1, Yo[:1]) < 2e-2


def test_start_points_batch_equals_single_calls(torch_cuda):
    torch = torch_cuda
    cfs, s, params, _, _ = _setup(torch, 64)
    frs = W.animation_frames(n_frames=5, seed=6)
    systems = [cfs.System(f.system) for f in frs]
    counts = [1, 17, 300, 4096, 33]
    outs = [torch.empty((2, c), dtype=torch.float32, device="cuda") for c in counts]
    s.start_points_batch(systems, [f.t for f in frs], outs, [11, 12, 13, 14, 15])
    for j, f in enumerate(frs):
        one = s.start_points(systems[j], f.t, counts[j], seed=11 + j)
        torch.cuda.synchronize()
        assert torch.equal(one, outs[j]), j


def _family(n, seed=0):
    frames = W.animation_frames(n_frames=n, seed=seed)
    return frames


def _hist(pts, W_=128, view=(-4.8, 4.8, -4.8, 4.8)):
    x, y = pts
    h, _, _ = np.histogram2d(y, x, bins=W_, range=[[view[2], view[3]], [view[0], view[1]]])
    return h / max(h.sum(), 1)


def test_training_reduces_loss_and_beats_uniform_start(torch_cuda):
    torch = torch_cuda
    from paper_2606_02226_gb300 import cfs
    frames = _family(16, seed=11)
    systems = [cfs.System(f.system) for f in frames]
    t = np.array([f.t for f in frames], np.float32)
    s = cfs.Sampler(seed=5)
    hist = s.train(systems, t, 1500, systems_per_step=16, points_per_system=512, n_proj=32,
                   lr=2e-3, seed=1)
    assert np.all(np.isfinite(hist))
    assert hist[-100:].mean() < 0.5 * hist[:20].mean(), (hist[:20].mean(), hist[-100:].mean())
    # gain: points after k cleanup steps vs the attractor (full burn-in)
    n = 1 << 16
    wins = 0
    for f in (0, 5, 9):
        sysd = frames[f].system
        sh = systems[f]
        ref = O.trace(sysd, [W.Op("splat", (0,))], np.arange(20000, dtype=np.uint32),
                      iters=60)[1][:, -1, :2].T
        href = _hist(ref)
        start = s.start_points(sh, float(t[f]), n, seed=123)
        st = start.cpu().numpy().T.copy()
        uni = W.uniform_points(n, 2, f)
        for k in (0, 2, 4, 8):
            # k plain chaos-game steps from each start, same map choices
            ids = np.arange(n, dtype=np.uint32)
            if k == 0:
                ps, pu = st, uni
            else:
                ps = O.trace(sysd, [W.Op("splat", (0,))], ids, iters=k, start=st)[1][:, -1, :2]
                pu = O.trace(sysd, [W.Op("splat", (0,))], ids, iters=k, start=uni)[1][:, -1, :2]
            l1s = np.abs(_hist(ps.T) - href).sum()
            l1u = np.abs(_hist(pu.T) - href).sum()
            if k <= 4:
                assert l1s < l1u, (f, k, l1s, l1u)
            wins += l1s < l1u
    assert wins >= 9


def test_train_ex_schedule(torch_cuda):
    """cfs_sampler_train_ex: a constant schedule trains as cfs_sampler_train
    does (the weight gradients are sums of FP32 atomics, so two runs agree to
    rounding, not bit for bit); a cosine decay trains too (finite, falling
    loss) and ends at other parameters."""
    from paper_2606_02226_gb300 import cfs
    frames = _family(8, seed=3)
    systems = [cfs.System(f.system) for f in frames]
    t = np.array([f.t for f in frames], np.float32)
    a = cfs.Sampler(seed=2)
    b = cfs.Sampler(seed=2)
    c = cfs.Sampler(seed=2)
    ha = a.train(systems, t, 60, systems_per_step=8, points_per_system=256, n_proj=16, seed=4)
    hb = b.train(systems, t, 60, systems_per_step=8, points_per_system=256, n_proj=16, seed=4,
                 lr_final=1e-3)
    hc = c.train(systems, t, 60, systems_per_step=8, points_per_system=256, n_proj=16, seed=4,
                 lr_final=1e-5)
    wa, wb_, wc = a.get_params()[0], b.get_params()[0], c.get_params()[0]
    same = np.abs(wa - wb_).max()
    assert same < 2e-4 and np.allclose(ha, hb, rtol=1e-3, atol=1e-6), same
    assert np.all(np.isfinite(hc)) and np.abs(wa - wc).max() > 10 * max(same, 1e-6)
    assert hc[-10:].mean() < hc[:5].mean()
    with pytest.raises(cfs.CfsError):
        c.train(systems, t, 2, systems_per_step=8, points_per_system=256, lr_final=0.0)
