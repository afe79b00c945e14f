"""GPU parity of the stored point-cloud path (generation, then streaming the
cloud through an 8-transform chain into a depth+colour layer) against the
CPU oracle on the same inputs."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_02226_gb300 import workloads as W

from _parity import EMPTY, check_depth_close, depth_of, fixed_margin

POS_TOL = 1e-5

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _cfs():
    from paper_2606_02226_gb300 import cfs
    return cfs


@pytest.mark.parametrize("n,iters", [(10001, 32), (4096, 5), (1, 3)])
def test_cloud_generation_bit_exact(torch_cuda, n, iters):
    cfs = _cfs()
    sysd = W.cloud_system()
    xyz, fn = cfs.pointcloud_generate(cfs.System(sysd), n, iters, seed=3, system_id=2)
    torch_cuda.cuda.synchronize()
    ox, ofn = O.pointcloud_generate(sysd, n, iters, seed=3, system_id=2)
    assert np.array_equal(xyz.cpu().numpy().T, ox)
    assert np.array_equal(fn.cpu().numpy(), ofn)


def _stream_parity(frame, n, W_, fast_trig=False, fold=False):
    torch = pytest.importorskip("torch")
    cfs = _cfs()
    sysd = W.cloud_system()
    ox, ofn = O.pointcloud_generate(sysd, n, 32)
    chain = W.cloud_chain(frame)
    t = W.cloud_target(W_)
    ten = cfs.alloc_target(t)
    disc = torch.zeros(1, dtype=torch.int64, device="cuda")
    xyz = torch.from_numpy(np.ascontiguousarray(ox.T)).cuda()
    fn = torch.from_numpy(ofn).cuda()
    cfs.render_points(cfs.Chain(chain, 3, fast_trig=fast_trig, fold_linear=fold), xyz, fn, [t],
                      [ten], discards=disc)
    torch.cuda.synchronize()
    g = ten.cpu().numpy().view(np.uint64)
    # margin: the position tolerance in pixels (the [-1, 1] view has W/2
    # pixels per unit)
    o = O.render_points(ox, ofn, chain, [t], margin_px=fixed_margin([t], POS_TOL),
                        track=True)[0]
    check_depth_close(g, o)
    d = int(disc.item())
    assert abs(d - o.n_discard) <= o.n_amb
    assert int((g != EMPTY).sum()) > 0
    return g, o


@pytest.mark.parametrize("frame,fast_trig,fold", [(0, False, False), (21, False, False),
                                                  (63, False, False), (0, True, False),
                                                  (63, True, False), (0, False, True),
                                                  (40, True, True)])
def test_cloud_streaming_parity(torch_cuda, frame, fast_trig, fold):
    # fold: the four affines and the camera translation run as one affine op
    _stream_parity(frame, 1 << 15, 512, fast_trig=fast_trig, fold=fold)


def test_render_points_needs_multiple_of_4(torch_cuda):
    torch = torch_cuda
    cfs = _cfs()
    t = W.cloud_target(16)
    ten = cfs.alloc_target(t)
    xyz = torch.zeros((3, 6), dtype=torch.float32, device="cuda")
    fn = torch.zeros(6, dtype=torch.uint8, device="cuda")
    with pytest.raises(cfs.CfsError):
        cfs.render_points(cfs.Chain(W.cloud_chain(0), 3), xyz, fn, [t], [ten])


def test_cloud_full_size_sampled(torch_cuda):
    """The benchmark's cloud (2^26 points, 8192^2 layer): every sampled
    point's key bounds its pixel's minimum from above, and every stored key
    decodes to a palette colour."""
    torch = torch_cuda
    cfs = _cfs()
    sysd = W.cloud_system()
    n = 1 << 26
    xyz, fn = cfs.pointcloud_generate(cfs.System(sysd), n, 32)
    t = W.cloud_target(8192)
    ten = cfs.alloc_target(t)
    chain = W.cloud_chain(40)
    cfs.render_points(cfs.Chain(chain, 3), xyz, fn, [t], [ten])
    torch.cuda.synchronize()
    ids = np.linspace(0, n - 1, 257).astype(np.int64)
    sx = xyz[:, torch.from_numpy(ids).cuda()].cpu().numpy().T.copy()
    sfn = fn[torch.from_numpy(ids).cuda()].cpu().numpy()
    # the sampled stored points equal the oracle's trajectories' endpoints
    k, p, _ = O.trace(sysd, [W.Op("splat", (0,))], ids.astype(np.uint32), iters=32)
    assert np.array_equal(sx, p[:, -1, :]) and np.array_equal(sfn, k[:, -1])
    # each sampled point's depth bounds the layer's depth at the pixel it
    # surely lands in (relative 1e-5 for the chain's FP32 differences)
    r = O.render_points(sx, sfn, chain, [t], margin_px=fixed_margin([t], POS_TOL), track=True)[0]
    layer = ten.cpu().numpy().view(np.uint64)
    sure = np.isfinite(r.zhi)
    assert sure.sum() > 100
    assert np.all(layer[sure] != EMPTY)
    assert np.all(depth_of(layer[sure]).astype(np.float64) <=
                  r.zhi[sure].astype(np.float64) * (1 + 1e-5))
    keys = layer[layer != EMPTY]
    cols = set(np.unique((keys & np.uint64(0xFFFFFFFF)).astype(np.uint32)).tolist())
    assert cols <= set(W.palette_rgba8(16)[:8].tolist())
    z = depth_of(keys)
    assert np.all(z > 1e-3)


def _morton_keys(xyz):
    """Morton keys of a [dim, n] float32 cloud, computed as the reorder
    defines them (FP32 box, scale, quantization; x in the lowest bit)."""
    dim, n = xyz.shape
    key = np.zeros(n, dtype=np.uint64)
    for d in range(dim):
        v = xyz[d]
        fin = v[~np.isnan(v)]
        lo, hi = np.float32(fin.min()), np.float32(fin.max())
        ext = np.float32(hi - lo)
        scale = np.float32(np.float32(1024.0) / ext) if ext > 0 else np.float32(0.0)
        with np.errstate(invalid="ignore", over="ignore"):
            u = (v - lo).astype(np.float32) * scale
        q = np.zeros(n, dtype=np.int64)
        ok = u >= 0
        q[ok] = np.minimum(np.minimum(u[ok], 2**31 - 1).astype(np.int64), 1023)
        for b in range(10):
            key |= (((q >> b) & 1).astype(np.uint64)) << np.uint64(3 * b + d if dim == 3 else 2 * b + d)
    return key


@pytest.mark.parametrize("n,dim", [(100003, 3), (4096 * 3 + 17, 2), (1, 3)])
def test_reorder_is_the_stable_morton_sort(torch_cuda, n, dim):
    torch = torch_cuda
    cfs = _cfs()
    rng = np.random.default_rng(n)
    xyz = rng.normal(size=(dim, n)).astype(np.float32)
    if n > 10:
        xyz[:, 5] = xyz[:, 3]          # equal keys keep their order
        xyz[0, 7] = np.nan
    fn = rng.integers(0, 8, n).astype(np.uint8)
    xo, fo, perm = cfs.pointcloud_reorder(torch.from_numpy(xyz).cuda(), torch.from_numpy(fn).cuda(),
                                          want_perm=True)
    torch.cuda.synchronize()
    expect = np.argsort(_morton_keys(xyz), kind="stable")
    p = perm.cpu().numpy()
    assert np.array_equal(p, expect)
    assert np.array_equal(xo.cpu().numpy(), xyz[:, expect], equal_nan=True)
    assert np.array_equal(fo.cpu().numpy(), fn[expect])


def test_reordered_cloud_renders_the_same_layer(torch_cuda):
    torch = torch_cuda
    cfs = _cfs()
    n = 1 << 18
    xyz, fn = cfs.pointcloud_generate(cfs.System(W.cloud_system()), n, 32)
    xo, fo = cfs.pointcloud_reorder(xyz, fn)
    t = W.cloud_target(1024)
    a, b = cfs.alloc_target(t), cfs.alloc_target(t)
    ch = cfs.Chain(W.cloud_chain(30), 3)
    cfs.render_points(ch, xyz, fn, [t], [a])
    cfs.render_points(ch, xo, fo, [t], [b])
    torch.cuda.synchronize()
    assert torch.equal(a, b)
