"""GPU parity of the density-estimation display (log density, gamma, packed
RGBA8) against the CPU oracle, through the C ABI.

Both sides compute in FP32 with the same operation order; only logf/powf
differ between CUDA and the host libm (by a few ulps).  So every component
code must be equal, except components whose 255 x + 1/2 lies within 1e-3 of
an integer on the oracle side (the oracle flags them), which may differ by
one.  The density maximum is a plain maximum of identical FP32 sums: exact."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_02226_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _desc(kind, Wd, H, C=4):
    return W.Target(kind, Wd, H, C if kind == "hist_u32" else 1, (0.0, 1.0, 0.0, 1.0),
                    palette=W.palette_rgba(16))


def _upload(torch, kind, arr):
    dt = {"hist_u32": torch.int32, "rgba_f32": torch.float32, "depth_u64": torch.int64}[kind]
    host = arr.view({"hist_u32": np.int32, "rgba_f32": np.float32, "depth_u64": np.int64}[kind])
    return torch.from_numpy(np.ascontiguousarray(host)).to("cuda").view(dt)


def _check_codes(g, o, near):
    g = g.astype(np.uint32)
    diff_any = g != o
    if not diff_any.any():
        return 0
    gb = np.stack([(g >> (8 * c)) & 0xFF for c in range(4)], -1).astype(np.int32)
    ob = np.stack([(o >> (8 * c)) & 0xFF for c in range(4)], -1).astype(np.int32)
    nb = np.stack([(near >> c) & 1 for c in range(4)], -1).astype(bool)
    d = np.abs(gb - ob)
    assert not (d > 1).any(), "a component differs by more than one code"
    assert not ((d == 1) & ~nb).any(), "a component away from a rounding boundary differs"
    return int((d == 1).sum())


def _run(torch, kind, Wd, H, C=4, seed=0, **kw):
    from paper_2606_02226_gb300 import cfs
    desc = _desc(kind, Wd, H, C)
    arr = W.synthetic_layer(kind, Wd, H, C, seed=seed)
    t = _upload(torch, kind, arr)
    out, amax = cfs.tonemap(desc, t, **kw)
    torch.cuda.synchronize()
    o, near, used = O.tonemap(desc, arr, **kw)
    g = out.cpu().numpy().view(np.uint32)
    n_diff = _check_codes(g, o, near)
    if amax is not None:
        assert float(amax.cpu()[0]) == used
    return n_diff, o


@pytest.mark.parametrize("kind,Wd,H", [("rgba_f32", 640, 360), ("rgba_f32", 257, 131),
                                       ("hist_u32", 512, 512), ("hist_u32", 257, 131),
                                       ("depth_u64", 300, 200), ("depth_u64", 257, 131)])
def test_display_matches_oracle(torch_cuda, kind, Wd, H):
    n_diff, o = _run(torch_cuda, kind, Wd, H, seed=3, gamma=2.2, background=0x10203040)
    assert n_diff <= 1e-3 * o.size


def test_display_parameters(torch_cuda):
    # fixed maximum, linear gamma, brightness that saturates, one channel
    _run(torch_cuda, "hist_u32", 128, 96, C=1, seed=5, gamma=1.0, brightness=3.0, a_max=40.0)
    _run(torch_cuda, "rgba_f32", 128, 96, seed=6, gamma=0.5, brightness=0.7)


def test_display_full_size_layers(torch_cuda):
    # the composed scene's 2048^2 RGBA layer and a 1920x1080 four-channel histogram
    n1, o1 = _run(torch_cuda, "rgba_f32", 2048, 2048, seed=7, gamma=2.2)
    n2, o2 = _run(torch_cuda, "hist_u32", 1920, 1080, seed=8, gamma=2.2)
    assert n1 <= 1e-3 * o1.size and n2 <= 1e-3 * o2.size


def test_display_empty_layer_is_background(torch_cuda):
    from paper_2606_02226_gb300 import cfs
    desc = _desc("hist_u32", 64, 64)
    t = cfs.alloc_target(desc)
    out, amax = cfs.tonemap(desc, t, background=0xFF000000)
    torch_cuda.cuda.synchronize()
    assert float(amax.cpu()[0]) == 0.0
    assert (out.cpu().numpy().view(np.uint32) == 0xFF000000).all()


def test_batch_display_matches_oracle(torch_cuda):
    from paper_2606_02226_gb300 import cfs
    torch = torch_cuda
    frames = W.animation_frames(n_frames=6, seed=0, min_log2=12, max_log2=13,
                                resolutions=(64, 128, 256))
    chain = cfs.Chain([W.Op("splat", (0,))], 2)
    items, arrs, descs = [], [], []
    for f, fr in enumerate(frames):
        d = W.animation_target(fr.W)
        d.palette = W.palette_rgba(16)
        a = W.synthetic_layer("hist_u32", fr.W, fr.W, d.C, seed=100 + f)
        items.append((cfs.System(fr.system), fr.n_points, 0, f, [d], [_upload(torch, "hist_u32", a)]))
        arrs.append(a)
        descs.append(d)
    b = cfs.Batch(chain, items, iters=30, burn_in=20)
    outs = [torch.empty((d.H, d.W), dtype=torch.int32, device="cuda") for d in descs]
    amax = torch.empty(len(frames), dtype=torch.float32, device="cuda")
    for rep in range(2):                      # two calls in a row reuse the staging
        b.display(outs, gamma=2.2, background=7, a_max_out=amax)
        torch.cuda.synchronize()
        for f, d in enumerate(descs):
            o, near, used = O.tonemap(d, arrs[f], gamma=2.2, background=7)
            _check_codes(outs[f].cpu().numpy().view(np.uint32), o, near)
            assert float(amax[f].cpu()) == used


def test_display_rejects_bad_arguments(torch_cuda):
    from paper_2606_02226_gb300 import cfs
    desc = _desc("rgba_f32", 32, 32)
    t = cfs.alloc_target(desc)
    with pytest.raises(cfs.CfsError):
        cfs.tonemap(desc, t, gamma=0.0)
    buf = torch_cuda.empty(32 * 32 + 1, dtype=torch_cuda.int32, device="cuda")
    with pytest.raises(cfs.CfsError):                 # output not 16-byte aligned
        cfs.tonemap(desc, t, out=buf[1:].view(32, 32))
