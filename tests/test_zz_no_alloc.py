"""The batched-histogram entry point that allocates nothing.

Some callers cannot allocate device memory while they render: a real-time
or embedded host whose memory budget is fixed after start-up, or a process
whose GPU memory belongs to another allocator.  cfs_render_batch_noalloc
keeps its workspace in a device array built into the library.  These checks
call it through the C ABI and compare its histograms and discard counts with
those of the allocating batch entry point and with the oracle, on two calls
in a row (the shared workspace keeps the previous call's contents, so the
second call checks that the counters are reset), and check that a call
leaves the device's free memory unchanged.  The file is collected last on
purpose: a failure here leaves every other test already run."""
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


def _items(cfs, frames, view):
    items, tens, descs, begin = [], [], [], 0
    for f, fr in enumerate(frames):
        t = W.animation_target(fr.W)
        t.view = view
        ten = cfs.alloc_target(t)
        items.append((cfs.System(fr.system), fr.n_points, begin, f, [t], [ten]))
        tens.append(ten)
        descs.append(t)
        begin += fr.n_points
    return items, tens, descs


def test_noalloc_batch_matches_allocating_batch_and_oracle_on_two_calls(torch_cuda):
    torch = torch_cuda
    from paper_2606_02226_gb300 import cfs
    frames = W.animation_frames(n_frames=24, seed=8, min_log2=10, max_log2=14,
                                resolutions=(64, 128, 256))
    view = (-2.0, 2.0, -2.0, 2.0)            # crops some attractors: discards
    chain_ops = [W.Op("splat", (0,))]
    chain = cfs.Chain(chain_ops, 2)
    ref_items, ref_tens, descs = _items(cfs, frames, view)
    b = cfs.Batch(chain, ref_items, iters=70, burn_in=20, seed=3)
    b.launch(clear=True)
    torch.cuda.synchronize()
    ref_disc = b.discards()[:, 0].astype(np.int64)
    ref = [t.cpu().numpy().view(np.uint32).copy() for t in ref_tens]
    assert ref_disc.sum() > 0
    # the oracle, frame by frame (exact affine arithmetic: bit for bit)
    begin = 0
    for f, fr in enumerate(frames):
        o = O.render(fr.system, chain_ops, [descs[f]], n_points=fr.n_points, iters=70,
                     burn_in=20, seed=3, system_id=f, point_begin=begin)[0]
        assert np.array_equal(o.buf, ref[f]), f
        assert o.n_discard == ref_disc[f], f
        begin += fr.n_points

    items, tens, _ = _items(cfs, frames, view)
    for call in range(2):
        for t in tens:
            t.fill_(7)                           # garbage: clear must remove it
        disc = torch.full((len(frames),), -1, dtype=torch.int64, device="cuda")
        cfs.render_batch_noalloc(items, iters=70, burn_in=20, seed=3, clear=True,
                                 discards=disc)
        torch.cuda.synchronize()
        for f in range(len(frames)):
            got = tens[f].cpu().numpy().view(np.uint32)
            assert np.array_equal(got, ref[f]), (call, f)
        assert np.array_equal(disc.cpu().numpy(), ref_disc), call


def test_noalloc_batch_leaves_free_memory_unchanged(torch_cuda):
    torch = torch_cuda
    from paper_2606_02226_gb300 import cfs
    view = (-2.0, 2.0, -2.0, 2.0)
    warm = W.animation_frames(n_frames=3, seed=4, min_log2=9, max_log2=10, resolutions=(32,))
    items, _, _ = _items(cfs, warm, view)
    cfs.render_batch_noalloc(items, iters=30, burn_in=5, seed=1, clear=True)
    torch.cuda.synchronize()
    # new frame shapes (more frames, other sizes), every buffer made up front
    frames = W.animation_frames(n_frames=40, seed=6, min_log2=10, max_log2=13,
                                resolutions=(64, 96, 200))
    items, tens, _ = _items(cfs, frames, view)
    disc = torch.zeros(len(frames), dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    cfs.render_batch_noalloc(items, iters=50, burn_in=10, seed=2, clear=True, discards=disc)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert int(sum(int(t.view(torch.int32).sum().item()) for t in tens)) + \
        int(disc.sum().item()) == sum(fr.n_points for fr in frames) * 40


def test_noalloc_batch_rejects_too_many_frames(torch_cuda):
    from paper_2606_02226_gb300 import cfs
    fr = W.animation_frames(n_frames=1, seed=1, min_log2=8, max_log2=8, resolutions=(16,))[0]
    t = W.animation_target(16)
    ten = cfs.alloc_target(t)
    s = cfs.System(fr.system)
    items = [(s, 16, 16 * j, j, [t], [ten]) for j in range(257)]
    with pytest.raises(cfs.CfsError):
        cfs.render_batch_noalloc(items, iters=10, burn_in=2)
