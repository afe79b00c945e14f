"""GPU parity of the batched renderer (many frames of different systems in one
persistent launch, replayed as a CUDA graph) against the CPU oracle, frame by
frame.  The animation frames are affine with a splat-only chain, so every
histogram is bit-exact."""
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


def _setup(frames, view=None):
    from paper_2606_02226_gb300 import cfs
    chain = cfs.Chain([W.Op("splat", (0,))], 2)
    items, descs, tens, systems = [], [], [], []
    begin = 0
    for f, fr in enumerate(frames):
        t = W.animation_target(fr.W)
        if view is not None:
            t.view = view
        ten = cfs.alloc_target(t)
        s = cfs.System(fr.system)
        systems.append(s)
        items.append((s, fr.n_points, begin, f, [t], [ten]))
        descs.append(t)
        tens.append(ten)
        begin += fr.n_points
    return cfs, chain, items, descs, tens


def _oracle(frames, descs, iters, burn_in, seed):
    out, disc = [], []
    begin = 0
    for f, (fr, t) in enumerate(zip(frames, descs)):
        r = O.render(fr.system, [W.Op("splat", (0,))], [t], n_points=fr.n_points,
                     point_begin=begin, system_id=f, iters=iters, burn_in=burn_in, seed=seed)
        out.append(r[0].buf)
        disc.append(r[0].n_discard)
        begin += fr.n_points
    return out, disc


def _host(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("words,warp_agg,window,ilp,iters,chunk",
                         [(8192, 1, 1, 1, 60, 4096), (1024, 1, 1, 1, 60, 4096),
                          (1024, 0, 1, 1, 60, 64), (8192, 1, 0, 1, 60, 4096),
                          (8192, 1, 1, 2, 60, 2048), (1024, 1, 1, 2, 63, 96),
                          (8192, 1, 0, 2, 61, 4096), (53248, 0, 1, 2, 62, 16384)])
def test_batch_matches_oracle_frame_by_frame(torch_cuda, words, warp_agg, window, ilp, iters,
                                             chunk):
    # plans passed through the C ABI: the privatized window at its default
    # size, at a size smaller than most attractors (splats split between
    # shared and global memory), without warp aggregation, and switched off;
    # one or two trajectories per thread (with step counts that cut the last
    # Philox block); items from 64 points to more than a frame
    frames = W.animation_frames(n_frames=14, seed=2, min_log2=8, max_log2=12,
                                resolutions=(64, 128))
    cfs, chain, items, descs, tens = _setup(frames)
    b = cfs.Batch(chain, items, iters=iters, burn_in=20, seed=4)
    b.set_plan(ilp=ilp, window=window, window_words=words, warp_agg=warp_agg, chunk=chunk)
    assert b.plan() == {"ilp": ilp, "window": window, "window_words": words,
                        "warp_agg": warp_agg, "chunk": chunk}
    info = b.info()
    assert info["n_items"] >= len(frames) and info["grid"] >= 1 and info["chunk"] == chunk
    b.launch(clear=True)
    torch_cuda.cuda.synchronize()
    ref, rdisc = _oracle(frames, descs, iters, 20, 4)
    for f in range(len(frames)):
        assert np.array_equal(_host(tens[f]), ref[f]), f
        assert int(_host(tens[f]).sum()) == frames[f].n_points * (iters - 20)
    assert list(b.discards()[:, 0]) == rdisc == [0] * len(frames)


@pytest.mark.parametrize("ilp,burn_in", [(1, 18), (2, 18), (1, 0), (2, 0), (2, 60)])
def test_batch_burn_in_on_and_off_block_boundaries(torch_cuda, ilp, burn_in):
    # whole Philox blocks with the burn-in on a block boundary take the
    # guard-free loop (0, 60), elsewhere (18) the general one; both must give
    # the oracle's histograms, including a burn-in that covers every step
    frames = W.animation_frames(n_frames=6, seed=9, min_log2=8, max_log2=11,
                                resolutions=(64, 128))
    cfs, chain, items, descs, tens = _setup(frames)
    b = cfs.Batch(chain, items, iters=60, burn_in=burn_in, seed=6)
    b.set_plan(ilp=ilp, chunk=256)
    b.launch(clear=True)
    torch_cuda.cuda.synchronize()
    ref, rdisc = _oracle(frames, descs, 60, burn_in, 6)
    for f in range(len(frames)):
        assert np.array_equal(_host(tens[f]), ref[f]), f
        assert int(_host(tens[f]).sum()) == frames[f].n_points * max(0, 60 - burn_in)


@pytest.mark.parametrize("C,words,ilp", [(1, 1024, 2), (1, 4096, 1), (16, 1024, 2),
                                         (16, 8192, 1), (3, 2048, 2)])
def test_batch_windows_with_other_channel_counts(torch_cuda, C, words, ilp):
    # one window per channel of a C-channel histogram (channel = map index
    # mod C; with 16 channels and at most 8 maps half of them stay empty),
    # the windows' counters packed one channel after the other: the
    # histograms are the oracle's bit for bit
    from paper_2606_02226_gb300 import cfs
    frames = W.animation_frames(n_frames=8, seed=11, min_log2=9, max_log2=12,
                                resolutions=(64, 128))
    chain = cfs.Chain([W.Op("splat", (0,))], 2)
    items, descs, tens, begin = [], [], [], 0
    for f, fr in enumerate(frames):
        t = W.Target("hist_u32", fr.W, fr.W, C, W.ANIMATION_VIEW)
        ten = cfs.alloc_target(t)
        items.append((cfs.System(fr.system), fr.n_points, begin, f, [t], [ten]))
        descs.append(t)
        tens.append(ten)
        begin += fr.n_points
    b = cfs.Batch(chain, items, iters=60, burn_in=20, seed=8)
    b.set_plan(ilp=ilp, window=1, window_words=words, chunk=256)
    b.launch(clear=True)
    torch_cuda.cuda.synchronize()
    win = b.windows()
    assert win.shape == (len(frames), C, 4)
    for f in range(len(frames)):
        area = [(int(x1) - int(x0) + 1) * (int(y1) - int(y0) + 1)
                for x0, y0, x1, y1 in win[f] if x1 >= x0]
        assert 0 < sum(area) <= words, (f, area)
    ref, rdisc = _oracle(frames, descs, 60, 20, 8)
    for f in range(len(frames)):
        assert np.array_equal(_host(tens[f]), ref[f]), f


@pytest.mark.parametrize("words", [1024, 4096, 53248])
def test_batch_windows_lie_in_the_counter_budget(torch_cuda, words):
    # the pre-pass places one window per histogram channel: inside the
    # target, all of a frame's windows within window_words counters, and,
    # where a channel's sampled splats exceed its share, over denser regions
    # than centred windows
    frames = W.animation_frames(n_frames=10, seed=5, min_log2=11, max_log2=13,
                                resolutions=(128, 256))
    cfs, chain, items, descs, tens = _setup(frames)
    b = cfs.Batch(chain, items, iters=60, burn_in=20, seed=2)
    with pytest.raises(cfs.CfsError):
        b.windows()                      # before the first launch
    b.set_plan(window=1, window_words=words, chunk=512)
    b.launch(clear=True)
    torch_cuda.cuda.synchronize()
    win = b.windows()
    C = descs[0].C
    assert win.shape == (len(frames), C, 4)
    tot_inside = tot_centred = 0
    for f, fr in enumerate(frames):
        h = _host(tens[f]).reshape(C, fr.W, fr.W)
        assert int(h.sum()) == fr.n_points * 40
        # the channels share the counters
        area = [(int(x1) - int(x0) + 1) * (int(y1) - int(y0) + 1)
                for x0, y0, x1, y1 in win[f] if x1 >= x0]
        assert sum(area) <= words, (f, area)
        for c in range(C):
            x0, y0, x1, y1 = (int(v) for v in win[f, c])
            if x1 < x0:
                assert (x0, y0, x1, y1) == (0, 0, -1, -1)
                continue
            assert 0 <= x0 <= x1 < fr.W and 0 <= y0 <= y1 < fr.W
            ys, xs = np.nonzero(h[c])
            if len(xs) == 0:
                continue
            inside = int(h[c, y0:y1 + 1, x0:x1 + 1].sum())
            # the centred window of the same shape over the channel's
            # splats' box
            ww, wh = x1 - x0 + 1, y1 - y0 + 1
            cx = xs.min() + max(0, (xs.max() - xs.min() + 1 - ww) // 2)
            cy = ys.min() + max(0, (ys.max() - ys.min() + 1 - wh) // 2)
            centred = int(h[c, cy:cy + wh, cx:cx + ww].sum())
            tot_inside += inside
            tot_centred += centred
            share = words * h[c].sum() / h.sum()     # about the channel's counters
            if (xs.max() - xs.min() + 1) * (ys.max() - ys.min() + 1) <= 0.4 * share:
                # a channel whose splats fit with room to spare: the sampled
                # box catches nearly all of them
                assert inside >= 0.97 * h[c].sum(), (f, c)
    # summed over the frames' channels, the sampled choice holds more splats
    # than centred windows of the same shapes
    print(f"window_words {words}: {tot_inside} splats in the chosen windows, "
          f"{tot_centred} in centred ones")
    assert tot_inside >= tot_centred


def test_batch_plan_validation(torch_cuda):
    frames = W.animation_frames(n_frames=2, seed=2, min_log2=8, max_log2=9, resolutions=(32,))
    cfs, chain, items, descs, tens = _setup(frames)
    b = cfs.Batch(chain, items, iters=30, burn_in=10, seed=1)
    for bad in ({"ilp": 3}, {"window": 2}, {"window_words": 1000}, {"window_words": 60000},
                {"warp_agg": 5}, {"chunk": 33}, {"chunk": 0}):
        with pytest.raises(cfs.CfsError):
            b.set_plan(**bad)
    assert b.plan()["ilp"] == 2              # unchanged by the rejected plans


def test_batch_graph_replay_clear_and_accumulate(torch_cuda):
    frames = W.animation_frames(n_frames=5, seed=3, min_log2=9, max_log2=11, resolutions=(64,))
    cfs, chain, items, descs, tens = _setup(frames)
    b = cfs.Batch(chain, items, iters=40, burn_in=8, seed=1)
    b.launch(clear=True)
    b.launch(clear=True)          # replay: same image
    torch_cuda.cuda.synchronize()
    first = [_host(t).copy() for t in tens]
    b.launch(clear=False)         # accumulate: doubles every bin
    torch_cuda.cuda.synchronize()
    for f in range(len(frames)):
        assert np.array_equal(_host(tens[f]), 2 * first[f])
    ref, _ = _oracle(frames, descs, 40, 8, 1)
    for f in range(len(frames)):
        assert np.array_equal(first[f], ref[f])


def test_batch_discards_and_set_system(torch_cuda):
    frames = W.animation_frames(n_frames=6, seed=5, min_log2=9, max_log2=10, resolutions=(64,))
    view = (-1.0, 1.0, -1.0, 1.0)      # crops the attractors: discards
    cfs, chain, items, descs, tens = _setup(frames, view=view)
    b = cfs.Batch(chain, items, iters=30, burn_in=10, seed=2)
    b.launch()
    torch_cuda.cuda.synchronize()
    ref, rdisc = _oracle(frames, descs, 30, 10, 2)
    assert [int(v) for v in b.discards()[:, 0]] == rdisc
    assert sum(rdisc) > 0
    for f in range(len(frames)):
        assert np.array_equal(_host(tens[f]), ref[f])
    # animate frame 2: give it frame 4's system
    b.set_system(2, cfs.System(frames[4].system))
    b.launch()
    torch_cuda.cuda.synchronize()
    frames2 = list(frames)
    frames2[2] = W.Frame(frames[4].system, frames[2].n_points, frames[2].W, frames[2].t)
    ref2, _ = _oracle(frames2, descs, 30, 10, 2)
    assert np.array_equal(_host(tens[2]), ref2[2])
    assert not np.array_equal(ref2[2], ref[2])


def test_batch_equals_single_renders_and_one_shot(torch_cuda):
    frames = W.animation_frames(n_frames=4, seed=6, min_log2=10, max_log2=12, resolutions=(128,))
    cfs, chain, items, descs, tens = _setup(frames)
    cfs.render_batch(chain, items, iters=50, burn_in=20, seed=7)
    torch_cuda.cuda.synchronize()
    got = [_host(t).copy() for t in tens]
    begin = 0
    for f, fr in enumerate(frames):
        single = cfs.alloc_target(descs[f])
        cfs.render(cfs.System(fr.system), chain, [descs[f]], [single], n_points=fr.n_points,
                   point_begin=begin, system_id=f, iters=50, burn_in=20, seed=7)
        torch_cuda.cuda.synchronize()
        assert np.array_equal(_host(single), got[f])
        begin += fr.n_points


def test_batch_rejects_mixed_kinds(torch_cuda):
    from paper_2606_02226_gb300 import cfs
    t = W.Target("hist_u32", 16, 16, 4)
    ten = cfs.alloc_target(t)
    sq = W.square_system()
    mixed = W.System(2, sq.maps[:2] + [W.Map("circle", (0.0,))], [0.3, 0.3, 0.4])
    chain = cfs.Chain([W.Op("splat", (0,))], 2)
    with pytest.raises(cfs.CfsError):
        cfs.Batch(chain, [(cfs.System(mixed), 10, 0, 0, [t], [ten])], iters=5, burn_in=1)


def test_batch_start_points_and_step_begin(torch_cuda):
    """Frames carrying their own start points (fewer than their points:
    point j starts at start j mod m) and a first step of 12: bit-exact
    against the oracle run from the repeated starts."""
    torch = torch_cuda
    frames = W.animation_frames(n_frames=5, seed=9, min_log2=9, max_log2=11, resolutions=(64,))
    cfs, chain, items, descs, tens = _setup(frames)
    starts, full = [], []
    for f, fr in enumerate(frames):
        m = max(1, fr.n_points // 3)
        st = (W.uniform_points(m, 2, 100 + f) * 2 - 1).astype(np.float32)
        starts.append(torch.from_numpy(np.ascontiguousarray(st.T)).cuda())
        full.append(st[np.arange(fr.n_points) % m])
    items = [tuple(it) + (starts[f],) for f, it in enumerate(items)]
    b = cfs.Batch(chain, items, iters=50, burn_in=20, seed=6, step_begin=12)
    b.launch()
    torch.cuda.synchronize()
    begin = 0
    for f, fr in enumerate(frames):
        o = O.render(fr.system, [W.Op("splat", (0,))], [descs[f]], n_points=fr.n_points,
                     point_begin=begin, system_id=f, iters=50, burn_in=20, seed=6,
                     step_begin=12, start=full[f])[0].buf
        assert np.array_equal(_host(tens[f]), o), f
        begin += fr.n_points


def test_batch_autotuner_keeps_results_exact(torch_cuda, tmp_path):
    # tuning changes the plan (program knobs, per-class item sizes and
    # windows), never the frames: the tuned launch is still the oracle's, bit
    # for bit; a second tune of the same batch takes every choice from the
    # cache, which survives a save / clear / load round trip
    frames = W.animation_frames(n_frames=9, seed=6, min_log2=8, max_log2=12,
                                resolutions=(64, 128))
    cfs, chain, items, descs, tens = _setup(frames)
    cfs.tune_cache_clear()
    b = cfs.Batch(chain, items, iters=44, burn_in=20, seed=3)
    choice = b.tune(trial_iters=24)
    assert choice["trials"] >= 8 and choice["chunk"] in (2048, 4096, 8192, 16384)
    assert choice["ilp"] in (1, 2) and choice["tile"] in (0, 1) and choice["trial_ms"] > 0
    assert choice["n_classes"] >= 2 and not choice["from_cache"]
    assert choice["window_words"] in ((13312, 26624, 53248) if choice["tile"] else (0,))
    b.launch(clear=True)
    torch_cuda.cuda.synchronize()
    ref, rdisc = _oracle(frames, descs, 44, 20, 3)
    for f in range(len(frames)):
        assert np.array_equal(_host(tens[f]), ref[f]), f
    assert list(b.discards()[:, 0]) == rdisc
    n = cfs.tune_cache_size()
    assert n == 2 + choice["n_classes"]      # program, classes, and whether to use them
    path = str(tmp_path / "tune.txt")
    cfs.tune_cache_save(path)
    cfs.tune_cache_clear()
    assert cfs.tune_cache_size() == 0
    cfs.tune_cache_load(path)
    assert cfs.tune_cache_size() == n
    b2 = cfs.Batch(chain, items, iters=44, burn_in=20, seed=3)
    again = b2.tune(trial_iters=24)
    assert again["from_cache"] and again["trials"] == 0
    for k in ("ilp", "tile", "chunk", "window_words", "warp_agg", "classes_windowed",
              "classes_used"):
        assert again[k] == choice[k], k
    b2.launch(clear=True)
    torch_cuda.cuda.synchronize()
    for f in range(len(frames)):
        assert np.array_equal(_host(tens[f]), ref[f]), f
    forced = b2.tune(trial_iters=24, retune=True)
    assert not forced["from_cache"] and forced["trials"] >= 8
    cfs.tune_cache_clear()
