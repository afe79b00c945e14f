"""Multi-process (world_size 2, gloo, CPU) checks of how the path shards.

Points are independent and their Philox streams depend only on (point,
step, system), so ranks can render disjoint ranges of point indices; the
only exchange is an order-free reduction of the layers (integer sums of
histograms, minimum of depth keys).  Here two gloo ranks each render half of
a frame with the oracle, reduce, and rank 0 checks the result against the
whole frame rendered in one process -- exactly, since every operation
involved is an integer sum or a minimum.  The benchmark's rank partition
(weak scaling: every rank its own range) is checked the same way.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from oracle import oracle as O
    from paper_2606_02226_gb300 import workloads as W

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # 1) shard one frame of the composed scene by point index
        wl = W.composed_render(n_points=2000, iters=40, W=64)
        bufs = [O.alloc_target_buffer(t) for t in wl.targets]
        for job in wl.jobs:
            per = (job.n_points + world - 1) // world
            lo = min(job.n_points, rank * per)
            hi = min(job.n_points, lo + per)
            if hi > lo:
                O.render(job.system, wl.chain, wl.targets, n_points=hi - lo,
                         point_begin=job.point_begin + lo, iters=wl.iters, burn_in=wl.burn_in,
                         seed=wl.seed, bufs=bufs)
        rgba = torch.from_numpy(bufs[0].copy())
        depth = torch.from_numpy(bufs[1].view(np.int64).copy())
        # the RGBA sums are exact in FP32 (palette in {0, .5, 1}, small counts)
        dist.all_reduce(rgba, op=dist.ReduceOp.SUM)
        # depth keys: unsigned minimum == signed minimum after flipping the top bit
        flipped = depth ^ torch.tensor(-(1 << 63), dtype=torch.int64)
        dist.all_reduce(flipped, op=dist.ReduceOp.MIN)
        depth_min = flipped ^ torch.tensor(-(1 << 63), dtype=torch.int64)
        # 2) the benchmark's weak-scaling partition: rank r takes its own
        #    range of point indices, no overlap, no data-path collective
        n_total = sum(j.n_points for j in wl.jobs)
        ranges = [[j.point_begin + rank * n_total, j.n_points] for j in wl.jobs]
        allr = [None] * world
        dist.all_gather_object(allr, ranges)
        if rank == 0:
            np.save(os.path.join(out_dir, "rgba.npy"), rgba.numpy())
            np.save(os.path.join(out_dir, "depth.npy"), depth_min.numpy().view(np.uint64))
            np.save(os.path.join(out_dir, "ranges.npy"), np.array(allr, dtype=np.int64))
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_to_the_whole_frame(tmp_path):
    from oracle import oracle as O
    from paper_2606_02226_gb300 import workloads as W
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    wl = W.composed_render(n_points=2000, iters=40, W=64)
    bufs = [O.alloc_target_buffer(t) for t in wl.targets]
    for job in wl.jobs:
        O.render(job.system, wl.chain, wl.targets, n_points=job.n_points,
                 point_begin=job.point_begin, iters=wl.iters, burn_in=wl.burn_in, seed=wl.seed,
                 bufs=bufs)
    assert np.array_equal(np.load(tmp_path / "rgba.npy"), bufs[0])
    assert np.array_equal(np.load(tmp_path / "depth.npy"), bufs[1])
    ranges = np.load(tmp_path / "ranges.npy")          # [rank][job][begin, n]
    spans = sorted((int(b), int(b + n)) for r in ranges for b, n in r)
    for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
        assert a1 <= b0                                  # disjoint point ranges
