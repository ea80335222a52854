"""The N > 1 path of bench.py on CPU: two ranks over gloo.  Each GPU of a
multi-GPU run is an independent replica; the only cross-rank step is the
reduction of the timing and of the units processed, which these tests run
with the same helpers bench.py uses (gloo instead of NCCL, CPU tensors)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, w, local = bench.dist_setup()
    assert (r, w, local) == (rank, world, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.dist_barrier(world)
        # rank k: slowest time 10 + k ms, 100 * (k + 1) units, latencies (k, 5 - k)
        t, units, extra = bench.reduce_over_ranks(world, "cpu", 10.0 + rank, 100.0 * (rank + 1),
                                                  (float(rank), 5.0 - rank))
        out[rank] = (t, units, tuple(extra))
    finally:
        dist.destroy_process_group()


def test_two_rank_reduction_over_gloo():
    world = 2
    out = mp.get_context("spawn").Manager().dict()   # no fork of this (threaded) process
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        t, units, extra = out[rank]
        assert t == 11.0                  # the slowest rank's time
        assert units == 300.0             # units of all ranks
        assert extra == (1.0, 5.0)        # worst latency percentiles


def test_single_rank_passes_values_through():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(1, "cpu", 3.5, 7.0, (1.0, 2.0)) == (3.5, 7.0, [1.0, 2.0])
    bench.dist_barrier(1)
    bench.dist_init(1, "cpu")
    bench.dist_done(1)


def test_reference_arm_other_ranks_exit_without_work():
    import sys
    sys.path.insert(0, ROOT)
    import bench

    class A:
        workload = "uniform_small"
        outputs = None
        steps = 1
        warmup = 3
    assert bench.run_reference(A(), 1, 2) == 0
