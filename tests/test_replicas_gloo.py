"""The multi-rank path of the benchmark, on CPU with gloo (world size 2).

With N GPUs every rank evaluates its own replica of the workload (the ranks
share nothing on the data path); the job's time is the slowest rank's, taken
by an all-reduce MAX after a barrier, and the reported value is the units of
all ranks over that time.  These tests run that host logic in two gloo
processes: the maximum reaches every rank, and the whole-job rate counts both
replicas.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, local_ms, out_dir):
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms_max = bench.max_over_ranks(local_ms[rank], dist, "cpu")
        rate = bench.whole_job_rate(1.0e9, world, ms_max)
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{ms_max!r} {rate!r}\n")
    finally:
        dist.destroy_process_group()


def test_slowest_rank_sets_the_time_and_rate_counts_all_replicas(tmp_path):
    world = 2
    local_ms = [3.0, 5.0]
    mp.spawn(_rank, args=(world, _free_port(), local_ms, str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        ms_max, rate = map(float, (tmp_path / f"rank{r}.txt").read_text().split())
        assert ms_max == 5.0
        assert rate == pytest.approx(world * 1.0e9 / 5.0e-3)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(4.5) == 4.5
    assert bench.whole_job_rate(2.0e9, 1, 4.0) == pytest.approx(5.0e11)
