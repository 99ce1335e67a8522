"""Host logic of bench.py's multi-process (replica) path, on CPU with two gloo ranks: the timed
region is the slowest rank's, and the whole-job throughput counts every rank's builds."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = 100.0 + 50.0 * rank            # rank 1 is the slower one
        ms_step, value = bench.job_throughput(ms_local, 5, world, 2.0e12, dist, "cpu")
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{ms_step!r} {value!r}\n")
    finally:
        dist.destroy_process_group()


def test_job_throughput_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        ms_step, value = map(float, (tmp_path / f"r{r}.txt").read_text().split())
        assert ms_step == pytest.approx(150.0 / 5)                   # the slowest rank's time
        assert value == pytest.approx(world * 2.0e12 / 0.030 / 1e12)  # both ranks' work


def test_job_throughput_one_process():
    sys.path.insert(0, ROOT)
    import bench
    ms_step, value = bench.job_throughput(200.0, 4, 1, 1.0e12)
    assert ms_step == 50.0 and value == pytest.approx(1.0e12 / 0.05 / 1e12)
