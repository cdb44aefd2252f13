"""The multi-rank timing of bench.py (independent replicas, slowest rank) on CPU gloo ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r pretends its timed steps took 100 + 10 r ms in total
    t = bench.max_over_ranks(100.0 + 10.0 * rank, dist)
    value = bench.job_throughput(1000, world, 4, t)
    out[rank] = (t, value)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value_on_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, v = res[r]
        assert t == 110.0                               # the slowest rank
        assert v == pytest.approx(1000 * 2 * 4 / 0.110)


def test_single_process_passes_values_through():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_throughput(10, 1, 2, 1000.0) == pytest.approx(20.0)
