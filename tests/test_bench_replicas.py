"""The multi-GPU path of bench.py is replicas (each rank advances its own system; nothing is
exchanged on the data path): two gloo ranks on the CPU check the timing reduction (the slowest
rank's time, max over ranks), the barrier, and the whole-job rate."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench._barrier(world)
    step_ms = [0.40, 0.55][rank]  # rank 1 is the slow replica
    t = bench._max_over_ranks(world, step_ms)
    out[rank] = (t, bench._job_rate(world, 786432, t))
    bench._barrier(world)
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, rate = res[r]
        assert t == pytest.approx(0.55)
        assert rate == pytest.approx(2 * 786432 / 0.55e-3)


def test_single_rank_is_identity():
    import bench
    assert bench._max_over_ranks(1, 0.37) == 0.37
    assert bench._job_rate(1, 1000, 1.0) == pytest.approx(1e6)
