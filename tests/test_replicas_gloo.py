"""bench.py at N > 1 runs independent replicas: the whole-job time is the slowest rank's and
the work is every rank's.  Checked with two gloo ranks on the CPU (no GPU, no NCCL)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms, emb = bench.replica_totals(1000.0 + 250.0 * rank, 10 ** 9 * (rank + 1), world, "cpu")
        out[rank] = (ms, emb)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_max_time_and_summed_work():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, emb = res[rank]
        assert ms == 1250.0
        assert emb == 3.0e9
    # value = units all ranks processed / the whole job's time
    assert res[0][1] / (res[0][0] / 1e3) == pytest.approx(2.4e9)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_totals(5.0, 7, 1, "cpu") == (5.0, 7.0)
