"""bench.py's replica mode (--gpus N) across ranks, on CPU with the gloo backend: every rank
times its own copy of the workload, the reported step time is the slowest rank's and the
value counts the units of all ranks.  Two processes rendezvous on 127.0.0.1."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    ms, kms, value = bench.aggregate_over_ranks(10.0 * (rank + 1), 5.0 + rank, 1000, world, dist, "cpu")
    out.put((rank, ms, kms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_is_the_slowest_rank_and_units_add_up():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, kms, value in res:
        assert ms == pytest.approx(20.0) and kms == pytest.approx(6.0)
        assert value == pytest.approx(1000 * 2 / 20e-3)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks(4.0, 3.0, 500, 1, None, "cpu") == (4.0, 3.0, pytest.approx(500 / 4e-3))
