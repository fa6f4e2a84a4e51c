"""The N > 1 replica path of bench.py on CPU (gloo, world_size 2).

bench.py runs one independent replica per GPU (the method needs no exchange
between replicas on this path) and reports the whole job: units summed over
ranks, time = the slowest rank. This checks that aggregation with real
processes and a real process group; no GPU is used.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [4.0, 7.5][rank]          # per-rank step time
    cells = [1.0e10, 1.2e10][rank]  # per-rank work
    out[rank] = bench.aggregate_ranks(ms, cells, dist)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        ms, cells, world = out[r]
        assert world == 2
        assert ms == pytest.approx(7.5)           # the slowest rank
        assert cells == pytest.approx(2.2e10)     # every rank's work


def test_single_process_aggregation_is_identity():
    import bench
    assert bench.aggregate_ranks(3.0, 5.0, None) == (3.0, 5.0, 1)
