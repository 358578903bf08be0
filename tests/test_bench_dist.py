"""Replica aggregation of bench.py across ranks (world size 2, gloo, CPU):
whole-job throughput = units of all ranks / slowest rank's time, and the
max-over-ranks reduction every rank agrees on."""
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
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), SDSL_BENCH_BACKEND="gloo")
    sys.path.insert(0, ROOT)
    import bench

    ws, r, local = bench.dist_init(None)
    bench.barrier(ws)
    secs = 2.0 if r == 0 else 3.0           # rank 1 is the slowest
    value, slowest = bench.aggregate(ws, 5, secs)
    out[r] = (ws, value, slowest, bench.max_over_ranks(ws, float(r + 10)))
    import torch.distributed as dist

    dist.destroy_process_group()


def test_two_rank_aggregation():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    for r in (0, 1):
        ws, value, slowest, mx = out[r]
        assert ws == 2
        assert slowest == 3.0
        assert value == pytest.approx(10 / 3.0)   # 5 units per rank, 2 ranks, slowest 3 s
        assert mx == 11.0
