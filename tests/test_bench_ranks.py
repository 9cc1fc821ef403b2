"""The multi-replica path of bench.py on CPU: two gloo ranks, as torchrun would launch them on
two GPUs.  The whole-job time is the slowest rank's, entries add up, and every rank colours its
own trials."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, ent = bench.over_ranks(dist, torch, 100.0 + 50.0 * rank, 1000 * (rank + 1), "cpu")
        out.put((rank, ms, ent, bench.rank_seed(7, rank)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, ent, seed in res:
        assert ms == 150.0 and ent == 3000.0  # max of the times, sum of the entries
    assert res[0][3] != res[1][3]  # independent colourings per replica


def test_one_process():
    assert bench.over_ranks(None, torch, 12.5, 7, "cpu") == (12.5, 7.0)
