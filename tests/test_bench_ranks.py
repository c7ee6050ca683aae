"""The multi-GPU form of the bench is replicas only: every rank solves its own
system and the job's time is the slowest rank's.  The rank bookkeeping and the
max-over-ranks reduction run here on CPU with two gloo ranks."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, values, out):
    import torch
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    ws, r, local = bench.dist_env()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out.put((rank, (ws, r, local), bench.max_over_ranks(values[rank], torch.device("cpu"))))
    finally:
        dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    values = [7.5, 9.25]
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, values, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [(2, 0, 0), (2, 1, 1)]
    assert [g[2] for g in got] == [9.25, 9.25]


def test_single_rank_is_the_identity():
    import torch

    import bench

    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        os.environ.pop(k, None)
    assert bench.dist_env() == (1, 0, 0)
    assert bench.max_over_ranks(3.0, torch.device("cpu")) == 3.0
