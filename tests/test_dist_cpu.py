"""Multi-process host logic of bench.py's replica path on CPU (gloo, world size 2):
max-over-ranks time, summed pivots, distinct problems per rank."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.reduce_max(10.0 + rank, torch.device("cpu"), world)
    piv = bench.reduce_sum(800 + rank, torch.device("cpu"), world)
    seed = bench.replica_seed("ks200k", rank)
    dist.barrier()
    q.put((rank, ms, piv, seed))
    dist.destroy_process_group()


def test_replica_aggregation_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(ms == 11.0 for _, ms, _, _ in res)          # max over ranks
    assert all(piv == 1601.0 for _, _, piv, _ in res)      # sum over ranks
    assert res[0][3] != res[1][3]                          # independent problem per rank


def test_single_process_is_identity():
    import bench
    assert bench.reduce_max(3.5, torch.device("cpu"), 1) == 3.5
    assert bench.reduce_sum(7, torch.device("cpu"), 1) == 7.0
