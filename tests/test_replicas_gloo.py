"""The multi-GPU bench path runs independent replicas: per-rank times are
reduced with a MAX over ranks and the value is world x per-rank work / that
time.  This checks the reduction logic with two gloo ranks on the CPU."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    secs = [2.0, 3.0][rank]
    t = bench.max_over_ranks(secs, device="cpu", world=world)
    value = bench.replica_value(work_per_rank=10.0, seconds=t, world=world)
    out[rank] = (t, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_reduce_max_time():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert out[0] == out[1] == (3.0, 2 * 10.0 / 3.0)
