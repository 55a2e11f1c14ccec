"""Multi-rank logic of bench.py on CPU (gloo, world size 2).

On this pool every box has one GPU, so the N-GPU bench runs N independent
replicas (no data-path collective); what needs checking is the host side:
the barrier, the max-over-ranks reduction of the step time, and the whole-job
throughput = all ranks' updates / max time.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    per_rank_ms = [12.0, 20.0][rank]            # rank 1 is the slow one
    t = torch.tensor([per_rank_ms])
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    updates = 8192 * 8192 * 1000
    value, tmax = bench.aggregate([float(t.item())] * world, [updates] * world)
    q.put((rank, float(t.item()), value, tmax))
    dist.destroy_process_group()


def test_two_rank_max_time_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tmax, value, tm in out:
        assert tmax == 20.0 and tm == 20.0
        assert value == pytest.approx(2 * 8192 * 8192 * 1000 / 20e-3 / 1e9)


def test_aggregate_single_rank():
    v, t = bench.aggregate([5.0], [10 ** 9])
    assert t == 5.0 and v == pytest.approx(200.0)
