"""Slab decomposition with halo exchange (the multi-GPU plan), on CPU ranks.

Every run here has one GPU, so the library has no multi-GPU path; the
decomposition itself is checked here, across torch.distributed gloo ranks
(processes) and across ranks run as threads of one process (randomised
shapes, rank counts, depths and boundaries).
Each rank owns a contiguous block of rows and exchanges K halo rows with its
neighbours every K steps.  The assembled result must equal the direct update
of the whole grid bit for bit, in FP32 and FP64, for periodic (a ring of
ranks) and Dirichlet boundaries, ragged row splits and a partial last block
of steps.  A run whose exchanges stop after the first block must not.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import workloads as W
from oracle import slab


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


# (seed, nx, ny, steps, bc, K, precision): row splits that are ragged, a last
# block shorter than K, and ranks that own exactly K rows.
CASES = {
    2: [(1, 41, 23, 10, W.PERIODIC, 3, "f32"), (2, 41, 23, 10, W.DIRICHLET, 3, "f32"),
        (3, 19, 16, 9, W.PERIODIC, 8, "f64"), (4, 33, 9, 7, W.DIRICHLET, 4, "f64"),
        (5, 7, 4, 5, W.PERIODIC, 2, "f32")],
    3: [(6, 17, 10, 7, W.PERIODIC, 3, "f32"), (7, 25, 31, 12, W.DIRICHLET, 5, "f32"),
        (8, 12, 9, 6, W.PERIODIC, 3, "f64")],
}


def _grid(case):
    seed, nx, ny, steps, bc, K, prec = case
    return W.random_grid(seed, nx, ny, steps, bc)


def _worker(rank, world, port, cases, skip_after, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for i, case in enumerate(cases):
            g = _grid(case)
            K, prec = case[5], case[6]
            ex = slab.TorchDistExchange(rank, world, g.bc == W.PERIODIC, skip_after=skip_after)
            own = slab.run_slab(g.u, g.kappa, g.src, g.steps, g.dt, g.bc, K, rank, world, ex, prec)
            q.put((i, rank, own))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _run_ranks(world, cases, skip_after=None):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, cases, skip_after, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(world * len(cases)):
        i, rank, own = q.get(timeout=180)
        got[(i, rank)] = own
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return [np.concatenate([got[(i, r)] for r in range(world)], axis=0) for i in range(len(cases))]


def _direct(case):
    g = _grid(case)
    return oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, g.bc, case[6])


@pytest.mark.parametrize("world", sorted(CASES))
def test_ranks_equal_direct_bit_for_bit(world):
    results = _run_ranks(world, CASES[world])
    for case, res in zip(CASES[world], results):
        ref = _direct(case)
        assert res.dtype == ref.dtype and res.shape == ref.shape
        assert np.array_equal(res, ref), f"world {world}, case {case}"


def test_exchange_that_stops_is_wrong():
    # κ and s are swapped once each, then one swap of u per block of K steps:
    # allowing 3 swaps keeps only the first block's u exchange.
    case = (9, 24, 12, 9, W.PERIODIC, 3, "f64")
    (res,) = _run_ranks(2, [case], skip_after=3)
    assert not np.array_equal(res, _direct(case))


@pytest.mark.parametrize("bc", [W.PERIODIC, W.DIRICHLET])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_single_rank_equals_direct(bc, prec):
    g = W.random_grid(10, 29, 13, 11, bc)
    own = slab.run_slab(g.u, g.kappa, g.src, g.steps, g.dt, g.bc, 4, 0, 1,
                        slab.LocalExchange(bc == W.PERIODIC), prec)
    assert np.array_equal(own, oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, g.bc, prec))


def test_single_rank_zero_steps_and_one_column():
    g = W.random_grid(11, 1, 6, 0, W.PERIODIC)
    own = slab.run_slab(g.u, g.kappa, g.src, 0, g.dt, g.bc, 2, 0, 1, slab.LocalExchange(True), "f32")
    assert np.array_equal(own, g.u)
    g = W.random_grid(12, 1, 6, 5, W.DIRICHLET)
    own = slab.run_slab(g.u, g.kappa, g.src, g.steps, g.dt, g.bc, 2, 0, 1, slab.LocalExchange(False), "f32")
    assert np.array_equal(own, oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, g.bc, "f32"))


def test_split_rows():
    assert slab.split_rows(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert slab.split_rows(5, 5) == [(i, i + 1) for i in range(5)]
    for ny, w in ((23, 2), (31, 3), (1000, 7)):
        parts = slab.split_rows(ny, w)
        sizes = [b - a for a, b in parts]
        assert parts[0][0] == 0 and parts[-1][1] == ny and max(sizes) - min(sizes) <= 1
        assert all(parts[i][1] == parts[i + 1][0] for i in range(w - 1))
    with pytest.raises(ValueError):
        slab.split_rows(2, 3)


def test_too_few_rows_per_rank_is_rejected():
    g = W.random_grid(13, 8, 5, 4, W.PERIODIC)
    with pytest.raises(ValueError):  # 2 + 3 rows over two ranks, K = 3
        slab.run_slab(g.u, g.kappa, g.src, 4, g.dt, g.bc, 3, 0, 2, slab.LocalExchange(True), "f32")
    with pytest.raises(ValueError):  # one periodic rank with fewer rows than K
        slab.run_slab(g.u, g.kappa, g.src, 4, g.dt, g.bc, 6, 0, 1, slab.LocalExchange(True), "f32")


def test_thread_ranks_equal_direct():
    # ranks as threads (mailbox per direction), a few fixed cases
    for seed, nx, ny, steps, bc, K, world, prec in [(20, 30, 17, 9, W.PERIODIC, 3, 4, "f32"),
                                                    (21, 9, 40, 13, W.DIRICHLET, 5, 7, "f64"),
                                                    (22, 64, 8, 6, W.PERIODIC, 4, 2, "f32")]:
        g = W.random_grid(seed, nx, ny, steps, bc)
        res = slab.run_threads(g.u, g.kappa, g.src, steps, g.dt, bc, K, world, prec)
        assert np.array_equal(res, oracle.direct(g.u, g.kappa, g.src, steps, g.dt, bc, prec))

