"""Argument validation of the C ABI, on the CPU.

Every entry point checks its arguments before any CUDA call, so the error
paths can be exercised without a GPU: the pointers below are fake device
addresses (never dereferenced), aligned or misaligned on purpose.  The host
queue order of the batched launch (LPT) needs no GPU either.
"""
import ctypes as C

import pytest

cpb = pytest.importorskip("paper_2206_07896_gb300")

U, O, K, S, X = 0x10000, 0x20000000, 0x40000000, 0x60000000, 0x70000000   # 256-byte aligned
INV, UNS, SHM, WS = (cpb.CPB_ERR_INVALID_VALUE, cpb.CPB_ERR_UNSUPPORTED_CONFIG, cpb.CPB_ERR_SHARED_MEM,
                     cpb.CPB_ERR_WORKSPACE)
D, P, F32, BF = cpb.CPB_DIRICHLET0, cpb.CPB_PERIODIC, cpb.CPB_F32, cpb.CPB_BF16_KAHAN


@pytest.fixture(scope="module")
def L():
    return cpb.Library(cpb.build.lib_path("libcpb.so"))


def status(fn, *args, **kw):
    with pytest.raises(cpb.CpbError) as e:
        fn(*args, **kw)
    return e.value.status


def test_stencil_launch_validation(L):
    g, b, shm = (4, 4, 1), (16, 16, 1), 2 * 18 * 18 * 4
    f = L.cpb_stencil_launch
    assert status(f, U, O, K, S, 0, 64, 1, 0.1, D, F32, g, b, shm, stream=0) == INV         # nx < 1
    assert status(f, U, O, K, S, 64, 64, -1, 0.1, D, F32, g, b, shm, stream=0) == INV       # steps < 0
    assert status(f, U, O, K, S, 64, 64, 1, 0.0, D, F32, g, b, shm, stream=0) == INV        # dt <= 0
    assert status(f, U, O, K, S, 64, 64, 1, float("nan"), D, F32, g, b, shm, stream=0) == INV
    assert status(f, U, O, K, S, 64, 64, 1, 0.1, 7, F32, g, b, shm, stream=0) == INV        # boundary
    assert status(f, U, O, K, S, 64, 64, 1, 0.1, D, 9, g, b, shm, stream=0) == INV          # storage
    assert status(f, None, O, K, S, 64, 64, 1, 0.1, D, F32, g, b, shm, stream=0) == INV     # null u_in
    assert status(f, U, U + 64, K, S, 64, 64, 1, 0.1, D, F32, g, b, shm, stream=0) == INV   # overlap
    assert status(f, U + 2, O, K, S, 64, 64, 1, 0.1, D, F32, g, b, shm, stream=0) == INV    # misaligned
    assert status(f, U, O, K, S, 64, 64, 1, 0.1, D, F32, g, (16, 16, 2), shm, stream=0) == UNS
    assert status(f, U, O, K, S, 64, 64, 1, 0.1, D, F32, g, (64, 32, 1), 1 << 20, stream=0) == UNS
    assert status(f, U, O, K, S, 64, 64, 1, 0.1, D, F32, (5, 4, 1), b, shm, stream=0) == INV  # grid
    assert status(f, U, O, K, S, 64, 64, 1, 0.1, D, F32, g, b, shm - 1, stream=0) == SHM
    assert status(f, U, O, K, None, 64, 64, 1, 0.1, D, F32, g, b, shm, stream=0) == INV     # tiled: src
    assert status(f, U, O, K, S, 64, 64, 1, 0.1, D, BF, g, b, shm, stream=0) == UNS         # tiled: f32


def test_tuned_launch_and_tuning_validation(L):
    bad = {"k": 9, "chunk_rows": 64, "warps_per_block": 1, "variant": 1, "stages": 2}
    assert status(L.cpb_stencil_launch_tuned, U, O, K, S, 64, 64, 4, 0.1, D, F32, tuning=bad, stream=0) == UNS
    for t in ({"k": 4, "chunk_rows": 0, "warps_per_block": 1, "variant": 1, "stages": 2},
              {"k": 4, "chunk_rows": 64, "warps_per_block": 9, "variant": 1, "stages": 2},
              {"k": 4, "chunk_rows": 64, "warps_per_block": 1, "variant": 1, "stages": 3},
              {"k": 4, "chunk_rows": 64, "warps_per_block": 1, "variant": 2, "stages": 2}):
        assert status(L.cpb_set_tuning, 64, 64, F32, D, t) == INV
    assert status(L.cpb_set_tuning, 0, 64, F32, D, {"k": 4, "chunk_rows": 64}) == INV


def test_3d_and_tile_blocked_validation(L):
    shm3 = L.cpb_stencil3d_shared_bytes(8)
    f3 = L.cpb_stencil3d_launch
    assert status(f3, U, O, K, S, 64, 8, 0, 1, 0.1, D, (1, 1, 1), (32, 8, 1), shm3, stream=0) == INV
    assert status(f3, U, O, K, S, 64, 8, 4, 1, 0.1, D, (1, 1, 1), (16, 8, 1), shm3, stream=0) == UNS
    assert status(f3, U, O, K, S, 64, 8, 4, 1, 0.1, D, (1, 1, 5), (32, 8, 1), shm3, stream=0) == INV
    assert status(f3, U, O, K, S, 64, 8, 4, 1, 0.1, D, (1, 1, 1), (32, 8, 1), shm3 - 1, stream=0) == SHM
    fb = L.cpb_stencil_tile_blocked
    shmb = L.cpb_tile_blocked_shared_bytes(16, 16, 2)
    assert status(fb, U, O, K, S, 64, 32, 2, 0, 0.1, D, (4, 2, 1), (16, 16, 1), shmb, stream=0) == INV
    assert status(fb, U, O, K, S, 64, 32, 2, 2, 0.1, D, (4, 2, 1), (16, 16, 1), shmb - 1, stream=0) == SHM
    assert status(fb, U, O, K, S, 64, 32, 2, 2, 0.1, D, (4, 3, 1), (16, 16, 1), shmb, stream=0) == INV
    big = L.cpb_tile_blocked_shared_bytes(32, 32, 16)
    assert big == 16 * 64 * 64 and L.cpb_tile_blocked_shared_bytes(32, 32, 17) == 0


def test_heat_sum_adjoint_host_validation(L):
    wsb = L.cpb_heat_sum_workspace_bytes(64, 64)
    assert status(L.cpb_heat_sum, U, 64, 64, F32, None, X, wsb, stream=0) == INV            # null out
    assert status(L.cpb_heat_sum, U, 64, 64, F32, O, None, 0, stream=0) == WS               # no workspace
    assert status(L.cpb_heat_sum, U, 64, 64, F32, O, X, wsb - 8, stream=0) == WS
    assert status(L.cpb_heat_sum_noalloc, U, 16384, 8192, F32, O, stream=0) == WS           # > 2^26 cells
    awsb = L.cpb_adjoint_workspace_bytes(64, 64, 10, 5)
    assert awsb > 0
    assert status(L.cpb_adjoint_forward, U, K, None, 64, 64, 10, 0.1, D, 0, O, X, awsb, stream=0) == INV
    assert status(L.cpb_adjoint_forward, U, K, None, 64, 64, 10, 0.1, D, 5, O, X, awsb - 1, stream=0) == WS
    assert status(L.cpb_adjoint_forward, U, K, None, 64, 64, 10, 0.1, D, 5, O, X + 16, awsb, stream=0) == WS
    hwsb = L.cpb_host_workspace_bytes(64, 64, F32)
    assert hwsb > 0
    import numpy as np
    h = np.zeros((64, 64), np.float32)
    assert status(L.cpb_stencil_host, h, h, h, h, 64, 64, 1, 0.1, D, F32, X, hwsb - 1, stream=0) == WS


def test_batch_order_is_host_only_lpt(L):
    n = 6
    descs = (cpb.cpb_grid_desc * n)()
    shapes = [(32, 32, 10), (100, 80, 50), (8, 8, 300), (64, 64, 64), (200, 10, 5), (16, 16, 16)]
    for i, (nx, ny, st) in enumerate(shapes):
        descs[i] = cpb.cpb_grid_desc(U + i * 0x100000, O + i * 0x100000, K + i * 0x100000, None, nx, ny, st, 0.1)
    order, n_large = L.cpb_batch_order(descs, {"grain": 1, "team_cells": 1000})
    cost = [nx * ny * st for nx, ny, st in shapes]
    large = [i for i in range(n) if shapes[i][0] * shapes[i][1] >= 1000]
    assert n_large == len(large) and sorted(order[:n_large]) == sorted(large)
    assert all(cost[a] >= cost[b] for a, b in zip(order[:n_large], order[1:n_large]))
    assert all(cost[a] >= cost[b] for a, b in zip(order[n_large:], order[n_large + 1:]))
    descs[3].dt = -1.0
    assert status(L.cpb_batch_order, descs, None) == INV
    assert status(L.cpb_batch_order, descs, {"grain": 0}) == INV
    assert status(L.cpb_batch_order, descs, {"grain": 1, "depth": 8, "threads": 384}) == INV
    descs[3].dt = 0.1
    # multi-warp teams must tile the CTA: a divisor of its warps, at most 15 teams
    for threads, tw in ((384, 4), (384, 3), (384, 12), (256, 2), (128, 4), (384, 1), (384, 0)):
        L.cpb_batch_order(descs, {"grain": 1, "threads": threads, "team_warps": tw})
    for threads, tw in ((384, 5), (384, 13), (256, 3), (128, 8)):
        assert status(L.cpb_batch_order, descs, {"grain": 1, "threads": threads, "team_warps": tw}) == INV
    assert L.cpb_batch_plan_default()["team_warps"] == 1


def test_slab_rows_match_the_row_split(L):
    # The library's split rule against the slab decomposition of the oracle's
    # CPU ranks (sizes differ by at most one, in rank order) and the halo rule.
    from oracle.slab import split_rows
    for ny in (8, 15, 61, 100, 1000):
        for world in (1, 2, 3, 5):
            for depth in (1, 2, 3):
                if world * depth > ny:
                    assert status(L.cpb_slab_rows, ny, world, 0, depth, D) == INV
                    continue
                parts = split_rows(ny, world)
                for rank in range(world):
                    for bc in (D, P):
                        r = L.cpb_slab_rows(ny, world, rank, depth, bc)
                        assert (r["row_lo"], r["row_hi"]) == parts[rank]
                        assert r["halo_lo"] == (depth if (bc == P or rank > 0) else 0)
                        assert r["halo_hi"] == (depth if (bc == P or rank < world - 1) else 0)
    assert status(L.cpb_slab_rows, 10, 2, 2, 1, D) == INV
    assert status(L.cpb_slab_rows, 10, 2, 0, 0, D) == INV
    assert status(L.cpb_slab_rows, 10, 2, 0, 1, 7) == INV


def test_slab_exchange_and_step_validation(L):
    assert status(L.cpb_slab_exchange, None, 64, 10, 2, 2, U, 2, 10, U, 2, 10, F32, stream=0) == INV
    assert status(L.cpb_slab_exchange, X, 64, 10, 2, 2, None, 2, 10, U, 2, 10, F32, stream=0) == INV
    assert status(L.cpb_slab_exchange, X, 64, 10, 2, 2, U, 2, 1, U, 2, 10, F32, stream=0) == INV  # neighbour too small
    assert status(L.cpb_slab_exchange, X, 64, 10, 11, 0, U, 2, 20, None, 0, 0, F32, stream=0) == INV
    assert status(L.cpb_slab_exchange, X, 64, 10, 2, 2, U, 2, 10, U, 2, 10, 9, stream=0) == INV
    # the exchange by row size: the same checks, and a row of at least one byte
    assert status(L.cpb_slab_exchange_rows, X, 0, 10, 2, 2, U, 2, 10, U, 2, 10, stream=0) == INV
    assert status(L.cpb_slab_exchange_rows, None, 128, 10, 2, 2, U, 2, 10, U, 2, 10, stream=0) == INV
    assert status(L.cpb_slab_exchange_rows, X, 128, 10, 2, 2, U, 2, 1, U, 2, 10, stream=0) == INV
    assert status(L.cpb_slab_exchange_rows, X, 128, 10, 2, 2, None, 2, 10, U, 2, 10, stream=0) == INV
    assert status(L.cpb_slab_exchange_rows, X, 128, 10, 11, 0, U, 2, 20, None, 0, 0, stream=0) == INV
    assert status(L.cpb_slab_step, U, O, K, S, 64, 14, 2, 2, 3, 0.1, D, F32, stream=0) == INV      # steps > halo
    assert status(L.cpb_slab_step, U, O, K, S, 64, 14, 2, 2, 0, 0.1, D, F32, stream=0) == INV
    assert status(L.cpb_slab_step, U, O, K, S, 64, 4, 2, 2, 1, 0.1, D, F32, stream=0) == INV       # no own rows
    assert status(L.cpb_slab_step, U, U, K, S, 64, 14, 2, 2, 2, 0.1, D, F32, stream=0) == INV      # in place


def test_bf16_block_dtype_is_accepted_and_validated(L):
    BB = cpb.CPB_BF16_KAHAN_BLOCK
    assert status(L.cpb_stencil_launch_tuned, U, U, K, S, 64, 32, 4, 0.1, D, BB, stream=0) == INV   # in place
    assert status(L.cpb_stencil_launch_tuned, U, O, K, S, 64, 32, 4, 0.1, D, 3, stream=0) == INV    # unknown dtype
    assert status(L.cpb_stencil_launch, U, O, K, S, 64, 32, 4, 0.1, D, BB, (4, 2, 1), (16, 16, 1),
                  2 * 18 * 18 * 4, stream=0) == UNS                                            # tiled kernel: FP32 only
    assert L.cpb_host_workspace_bytes(64, 64, BB) == L.cpb_host_workspace_bytes(64, 64, BF)
