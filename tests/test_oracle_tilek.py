"""Pins for the multi-barrier kernel in the oracle: the shared-memory
temporal-blocked tiled kernel (depth steps per launch, depth + 1 barriers,
depth of them inside its time loop -- the paper's srad class has nine block
synchronisations, Sec. V) executed with loop fission (Sec. III "SPMD to MPMD"): the time
loop is kept and each barrier-free region inside it becomes a thread loop.

Pinned to the direct loop bit for bit over depths, block shapes, ragged
grids, pools and both boundaries, and to the failure of the same kernel run
without the split at its barriers.
"""
import numpy as np
import pytest

import oracle
import workloads as W


@pytest.mark.parametrize("bc", [W.DIRICHLET, W.PERIODIC])
@pytest.mark.parametrize("shape,block,depth,steps", [((100, 37), (16, 8), 3, 7), ((64, 64), (32, 8), 8, 17),
                                                     ((7, 3), (16, 16), 5, 5), ((1, 1), (4, 4), 2, 3),
                                                     ((130, 45), (8, 4), 1, 4), ((33, 90), (32, 2), 8, 8)])
def test_tile_blocked_equals_direct(bc, shape, block, depth, steps):
    nx, ny = shape
    g = W.random_grid(nx + 3 * ny + depth, nx, ny, steps, bc)
    ref = oracle.direct(g.u, g.kappa, g.src, steps, g.dt, bc, "f32")
    got = oracle.tile_blocked(g.u, g.kappa, g.src, steps, g.dt, bc, "f32", depth=depth, block=block, pool=3)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("bc", [W.DIRICHLET, W.PERIODIC])
def test_tile_blocked_f64(bc):
    g = W.random_grid(77, 90, 50, 11, bc)
    u, k, s = (x.astype(np.float64) for x in (g.u, g.kappa, g.src))
    np.testing.assert_array_equal(
        oracle.tile_blocked(u, k, s, 11, float(g.dt), bc, "f64", depth=4, block=(16, 16), pool=2),
        oracle.direct(u, k, s, 11, float(g.dt), bc, "f64"))


@pytest.mark.parametrize("depth", [1, 4])
def test_tile_blocked_without_split_at_barriers_is_wrong(depth):
    # All regions of a thread before the next thread starts: a thread reads
    # tile positions that later threads have not staged or updated yet.
    g = W.random_grid(78, 60, 40, 2 * depth, W.PERIODIC)
    ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, g.bc, "f32")
    got = oracle.tile_blocked(g.u, g.kappa, g.src, g.steps, g.dt, g.bc, "f32", depth=depth, block=(16, 8),
                              fission=False)
    assert not np.array_equal(got, ref)
