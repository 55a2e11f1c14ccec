"""Pins for the warp-level executor of the oracle.

Sec. III "SPMD to MPMD": a kernel that uses warp-level functions (shuffles) is wrapped in
nested loops -- an outer loop over the ceil(block_size / 32) warps of a block
and an inner loop over the 32 lanes of a warp -- split at every warp function.
The oracle runs the shuffle-based, temporal-blocked strip kernel (a warp per
128-column strip, 4 cells per lane, K time levels per pass, x-neighbours of a
lane's edge cells by shuffle) that way.  Pinned here to the direct loop (the
stencil's definition, itself pinned in test_oracle_pins.py) bit for bit, and
to the failure of the same kernel when the lane loops are not split at the
shuffles.
"""
import numpy as np
import pytest

import oracle
import workloads as W


@pytest.mark.parametrize("nx,ny,bc", [(300, 97, W.PERIODIC), (300, 97, W.DIRICHLET),
                                      (129, 40, W.DIRICHLET), (520, 33, W.PERIODIC),
                                      (50, 7, W.PERIODIC), (50, 7, W.DIRICHLET),
                                      (1, 1, W.DIRICHLET), (5, 300, W.PERIODIC)])
@pytest.mark.parametrize("k", [1, 2, 4, 7, 8])
def test_strip_warp_equals_direct_f32(nx, ny, bc, k):
    g = W.random_grid(11, nx, ny, 2 * k + 1, bc)
    ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, g.bc, "f32")
    got = oracle.strip_warp(g.u, g.kappa, g.src, g.steps, g.dt, g.bc, "f32", k=k, chunk=16, warps=2,
                            pool=3)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("bc", [W.PERIODIC, W.DIRICHLET])
def test_strip_warp_equals_direct_f64(bc):
    g = W.random_grid(12, 260, 45, 9, bc)
    u, k, s = (x.astype(np.float64) for x in (g.u, g.kappa, g.src))
    ref = oracle.direct(u, k, s, g.steps, float(g.dt), g.bc, "f64")
    got = oracle.strip_warp(u, k, s, g.steps, float(g.dt), g.bc, "f64", k=4, chunk=10, warps=3, pool=2)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("chunk,warps,pool", [(1, 1, 1), (7, 4, 5), (1000, 32, 2)])
def test_strip_warp_geometry_does_not_change_bits(chunk, warps, pool):
    # Chunk height, warps per block and pool size only regroup the same cells.
    g = W.random_grid(13, 777, 61, 10, W.PERIODIC)
    ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, g.bc, "f32")
    got = oracle.strip_warp(g.u, g.kappa, g.src, g.steps, g.dt, g.bc, "f32", k=3, chunk=chunk,
                            warps=warps, pool=pool)
    np.testing.assert_array_equal(got, ref)


def test_strip_warp_zero_steps_is_identity():
    g = W.random_grid(14, 64, 9, 0, W.DIRICHLET)
    got = oracle.strip_warp(g.u, g.kappa, g.src, 0, g.dt, g.bc, "f32", k=4)
    np.testing.assert_array_equal(got, g.u)


@pytest.mark.parametrize("bc", [W.PERIODIC, W.DIRICHLET])
def test_strip_warp_without_split_at_shuffles_is_wrong(bc):
    # One lane loop per section, not split at the shuffles: a lane reads its
    # east neighbour's exchange slot before that lane has written it.
    g = W.random_grid(15, 300, 40, 6, bc)
    ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, g.bc, "f32")
    got = oracle.strip_warp(g.u, g.kappa, g.src, g.steps, g.dt, g.bc, "f32", k=3, fission=False)
    assert not np.array_equal(got, ref)


def test_strip_warp_rejects_depth_beyond_its_rings():
    g = W.random_grid(16, 64, 9, 9, W.PERIODIC)
    with pytest.raises(RuntimeError):
        oracle.strip_warp(g.u, g.kappa, g.src, 9, g.dt, g.bc, "f32", k=9)
