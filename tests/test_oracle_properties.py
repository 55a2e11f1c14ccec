"""Randomised properties of the oracle's executors (CPU; skipped where
hypothesis is not installed).

Every executor of the paper's execution model -- the tiled kernel run with
loop fission on the thread pool (Sec. III "SPMD to MPMD", Sec. IV), the warp-level strip
kernel (nested warp / lane loops split at every shuffle, Sec. III "SPMD to MPMD"), the
3-D z-marching kernel with barriers inside its plane loop and the
temporal-blocked tile with a barrier per time step -- must equal the
direct loop (the stencil's definition) bit for bit for any grid shape, launch
geometry, pool size, grain and depth.
"""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")

import oracle  # noqa: E402
import workloads as W  # noqa: E402

given, settings = hyp.given, hyp.settings
bcs = st.sampled_from([W.DIRICHLET, W.PERIODIC])


@settings(max_examples=40, deadline=None)
@given(nx=st.integers(1, 70), ny=st.integers(1, 40), steps=st.integers(0, 6), bc=bcs,
       bx=st.integers(1, 33), by=st.integers(1, 9), pool=st.integers(1, 5), grain=st.integers(0, 7),
       seed=st.integers(0, 2 ** 16))
def test_fission_equals_direct(nx, ny, steps, bc, bx, by, pool, grain, seed):
    g = W.random_grid(seed, nx, ny, steps, bc)
    ref = oracle.direct(g.u, g.kappa, g.src, steps, g.dt, bc, "f32")
    got = oracle.fission(g.u, g.kappa, g.src, steps, g.dt, bc, "f32", block=(bx, by), pool=pool,
                         block_per_fetch=grain)
    np.testing.assert_array_equal(got, ref)


@settings(max_examples=40, deadline=None)
@given(nx=st.integers(1, 300), ny=st.integers(1, 30), steps=st.integers(0, 9), bc=bcs,
       k=st.integers(1, 8), chunk=st.integers(1, 40), warps=st.integers(1, 4), pool=st.integers(1, 4),
       seed=st.integers(0, 2 ** 16))
def test_strip_warp_equals_direct(nx, ny, steps, bc, k, chunk, warps, pool, seed):
    g = W.random_grid(seed, nx, ny, steps, bc)
    ref = oracle.direct(g.u, g.kappa, g.src, steps, g.dt, bc, "f32")
    got = oracle.strip_warp(g.u, g.kappa, g.src, steps, g.dt, bc, "f32", k=k, chunk=chunk, warps=warps,
                            pool=pool)
    np.testing.assert_array_equal(got, ref)


@settings(max_examples=30, deadline=None)
@given(nx=st.integers(1, 40), ny=st.integers(1, 20), nz=st.integers(1, 12), steps=st.integers(0, 4),
       bc=bcs, bx=st.integers(1, 33), by=st.integers(1, 9), zc=st.integers(1, 6), pool=st.integers(1, 4),
       seed=st.integers(0, 2 ** 16))
def test_fission3_equals_direct3(nx, ny, nz, steps, bc, bx, by, zc, pool, seed):
    g = W.random_grid3(seed, nx, ny, nz, steps, bc)
    ref = oracle.direct3(g.u, g.kappa, g.src, steps, g.dt, bc, "f32")
    got = oracle.fission3(g.u, g.kappa, g.src, steps, g.dt, bc, "f32", block=(bx, by), zchunks=min(zc, nz),
                          pool=pool)
    np.testing.assert_array_equal(got, ref)


@settings(max_examples=30, deadline=None)
@given(nx=st.integers(1, 60), ny=st.integers(1, 30), steps=st.integers(0, 9), bc=bcs, depth=st.integers(1, 8),
       bx=st.integers(1, 33), by=st.integers(1, 9), pool=st.integers(1, 4), seed=st.integers(0, 2 ** 16))
def test_tile_blocked_equals_direct(nx, ny, steps, bc, depth, bx, by, pool, seed):
    g = W.random_grid(seed, nx, ny, steps, bc)
    ref = oracle.direct(g.u, g.kappa, g.src, steps, g.dt, bc, "f32")
    got = oracle.tile_blocked(g.u, g.kappa, g.src, steps, g.dt, bc, "f32", depth=depth, block=(bx, by),
                              pool=pool)
    np.testing.assert_array_equal(got, ref)
