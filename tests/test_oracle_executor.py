"""Pins for the oracle's execution model (the paper's CPU runtime).

The executor follows the paper's SPMD-to-MPMD scheme (Sec. III "SPMD to MPMD": one loop over
a block's threads per barrier-free region) and its runtime (Sec. IV: thread pool,
mutex task queue of kernel structures, coarse-grained fetching).  Each test pins
it to a result fixed by definition, not by the oracle itself.
"""
import numpy as np
import pytest

import oracle


def test_vecadd_paper_example():
    # Listings 1-2: gridSize = 2, blockSize = 2, c = a + b.
    a = np.array([1.0, 2.0, 3.0, 4.0])
    b = np.array([10.0, 20.0, 30.0, 40.0])
    np.testing.assert_array_equal(oracle.vecadd(a, b, grid=2, block=2, pool=2), a + b)


@pytest.mark.parametrize("n,block,pool", [(1000, 64, 3), (777, 32, 5), (5, 8, 1)])
def test_vecadd_ragged(n, block, pool):
    rng = np.random.default_rng(n)
    a, b = rng.random(n), rng.random(n)
    grid = (n + block - 1) // block
    np.testing.assert_array_equal(oracle.vecadd(a, b, grid, block, pool), a + b)


@pytest.mark.parametrize("n", [1, 2, 7, 64, 256])
def test_dynamic_reverse_fissioned(n):
    # Listing 3: dynamic shared memory + one barrier reverses d.
    d = np.arange(n, dtype=np.int32) * 3 + 1
    np.testing.assert_array_equal(oracle.dynamic_reverse(d, fission=True), d[::-1])


@pytest.mark.parametrize("n", [2, 7, 64])
def test_dynamic_reverse_without_fission_is_wrong(n):
    # Ignoring the barrier (each thread runs both regions in turn) reads shared
    # slots before they are written: the result must differ from the reversal.
    d = np.arange(n, dtype=np.int32) * 3 + 1
    assert not np.array_equal(oracle.dynamic_reverse(d, fission=False), d[::-1])


@pytest.mark.parametrize("grid", [1, 7, 12, 100, 1000])
@pytest.mark.parametrize("pool", [1, 2, 3, 6])
def test_every_block_runs_once(grid, pool):
    avg = -(-grid // pool)  # average coarse-grained fetching: ceil(grid / pool)
    for grain in (1, 0, 2 * avg, grid):
        rc, counts, fetches = oracle.fetch_accounting(grid, pool, grain)
        assert rc == 0
        assert counts.shape == (grid,) and np.all(counts == 1)
        g = avg if grain == 0 else grain
        assert fetches == -(-grid // g)


def test_average_fetch_uses_pool_size_fetches():
    # Sec. IV: average coarse-grained fetching needs threadPoolSize fetches
    # (Fig. runtime_opt(a): grid 12, pool 3 -> 4 blocks per fetch, 3 fetches);
    # aggressive fetching with 6 blocks per fetch needs 2 (Fig. runtime_opt(b)).
    assert oracle.fetch_accounting(12, 3, 0)[2] == 3
    assert oracle.fetch_accounting(12, 3, 6)[2] == 2


def test_injected_block_error_propagates_without_deadlock():
    rc, counts, _ = oracle.fetch_accounting(50, 4, 3, fail_block=17)
    assert rc == 7
    assert np.all(counts == 1)          # the other blocks still ran exactly once
    rc2, counts2, _ = oracle.fetch_accounting(50, 4, 3)   # pool still usable
    assert rc2 == 0 and np.all(counts2 == 1)


def test_empty_grid():
    rc, counts, fetches = oracle.fetch_accounting(0, 3)
    assert rc == 0 and counts.size == 0 and fetches == 0
