"""The paper's worked examples, stored as text fixtures under tests/golden/.

Each fixture line is a value the paper states for an example (its section and
figure or listing are named in the fixture's header); the oracle's executor
must reproduce it.
"""
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_runtime_opt_fetching_example():
    # Sec. IV "Runtime Optimizations", Fig. runtime_opt (a) and (b).
    rows = _rows("runtime_opt_fetching.txt")
    assert [r[0] for r in rows] == ["average", "aggressive"]
    for mode, grid, pool, bpf, fetches, used in rows:
        grid, pool, bpf, fetches, used = map(int, (grid, pool, bpf, fetches, used))
        grain = 0 if mode == "average" else bpf   # 0 selects ceil(grid / pool)
        if mode == "average":
            assert -(-grid // pool) == bpf
        rc, counts, got = oracle.fetch_accounting(grid, pool, grain)
        assert rc == 0 and np.all(counts == 1)
        assert got == fetches
        # each fetch is served by one worker, so at most `fetches` workers run
        assert min(pool, got) == used


def test_paper_listing_examples():
    rows = {r[0]: r[1:] for r in _rows("paper_listings.txt")}
    # vecAdd, Listings 1-2: grid 2 x block 2 covers ids 0..3.
    grid, block = int(rows["vecAdd"][0]), int(rows["vecAdd"][1])
    a = np.arange(grid * block, dtype=np.float64) + 1.0
    b = 10.0 * a
    np.testing.assert_array_equal(oracle.vecadd(a, b, grid=grid, block=block, pool=2), a + b)
    # dynamicReverse, Listing 3: <<<1, n, n * sizeof(int)>>>, one barrier ->
    # two regions; the fissioned run reverses, an unfissioned one does not.
    assert rows["dynamicReverse"][0] == "1" and rows["dynamicReverse"][1] == "n"
    assert int(rows["dynamicReverse"][3]) == 2
    for n in (3, 64):
        d = np.arange(n, dtype=np.int32) * 5 - 7
        np.testing.assert_array_equal(oracle.dynamic_reverse(d, fission=True), d[::-1])
        assert not np.array_equal(oracle.dynamic_reverse(d, fission=False), d[::-1])
