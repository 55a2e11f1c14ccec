"""Randomised slab decompositions (ranks as threads) against the direct update, bit for bit."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import slab

hypothesis = pytest.importorskip("hypothesis")
st = hypothesis.strategies


@hypothesis.settings(max_examples=40, deadline=None)
@hypothesis.given(nx=st.integers(1, 24), world=st.integers(1, 5), K=st.integers(1, 6), extra=st.integers(0, 12),
                  steps=st.integers(0, 15), bc=st.sampled_from([W.PERIODIC, W.DIRICHLET]),
                  prec=st.sampled_from(["f32", "f64"]), seed=st.integers(0, 10 ** 6))
def test_thread_ranks_random_shapes(nx, world, K, extra, steps, bc, prec, seed):
    ny = world * K + extra  # every rank owns at least K rows
    g = W.random_grid(seed, nx, ny, steps, bc)
    res = slab.run_threads(g.u, g.kappa, g.src, steps, g.dt, bc, K, world, prec)
    assert np.array_equal(res, oracle.direct(g.u, g.kappa, g.src, steps, g.dt, bc, prec))
