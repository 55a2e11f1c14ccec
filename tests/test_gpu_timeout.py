"""Failure detection without a GPU fault: a bounded device wait that runs out.

The TMA-ring kernels wait on an mbarrier per row slot.  The test hook withholds
the copies of one row (its slot's barrier is told the row's byte count, but no
copy is issued, so the phase never completes), with a short wait limit: the
kernel must record CPB_ERR_TIMEOUT in the device status word, drain its own
copies and return; the context stays usable.
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
cpb = pytest.importorskip("paper_2206_07896_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.mark.parametrize("depth,bc", [(4, W.PERIODIC), (8, W.PERIODIC),   # single rows / rows in pairs
                                      (4, W.DIRICHLET), (8, W.DIRICHLET)])
def test_wait_timeout_is_reported_and_context_survives(dev, depth, bc):
    L = cpb.lib(fma=False)
    g = W.random_grid(3, 256, 64, depth, bc)
    u = torch.from_numpy(g.u).to(dev)
    k = torch.from_numpy(g.kappa).to(dev)
    s = torch.from_numpy(g.src).to(dev)
    t = {"k": depth, "chunk_rows": 16, "warps_per_block": 4, "variant": 1, "stages": 4}
    assert L.cpb_device_status() == 0
    out = torch.empty_like(u)
    try:
        L.cpb_debug_set(2000, 10)      # short wait; row 10's copies never complete
        L.cpb_stencil_launch_tuned(u, out, k, s, g.nx, g.ny, g.steps, float(g.dt), g.bc,
                                   cpb.CPB_F32, tuning=t, scratch=torch.empty_like(u))
        assert L.cpb_device_status() == cpb.CPB_ERR_TIMEOUT
    finally:
        L.cpb_debug_set(0, -1)
    assert L.cpb_device_status() == 0   # cleared by the read
    # The context is still usable and the next run is correct.
    L.cpb_stencil_launch_tuned(u, out, k, s, g.nx, g.ny, g.steps, float(g.dt), g.bc, cpb.CPB_F32,
                               tuning=t, scratch=torch.empty_like(u))
    torch.cuda.synchronize()
    ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, g.bc, "f32")
    np.testing.assert_array_equal(out.cpu().numpy(), ref)
    assert L.cpb_device_status() == 0
