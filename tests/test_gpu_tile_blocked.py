"""GPU parity of the multi-barrier kernel (cpb_stencil_tile_blocked): the
shared-memory temporal-blocked tile with a barrier after staging and after
every time step, on the caller's launch geometry.  --fmad=false build bit for
bit against the oracle (the direct loop and the same kernel run with loop
fission) over depths, block shapes, ragged grids, both boundaries and both
scratch modes; error codes."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
cpb = pytest.importorskip("paper_2206_07896_gb300")

pytestmark = pytest.mark.gpu
D, P = W.DIRICHLET, W.PERIODIC


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def run(L, g, dev, depth, block, steps=None, scratch=True, src=True):
    steps = g.steps if steps is None else steps
    u = torch.from_numpy(g.u).to(dev)
    k = torch.from_numpy(g.kappa).to(dev)
    s = torch.from_numpy(g.src).to(dev) if src else None
    u_in, out = u.clone(), torch.empty_like(u)
    scr = torch.empty_like(u) if scratch else None
    bx, by = block
    L.cpb_stencil_tile_blocked(u_in, out, k, s, g.nx, g.ny, steps, depth, float(g.dt), g.bc,
                               ((g.nx + bx - 1) // bx, (g.ny + by - 1) // by, 1), (bx, by, 1),
                               L.cpb_tile_blocked_shared_bytes(bx, by, depth), scratch=scr)
    torch.cuda.synchronize()
    if scratch:
        assert torch.equal(u_in, u)
    return out.cpu().numpy()


@pytest.mark.parametrize("bc", [D, P])
@pytest.mark.parametrize("shape,block,depth,steps", [((300, 97), (32, 8), 4, 9), ((100, 37), (16, 8), 3, 7),
                                                     ((64, 64), (32, 32), 8, 17), ((7, 3), (16, 16), 5, 5),
                                                     ((1, 1), (4, 4), 2, 3), ((130, 45), (8, 4), 1, 4),
                                                     ((257, 90), (64, 16), 16, 33)])
def test_tile_blocked_bit_exact(dev, bc, shape, block, depth, steps):
    L = cpb.lib(fma=False)
    nx, ny = shape
    g = W.random_grid(nx + 5 * ny + depth, nx, ny, steps, bc)
    ref = oracle.direct(g.u, g.kappa, g.src, steps, g.dt, bc, "f32")
    for scratch in (True, False):
        np.testing.assert_array_equal(run(L, g, dev, depth, block, scratch=scratch), ref)


@pytest.mark.parametrize("bc", [D, P])
def test_tile_blocked_matches_fission_executor_and_null_source(dev, bc):
    L = cpb.lib(fma=False)
    g = W.random_grid(91, 200, 150, 12, bc)
    ref = oracle.tile_blocked(g.u, g.kappa, g.src, 12, g.dt, bc, "f32", depth=6, block=(32, 8), pool=4)
    np.testing.assert_array_equal(run(L, g, dev, 6, (32, 8)), ref)
    ref0 = oracle.direct(g.u, g.kappa, np.zeros_like(g.src), 12, g.dt, bc, "f32")
    np.testing.assert_array_equal(run(L, g, dev, 6, (32, 8), src=False), ref0)


def test_tile_blocked_fma_build_within_tolerance(dev):
    g = W.random_grid(92, 512, 256, 400, P, r=0.24)
    ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, P, "f64", pool=8)
    got = run(cpb.lib(fma=True), g, dev, 8, (32, 16))
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 1e-5


def test_tile_blocked_error_codes(dev):
    L = cpb.lib(fma=False)
    g = W.random_grid(93, 64, 32, 2, D)
    u = torch.from_numpy(g.u).to(dev)
    k = torch.from_numpy(g.kappa).to(dev)
    out = torch.empty_like(u)

    def call(grid, block, shm, depth=2, uo=out):
        with pytest.raises(cpb.CpbError) as e:
            L.cpb_stencil_tile_blocked(u, uo, k, None, 64, 32, 2, depth, float(g.dt), D, grid, block, shm)
        return e.value.status

    shm = L.cpb_tile_blocked_shared_bytes(16, 16, 2)
    assert shm == 16 * 20 * 20
    assert call((4, 2, 1), (64, 32, 1), 1 << 20) == cpb.CPB_ERR_UNSUPPORTED_CONFIG   # 2048 threads
    assert call((3, 2, 1), (16, 16, 1), shm) == cpb.CPB_ERR_INVALID_VALUE            # grid.x wrong
    assert call((4, 2, 1), (16, 16, 1), shm - 1) == cpb.CPB_ERR_SHARED_MEM
    assert call((4, 2, 1), (16, 16, 1), shm, depth=0) == cpb.CPB_ERR_INVALID_VALUE
    assert call((4, 2, 1), (16, 16, 1), shm, depth=17) == cpb.CPB_ERR_INVALID_VALUE
    assert call((4, 2, 1), (16, 16, 1), shm, uo=u) == cpb.CPB_ERR_INVALID_VALUE        # in place
    assert L.cpb_tile_blocked_shared_bytes(32, 33, 1) == 0 and L.cpb_tile_blocked_shared_bytes(8, 8, 17) == 0
