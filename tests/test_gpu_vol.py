"""GPU parity of the 3-D 7-point variant (cpb_stencil3d_launch) against the oracle.

The --fmad=false build must equal the oracle's FP32 3-D update bit for bit on
every launch geometry (ragged tiles in x and y, z-chunks that split the
planes unevenly, both boundaries, with and without scratch, the 16-byte and
the scalar access paths); the default build stays within 1e-5 relative L-inf
of the FP64 oracle.
"""
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


def run3(L, g, dev, block=(0, 0, 0), zc=None, scratch=True, steps=None, src=True):
    steps = g.steps if steps is None else steps
    u = torch.from_numpy(g.u).to(dev)
    k = torch.from_numpy(g.kappa).to(dev)
    s = torch.from_numpy(g.src).to(dev) if src else None
    u_in, out = u.clone(), torch.empty_like(u)
    scr = torch.empty_like(u) if scratch else None
    if block == (0, 0, 0):
        grid, shm = (0, 0, 0), 0
    else:
        by = block[1]
        grid = ((g.nx + 127) // 128, (g.ny + by - 1) // by, zc)
        shm = L.cpb_stencil3d_shared_bytes(by)
    L.cpb_stencil3d_launch(u_in, out, k, s, g.nx, g.ny, g.nz, steps, float(g.dt), g.bc, grid, block, shm,
                           scratch=scr)
    torch.cuda.synchronize()
    if scratch:
        assert torch.equal(u_in, u)
    return out.cpu().numpy()


@pytest.mark.parametrize("bc", [D, P])
@pytest.mark.parametrize("shape,by,zc", [((200, 37, 19), 8, 3), ((130, 9, 5), 4, 2), ((256, 16, 40), 8, 7),
                                         ((1, 1, 1), 1, 1), ((52, 70, 3), 2, 3), ((384, 5, 9), 8, 1)])
@pytest.mark.parametrize("steps", [1, 4])
def test_vol_bit_exact(dev, bc, shape, by, zc, steps):
    L = cpb.lib(fma=False)
    nx, ny, nz = shape
    g = W.random_grid3(nx + 7 * ny + nz, nx, ny, nz, steps, bc)
    ref = oracle.direct3(g.u, g.kappa, g.src, steps, g.dt, bc, "f32")
    for scratch in (True, False):
        got = run3(L, g, dev, block=(32, by, 1), zc=zc, scratch=scratch)
        np.testing.assert_array_equal(got, ref, err_msg=f"{shape} by={by} zc={zc} scratch={scratch}")


@pytest.mark.parametrize("bc", [D, P])
def test_vol_default_geometry_and_null_source(dev, bc):
    L = cpb.lib(fma=False)
    g = W.random_grid3(41, 160, 44, 33, 3, bc)
    ref = oracle.fission3(g.u, g.kappa, g.src, g.steps, g.dt, bc, "f32", block=(32, 8), zchunks=4, pool=4)
    np.testing.assert_array_equal(run3(L, g, dev), ref)
    ref0 = oracle.direct3(g.u, g.kappa, np.zeros_like(g.src), g.steps, g.dt, bc, "f32")
    np.testing.assert_array_equal(run3(L, g, dev, src=False), ref0)


def test_vol_misaligned_takes_scalar_path(dev):
    L = cpb.lib(fma=False)
    g = W.random_grid3(42, 132, 10, 6, 2, D)
    ref = oracle.direct3(g.u, g.kappa, g.src, g.steps, g.dt, D, "f32")
    n = g.u.size
    buf = [torch.empty(n + 1, device=dev) for _ in range(4)]
    u, k, s, out = (b[1:] for b in buf)   # 4-byte aligned, not 16
    u.copy_(torch.from_numpy(g.u.reshape(-1)))
    k.copy_(torch.from_numpy(g.kappa.reshape(-1)))
    s.copy_(torch.from_numpy(g.src.reshape(-1)))
    L.cpb_stencil3d_launch(u, out, k, s, g.nx, g.ny, g.nz, g.steps, float(g.dt), D, (2, 2, 2), (32, 8, 1),
                           L.cpb_stencil3d_shared_bytes(8))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy().reshape(g.u.shape), ref)


@pytest.mark.parametrize("bc", [D, P])
def test_vol_fma_build_within_tolerance(dev, bc):
    g = W.random_grid3(43, 96, 96, 96, 200, bc)
    u, k, s = (x.astype(np.float64) for x in (g.u, g.kappa, g.src))
    ref = oracle.direct3(u, k, s, g.steps, float(g.dt), bc, "f64", pool=8)
    got = run3(cpb.lib(fma=True), g, dev)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err <= 1e-5, err


def test_vol_conservation_periodic(dev):
    g = W.random_grid3(44, 128, 64, 64, 300, P, zero_source=True)
    got = run3(cpb.lib(fma=True), g, dev)
    s0 = float(np.sum(g.u.astype(np.float64)))
    assert abs(float(np.sum(got.astype(np.float64))) - s0) <= 1e-6 * s0


def test_vol_error_codes(dev):
    L = cpb.lib(fma=False)
    g = W.random_grid3(45, 64, 8, 4, 1, D)
    u = torch.from_numpy(g.u).to(dev)
    k = torch.from_numpy(g.kappa).to(dev)
    out = torch.empty_like(u)

    def call(grid, block, shm, nx=64, ny=8, nz=4, steps=1, dt=0.1, uo=out):
        with pytest.raises(cpb.CpbError) as e:
            L.cpb_stencil3d_launch(u, uo, k, None, nx, ny, nz, steps, dt, D, grid, block, shm)
        return e.value.status

    shm = L.cpb_stencil3d_shared_bytes(8)
    assert shm > 0 and L.cpb_stencil3d_shared_bytes(9) == 0 and L.cpb_stencil3d_shared_bytes(0) == 0
    assert call((1, 1, 1), (33, 8, 1), shm) == cpb.CPB_ERR_UNSUPPORTED_CONFIG
    assert call((1, 1, 1), (32, 9, 1), 1 << 16) == cpb.CPB_ERR_UNSUPPORTED_CONFIG
    assert call((2, 1, 1), (32, 8, 1), shm) == cpb.CPB_ERR_INVALID_VALUE     # grid.x != ceil(nx/128)
    assert call((1, 1, 5), (32, 8, 1), shm) == cpb.CPB_ERR_INVALID_VALUE     # grid.z > nz
    assert call((1, 1, 1), (32, 8, 1), shm - 1) == cpb.CPB_ERR_SHARED_MEM
    assert call((1, 1, 1), (32, 8, 1), shm, nz=0) == cpb.CPB_ERR_INVALID_VALUE
    assert call((1, 1, 1), (32, 8, 1), shm, dt=-1.0) == cpb.CPB_ERR_INVALID_VALUE
    assert call((1, 1, 1), (32, 8, 1), shm, uo=u) == cpb.CPB_ERR_INVALID_VALUE  # in place
