"""GPU adjoint (FP32, checkpointed) against the FP64 CPU adjoint, and the autograd wrapper."""
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


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu_adjoint(L, g, dev, steps, ckpt, bc, lam_T, src=None):
    u0 = torch.from_numpy(g.u).to(dev)
    k = torch.from_numpy(g.kappa).to(dev)
    s = torch.from_numpy(src).to(dev) if src is not None else None
    lam = torch.from_numpy(lam_T.astype(np.float32)).to(dev)
    wsb = L.cpb_adjoint_workspace_bytes(g.nx, g.ny, steps, ckpt)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    gu, gk = torch.empty_like(u0), torch.empty_like(u0)
    L.cpb_stencil_adjoint(u0, k, s, lam, g.nx, g.ny, steps, float(g.dt), bc, ckpt, gu, gk, ws, wsb)
    torch.cuda.synchronize()
    return gu.cpu().numpy().astype(np.float64), gk.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("bc", [W.DIRICHLET, W.PERIODIC])
@pytest.mark.parametrize("shape,steps,ckpt", [((256, 192), 60, 7), ((130, 50), 23, 23),
                                              ((64, 64), 5, 20), ((1, 17), 9, 4)])
def test_adjoint_matches_fp64_oracle(dev, bc, shape, steps, ckpt):
    nx, ny = shape
    g = W.differentiation(seed=nx + ny, n=nx, ny=ny, steps=steps, ckpt=ckpt)
    tgt = g.extras["target"].astype(np.float64)
    s = np.zeros_like(g.u, dtype=np.float64)
    # lambda_T from the FP64 oracle's u_T, so both sides see the same lambda_T
    L64, gu_ref, gk_ref = oracle.adjoint_f64(g.u, g.kappa, s, tgt, steps, float(g.dt), bc, ckpt)
    uT = oracle.direct(g.u, g.kappa, s, steps, g.dt, bc, "f64")
    lam_T = uT - tgt
    for fma in (False, True):
        gu, gk = gpu_adjoint(cpb.lib(fma=fma), g, dev, steps, ckpt, bc, lam_T)
        assert rel_l2(gu, gu_ref) <= 1e-4
        assert rel_l2(gk, gk_ref) <= 1e-4


@pytest.mark.parametrize("with_src", [False, True])
@pytest.mark.parametrize("bc", [W.DIRICHLET, W.PERIODIC])
@pytest.mark.parametrize("nx,ny,steps,ckpts", [(200, 90, 31, (5, 31, 64)), (260, 70, 23, (2, 6, 23)),
                                               (130, 40, 11, (3, 11))])
def test_adjoint_checkpoint_interval_invariant(dev, bc, nx, ny, steps, ckpts, with_src):
    # Checkpoints every step recompute nothing; longer intervals recompute
    # each segment (depth-4 passes that store their levels where nx % 4 == 0,
    # one-step passes otherwise) and must give the same bits, with or
    # without a source term in the states.
    g = W.differentiation(seed=3, n=nx, ny=ny, steps=steps, ckpt=5)
    rng = np.random.default_rng(0)
    lam_T = rng.standard_normal(g.u.shape)
    src = (rng.random(g.u.shape, dtype=np.float32) * np.float32(1e-3)) if with_src else None
    L = cpb.lib(fma=False)  # the build whose rounding does not depend on the pass depth
    ref = gpu_adjoint(L, g, dev, steps, 1, bc, lam_T, src=src)
    for ck in ckpts:
        got = gpu_adjoint(L, g, dev, steps, ck, bc, lam_T, src=src)
        np.testing.assert_array_equal(got[0], ref[0])
        np.testing.assert_array_equal(got[1], ref[1])
    assert L.cpb_device_status() == 0


def test_autograd_function(dev):
    g = W.differentiation(seed=9, n=96, ny=80, steps=40, ckpt=10)
    tgt = torch.from_numpy(g.extras["target"]).to(dev)
    u0 = torch.from_numpy(g.u).to(dev).requires_grad_(True)
    k = torch.from_numpy(g.kappa).to(dev).requires_grad_(True)
    uT = cpb.StencilFn.apply(u0, k, None, 40, float(g.dt), W.DIRICHLET, 10)
    loss = 0.5 * ((uT - tgt) ** 2).sum()
    loss.backward()
    Lref, gu_ref, gk_ref = oracle.adjoint_f64(g.u, g.kappa, np.zeros_like(g.u, np.float64),
                                             g.extras["target"].astype(np.float64), 40,
                                             float(g.dt), W.DIRICHLET, 10)
    assert abs(float(loss) - Lref) <= 1e-5 * Lref
    assert rel_l2(u0.grad.cpu().numpy().astype(np.float64), gu_ref) <= 1e-4
    assert rel_l2(k.grad.cpu().numpy().astype(np.float64), gk_ref) <= 1e-4
    # forward value equals the plain stencil
    plain = cpb.stencil(u0.detach(), k.detach(), None, 40, float(g.dt), W.DIRICHLET)
    torch.testing.assert_close(uT.detach(), plain, rtol=0, atol=0)


@pytest.mark.slow
def test_adjoint_full_size_differentiation_workload(dev):
    g = W.differentiation()       # 2048^2, 200 steps, checkpoint every 20
    tgt = g.extras["target"].astype(np.float64)
    s = np.zeros_like(g.u, dtype=np.float64)
    _, gu_ref, gk_ref = oracle.adjoint_f64(g.u, g.kappa, s, tgt, g.steps, float(g.dt), g.bc,
                                           g.extras["ckpt"], pool=oracle.host_cores())
    uT = oracle.direct(g.u, g.kappa, s, g.steps, g.dt, g.bc, "f64", pool=oracle.host_cores())
    gu, gk = gpu_adjoint(cpb.lib(fma=True), g, dev, g.steps, g.extras["ckpt"], g.bc, uT - tgt)
    assert rel_l2(gu, gu_ref) <= 1e-4
    assert rel_l2(gk, gk_ref) <= 1e-4


@pytest.mark.parametrize("bc", [W.DIRICHLET, W.PERIODIC])
@pytest.mark.parametrize("nx,ny,steps,ckpt", [(256, 130, 37, 20), (520, 77, 10, 10), (128, 40, 7, 3),
                                              (384, 9, 13, 13)])
def test_blocked_adjoint_passes_equal_one_step_launches(dev, bc, nx, ny, steps, ckpt):
    # Where every field allows 16-byte rows the backward sweep runs passes of
    # up to 4 steps; a gradient buffer off the 16-byte grid makes it launch one
    # step at a time.  The pass adds each row's gradient terms in step order,
    # so both give the same bits (--fmad=false build), for every depth the
    # segment lengths produce (4, and the remainders 3, 2, 1).
    L = cpb.lib(fma=False)
    g = W.differentiation(seed=nx + steps, n=nx, ny=ny, steps=steps, ckpt=ckpt)
    rng = np.random.default_rng(1)
    lam = torch.from_numpy(rng.standard_normal(g.u.shape).astype(np.float32)).to(dev)
    u0 = torch.from_numpy(g.u).to(dev)
    k = torch.from_numpy(g.kappa).to(dev)
    s = torch.from_numpy((rng.random(g.u.shape, dtype=np.float32) * np.float32(1e-3))).to(dev)
    wsb = L.cpb_adjoint_workspace_bytes(nx, ny, steps, ckpt)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    n = nx * ny
    out = []
    for off in (0, 1):   # gradient buffer 16-byte aligned, then 4 bytes past it
        gu = torch.empty_like(u0)
        gk_buf = torch.empty(n + 4, dtype=torch.float32, device=dev)
        gk = gk_buf[off:off + n]
        L.cpb_stencil_adjoint(u0, k, s, lam, nx, ny, steps, float(g.dt), bc, ckpt, gu, gk, ws, wsb)
        torch.cuda.synchronize()
        out.append((gu.cpu().numpy(), gk.cpu().numpy().reshape(ny, nx)))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert L.cpb_device_status() == 0
