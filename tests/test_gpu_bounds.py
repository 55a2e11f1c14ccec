"""Every kernel under the bounds-checked build (libcpb_check.so).

In that build each global element range a kernel reads or writes is checked
against its field; an access outside is recorded (translation unit and
source line, read by cpb_bounds_status) and clamped into the field, so a
failing check touches nothing outside its buffers.  The kernels run here on
ragged, tiny and misaligned shapes, both boundary rules and every path
(both row-load variants at every depth, both BF16 roundings, the tiled and
multi-barrier kernels, the 3-D kernels, the batched launch, the adjoint in
passes and in single steps, the heat sums, the slab calls): no access may
fall outside its field, and the results must still equal the oracle (bit for
bit where the --fmad=false arithmetic fixes them, which the checked build
has).
"""
import numpy as np
import pytest

import oracle
import workloads as W
from test_gpu_batched import pack, run_batch, small_batch
from test_gpu_slab import run_slabs

torch = pytest.importorskip("torch")
cpb = pytest.importorskip("paper_2206_07896_gb300")

pytestmark = pytest.mark.gpu
D, P = W.DIRICHLET, W.PERIODIC


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def L(dev):
    lib = cpb.lib_checked()
    lib.cpb_bounds_status()   # read and clear
    return lib


def clean(L):
    torch.cuda.synchronize()
    assert L.cpb_device_status() == 0
    assert L.cpb_bounds_status() == (0, 0)


def to_dev(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_the_other_builds_do_not_check(dev):
    for fma in (True, False):
        with pytest.raises(cpb.CpbError) as e:
            cpb.lib(fma=fma).cpb_bounds_status()
        assert e.value.status == cpb.CPB_ERR_UNSUPPORTED_CONFIG


@pytest.mark.parametrize("bc", [D, P])
@pytest.mark.parametrize("k", [1, 3, 4, 6, 8])
def test_stream_kernels_in_bounds(dev, L, bc, k):
    for (nx, ny) in [(256, 130), (272, 33), (121, 5), (5, 3), (1, 1), (130, 1), (1000, 19)]:
        g = W.random_grid(nx + ny + k, nx, ny, 2 * k + 1, bc)
        ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, bc, "f32")
        u, kap, s = to_dev(g.u, dev), to_dev(g.kappa, dev), to_dev(g.src, dev)
        for variant, chunk, wpb, stages in ((0, 7, 2, 2), (1, 16, 4, 2), (1, 300, 1, 8)):
            t = {"k": k, "chunk_rows": chunk, "warps_per_block": wpb, "variant": variant, "stages": stages}
            for scratch in (True, False):
                out = torch.empty_like(u)
                L.cpb_stencil_launch_tuned(u.clone(), out, kap, s, nx, ny, g.steps, float(g.dt), bc, cpb.CPB_F32,
                                           tuning=t, scratch=torch.empty_like(u) if scratch else None)
                torch.cuda.synchronize()
                np.testing.assert_array_equal(out.cpu().numpy(), ref, err_msg=f"{nx}x{ny} {t}")
        clean(L)


def test_stream_misaligned_fields_in_bounds(dev, L):
    # fields 4 bytes off a 16-byte boundary take the scalar row path
    for bc in (D, P):
        g = W.random_grid(9, 64, 40, 6, bc)
        n = g.nx * g.ny
        big = torch.zeros(4 * n + 16, dtype=torch.float32, device=dev)
        u, kap, s = big[1:1 + n], big[n + 2:2 * n + 2], big[2 * n + 3:3 * n + 3]
        u.copy_(to_dev(g.u, dev).reshape(-1))
        kap.copy_(to_dev(g.kappa, dev).reshape(-1))
        s.copy_(to_dev(g.src, dev).reshape(-1))
        out = torch.empty(n, dtype=torch.float32, device=dev)
        L.cpb_stencil_launch_tuned(u, out, kap, s, g.nx, g.ny, g.steps, float(g.dt), bc, cpb.CPB_F32,
                                   tuning={"k": 4, "chunk_rows": 16, "warps_per_block": 2, "variant": 1,
                                           "stages": 2})
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy().reshape(g.ny, g.nx),
                                      oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, bc, "f32"))
    clean(L)


@pytest.mark.parametrize("bc", [D, P])
def test_bf16_kernels_in_bounds(dev, L, bc):
    for (nx, ny) in [(272, 50), (300, 9), (6, 5)]:
        g = W.random_grid(nx * 2 + ny, nx, ny, 9, bc)
        st = oracle.bf16k_pack(g.u)
        kb, sb = oracle.bf16_round(g.kappa), oracle.bf16_round(g.src)
        fields = (to_dev(st.view(np.int32), dev), to_dev(kb.view(np.int16), dev), to_dev(sb.view(np.int16), dev))
        ref_step = oracle.direct_bf16k(st, kb, sb, g.steps, g.dt, bc)
        ref_pass = oracle.direct_bf16k_block(st, kb, sb, oracle.pass_schedule(g.steps, 4), g.dt, bc)
        for variant in (0, 1):
            t = {"k": 4, "chunk_rows": 16, "warps_per_block": 2, "variant": variant, "stages": 2}
            for dtype, ref in ((cpb.CPB_BF16_KAHAN, ref_step), (cpb.CPB_BF16_KAHAN_BLOCK, ref_pass)):
                out = torch.empty_like(fields[0])
                L.cpb_stencil_launch_tuned(fields[0].clone(), out, fields[1], fields[2], nx, ny, g.steps,
                                           float(g.dt), bc, dtype, tuning=t, scratch=torch.empty_like(fields[0]))
                torch.cuda.synchronize()
                np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), ref,
                                              err_msg=f"{nx}x{ny} dtype {dtype} variant {variant}")
    clean(L)


@pytest.mark.parametrize("bc", [D, P])
def test_tiled_and_multi_barrier_kernels_in_bounds(dev, L, bc):
    for (nx, ny), (bx, by) in (((37, 29), (16, 16)), ((50, 17), (8, 4)), ((1, 1), (16, 16)), ((130, 3), (32, 2))):
        g = W.random_grid(nx + 3 * ny, nx, ny, 6, bc)
        ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, bc, "f32")
        u, kap, s = to_dev(g.u, dev), to_dev(g.kappa, dev), to_dev(g.src, dev)
        grid = ((nx + bx - 1) // bx, (ny + by - 1) // by, 1)
        out = torch.empty_like(u)
        L.cpb_stencil_launch(u.clone(), out, kap, s, nx, ny, g.steps, float(g.dt), bc, cpb.CPB_F32, grid,
                             (bx, by, 1), 2 * 4 * (bx + 2) * (by + 2), scratch=torch.empty_like(u))
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref)
        for d in (1, 3):
            out2 = torch.empty_like(u)
            L.cpb_stencil_tile_blocked(u.clone(), out2, kap, s, nx, ny, g.steps, d, float(g.dt), bc, grid,
                                       (bx, by, 1), L.cpb_tile_blocked_shared_bytes(bx, by, d),
                                       scratch=torch.empty_like(u))
            torch.cuda.synchronize()
            np.testing.assert_array_equal(out2.cpu().numpy(), ref)
    clean(L)


@pytest.mark.parametrize("bc", [D, P])
def test_3d_kernels_in_bounds(dev, L, bc):
    for (nx, ny, nz) in [(132, 20, 9), (130, 7, 5), (64, 9, 3), (4, 1, 1)]:  # ring path (nx % 4 == 0) and scalar
        g = W.random_grid3(nx + ny + nz, nx, ny, nz, 4, bc)
        ref = oracle.direct3(g.u, g.kappa, g.src, g.steps, g.dt, bc, "f32")
        u, kap, s = to_dev(g.u, dev), to_dev(g.kappa, dev), to_dev(g.src, dev)
        out = torch.empty_like(u)
        L.cpb_stencil3d_launch(u.clone(), out, kap, s, nx, ny, nz, g.steps, float(g.dt), bc,
                               scratch=torch.empty_like(u))
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref, err_msg=f"{nx}x{ny}x{nz}")
    clean(L)


@pytest.mark.parametrize("bc", [D, P])
@pytest.mark.parametrize("plan", [{"grain": 1, "threads": 384, "team_cells": 4096},
                                  {"grain": 2, "threads": 128, "team_cells": 1, "depth": 8},
                                  {"grain": 1, "threads": 384, "team_cells": 20000, "team_warps": 4}])
def test_batched_launch_in_bounds(dev, L, bc, plan):
    grids = small_batch(11 + bc, bc)
    u, k, s, off = pack(grids, dev)
    uo, _ = run_batch(L, grids, dev, bc, plan, u, k, s, off)
    out = uo.cpu().numpy()
    for g, o in zip(grids, off):
        ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, bc, "f32")
        np.testing.assert_array_equal(out[o:o + g.nx * g.ny].reshape(g.ny, g.nx), ref)
    clean(L)


@pytest.mark.parametrize("bc", [D, P])
def test_adjoint_in_bounds(dev, L, bc):
    for (nx, ny, steps, ckpt) in [(256, 70, 13, 5), (132, 17, 9, 4), (5, 3, 4, 2)]:
        g = W.differentiation(seed=nx, n=nx, ny=ny, steps=steps, ckpt=ckpt)
        tgt = g.extras["target"].astype(np.float64)
        src = np.random.default_rng(nx).random(g.u.shape, dtype=np.float32) * np.float32(1e-3)
        _, gu_ref, gk_ref = oracle.adjoint_f64(g.u, g.kappa, src.astype(np.float64), tgt, steps, float(g.dt),
                                               bc, ckpt)
        lam_T = oracle.direct(g.u, g.kappa, src, steps, g.dt, bc, "f64") - tgt
        u0, kap, s = to_dev(g.u, dev), to_dev(g.kappa, dev), to_dev(src, dev)
        lam = to_dev(lam_T.astype(np.float32), dev)
        wsb = L.cpb_adjoint_workspace_bytes(nx, ny, steps, ckpt)
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
        got = []
        for off in (0, 1):   # aligned: passes of up to 4 steps; 4 bytes off: one step per launch
            gu = torch.empty_like(u0)
            gbuf = torch.empty(nx * ny + 4, dtype=torch.float32, device=dev)
            L.cpb_stencil_adjoint(u0, kap, s, lam, nx, ny, steps, float(g.dt), bc, ckpt, gu,
                                  gbuf[off:off + nx * ny], ws, wsb)
            torch.cuda.synchronize()
            got.append((gu.cpu().numpy(), gbuf[off:off + nx * ny].cpu().numpy().reshape(ny, nx)))
        np.testing.assert_array_equal(got[0][0], got[1][0])
        np.testing.assert_array_equal(got[0][1], got[1][1])
        assert rel_l2(got[0][0].astype(np.float64), gu_ref) <= 1e-4
        assert rel_l2(got[0][1].astype(np.float64), gk_ref) <= 1e-4
    clean(L)


def test_heat_sums_in_bounds(dev, L):
    for shape in [(70, 256), (3, 5), (1, 1), (1, 7), (129, 130)]:
        u = np.random.default_rng(shape[1]).random(shape, dtype=np.float32)
        ud = to_dev(u, dev)
        tol = u.size * 2.0 ** -52
        assert abs(float(cpb.heat_sum(ud, library=L)) - oracle.heat_sum_f32(u)) <= tol
        if u.size > 1:
            flat = ud.reshape(-1)[1:]   # scalar head and tail around the aligned body
            got = float(cpb.heat_sum(flat.reshape(1, -1), library=L))
            assert abs(got - oracle.heat_sum_f32(u.reshape(-1)[1:])) <= tol
        st = oracle.bf16k_pack(u)
        got = float(cpb.heat_sum(to_dev(st.view(np.int32), dev), dtype=cpb.CPB_BF16_KAHAN, library=L))
        assert abs(got - oracle.heat_sum_bf16k(st)) <= tol
        out = torch.empty((), dtype=torch.float64, device=dev)
        L.cpb_heat_sum_noalloc(ud, shape[1], shape[0], cpb.CPB_F32, out)
        torch.cuda.synchronize()
        assert abs(float(out) - oracle.heat_sum_f32(u)) <= tol
    clean(L)


@pytest.mark.parametrize("bc", [P, D])
@pytest.mark.parametrize("world,K,nx,ny,steps", [(3, 4, 260, 61, 9), (2, 8, 384, 40, 11), (4, 2, 203, 21, 5)])
def test_slab_calls_in_bounds(dev, L, bc, world, K, nx, ny, steps):
    g = W.random_grid(44 + world, nx, ny, steps, bc)
    res = run_slabs(L, g, world, K, dev, {"k": K, "chunk_rows": 16, "warps_per_block": 2,
                                           "variant": 1 if nx % 4 == 0 else 0, "stages": 2})
    np.testing.assert_array_equal(res, oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, bc, "f32"))
    clean(L)
