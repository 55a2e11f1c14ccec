"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

The --fmad=false build must equal the oracle's FP32 mode bit for bit (same
per-cell rounding sequence); the default build must stay within the stated
tolerance of the FP64 oracle.  Sizes span several strips / tiles with ragged
tails, both boundary rules, both pass-count parities and both scratch modes.
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


@pytest.fixture(scope="module")
def exact():
    return cpb.lib(fma=False)


@pytest.fixture(scope="module")
def fast():
    return cpb.lib(fma=True)


def to_dev(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def run_tuned(L, g, dev, tuning, steps=None, scratch=True, dtype=cpb.CPB_F32, fields=None):
    steps = g.steps if steps is None else steps
    if fields is None:
        u, k, s = to_dev(g.u, dev), to_dev(g.kappa, dev), to_dev(g.src, dev)
    else:
        u, k, s = fields
    u_in = u.clone()
    out = torch.empty_like(u)
    scr = torch.empty_like(u) if scratch else None
    L.cpb_stencil_launch_tuned(u_in, out, k, s, g.nx, g.ny, steps, float(g.dt), g.bc, dtype,
                               tuning=tuning, scratch=scr)
    torch.cuda.synchronize()
    if scratch:
        assert torch.equal(u_in, u), "u_in must be untouched when scratch is given"
    return out.cpu().numpy()


# ---------------------------------------------------------------------------
# the tiled one-step kernel (caller's launch geometry)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("bc", [D, P])
@pytest.mark.parametrize("shape,block,steps", [((512, 512), (16, 16), 100), ((37, 29), (16, 16), 7),
                                               ((50, 17), (8, 4), 6), ((130, 3), (32, 2), 5),
                                               ((1, 1), (16, 16), 3)])
def test_tile_kernel_bit_exact(dev, exact, bc, shape, block, steps):
    nx, ny = shape
    g = W.random_grid(3, nx, ny, steps, bc) if shape != (512, 512) else W.plain_small()
    if shape == (512, 512):
        g.bc = bc
    ref = oracle.fission(g.u, g.kappa, g.src, g.steps, g.dt, bc, "f32", block=block, pool=4)
    bx, by = block
    u, k, s = to_dev(g.u, dev), to_dev(g.kappa, dev), to_dev(g.src, dev)
    for scratch in (False, True):
        u_in = u.clone()
        out = torch.empty_like(u)
        scr = torch.empty_like(u) if scratch else None
        exact.cpb_stencil_launch(u_in, out, k, s, nx, ny, g.steps, float(g.dt), bc, cpb.CPB_F32,
                                 ((nx + bx - 1) // bx, (ny + by - 1) // by, 1), (bx, by, 1),
                                 2 * 4 * (bx + 2) * (by + 2), scratch=scr)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref)


# ---------------------------------------------------------------------------
# the streaming temporal-blocked kernel
# ---------------------------------------------------------------------------
SHAPES = [(256, 130), (300, 97), (121, 5), (8, 8), (1, 1), (5, 3), (1000, 33), (64, 300)]


@pytest.mark.parametrize("bc", [D, P])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7, 8])
def test_stream_bit_exact_all_depths(dev, exact, bc, k):
    for (nx, ny) in SHAPES:
        for steps in (1, 2 * k + 1, 3 * k):
            g = W.random_grid(nx * 7 + ny, nx, ny, steps, bc)
            ref = oracle.direct(g.u, g.kappa, g.src, steps, g.dt, bc, "f32")
            for chunk, wpb in ((16, 4), (7, 1), (64, 8)):
                t = {"k": k, "chunk_rows": chunk, "warps_per_block": wpb}
                for scratch in (True, False):
                    got = run_tuned(exact, g, dev, t, scratch=scratch)
                    np.testing.assert_array_equal(got, ref, err_msg=f"{nx}x{ny} steps={steps} {t}")


@pytest.mark.parametrize("bc", [D, P])
def test_stream_zero_steps_copies(dev, exact, bc):
    g = W.random_grid(1, 40, 20, 0, bc)
    got = run_tuned(exact, g, dev, {"k": 4, "chunk_rows": 16, "warps_per_block": 4}, steps=0)
    np.testing.assert_array_equal(got, g.u)


@pytest.mark.parametrize("bc", [D, P])
def test_stream_null_source_means_zero(dev, exact, bc):
    g = W.random_grid(5, 200, 60, 9, bc, zero_source=True)
    ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, bc, "f32")
    u, k = to_dev(g.u, dev), to_dev(g.kappa, dev)
    out = torch.empty_like(u)
    exact.cpb_stencil_launch_tuned(u.clone(), out, k, None, g.nx, g.ny, g.steps, float(g.dt), bc,
                                   cpb.CPB_F32, tuning={"k": 3, "chunk_rows": 20})
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), ref)


def test_stream_misaligned_pointers_take_scalar_path(dev, exact):
    g = W.random_grid(9, 64, 40, 6, P)
    ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, P, "f32")
    n = g.nx * g.ny
    big = torch.zeros(4 * n + 16, dtype=torch.float32, device=dev)
    u = big[1:1 + n]
    k = big[n + 2:2 * n + 2]
    s = big[2 * n + 3:3 * n + 3]
    u.copy_(to_dev(g.u, dev).reshape(-1))
    k.copy_(to_dev(g.kappa, dev).reshape(-1))
    s.copy_(to_dev(g.src, dev).reshape(-1))
    out = torch.empty(n, dtype=torch.float32, device=dev)
    exact.cpb_stencil_launch_tuned(u, out, k, s, g.nx, g.ny, g.steps, float(g.dt), P, cpb.CPB_F32,
                                   tuning={"k": 4, "chunk_rows": 16})
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy().reshape(g.ny, g.nx), ref)


def test_default_tuning_path(dev, exact):
    g = W.plain_small()
    ref = oracle.fission(g.u, g.kappa, g.src, g.steps, g.dt, g.bc, "f32", pool=4)
    u, k, s = to_dev(g.u, dev), to_dev(g.kappa, dev), to_dev(g.src, dev)
    out = torch.empty_like(u)
    exact.cpb_stencil_launch(u.clone(), out, k, s, g.nx, g.ny, g.steps, float(g.dt), g.bc,
                             cpb.CPB_F32, (0, 0, 0), (0, 0, 0), 0)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), ref)


@pytest.mark.parametrize("bc", [D, P])
def test_fma_build_within_tolerance(dev, fast, bc):
    g = W.random_grid(12, 512, 384, 1000, bc, r=0.24)
    ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, bc, "f64", pool=8)
    got = run_tuned(fast, g, dev, {"k": 4, "chunk_rows": 64, "warps_per_block": 4})
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err <= 1e-5, err


# ---------------------------------------------------------------------------
# BF16-Kahan storage
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("bc", [D, P])
@pytest.mark.parametrize("k", [1, 3, 4, 8])
def test_bf16k_bit_exact(dev, exact, bc, k):
    for (nx, ny) in [(256, 70), (300, 45), (6, 5)]:
        g = W.random_grid(nx + ny + k, nx, ny, 2 * k + 1, bc)
        st = oracle.bf16k_pack(g.u)
        kb, sb = oracle.bf16_round(g.kappa), oracle.bf16_round(g.src)
        ref = oracle.direct_bf16k(st, kb, sb, g.steps, g.dt, bc)
        fields = (to_dev(st.view(np.int32), dev), to_dev(kb.view(np.int16), dev),
                  to_dev(sb.view(np.int16), dev))
        for scratch in (True, False):
            got = run_tuned(exact, g, dev, {"k": k, "chunk_rows": 24, "warps_per_block": 2},
                            dtype=cpb.CPB_BF16_KAHAN, fields=fields, scratch=scratch)
            np.testing.assert_array_equal(got.view(np.uint32), ref)


@pytest.mark.parametrize("bc", [D, P])
@pytest.mark.parametrize("k", [1, 2, 4, 6, 8])
def test_bf16k_block_bit_exact(dev, exact, bc, k):
    # BF16-Kahan storage rounded only where a pass stores: both row-load
    # variants, both scratch modes (the pass schedule differs), ragged sizes.
    for (nx, ny) in [(272, 70), (300, 45), (136, 50), (6, 5), (1088, 33)]:
        for steps in (2 * k + 1, 4 * k):
            g = W.random_grid(nx + 3 * ny + k, nx, ny, steps, bc)
            st = oracle.bf16k_pack(g.u)
            kb, sb = oracle.bf16_round(g.kappa), oracle.bf16_round(g.src)
            fields = (to_dev(st.view(np.int32), dev), to_dev(kb.view(np.int16), dev),
                      to_dev(sb.view(np.int16), dev))
            for variant, stages in ((0, 2), (1, 2), (1, 8)):
                for scratch in (True, False):
                    ref = oracle.direct_bf16k_block(st, kb, sb, oracle.pass_schedule(steps, k, scratch),
                                                    g.dt, bc)
                    got = run_tuned(exact, g, dev, {"k": k, "chunk_rows": 24, "warps_per_block": 2,
                                                    "variant": variant, "stages": stages},
                                    dtype=cpb.CPB_BF16_KAHAN_BLOCK, fields=fields, scratch=scratch)
                    np.testing.assert_array_equal(got.view(np.uint32), ref,
                                                  err_msg=f"{nx}x{ny} steps={steps} v{variant} scratch={scratch}")
    assert exact.cpb_device_status() == 0


def test_bf16_conversions_match_oracle(dev, exact):
    x = np.random.default_rng(4).standard_normal(100003).astype(np.float32)
    xd = to_dev(x, dev)
    r = torch.empty(x.size, dtype=torch.int16, device=dev)
    exact.cpb_bf16_round(xd, r, x.size)
    st = torch.empty(x.size, dtype=torch.int32, device=dev)
    exact.cpb_bf16k_pack(xd, st, x.size)
    back = torch.empty_like(xd)
    exact.cpb_bf16k_unpack(st, back, x.size)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(r.cpu().numpy().view(np.uint16), oracle.bf16_round(x))
    np.testing.assert_array_equal(st.cpu().numpy().view(np.uint32), oracle.bf16k_pack(x))
    ref_back = oracle.bf16k_value(oracle.bf16k_pack(x)).astype(np.float32)
    np.testing.assert_array_equal(back.cpu().numpy(), ref_back)


# ---------------------------------------------------------------------------
# heat sum
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(1, 1), (3, 7), (1000, 999), (4096, 4096)])
def test_heat_sum(dev, fast, shape):
    nx, ny = shape
    u = np.random.default_rng(nx).random((ny, nx), dtype=np.float32)
    ud = to_dev(u, dev)
    got = float(cpb.heat_sum(ud, library=fast))
    ref = oracle.heat_sum_f32(u)
    assert abs(got - ref) <= u.size * 2.0 ** -52 * float(u.max())
    # determinism: same bits again
    assert float(cpb.heat_sum(ud, library=fast)) == got
    # misaligned start exercises the scalar head
    if u.size > 8:
        flat = ud.reshape(-1)[1:]
        got2 = float(cpb.heat_sum(flat.reshape(1, -1), library=fast))
        assert abs(got2 - oracle.heat_sum_f32(u.reshape(-1)[1:])) <= u.size * 2.0 ** -52


def test_heat_sum_bf16k(dev, fast):
    u = np.random.default_rng(2).random((300, 200), dtype=np.float32)
    st = oracle.bf16k_pack(u)
    got = float(cpb.heat_sum(to_dev(st.view(np.int32), dev), dtype=cpb.CPB_BF16_KAHAN, library=fast))
    ref = oracle.heat_sum_bf16k(st)
    assert abs(got - ref) <= st.size * 2.0 ** -52


def test_conservation_periodic_gpu(dev, fast):
    g = W.plain_scale(seed=7, n=1024, steps=400, zero_source=True)
    u0 = to_dev(g.u, dev)
    out = cpb.stencil(u0, to_dev(g.kappa, dev), to_dev(g.src, dev), g.steps, float(g.dt), P,
                      library=fast)
    s0, s1 = float(cpb.heat_sum(u0, library=fast)), float(cpb.heat_sum(out, library=fast))
    assert abs(s1 - s0) <= 1e-6 * abs(s0)


# ---------------------------------------------------------------------------
# launch-model errors: a failed check enqueues nothing
# ---------------------------------------------------------------------------
def test_error_codes(dev, exact):
    g = W.random_grid(1, 64, 32, 2, D)
    u, k, s = to_dev(g.u, dev), to_dev(g.kappa, dev), to_dev(g.src, dev)
    out = torch.full_like(u, -7.0)
    L = exact

    def status(fn, *a, **kw):
        try:
            fn(*a, **kw)
        except cpb.CpbError as e:
            return e.status
        return 0

    tile = dict(grid=(4, 2, 1), block=(16, 16, 1), shared_bytes=2 * 18 * 18 * 4)
    args = (u, out, k, s, 64, 32, 2, float(g.dt), D, cpb.CPB_F32)
    assert status(L.cpb_stencil_launch, *args, **tile) == 0
    torch.cuda.synchronize()
    out.fill_(-7.0)
    bad = [
        ((u, out, k, s, 0, 32, 2, float(g.dt), D, cpb.CPB_F32), tile, cpb.CPB_ERR_INVALID_VALUE),
        ((u, out, k, s, 64, 32, -1, float(g.dt), D, cpb.CPB_F32), tile, cpb.CPB_ERR_INVALID_VALUE),
        ((u, out, k, s, 64, 32, 2, 0.0, D, cpb.CPB_F32), tile, cpb.CPB_ERR_INVALID_VALUE),
        ((u, out, k, s, 64, 32, 2, float("nan"), D, cpb.CPB_F32), tile, cpb.CPB_ERR_INVALID_VALUE),
        ((u, out, k, s, 64, 32, 2, float(g.dt), 5, cpb.CPB_F32), tile, cpb.CPB_ERR_INVALID_VALUE),
        ((u, u, k, s, 64, 32, 2, float(g.dt), D, cpb.CPB_F32), tile, cpb.CPB_ERR_INVALID_VALUE),
        ((None, out, k, s, 64, 32, 2, float(g.dt), D, cpb.CPB_F32), tile, cpb.CPB_ERR_INVALID_VALUE),
        (args, dict(tile, grid=(5, 2, 1)), cpb.CPB_ERR_INVALID_VALUE),
        (args, dict(tile, block=(64, 32, 1), grid=(1, 1, 1)), cpb.CPB_ERR_UNSUPPORTED_CONFIG),
        (args, dict(tile, block=(16, 16, 2)), cpb.CPB_ERR_UNSUPPORTED_CONFIG),
        (args, dict(tile, shared_bytes=100), cpb.CPB_ERR_SHARED_MEM),
        ((u, out, k, s, 64, 32, 2, float(g.dt), D, cpb.CPB_BF16_KAHAN), tile,
         cpb.CPB_ERR_UNSUPPORTED_CONFIG),
    ]
    for a, geo, code in bad:
        assert status(L.cpb_stencil_launch, *a, **geo) == code, (a[4:], geo)
    assert status(L.cpb_stencil_launch_tuned, *args, tuning={"k": 9, "chunk_rows": 8}) == \
        cpb.CPB_ERR_UNSUPPORTED_CONFIG
    assert status(L.cpb_stencil_launch_tuned, *args, tuning={"k": 2, "chunk_rows": 0}) == \
        cpb.CPB_ERR_UNSUPPORTED_CONFIG
    ws = torch.empty(1, dtype=torch.float64, device=dev)
    d = torch.empty((), dtype=torch.float64, device=dev)
    assert status(L.cpb_heat_sum, u, 64, 32, cpb.CPB_F32, d, ws, 0) == cpb.CPB_ERR_WORKSPACE
    torch.cuda.synchronize()
    assert torch.all(out == -7.0), "a rejected call must not launch"


# ---------------------------------------------------------------------------
# graph capture, tuning cache, autotuner, host end-to-end call
# ---------------------------------------------------------------------------
def test_graph_replays_the_run(dev, exact):
    g = W.random_grid(6, 300, 200, 23, P)
    ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, P, "f32")
    u, k, s = to_dev(g.u, dev), to_dev(g.kappa, dev), to_dev(g.src, dev)
    out, scr = torch.empty_like(u), torch.empty_like(u)
    gr = exact.cpb_graph_create(u, out, k, s, g.nx, g.ny, g.steps, float(g.dt), P, cpb.CPB_F32,
                                tuning={"k": 4, "chunk_rows": 32}, scratch=scr)
    try:
        for _ in range(2):
            out.zero_()
            exact.cpb_graph_launch(gr)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(out.cpu().numpy(), ref)
    finally:
        exact.cpb_graph_destroy(gr)


@pytest.mark.parametrize("dtype", [cpb.CPB_F32, cpb.CPB_BF16_KAHAN])
@pytest.mark.parametrize("split", [1, 13, 37])
def test_resume_from_saved_state(dev, exact, dtype, split):
    # Checkpoint / resume: the state is u alone (the (hi, cmp) words for
    # BF16-Kahan), so stopping after `split` steps and resuming from the stored
    # state gives the same bits as one run, whatever the pass schedules.
    g = W.random_grid(31, 520, 77, 50, P)
    t = {"k": 8, "chunk_rows": 24, "warps_per_block": 2, "variant": 1, "stages": 2}
    if dtype == cpb.CPB_F32:
        fields = (to_dev(g.u, dev), to_dev(g.kappa, dev), to_dev(g.src, dev))
    else:
        fields = (to_dev(oracle.bf16k_pack(g.u).view(np.int32), dev),
                  to_dev(oracle.bf16_round(g.kappa).view(np.int16), dev),
                  to_dev(oracle.bf16_round(g.src).view(np.int16), dev))
    whole = run_tuned(exact, g, dev, t, steps=g.steps, dtype=dtype, fields=fields)
    first = run_tuned(exact, g, dev, t, steps=split, dtype=dtype, fields=fields)
    resumed = (torch.from_numpy(first).to(dev),) + fields[1:]
    second = run_tuned(exact, g, dev, t, steps=g.steps - split, dtype=dtype, fields=resumed)
    np.testing.assert_array_equal(second.view(np.uint32), whole.view(np.uint32))
    if dtype == cpb.CPB_F32:
        np.testing.assert_array_equal(whole, oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, P, "f32"))


def test_tuning_cache_and_autotune(dev, exact):
    g = W.random_grid(8, 640, 256, 12, P)
    ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, P, "f32")
    u, k, s = to_dev(g.u, dev), to_dev(g.kappa, dev), to_dev(g.src, dev)
    exact.cpb_set_tuning(640, 256, cpb.CPB_F32, P, {"k": 3, "chunk_rows": 40, "warps_per_block": 2})
    assert exact.cpb_get_tuning(640, 256, cpb.CPB_F32, P) == {"k": 3, "chunk_rows": 40,
                                                             "warps_per_block": 2, "variant": 0,
                                                             "stages": 8}
    best = exact.cpb_autotune(u.clone(), torch.empty_like(u), k, s, 640, 256, 8, float(g.dt), P,
                              cpb.CPB_F32)
    assert exact.cpb_get_tuning(640, 256, cpb.CPB_F32, P) == best
    out = torch.empty_like(u)
    exact.cpb_stencil_launch(u.clone(), out, k, s, 640, 256, g.steps, float(g.dt), P, cpb.CPB_F32,
                             (0, 0, 0), (0, 0, 0), 0)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), ref)


@pytest.mark.parametrize("dtype", [cpb.CPB_F32, cpb.CPB_BF16_KAHAN])
def test_host_end_to_end(dev, exact, dtype):
    g = W.random_grid(10, 260, 130, 11, D)
    if dtype == cpb.CPB_F32:
        u0, kk, ss = g.u, g.kappa, g.src
        ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, D, "f32")
        out = np.empty_like(g.u)
    else:
        u0, kk, ss = oracle.bf16k_pack(g.u), oracle.bf16_round(g.kappa), oracle.bf16_round(g.src)
        ref = oracle.direct_bf16k(u0, kk, ss, g.steps, g.dt, D)
        out = np.empty_like(u0)
    wsb = exact.cpb_host_workspace_bytes(g.nx, g.ny, dtype)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    exact.cpb_stencil_host(u0, kk, ss, out, g.nx, g.ny, g.steps, float(g.dt), D, dtype, ws, wsb)
    np.testing.assert_array_equal(out, ref)


# ---------------------------------------------------------------------------
# variant 1: TMA bulk-copy ring
# ---------------------------------------------------------------------------
BULK_SHAPES = [(256, 130), (272, 97), (1024, 33), (128, 300), (144, 8)]


@pytest.mark.parametrize("bc", [D, P])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7, 8])
def test_bulk_variant_bit_exact(dev, exact, bc, k):
    for (nx, ny) in BULK_SHAPES:
        for steps in (1, 2 * k + 1):
            g = W.random_grid(nx * 3 + ny + k, nx, ny, steps, bc)
            ref = oracle.direct(g.u, g.kappa, g.src, steps, g.dt, bc, "f32")
            for chunk, wpb, stages in ((16, 4, 8), (7, 1, 2), (64, 8, 4), (300, 2, 16)):
                t = {"k": k, "chunk_rows": chunk, "warps_per_block": wpb, "variant": 1,
                     "stages": stages}
                for scratch in (True, False):
                    got = run_tuned(exact, g, dev, t, scratch=scratch)
                    np.testing.assert_array_equal(got, ref, err_msg=f"{nx}x{ny} steps={steps} {t}")
    assert exact.cpb_device_status() == 0


@pytest.mark.parametrize("bc", [D, P])
@pytest.mark.parametrize("k", [1, 4, 6, 8])
def test_bulk_variant_bf16k_bit_exact(dev, exact, bc, k):
    for (nx, ny) in [(272, 70), (136, 50), (400, 9)]:
        g = W.random_grid(nx + ny + k, nx, ny, 2 * k + 1, bc)
        st = oracle.bf16k_pack(g.u)
        kb, sb = oracle.bf16_round(g.kappa), oracle.bf16_round(g.src)
        ref = oracle.direct_bf16k(st, kb, sb, g.steps, g.dt, bc)
        fields = (to_dev(st.view(np.int32), dev), to_dev(kb.view(np.int16), dev),
                  to_dev(sb.view(np.int16), dev))
        for stages in (2, 8):
            got = run_tuned(exact, g, dev, {"k": k, "chunk_rows": 24, "warps_per_block": 2,
                                            "variant": 1, "stages": stages},
                            dtype=cpb.CPB_BF16_KAHAN, fields=fields)
            np.testing.assert_array_equal(got.view(np.uint32), ref)
    assert exact.cpb_device_status() == 0


def test_bulk_variant_fma_build_within_tolerance(dev, fast):
    g = W.random_grid(21, 1024, 512, 1000, P, r=0.24)
    ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, P, "f64", pool=8)
    got = run_tuned(fast, g, dev, {"k": 6, "chunk_rows": 128, "warps_per_block": 4, "variant": 1,
                                   "stages": 8})
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err <= 1e-5, err


@pytest.mark.parametrize("bc", [D, P])
@pytest.mark.parametrize("k", [3, 8])
def test_stream_kernel_equals_warp_level_oracle(dev, exact, bc, k):
    # The tuned GPU kernel and the same kernel class run the paper's way for
    # kernels with warp functions (nested warp / lane loops split at every
    # shuffle), with the same depth and chunking: bit for bit.
    g = W.random_grid(61 + k, 520, 77, 2 * k + 3, bc)
    ref = oracle.strip_warp(g.u, g.kappa, g.src, g.steps, g.dt, bc, "f32", k=k, chunk=24, warps=2, pool=4)
    got = run_tuned(exact, g, dev, {"k": k, "chunk_rows": 24, "warps_per_block": 2, "variant": 1,
                                    "stages": 2})
    np.testing.assert_array_equal(got, ref)


def test_host_async_calls_overlap_and_stay_exact(dev, exact):
    # Three problems through the pipelined host call on alternating
    # workspaces (copy-in, compute and copy-out streams), the third reusing
    # the first one's workspace once that call's copy-out has passed: every
    # result equals the oracle bit for bit.
    grids = [W.random_grid(50 + i, 260, 130, 11 + i, D) for i in range(3)]
    wsb = exact.cpb_host_workspace_bytes(260, 130, cpb.CPB_F32)
    ws = [torch.empty(wsb, dtype=torch.uint8, device=dev) for _ in range(2)]
    s_in, s_c, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ins = [tuple(torch.from_numpy(x.copy()).pin_memory() for x in (g.u, g.kappa, g.src)) for g in grids]
    outs = [torch.empty((130, 260), dtype=torch.float32).pin_memory() for _ in grids]
    done = [None, None]
    for i, g in enumerate(grids):
        w = i % 2
        if done[w] is not None:
            s_in.wait_event(done[w])
        exact.cpb_stencil_host_async(*ins[i], outs[i], g.nx, g.ny, g.steps, float(g.dt), D, cpb.CPB_F32, ws[w],
                                     wsb, s_in, s_c, s_out)
        ev = torch.cuda.Event()
        ev.record(s_out)
        done[w] = ev
    torch.cuda.synchronize()
    for g, o in zip(grids, outs):
        np.testing.assert_array_equal(o.numpy(), oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, D, "f32"))
    with pytest.raises(cpb.CpbError) as e:
        exact.cpb_stencil_host_async(*ins[0], outs[0], 260, 130, 3, float(grids[0].dt), D, cpb.CPB_F32, ws[0], wsb,
                                     s_in, s_in, s_out)
    assert e.value.status == cpb.CPB_ERR_INVALID_VALUE
