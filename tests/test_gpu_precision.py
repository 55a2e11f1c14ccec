"""Accuracy of the GPU path against the FP64 oracle, and full-size parity checks.

* FP32 (default build, FMA contraction) within relative L-inf 1e-5 of FP64
  after 1000 steps on the 8192^2 periodic workload, and after 2000 steps on the
  precision workload's distributions.
* BF16-Kahan storage within 1e-2 of FP64 (error reported both against the
  original FP32 inputs and against the bf16-quantised inputs), on a 1024^2
  grid and on the full 16384^2 precision workload (2000 steps, both rounding
  readings, the autotuned configurations).
* Full-size launches in the benchmark's configuration: sampled cells equal the
  oracle's dependency-cone values bit for bit (--fmad=false build).
* Heat conservation at full size (periodic, s = 0) with the FP64 heat sum.
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


def rel_linf(a, ref):
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref)))


def run(L, g, dev, tuning=None, steps=None):
    u, k, s = (torch.from_numpy(x).to(dev) for x in (g.u, g.kappa, g.src))
    out, scr = torch.empty_like(u), torch.empty_like(u)
    L.cpb_stencil_launch_tuned(u, out, k, s, g.nx, g.ny, g.steps if steps is None else steps,
                               float(g.dt), g.bc, cpb.CPB_F32, tuning=tuning, scratch=scr)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def sample_idx(nx, ny, count=48, seed=0):
    rng = np.random.default_rng(seed)
    pts = [(0, 0), (nx - 1, 0), (0, ny - 1), (nx - 1, ny - 1), (nx // 2, 0), (0, ny // 2),
           (nx - 1, ny // 2), (nx // 2, ny - 1), (119, 7), (120, 8), (121, 9), (nx - 121, ny - 2)]
    pts += [(int(a), int(b)) for a, b in zip(rng.integers(0, nx, count), rng.integers(0, ny, count))]
    return np.array([j * nx + i for i, j in pts], np.int64)


def test_fp32_plain_scale_1000_steps_within_1e5(dev):
    g = W.plain_scale()                     # 8192^2, periodic, 1000 steps
    got = run(cpb.lib(fma=True), g, dev)
    ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, g.bc, "f64", pool=oracle.host_cores())
    err = rel_linf(got, ref)
    print(f"plain_scale FP32 rel L-inf vs FP64 after 1000 steps: {err:.3e}")
    assert err <= 1e-5


def test_fp32_and_bf16k_precision_distributions_2000_steps(dev):
    g = W.precision(n=1024, steps=2000)     # the 16384^2 workload's distributions, smaller grid
    pool = oracle.host_cores()
    ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, g.bc, "f64", pool=pool)
    got32 = run(cpb.lib(fma=True), g, dev)
    e32 = rel_linf(got32, ref)
    # BF16-Kahan on the device from the FP32 fields
    L = cpb.lib(fma=True)
    N = g.nx * g.ny
    u, k, s = (torch.from_numpy(x).to(dev) for x in (g.u, g.kappa, g.src))
    st = torch.empty(N, dtype=torch.int32, device=dev)
    kb = torch.empty(N, dtype=torch.int16, device=dev)
    sb = torch.empty(N, dtype=torch.int16, device=dev)
    L.cpb_bf16k_pack(u, st, N)
    L.cpb_bf16_round(k, kb, N)
    L.cpb_bf16_round(s, sb, N)
    out, scr = torch.empty_like(st), torch.empty_like(st)
    L.cpb_stencil_launch_tuned(st, out, kb, sb, g.nx, g.ny, g.steps, float(g.dt), g.bc,
                               cpb.CPB_BF16_KAHAN, scratch=scr)
    torch.cuda.synchronize()
    got16 = oracle.bf16k_value(out.cpu().numpy().view(np.uint32)).reshape(g.ny, g.nx)
    e16 = rel_linf(got16, ref)
    kq = oracle.bf16_to_f32(kb.cpu().numpy().view(np.uint16)).reshape(g.ny, g.nx)
    sq = oracle.bf16_to_f32(sb.cpu().numpy().view(np.uint16)).reshape(g.ny, g.nx)
    u0q = oracle.bf16k_value(st.cpu().numpy().view(np.uint32)).reshape(g.ny, g.nx)
    refq = oracle.direct(u0q, kq, sq, g.steps, g.dt, g.bc, "f64", pool=pool)
    e16q = rel_linf(got16, refq)
    print(f"precision 1024^2 x 2000: FP32 {e32:.3e}  BF16-Kahan {e16:.3e} "
          f"(vs FP64 on quantised inputs {e16q:.3e})")
    assert e32 <= 1e-5
    assert e16 <= 1e-2
    assert e16q <= 1e-3


def _bf16_fields(L, dev, g):
    N = g.nx * g.ny
    u, k, s = (torch.from_numpy(x).to(dev) for x in (g.u, g.kappa, g.src))
    st = torch.empty(N, dtype=torch.int32, device=dev)
    kb = torch.empty(N, dtype=torch.int16, device=dev)
    sb = torch.empty(N, dtype=torch.int16, device=dev)
    L.cpb_bf16k_pack(u, st, N)
    L.cpb_bf16_round(k, kb, N)
    L.cpb_bf16_round(s, sb, N)
    return st, kb, sb


def _run_tuned_dtype(L, dev, g, fields, dtype):
    """Autotune on copies (as the benchmark does), then the whole run."""
    u, k, s = fields
    a, b = torch.empty_like(u), torch.empty_like(u)
    a.copy_(u)
    t = L.cpb_autotune(a, b, k, s, g.nx, g.ny, 24, float(g.dt), g.bc, dtype)
    out = torch.empty_like(u)
    L.cpb_stencil_launch_tuned(u, out, k, s, g.nx, g.ny, g.steps, float(g.dt), g.bc, dtype, tuning=t,
                               scratch=a)
    torch.cuda.synchronize()
    del a, b
    return out.cpu().numpy(), t


@pytest.mark.slow
def test_precision_workload_full_size_against_fp64(dev):
    # The precision workload as stated: 16384^2, Dirichlet, 2000 steps, at the
    # autotuned configurations the benchmark times.  FP32 within 1e-5 and
    # BF16-Kahan storage (both rounding readings) within 1e-2 relative L-inf
    # of the FP64 oracle on the original FP32 inputs; the BF16 forms also
    # against FP64 on the bf16-quantised inputs (the storage error alone).
    g = W.precision()
    pool = oracle.host_cores()
    L = cpb.lib(fma=True)
    shape = (g.ny, g.nx)
    f32 = tuple(torch.from_numpy(x).to(dev) for x in (g.u, g.kappa, g.src))
    got32, t32 = _run_tuned_dtype(L, dev, g, f32, cpb.CPB_F32)
    del f32
    bf = _bf16_fields(L, dev, g)
    got16, t16 = _run_tuned_dtype(L, dev, g, bf, cpb.CPB_BF16_KAHAN)
    got16b, t16b = _run_tuned_dtype(L, dev, g, bf, cpb.CPB_BF16_KAHAN_BLOCK)
    st0, kb, sb = (x.cpu().numpy() for x in bf)
    del bf
    torch.cuda.empty_cache()
    v16 = oracle.bf16k_value(got16.view(np.uint32)).reshape(shape)
    v16b = oracle.bf16k_value(got16b.view(np.uint32)).reshape(shape)
    del got16, got16b
    ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, g.bc, "f64", pool=pool)
    e32, e16, e16b = rel_linf(got32.reshape(shape), ref), rel_linf(v16, ref), rel_linf(v16b, ref)
    del ref, got32
    kq = oracle.bf16_to_f32(kb.view(np.uint16)).reshape(shape)
    sq = oracle.bf16_to_f32(sb.view(np.uint16)).reshape(shape)
    u0q = oracle.bf16k_value(st0.view(np.uint32)).reshape(shape)
    del g.u, g.kappa, g.src
    refq = oracle.direct(u0q, kq, sq, g.steps, g.dt, g.bc, "f64", pool=pool)
    e16q, e16bq = rel_linf(v16, refq), rel_linf(v16b, refq)
    print(f"precision 16384^2 x 2000 rel L-inf vs FP64: FP32 {e32:.3e} (depth {t32['k']}), "
          f"BF16-Kahan every step {e16:.3e} (quantised inputs {e16q:.3e}, depth {t16['k']}), "
          f"BF16-Kahan per pass {e16b:.3e} (quantised inputs {e16bq:.3e}, depth {t16b['k']})")
    assert e32 <= 1e-5
    assert e16 <= 1e-2 and e16b <= 1e-2
    # The storage error alone is held to the same stated BF16 bound: rounded
    # every step it reached 1.16e-3 at this size (2000 roundings of the
    # ~16-bit hi + cmp state), rounded once per pass 1.3e-5.
    assert e16q <= 1e-2 and e16bq <= 1e-2


@pytest.mark.parametrize("which", ["plain_scale", "precision"])
def test_full_size_sampled_bit_exact(dev, which):
    L = cpb.lib(fma=False)
    if which == "plain_scale":
        g = W.plain_scale(steps=12)
    else:
        g = W.precision(steps=12)
    nx, ny = g.nx, g.ny
    u, k, s = (torch.from_numpy(x).to(dev) for x in (g.u, g.kappa, g.src))
    a, b = torch.empty_like(u), torch.empty_like(u)
    a.copy_(u)
    best = L.cpb_autotune(a, b, k, s, nx, ny, 24, float(g.dt), g.bc, cpb.CPB_F32)
    out, scr = torch.empty_like(u), torch.empty_like(u)
    L.cpb_stencil_launch_tuned(u, out, k, s, nx, ny, g.steps, float(g.dt), g.bc, cpb.CPB_F32,
                               tuning=best, scratch=scr)
    torch.cuda.synchronize()
    idx = sample_idx(nx, ny)
    got = out.reshape(-1)[torch.from_numpy(idx).to(dev)].cpu().numpy()
    ref = oracle.sample(g.u, g.kappa, g.src, g.steps, g.dt, g.bc, idx, "f32")
    np.testing.assert_array_equal(got, ref)
    assert L.cpb_device_status() == 0


def test_full_size_conservation(dev):
    g = W.plain_scale(zero_source=True)     # 8192^2, periodic, s = 0, 1000 steps
    L = cpb.lib(fma=True)
    u0 = torch.from_numpy(g.u).to(dev)
    out = cpb.stencil(u0, torch.from_numpy(g.kappa).to(dev), None, g.steps, float(g.dt), g.bc,
                      library=L)
    s0, s1 = float(cpb.heat_sum(u0, library=L)), float(cpb.heat_sum(out, library=L))
    drift = abs(s1 - s0) / abs(s0)
    print(f"heat drift after 1000 steps (FP32 storage, FP64 sum): {drift:.3e}")
    assert abs(s0 - oracle.heat_sum_f32(g.u)) <= g.u.size * 2.0 ** -52
    assert drift <= 1e-6
