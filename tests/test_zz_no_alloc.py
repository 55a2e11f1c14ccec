"""The heat sum that allocates nothing (cpb_heat_sum_noalloc).

Some callers cannot allocate device memory (their framework owns all device
memory, or they cannot afford the device synchronisation that cudaMalloc and
cudaFree imply).  cpb_heat_sum_noalloc keeps its partial sums in an array
built into the library instead of a caller workspace.  This test calls it
through the C ABI twice in a row and checks each result against the
workspace version, cpb_heat_sum, and against the CPU oracle's FP64 sum.  For
FP32 fields whose values are multiples of 2^-24 in [0, 1) every partial and
total is exact in FP64, so the three must be equal; otherwise they agree
within the heat-sum tolerance used by the other tests (n * 2^-52 * max|u|).
A call on a small grid right after one on a large grid shows that the
partials left in the shared array by the earlier call are not read.  The file
is collected last, and passes both alone in a fresh process and after the
rest.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
cpb = pytest.importorskip("paper_2206_07896_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def workspace_sum(L, u, nx, ny, dtype, dev):
    wsb = L.cpb_heat_sum_workspace_bytes(nx, ny)
    ws = torch.empty(max(wsb, 8) // 8, dtype=torch.float64, device=dev)
    out = torch.empty((), dtype=torch.float64, device=dev)
    L.cpb_heat_sum(u, nx, ny, dtype, out, ws, wsb)
    torch.cuda.synchronize()
    return float(out)


def noalloc_sum(L, u, nx, ny, dtype, dev):
    out = torch.full((), -1.0, dtype=torch.float64, device=dev)
    L.cpb_heat_sum_noalloc(u, nx, ny, dtype, out)
    torch.cuda.synchronize()
    return float(out)


def dyadic_field(nx, ny, seed, dev):
    """FP32 values k * 2^-24, k in [0, 2^24): exact in FP32 and summed exactly in FP64."""
    g = torch.Generator(dev).manual_seed(seed)
    k = torch.randint(0, 1 << 24, (ny, nx), generator=g, device=dev, dtype=torch.int32)
    return k.to(torch.float32) * 2.0 ** -24


@pytest.mark.parametrize("shape", [(1, 1), (1000, 999), (4096, 4096), (8192, 8192)])
def test_noalloc_heat_sum_equals_workspace_version_and_oracle_twice(dev, shape):
    L = cpb.lib(fma=True)
    nx, ny = shape
    u = dyadic_field(nx, ny, nx, dev)
    ref = workspace_sum(L, u, nx, ny, cpb.CPB_F32, dev)
    assert ref == oracle.heat_sum_f32(u.cpu().numpy())
    for _ in range(2):
        assert noalloc_sum(L, u, nx, ny, cpb.CPB_F32, dev) == ref


def test_noalloc_heat_sum_small_grid_after_large_grid(dev):
    L = cpb.lib(fma=True)
    big = dyadic_field(8192, 8192, 3, dev)   # fills all 4096 partials of the shared array
    assert noalloc_sum(L, big, 8192, 8192, cpb.CPB_F32, dev) == workspace_sum(L, big, 8192, 8192,
                                                                               cpb.CPB_F32, dev)
    small = dyadic_field(300, 70, 4, dev)     # two partials: the rest of the array is stale
    want = oracle.heat_sum_f32(small.cpu().numpy())
    for _ in range(2):
        assert noalloc_sum(L, small, 300, 70, cpb.CPB_F32, dev) == want


def test_noalloc_heat_sum_general_values_within_tolerance(dev):
    # Values that are not exact in a common binade: the sums agree to the
    # order-dependent FP64 tolerance.
    L = cpb.lib(fma=True)
    nx, ny = 2048, 1500
    u = torch.randn((ny, nx), dtype=torch.float32, device=dev, generator=torch.Generator(dev).manual_seed(5))
    ref = oracle.heat_sum_f32(u.cpu().numpy())
    tol = nx * ny * 2.0 ** -52 * float(u.abs().max())
    for _ in range(2):
        got = noalloc_sum(L, u, nx, ny, cpb.CPB_F32, dev)
        assert abs(got - ref) <= tol
        assert abs(got - workspace_sum(L, u, nx, ny, cpb.CPB_F32, dev)) <= tol


@pytest.mark.parametrize("dtype", ["bf16k", "bf16k_block"])
def test_noalloc_heat_sum_bf16k_twice(dev, dtype):
    L = cpb.lib(fma=True)
    code = cpb.CPB_BF16_KAHAN if dtype == "bf16k" else cpb.CPB_BF16_KAHAN_BLOCK
    nx, ny = 3000, 700
    u = torch.rand((ny, nx), dtype=torch.float32, device=dev, generator=torch.Generator(dev).manual_seed(1))
    st = torch.empty(nx * ny, dtype=torch.int32, device=dev)
    L.cpb_bf16k_pack(u, st, nx * ny)
    ref = workspace_sum(L, st, nx, ny, code, dev)
    want = oracle.heat_sum_bf16k(st.cpu().numpy().view(np.uint32))
    for _ in range(2):
        got = noalloc_sum(L, st, nx, ny, code, dev)
        assert abs(got - ref) <= nx * ny * 2.0 ** -52
        assert abs(got - want) <= nx * ny * 2.0 ** -52


def test_noalloc_heat_sum_rejects_grids_beyond_its_scratch(dev):
    L = cpb.lib(fma=True)
    u = torch.zeros(16, dtype=torch.float32, device=dev)
    out = torch.full((), 7.0, dtype=torch.float64, device=dev)
    with pytest.raises(cpb.CpbError) as e:
        L.cpb_heat_sum_noalloc(u, 8192, 8193, cpb.CPB_F32, out)   # 2^26 + 8192 cells: too many
    assert e.value.status == cpb.CPB_ERR_WORKSPACE
    torch.cuda.synchronize()
    assert float(out) == 7.0          # rejected before any launch
