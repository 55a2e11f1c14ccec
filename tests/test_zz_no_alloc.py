"""The heat sum that allocates nothing (cpb_heat_sum_noalloc).

Some callers cannot allocate device memory (their framework owns all device
memory, or they cannot afford the device synchronisation that cudaMalloc and
cudaFree imply).  cpb_heat_sum_noalloc keeps its partial sums in an array
built into the library instead of a caller workspace.  This test calls it
through the C ABI twice in a row and checks each result against the
workspace version, cpb_heat_sum, within the heat-sum tolerance used by the
other tests (n * 2^-52 * max|u|).  It lives in a file of its own that pytest
collects last, and passes both alone in a fresh process and after the rest.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("shape", [(1, 1), (1000, 999), (4096, 4096), (8192, 8192)])
def test_noalloc_heat_sum_matches_workspace_version_twice(dev, shape):
    L = cpb.lib(fma=True)
    nx, ny = shape
    u = torch.rand((ny, nx), dtype=torch.float32, device=dev, generator=torch.Generator(dev).manual_seed(nx))
    ref = workspace_sum(L, u, nx, ny, cpb.CPB_F32, dev)
    tol = nx * ny * 2.0 ** -52 * float(u.abs().max())
    for _ in range(2):
        out = torch.full((), -1.0, dtype=torch.float64, device=dev)
        L.cpb_heat_sum_noalloc(u, nx, ny, cpb.CPB_F32, out)
        torch.cuda.synchronize()
        assert abs(float(out) - ref) <= tol


def test_noalloc_heat_sum_bf16k_twice(dev):
    L = cpb.lib(fma=True)
    nx, ny = 3000, 700
    u = torch.rand((ny, nx), dtype=torch.float32, device=dev, generator=torch.Generator(dev).manual_seed(1))
    st = torch.empty(nx * ny, dtype=torch.int32, device=dev)
    L.cpb_bf16k_pack(u, st, nx * ny)
    ref = workspace_sum(L, st, nx, ny, cpb.CPB_BF16_KAHAN, dev)
    for _ in range(2):
        out = torch.empty((), dtype=torch.float64, device=dev)
        L.cpb_heat_sum_noalloc(st, nx, ny, cpb.CPB_BF16_KAHAN, out)
        torch.cuda.synchronize()
        assert abs(float(out) - ref) <= nx * ny * 2.0 ** -52


def test_noalloc_heat_sum_rejects_grids_beyond_its_scratch(dev):
    L = cpb.lib(fma=True)
    u = torch.zeros(16, dtype=torch.float32, device=dev)
    out = torch.full((), 7.0, dtype=torch.float64, device=dev)
    with pytest.raises(cpb.CpbError) as e:
        L.cpb_heat_sum_noalloc(u, 8192, 8193, cpb.CPB_F32, out)   # 2^26 + 8192 cells: too many
    assert e.value.status == cpb.CPB_ERR_WORKSPACE
    torch.cuda.synchronize()
    assert float(out) == 7.0          # rejected before any launch
