"""The slab decomposition on one GPU with the library's own kernels.

Ranks are emulated in one process, one after another, with no kernel waiting
on another.  Rank r's slab lives in its own device buffer: its own rows plus
K halo rows on each side that has a neighbour.  Every K steps the halos are
filled by device-to-device copies of the neighbours' own rows (a ring for
periodic boundaries).  Then one depth-K pass of the stream kernel runs on
each slab under the grid's own boundary rule.  The rows at a slab's cut
edges see a wrong boundary, but the error moves inward by one row per step,
so after K steps the own rows are exact.  A slab at a Dirichlet edge has no
halo on that side: its buffer edge is the true boundary.

The assembled result of the --fmad=false build must equal the FP32 oracle bit
for bit, and the whole-grid run of the same library.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle.slab import split_rows

torch = pytest.importorskip("torch")
cpb = pytest.importorskip("paper_2206_07896_gb300")

pytestmark = pytest.mark.gpu
D, P = W.DIRICHLET, W.PERIODIC


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def run_slabs(L, g, world, K, dev, tuning_extra):
    ny, nx = g.u.shape
    periodic = g.bc == P
    parts = split_rows(ny, world)
    # halo rows below / above each rank's own rows (none past a Dirichlet edge)
    lo_h = [K if (periodic or r > 0) else 0 for r in range(world)]
    hi_h = [K if (periodic or r < world - 1) else 0 for r in range(world)]

    def rows(r):  # global row of every local row of rank r (wrapped)
        lo, hi = parts[r]
        return np.arange(lo - lo_h[r], hi + hi_h[r]) % ny

    u, kap, src, out = [], [], [], []
    for r in range(world):
        idx = rows(r)
        u.append(torch.from_numpy(np.ascontiguousarray(g.u[idx])).to(dev))
        kap.append(torch.from_numpy(np.ascontiguousarray(g.kappa[idx])).to(dev))  # static halos, once
        src.append(torch.from_numpy(np.ascontiguousarray(g.src[idx])).to(dev))
        out.append(torch.empty_like(u[-1]))
    n = [hi - lo for lo, hi in parts]

    def own(r, t):
        return t[r][lo_h[r]:lo_h[r] + n[r]]

    done = 0
    while done < g.steps:
        k = min(K, g.steps - done)
        for r in range(world):  # halo exchange: neighbours' own rows into this slab's halos
            if lo_h[r]:
                below = (r - 1) % world
                u[r][:K].copy_(own(below, u)[n[below] - K:])
            if hi_h[r]:
                above = (r + 1) % world
                u[r][lo_h[r] + n[r]:].copy_(own(above, u)[:K])
        for r in range(world):
            t = {"k": K, **tuning_extra}
            L.cpb_stencil_launch_tuned(u[r], out[r], kap[r], src[r], nx, u[r].shape[0], k, float(g.dt), g.bc,
                                       cpb.CPB_F32, tuning=t)
        for r in range(world):
            own(r, u).copy_(own(r, out))
        done += k
    torch.cuda.synchronize()
    return np.concatenate([own(r, u).cpu().numpy() for r in range(world)], axis=0)


@pytest.mark.parametrize("bc", [P, D])
@pytest.mark.parametrize("world,K,nx,ny,steps", [
    (2, 4, 520, 150, 13),   # TMA row ring (nx % 4 == 0), partial last block
    (3, 8, 384, 100, 17),   # depth 8 (rows in pairs)
    (4, 2, 203, 61, 7),     # register-prefetch rows (nx % 4 != 0), ragged split
    (5, 3, 256, 15, 9),     # ranks owning exactly K rows
])
def test_slabs_equal_oracle_and_whole_grid(dev, bc, world, K, nx, ny, steps):
    L = cpb.lib(fma=False)
    g = W.random_grid(40 + world, nx, ny, steps, bc)
    variant = 1 if nx % 4 == 0 else 0
    res = run_slabs(L, g, world, K, dev, {"chunk_rows": 64, "warps_per_block": 2, "variant": variant,
                                           "stages": 4})
    ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, g.bc, "f32")
    assert np.array_equal(res, ref)
    whole = cpb.stencil(torch.from_numpy(g.u).to(dev), torch.from_numpy(g.kappa).to(dev),
                        torch.from_numpy(g.src).to(dev), g.steps, float(g.dt), g.bc, library=L).cpu().numpy()
    assert np.array_equal(res, whole)
    assert L.cpb_device_status() == 0
