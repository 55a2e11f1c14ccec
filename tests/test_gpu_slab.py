"""The slab decomposition on one GPU through the library's slab calls.

Ranks are emulated in one process, one after another, with no kernel waiting
on another.  cpb_slab_rows gives rank r its own rows and halo sizes; rank r's
slab lives in its own device buffers (u, kappa, s): its own rows plus K halo
rows on each side that has a neighbour.  kappa and s halos are exchanged once
(they never change); every K steps cpb_slab_exchange fills the u halos from
the neighbours' own rows (a ring for periodic boundaries), then cpb_slab_step
runs one pass of up to K steps on each slab under the grid's own boundary
rule.  The rows at a slab's cut edges see a wrong boundary, but the error
moves inward by one row per step, so after the pass the own rows are exact.
A slab at a Dirichlet edge has no halo on that side: its buffer edge is the
true boundary.

The assembled result of the --fmad=false build must equal the FP32 oracle bit
for bit, and the whole-grid run of the same library.
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


def run_slabs(L, g, world, K, dev, tuning):
    ny, nx = g.u.shape
    F = cpb.CPB_F32
    lay = [L.cpb_slab_rows(ny, world, r, K, g.bc) for r in range(world)]
    n = [x["row_hi"] - x["row_lo"] for x in lay]
    hl = [x["halo_lo"] for x in lay]
    hh = [x["halo_hi"] for x in lay]
    rows = [hl[r] + n[r] + hh[r] for r in range(world)]

    def slab_of(field):  # own rows placed, halos zero (filled by the exchange)
        out = []
        for r in range(world):
            t = torch.zeros((rows[r], nx), dtype=torch.float32, device=dev)
            t[hl[r]:hl[r] + n[r]] = torch.from_numpy(field[lay[r]["row_lo"]:lay[r]["row_hi"]]).to(dev)
            out.append(t)
        return out

    def exchange(bufs):
        for r in range(world):
            b, a = (r - 1) % world, (r + 1) % world
            L.cpb_slab_exchange(bufs[r], nx, n[r], hl[r], hh[r], bufs[b] if hl[r] else None, hl[b], n[b],
                                bufs[a] if hh[r] else None, hl[a], n[a], F)

    u, kap, src = slab_of(g.u), slab_of(g.kappa), slab_of(g.src)
    exchange(kap)        # static fields: halos once
    exchange(src)
    out = [torch.empty_like(x) for x in u]
    done = 0
    while done < g.steps:
        k = min(K, g.steps - done)
        exchange(u)
        for r in range(world):
            L.cpb_slab_step(u[r], out[r], kap[r], src[r], nx, rows[r], hl[r], hh[r], k, float(g.dt), g.bc, F,
                            tuning=tuning)
        u, out = out, u
        done += k
    torch.cuda.synchronize()
    return np.concatenate([u[r][hl[r]:hl[r] + n[r]].cpu().numpy() for r in range(world)], axis=0)


@pytest.mark.parametrize("bc", [P, D])
@pytest.mark.parametrize("world,K,nx,ny,steps", [
    (2, 4, 520, 150, 13),   # TMA row ring (nx % 4 == 0), partial last block
    (3, 8, 384, 100, 17),   # depth 8 (rows in pairs)
    (4, 2, 203, 61, 7),     # register-prefetch rows (nx % 4 != 0), ragged split
    (5, 3, 256, 15, 9),     # ranks owning exactly K rows
    (1, 4, 256, 40, 10),    # one rank: a periodic slab's halos are its own wrapped rows
])
def test_slabs_equal_oracle_and_whole_grid(dev, bc, world, K, nx, ny, steps):
    L = cpb.lib(fma=False)
    g = W.random_grid(40 + world, nx, ny, steps, bc)
    variant = 1 if nx % 4 == 0 else 0
    res = run_slabs(L, g, world, K, dev, {"k": K, "chunk_rows": 64, "warps_per_block": 2, "variant": variant,
                                           "stages": 4})
    ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, g.bc, "f32")
    assert np.array_equal(res, ref)
    whole = cpb.stencil(torch.from_numpy(g.u).to(dev), torch.from_numpy(g.kappa).to(dev),
                        torch.from_numpy(g.src).to(dev), g.steps, float(g.dt), g.bc, library=L).cpu().numpy()
    assert np.array_equal(res, whole)
    assert L.cpb_device_status() == 0


def run_slabs_bf16k(L, g, world, K, dev, dtype, tuning):
    """The same decomposition with BF16-Kahan storage: u as 32-bit (hi, cmp)
    words exchanged by cpb_slab_exchange, kappa and s as 2-byte bf16 fields
    whose halos go through cpb_slab_exchange_rows (2 nx bytes per row)."""
    ny, nx = g.u.shape
    lay = [L.cpb_slab_rows(ny, world, r, K, g.bc) for r in range(world)]
    n = [x["row_hi"] - x["row_lo"] for x in lay]
    hl = [x["halo_lo"] for x in lay]
    hh = [x["halo_hi"] for x in lay]
    rows = [hl[r] + n[r] + hh[r] for r in range(world)]
    st = oracle.bf16k_pack(g.u).view(np.int32)
    kb = oracle.bf16_round(g.kappa).view(np.int16)
    sb = oracle.bf16_round(g.src).view(np.int16)

    def slab_of(field, tdt):
        out = []
        for r in range(world):
            t = torch.zeros((rows[r], nx), dtype=tdt, device=dev)
            t[hl[r]:hl[r] + n[r]] = torch.from_numpy(field[lay[r]["row_lo"]:lay[r]["row_hi"]]).to(dev)
            out.append(t)
        return out

    def neighbours(r):
        return (r - 1) % world, (r + 1) % world

    def exchange_u(bufs):
        for r in range(world):
            b, a = neighbours(r)
            L.cpb_slab_exchange(bufs[r], nx, n[r], hl[r], hh[r], bufs[b] if hl[r] else None, hl[b], n[b],
                                bufs[a] if hh[r] else None, hl[a], n[a], dtype)

    def exchange_ks(bufs):
        for r in range(world):
            b, a = neighbours(r)
            L.cpb_slab_exchange_rows(bufs[r], 2 * nx, n[r], hl[r], hh[r], bufs[b] if hl[r] else None, hl[b],
                                     n[b], bufs[a] if hh[r] else None, hl[a], n[a])

    u, kap, src = slab_of(st, torch.int32), slab_of(kb, torch.int16), slab_of(sb, torch.int16)
    exchange_ks(kap)
    exchange_ks(src)
    out = [torch.empty_like(x) for x in u]
    done, depths = 0, []
    while done < g.steps:
        k = min(K, g.steps - done)
        exchange_u(u)
        for r in range(world):
            L.cpb_slab_step(u[r], out[r], kap[r], src[r], nx, rows[r], hl[r], hh[r], k, float(g.dt), g.bc, dtype,
                            tuning=tuning)
        u, out = out, u
        done += k
        depths.append(k)
    torch.cuda.synchronize()
    res = np.concatenate([u[r][hl[r]:hl[r] + n[r]].cpu().numpy() for r in range(world)], axis=0)
    return res.view(np.uint32), depths, st, kb, sb


@pytest.mark.parametrize("dtype", [cpb.CPB_BF16_KAHAN, cpb.CPB_BF16_KAHAN_BLOCK])
@pytest.mark.parametrize("bc", [P, D])
@pytest.mark.parametrize("world,K,nx,ny,steps", [(3, 4, 272, 60, 11), (2, 8, 400, 40, 13), (4, 2, 206, 21, 5)])
def test_bf16k_slabs_equal_oracle(dev, bc, dtype, world, K, nx, ny, steps):
    # Every-step rounding does not depend on the decomposition; rounding once
    # per pass gives the oracle's per-pass form on the rounds' pass depths.
    L = cpb.lib(fma=False)
    g = W.random_grid(60 + world, nx, ny, steps, bc)
    variant = 1 if nx % 8 == 0 else 0
    res, depths, st, kb, sb = run_slabs_bf16k(L, g, world, K, dev, dtype,
                                              {"k": K, "chunk_rows": 32, "warps_per_block": 2, "variant": variant,
                                               "stages": 4})
    if dtype == cpb.CPB_BF16_KAHAN:
        ref = oracle.direct_bf16k(st.view(np.uint32), kb.view(np.uint16), sb.view(np.uint16), g.steps, g.dt, bc)
    else:
        ref = oracle.direct_bf16k_block(st.view(np.uint32), kb.view(np.uint16), sb.view(np.uint16), depths, g.dt, bc)
    np.testing.assert_array_equal(res, ref)
    assert L.cpb_device_status() == 0
