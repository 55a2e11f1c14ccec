"""CPU oracle for the barrier-tiled heat stencil (ctypes wrapper over liboracle.so).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of bench.py may import this package.  It shares no code with
the CUDA library and imports nothing from it.

Functions (all numpy in, numpy out):

* ``direct(g, precision, pool)``      the canonical update as a plain loop over
                                      cells (FP64 / FP32), the stencil's definition.
* ``fission(g, precision, block, pool, block_per_fetch)``
                                      the tiled SPMD kernel executed as the paper
                                      defines CUDA execution on CPUs: a loop over
                                      blocks run by a thread pool with a task queue
                                      and coarse-grained fetching (Sec. IV), and
                                      inside each block one thread loop per
                                      barrier-free region (Sec. III "SPMD to MPMD").
* ``direct_bf16k``                    BF16-Kahan storage, FP32 compute, every step
                                      rounded into storage.
* ``direct_bf16k_block``              BF16-Kahan storage rounded once per pass of
                                      a temporal-block schedule (``pass_schedule``).
* ``sample``                          sampled cells of a large run via their
                                      dependency cones (bit-identical to ``direct``).
* ``heat_sum_*``                      FP64 sums.
* ``adjoint_f64``                     gradient of 0.5||u_T - target||^2 w.r.t.
                                      u_0 and kappa (discrete adjoint, checkpointed).
* ``tile_blocked``                    the shared-memory temporal-blocked tiled
                                      kernel (depth steps per launch, a
                                      barrier after each) run with loop fission.
* ``direct3`` / ``fission3``          the 3-D 7-point variant: the plain loop,
                                      and the z-marching tiled kernel (two
                                      barriers inside its plane loop) run with
                                      loop fission.
* ``strip_warp``                      the shuffle-based temporal-blocked strip
                                      kernel run with nested warp / lane loops
                                      split at every shuffle (Sec. III "SPMD to MPMD").
* ``slab`` (module)                   the y-slab decomposition of the stencil
                                      across ranks with K-row halo exchange every
                                      K steps (torch.distributed gloo ranks, or
                                      ranks as threads, on CPU).
* ``vecadd`` / ``dynamic_reverse`` / ``fetch_accounting``
                                      the paper's example kernels (Listings 1-3)
                                      and runtime accounting, to test the executor.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_LIB = None

DIRICHLET = 0
PERIODIC = 1

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_fp = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_u32 = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_u16 = np.ctypeslib.ndpointer(dtype=np.uint16, flags="C_CONTIGUOUS")
_i32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = C.CDLL(path)
        i, d, f = C.c_int, C.c_double, C.c_float
        L.orc_direct_f64.argtypes = [_dp, _dp, _dp, i, i, i, d, i, i, _dp]
        L.orc_direct_f32.argtypes = [_fp, _fp, _fp, i, i, i, f, i, i, _fp]
        L.orc_fission_f64.argtypes = [_dp, _dp, _dp, i, i, i, d, i, i, i, i, i, _dp]
        L.orc_fission_f32.argtypes = [_fp, _fp, _fp, i, i, i, f, i, i, i, i, i, _fp]
        L.orc_direct_bf16k.argtypes = [_u32, _u16, _u16, i, i, i, f, i, i, i, _u32]
        L.orc_bf16_round.argtypes = [_fp, _u16, C.c_longlong]
        L.orc_bf16_round.restype = None
        L.orc_heat_sum_f32.argtypes = [_fp, C.c_longlong]
        L.orc_heat_sum_f32.restype = d
        L.orc_heat_sum_f64.argtypes = [_dp, C.c_longlong]
        L.orc_heat_sum_f64.restype = d
        L.orc_heat_sum_bf16k.argtypes = [_u32, C.c_longlong]
        L.orc_heat_sum_bf16k.restype = d
        L.orc_sample_f32.argtypes = [_fp, _fp, _fp, i, i, i, f, i, _i64, i, _fp]
        L.orc_sample_f64.argtypes = [_dp, _dp, _dp, i, i, i, d, i, _i64, i, _dp]
        L.orc_adjoint_f64.argtypes = [_dp, _dp, _dp, _dp, i, i, i, d, i, i, i, _dp, _dp,
                                      C.POINTER(C.c_double)]
        L.orc_strip_warp_f32.argtypes = [_fp, _fp, _fp, i, i, i, f, i, i, i, i, i, i, _fp]
        L.orc_strip_warp_f64.argtypes = [_dp, _dp, _dp, i, i, i, d, i, i, i, i, i, i, _dp]
        L.orc_tilek_f32.argtypes = [_fp, _fp, _fp, i, i, i, f, i, i, i, i, i, i, _fp]
        L.orc_tilek_f64.argtypes = [_dp, _dp, _dp, i, i, i, d, i, i, i, i, i, i, _dp]
        L.orc_direct3_f32.argtypes = [_fp, _fp, _fp, i, i, i, i, f, i, i, _fp]
        L.orc_direct3_f64.argtypes = [_dp, _dp, _dp, i, i, i, i, d, i, i, _dp]
        L.orc_fission3_f32.argtypes = [_fp, _fp, _fp, i, i, i, i, f, i, i, i, i, i, _fp]
        L.orc_fission3_f64.argtypes = [_dp, _dp, _dp, i, i, i, i, d, i, i, i, i, i, _dp]
        L.orc_vecadd.argtypes = [_dp, _dp, _dp, i, i, i, i]
        L.orc_dynamic_reverse.argtypes = [_i32, i, i]
        L.orc_fetch_accounting.argtypes = [i, i, i, i, _i32, C.POINTER(C.c_int)]
        _LIB = L
    return _LIB


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def direct(u, kappa, src, steps, dt, bc, precision="f64", pool=1):
    """Run `steps` steps of the direct loop.  precision: 'f64' or 'f32'."""
    ny, nx = u.shape
    if precision == "f64":
        out = np.empty((ny, nx), np.float64)
        _check(lib().orc_direct_f64(_c(u, np.float64), _c(kappa, np.float64), _c(src, np.float64),
                                    nx, ny, steps, float(dt), bc, pool, out), "direct_f64")
    else:
        out = np.empty((ny, nx), np.float32)
        _check(lib().orc_direct_f32(_c(u, np.float32), _c(kappa, np.float32), _c(src, np.float32),
                                    nx, ny, steps, float(np.float32(dt)), bc, pool, out), "direct_f32")
    return out


def fission(u, kappa, src, steps, dt, bc, precision="f32", block=(16, 16), pool=1,
            block_per_fetch=0):
    """The tiled kernel executed per the paper's CPU execution model."""
    ny, nx = u.shape
    bx, by = block
    if precision == "f64":
        out = np.empty((ny, nx), np.float64)
        _check(lib().orc_fission_f64(_c(u, np.float64), _c(kappa, np.float64), _c(src, np.float64),
                                     nx, ny, steps, float(dt), bc, bx, by, pool, block_per_fetch,
                                     out), "fission_f64")
    else:
        out = np.empty((ny, nx), np.float32)
        _check(lib().orc_fission_f32(_c(u, np.float32), _c(kappa, np.float32), _c(src, np.float32),
                                     nx, ny, steps, float(np.float32(dt)), bc, bx, by, pool,
                                     block_per_fetch, out), "fission_f32")
    return out


def strip_warp(u, kappa, src, steps, dt, bc, precision="f32", k=4, chunk=64, warps=1, pool=1,
               fission=True):
    """The shuffle-based temporal-blocked strip kernel (a warp per 128-column
    strip, 4 cells per lane, k time levels per pass) executed per the paper's
    execution model for kernels with warp-level functions: nested warp / lane
    loops split at every shuffle (Sec. III "SPMD to MPMD").  fission=False ignores the
    split at the shuffles (for the test showing it is needed).  k <= 8."""
    ny, nx = u.shape
    T, fn = (np.float64, "orc_strip_warp_f64") if precision == "f64" else (np.float32, "orc_strip_warp_f32")
    out = np.empty((ny, nx), T)
    dtv = float(dt) if precision == "f64" else float(np.float32(dt))
    _check(getattr(lib(), fn)(_c(u, T), _c(kappa, T), _c(src, T), nx, ny, steps, dtv, bc, k, chunk,
                              warps, pool, 1 if fission else 0, out), fn)
    return out


def tile_blocked(u, kappa, src, steps, dt, bc, precision="f32", depth=4, block=(32, 8), pool=1,
                 fission=True):
    """The shared-memory temporal-blocked tiled kernel (depth steps per
    launch, depth + 1 barriers, depth of them inside its time loop) executed
    with loop fission on the thread pool; fission=False ignores the barriers."""
    ny, nx = u.shape
    T, fn = (np.float64, "orc_tilek_f64") if precision == "f64" else (np.float32, "orc_tilek_f32")
    out = np.empty((ny, nx), T)
    dtv = float(dt) if precision == "f64" else float(np.float32(dt))
    _check(getattr(lib(), fn)(_c(u, T), _c(kappa, T), _c(src, T), nx, ny, steps, dtv, bc, depth, block[0],
                              block[1], pool, 1 if fission else 0, out), fn)
    return out


def direct3(u, kappa, src, steps, dt, bc, precision="f32", pool=1):
    """The 3-D 7-point update as a plain loop over cells; arrays [nz, ny, nx]."""
    nz, ny, nx = u.shape
    T, fn = (np.float64, "orc_direct3_f64") if precision == "f64" else (np.float32, "orc_direct3_f32")
    out = np.empty((nz, ny, nx), T)
    dtv = float(dt) if precision == "f64" else float(np.float32(dt))
    _check(getattr(lib(), fn)(_c(u, T), _c(kappa, T), _c(src, T), nx, ny, nz, steps, dtv, bc, pool, out),
           fn)
    return out


def fission3(u, kappa, src, steps, dt, bc, precision="f32", block=(32, 8), zchunks=1, pool=1):
    """The z-marching tiled 3-D kernel (two barriers inside its plane loop)
    executed with loop fission on the thread pool."""
    nz, ny, nx = u.shape
    T, fn = (np.float64, "orc_fission3_f64") if precision == "f64" else (np.float32, "orc_fission3_f32")
    out = np.empty((nz, ny, nx), T)
    dtv = float(dt) if precision == "f64" else float(np.float32(dt))
    _check(getattr(lib(), fn)(_c(u, T), _c(kappa, T), _c(src, T), nx, ny, nz, steps, dtv, bc, block[0],
                              block[1], zchunks, pool, out), fn)
    return out


def bf16_round(x) -> np.ndarray:
    """IEEE round-to-nearest-even float32 -> bfloat16 bit patterns (uint16)."""
    x = _c(x, np.float32)
    out = np.empty(x.shape, np.uint16)
    lib().orc_bf16_round(x.reshape(-1), out.reshape(-1), x.size)
    return out


def bf16_to_f32(h) -> np.ndarray:
    return (np.asarray(h, dtype=np.uint32) << 16).view(np.float32)


def bf16k_pack(u) -> np.ndarray:
    """Initial BF16-Kahan state of a float32 field: hi = rn(u), cmp = rn(hi - u)."""
    u = _c(u, np.float32)
    hi = bf16_round(u)
    cmp = bf16_round(bf16_to_f32(hi) - u)
    return (hi.astype(np.uint32) | (cmp.astype(np.uint32) << 16)).astype(np.uint32)


def bf16k_value(st) -> np.ndarray:
    """Exact value (float64) of a BF16-Kahan state: hi - cmp."""
    st = np.asarray(st, dtype=np.uint32)
    hi = bf16_to_f32((st & 0xFFFF).astype(np.uint16)).astype(np.float64)
    cm = bf16_to_f32((st >> 16).astype(np.uint16)).astype(np.float64)
    return hi - cm


def direct_bf16k(state, kappa_bf16, src_bf16, steps, dt, bc, pool=1, compensate=True):
    """BF16-Kahan steps.  compensate=False is the no-compensation diagnostic."""
    ny, nx = state.shape
    out = np.empty((ny, nx), np.uint32)
    _check(lib().orc_direct_bf16k(_c(state, np.uint32), _c(kappa_bf16, np.uint16),
                                  _c(src_bf16, np.uint16), nx, ny, steps, float(np.float32(dt)), bc,
                                  1 if compensate else 0, pool, out), "direct_bf16k")
    return out


def pass_schedule(steps, k, have_scratch=True):
    """Depths of the passes the library runs for `steps` steps at depth k: k
    each, then steps % k; without a scratch buffer an even pass count is made
    odd by splitting the last pass of depth >= 2 into d - d//2 and d//2 (the
    rule the C header states for CPB_BF16_KAHAN_BLOCK).  Host logic only: the
    input of direct_bf16k_block."""
    d = [k] * (steps // k) + ([steps % k] if steps % k else [])
    if not have_scratch and d and len(d) % 2 == 0:
        for i in range(len(d) - 1, -1, -1):
            if d[i] >= 2:
                d[i:i + 1] = [d[i] - d[i] // 2, d[i] // 2]
                break
    return d


def direct_bf16k_block(state, kappa_bf16, src_bf16, depths, dt, bc, pool=1):
    """BF16-Kahan storage rounded once per pass: for each pass depth d the
    state's value hi - cmp (exact in FP32) advances d steps of the FP32 direct
    update with the bf16 kappa and source widened to FP32, then is rounded back
    into (hi, cmp) = (rn(v), rn(hi - v)).  Composed of direct() and
    bf16k_pack(), both pinned on their own."""
    st = np.ascontiguousarray(state, dtype=np.uint32)
    k32 = bf16_to_f32(kappa_bf16).reshape(st.shape)
    s32 = bf16_to_f32(src_bf16).reshape(st.shape)
    for d in depths:
        u = bf16k_value(st).astype(np.float32)
        u = direct(u, k32, s32, int(d), dt, bc, "f32", pool=pool)
        st = bf16k_pack(u)
    return st


def heat_sum_f32(u) -> float:
    u = _c(u, np.float32).reshape(-1)
    return lib().orc_heat_sum_f32(u, u.size)


def heat_sum_f64(u) -> float:
    u = _c(u, np.float64).reshape(-1)
    return lib().orc_heat_sum_f64(u, u.size)


def heat_sum_bf16k(st) -> float:
    st = _c(st, np.uint32).reshape(-1)
    return lib().orc_heat_sum_bf16k(st, st.size)


def sample(u, kappa, src, steps, dt, bc, idx, precision="f32"):
    """Values after `steps` steps at flat indices idx (j*nx+i), from dependency cones."""
    ny, nx = u.shape
    idx = _c(idx, np.int64).reshape(-1)
    if precision == "f64":
        out = np.empty(idx.size, np.float64)
        _check(lib().orc_sample_f64(_c(u, np.float64), _c(kappa, np.float64), _c(src, np.float64),
                                    nx, ny, steps, float(dt), bc, idx, idx.size, out), "sample_f64")
    else:
        out = np.empty(idx.size, np.float32)
        _check(lib().orc_sample_f32(_c(u, np.float32), _c(kappa, np.float32), _c(src, np.float32),
                                    nx, ny, steps, float(np.float32(dt)), bc, idx, idx.size, out),
               "sample_f32")
    return out


def adjoint_f64(u0, kappa, src, target, steps, dt, bc, ckpt=20, pool=1):
    """Returns (loss, dL/du0, dL/dkappa) for L = 0.5 ||u_T - target||^2, FP64."""
    ny, nx = u0.shape
    gu = np.empty((ny, nx), np.float64)
    gk = np.empty((ny, nx), np.float64)
    loss = C.c_double(0.0)
    _check(lib().orc_adjoint_f64(_c(u0, np.float64), _c(kappa, np.float64), _c(src, np.float64),
                                 _c(target, np.float64), nx, ny, steps, float(dt), bc, ckpt, pool,
                                 gu, gk, C.byref(loss)), "adjoint_f64")
    return loss.value, gu, gk


def vecadd(a, b, grid, block, pool=1):
    a = _c(a, np.float64)
    b = _c(b, np.float64)
    c = np.zeros_like(a)
    _check(lib().orc_vecadd(a, b, c, a.size, grid, block, pool), "vecadd")
    return c


def dynamic_reverse(d, fission=True):
    d = _c(d, np.int32).copy()
    _check(lib().orc_dynamic_reverse(d, d.size, 1 if fission else 0), "dynamic_reverse")
    return d


def fetch_accounting(grid, pool, block_per_fetch=0, fail_block=-1):
    """Returns (rc, counts per block, number of fetches)."""
    counts = np.zeros(max(grid, 1), np.int32)
    fetches = C.c_int(0)
    rc = lib().orc_fetch_accounting(grid, pool, block_per_fetch, fail_block, counts, C.byref(fetches))
    return rc, counts[:grid], fetches.value
