"""Python binding of libcpb (ctypes), a barrier-tiled heat stencil for GB300.

The functions named ``cpb_*`` mirror the C ABI in ``include/cpb.h`` one to one:
they only marshal arguments (torch tensors or integer device addresses,
streams) and turn a non-success status into :class:`CpbError`.  Every step of
the computation runs in the CUDA kernels of the shared library; there is no
CPU path.  If the library has not been built the first call raises.

Two builds are available: ``lib()`` (default, FMA contraction allowed) and
``lib(fma=False)`` (``--fmad=false``: the library's FP32 rounding order bit for
bit).  Module-level ``cpb_*`` functions use the default build; pass
``library=lib(fma=False)`` or call the methods of that object for the other.

Higher-level helpers: :func:`stencil` (allocating wrapper) and
:class:`StencilFn` (autograd), both built from the ``cpb_*`` calls.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

CPB_SUCCESS = 0
CPB_ERR_INVALID_VALUE = 1
CPB_ERR_UNSUPPORTED_CONFIG = 2
CPB_ERR_SHARED_MEM = 3
CPB_ERR_LAUNCH = 4
CPB_ERR_TIMEOUT = 5
CPB_ERR_CUDA = 6
CPB_ERR_WORKSPACE = 7

CPB_F32 = 0
CPB_BF16_KAHAN = 1
CPB_BF16_KAHAN_BLOCK = 2
CPB_DIRICHLET0 = 0
CPB_PERIODIC = 1


class CpbError(RuntimeError):
    def __init__(self, status: int, func: str, detail: str = ""):
        self.status = status
        super().__init__(f"{func}: status {status}" + (f" ({detail})" if detail else ""))


class cpb_dim3(C.Structure):
    _fields_ = [("x", C.c_uint), ("y", C.c_uint), ("z", C.c_uint)]


class cpb_grid_desc(C.Structure):
    _fields_ = [("u_in", C.c_void_p), ("u_out", C.c_void_p), ("kappa", C.c_void_p),
                ("src", C.c_void_p), ("nx", C.c_int), ("ny", C.c_int), ("steps", C.c_int),
                ("dt", C.c_float)]


# Candidates of cpb_batch_autotune (include/cpb.h): depth, then grain, then threads.
BATCH_TUNE_DEPTHS = (4, 8)
BATCH_TUNE_GRAINS = (1, 2, 4, 8, 16)
BATCH_TUNE_THREADS = (128, 256, 384)
BATCH_TUNE_CANDIDATES = len(BATCH_TUNE_DEPTHS) * len(BATCH_TUNE_GRAINS) * len(BATCH_TUNE_THREADS)


class cpb_batch_plan(C.Structure):
    _fields_ = [("grain", C.c_int), ("blocks", C.c_int), ("threads", C.c_int),
                ("team_cells", C.c_int), ("depth", C.c_int), ("team_warps", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class cpb_tuning(C.Structure):
    _fields_ = [("k", C.c_int), ("chunk_rows", C.c_int), ("warps_per_block", C.c_int),
                ("variant", C.c_int), ("stages", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_vp, _i, _f, _sz, _ll = C.c_void_p, C.c_int, C.c_float, C.c_size_t, C.c_longlong

# name -> (restype, argtypes); mirrors include/cpb.h
_SIGS = {
    "cpb_version": (_i, []),
    "cpb_status_string": (C.c_char_p, [_i]),
    "cpb_last_error_detail": (C.c_char_p, []),
    "cpb_device_info": (_i, [C.POINTER(_i), C.POINTER(_i), C.POINTER(_i)]),
    "cpb_stencil_launch": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _f, _i, _i, cpb_dim3, cpb_dim3, _sz,
                                _vp, _vp]),
    "cpb_stencil_launch_tuned": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _f, _i, _i,
                                      C.POINTER(cpb_tuning), _vp, _vp]),
    "cpb_set_tuning": (_i, [_i, _i, _i, _i, C.POINTER(cpb_tuning)]),
    "cpb_get_tuning": (_i, [_i, _i, _i, _i, C.POINTER(cpb_tuning)]),
    "cpb_lookup_tuning": (_i, [_i, _i, _i, _i, C.POINTER(cpb_tuning), C.POINTER(_i)]),
    "cpb_tuning_save": (_i, [C.c_char_p, C.c_char_p]),
    "cpb_tuning_load": (_i, [C.c_char_p, C.c_char_p, C.POINTER(_i)]),
    "cpb_autotune": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _f, _i, _i, _vp, C.POINTER(cpb_tuning)]),
    "cpb_device_status": (_i, [C.POINTER(_i)]),
    "cpb_bounds_status": (_i, [C.POINTER(_i), C.POINTER(_i)]),
    "cpb_debug_set": (_i, [_i, _i]),
    "cpb_heat_sum_workspace_bytes": (_sz, [_i, _i]),
    "cpb_heat_sum": (_i, [_vp, _i, _i, _i, _vp, _vp, _sz, _vp]),
    "cpb_heat_sum_noalloc": (_i, [_vp, _i, _i, _i, _vp, _vp]),
    "cpb_bf16_round": (_i, [_vp, _vp, _ll, _vp]),
    "cpb_bf16k_pack": (_i, [_vp, _vp, _ll, _vp]),
    "cpb_bf16k_unpack": (_i, [_vp, _vp, _ll, _vp]),
    "cpb_host_workspace_bytes": (_sz, [_i, _i, _i]),
    "cpb_stencil_host": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _f, _i, _i, _vp, _sz, _vp]),
    "cpb_stencil_host_async": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _f, _i, _i, _vp, _sz, _vp, _vp, _vp]),
    "cpb_batch_plan_default": (_i, [C.POINTER(cpb_batch_plan)]),
    "cpb_batch_order": (_i, [_vp, _i, C.POINTER(cpb_batch_plan), _vp, C.POINTER(_i)]),
    "cpb_batch_work_bytes": (_sz, []),
    "cpb_stencil_batched": (_i, [_vp, _vp, _i, _i, _i, _i, C.POINTER(cpb_batch_plan), _vp, _vp]),
    "cpb_batch_status": (_i, [_vp, C.POINTER(_i), _vp]),
    "cpb_tile_blocked_shared_bytes": (_sz, [_i, _i, _i]),
    "cpb_stencil_tile_blocked": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _i, _f, _i, cpb_dim3, cpb_dim3, _sz,
                                      _vp, _vp]),
    "cpb_stencil3d_shared_bytes": (_sz, [_i]),
    "cpb_stencil3d_launch": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _i, _f, _i, cpb_dim3, cpb_dim3, _sz,
                                  _vp, _vp]),
    "cpb_batch_autotune": (_i, [_vp, _vp, _i, _i, _i, _i, _vp, _vp, C.POINTER(cpb_batch_plan), _vp]),
    "cpb_adjoint_workspace_bytes": (_sz, [_i, _i, _i, _i]),
    "cpb_adjoint_forward": (_i, [_vp, _vp, _vp, _i, _i, _i, _f, _i, _i, _vp, _vp, _sz, _vp]),
    "cpb_adjoint_backward": (_i, [_vp, _vp, _vp, _i, _i, _i, _f, _i, _i, _vp, _vp, _vp, _sz, _vp]),
    "cpb_stencil_adjoint": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _f, _i, _i, _vp, _vp, _vp, _sz,
                                 _vp]),
    "cpb_graph_create": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _f, _i, _i, C.POINTER(cpb_tuning),
                              _vp, C.POINTER(_vp)]),
    "cpb_slab_rows": (_i, [_i, _i, _i, _i, _i, C.POINTER(_i), C.POINTER(_i), C.POINTER(_i), C.POINTER(_i)]),
    "cpb_slab_exchange": (_i, [_vp, _i, _i, _i, _i, _vp, _i, _i, _vp, _i, _i, _i, _vp]),
    "cpb_slab_exchange_rows": (_i, [_vp, _sz, _i, _i, _i, _vp, _i, _i, _vp, _i, _i, _vp]),
    "cpb_slab_step": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _i, _i, _f, _i, _i, C.POINTER(cpb_tuning), _vp]),
    "cpb_graph_launch": (_i, [_vp, _vp]),
    "cpb_graph_destroy": (_i, [_vp]),
}

EXPORTED = tuple(_SIGS)


def ptr(x) -> int | None:
    """Device address of a torch tensor, or an int / None passed through."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def host_ptr(x) -> int | None:
    """Host address of a numpy array or pinned torch CPU tensor."""
    if x is None:
        return None
    if hasattr(x, "ctypes"):
        return int(x.ctypes.data)
    return int(x.data_ptr())


def stream_handle(stream=None) -> int | None:
    """cudaStream_t of a torch stream (default: torch's current stream)."""
    if isinstance(stream, int):
        return stream
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _dim3(v) -> cpb_dim3:
    if isinstance(v, cpb_dim3):
        return v
    v = tuple(v) + (1,) * (3 - len(tuple(v))) if len(tuple(v)) < 3 else tuple(v)
    return cpb_dim3(*[int(a) for a in v])


class Library:
    """One loaded build of libcpb; methods mirror the C ABI."""

    def __init__(self, path: str):
        if not os.path.exists(path):
            raise RuntimeError(f"libcpb is not built ({path} missing): run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        self.path = path
        self._lib = C.CDLL(path, mode=C.RTLD_LOCAL)
        for name, (res, args) in _SIGS.items():
            fn = getattr(self._lib, name)
            fn.restype = res
            fn.argtypes = args

    def _call(self, name, *args):
        st = getattr(self._lib, name)(*args)
        if st != CPB_SUCCESS:
            detail = self._lib.cpb_last_error_detail().decode()
            raise CpbError(st, name, detail or self._lib.cpb_status_string(st).decode())
        return st

    # -- C ABI mirrors -----------------------------------------------------
    def cpb_version(self) -> int:
        return self._lib.cpb_version()

    def cpb_status_string(self, status: int) -> str:
        return self._lib.cpb_status_string(status).decode()

    def cpb_last_error_detail(self) -> str:
        return self._lib.cpb_last_error_detail().decode()

    def cpb_device_info(self):
        a, b, c = _i(), _i(), _i()
        self._call("cpb_device_info", C.byref(a), C.byref(b), C.byref(c))
        return {"sm_count": a.value, "l2_bytes": b.value, "smem_optin_bytes": c.value}

    def cpb_stencil_launch(self, u_in, u_out, kappa, src, nx, ny, steps, dt, bc, dtype, grid,
                           block, shared_bytes, scratch=None, stream=None):
        self._call("cpb_stencil_launch", ptr(u_in), ptr(u_out), ptr(kappa), ptr(src), nx, ny, steps,
                   float(dt), bc, dtype, _dim3(grid), _dim3(block), shared_bytes, ptr(scratch),
                   stream_handle(stream))

    def cpb_tile_blocked_shared_bytes(self, bx, by, depth) -> int:
        return self._lib.cpb_tile_blocked_shared_bytes(bx, by, depth)

    def cpb_stencil_tile_blocked(self, u_in, u_out, kappa, src, nx, ny, steps, depth, dt, bc, grid, block,
                                 shared_bytes, scratch=None, stream=None):
        self._call("cpb_stencil_tile_blocked", ptr(u_in), ptr(u_out), ptr(kappa), ptr(src), nx, ny, steps,
                   depth, float(dt), bc, _dim3(grid), _dim3(block), shared_bytes, ptr(scratch),
                   stream_handle(stream))

    def cpb_stencil3d_shared_bytes(self, by) -> int:
        return self._lib.cpb_stencil3d_shared_bytes(by)

    def cpb_stencil3d_launch(self, u_in, u_out, kappa, src, nx, ny, nz, steps, dt, bc,
                             grid=(0, 0, 0), block=(0, 0, 0), shared_bytes=0, scratch=None, stream=None):
        self._call("cpb_stencil3d_launch", ptr(u_in), ptr(u_out), ptr(kappa), ptr(src), nx, ny, nz, steps,
                   float(dt), bc, _dim3(grid), _dim3(block), shared_bytes, ptr(scratch),
                   stream_handle(stream))

    def cpb_stencil_launch_tuned(self, u_in, u_out, kappa, src, nx, ny, steps, dt, bc, dtype,
                                 tuning=None, scratch=None, stream=None):
        t = C.byref(as_tuning(tuning)) if tuning is not None else None
        self._call("cpb_stencil_launch_tuned", ptr(u_in), ptr(u_out), ptr(kappa), ptr(src), nx, ny,
                   steps, float(dt), bc, dtype, t, ptr(scratch), stream_handle(stream))

    def cpb_set_tuning(self, nx, ny, dtype, bc, tuning):
        self._call("cpb_set_tuning", nx, ny, dtype, bc, C.byref(as_tuning(tuning)))

    def cpb_get_tuning(self, nx, ny, dtype, bc) -> dict:
        t = cpb_tuning()
        self._call("cpb_get_tuning", nx, ny, dtype, bc, C.byref(t))
        return t.as_dict()

    def cpb_lookup_tuning(self, nx, ny, dtype, bc):
        """The cached tuning (dict) for the key, or None."""
        t, found = cpb_tuning(), _i()
        self._call("cpb_lookup_tuning", nx, ny, dtype, bc, C.byref(t), C.byref(found))
        return t.as_dict() if found.value else None

    def cpb_tuning_save(self, path, device=None):
        self._call("cpb_tuning_save", os.fsencode(path), device.encode() if device else None)

    def cpb_tuning_load(self, path, device=None) -> int:
        n = _i()
        self._call("cpb_tuning_load", os.fsencode(path), device.encode() if device else None, C.byref(n))
        return n.value

    def cpb_autotune(self, u_a, u_b, kappa, src, nx, ny, steps, dt, bc, dtype, stream=None) -> dict:
        t = cpb_tuning()
        self._call("cpb_autotune", ptr(u_a), ptr(u_b), ptr(kappa), ptr(src), nx, ny, steps, float(dt),
                   bc, dtype, stream_handle(stream), C.byref(t))
        return t.as_dict()

    def cpb_device_status(self) -> int:
        st = _i()
        self._call("cpb_device_status", C.byref(st))
        return st.value

    def cpb_bounds_status(self):
        """(unit, line) of the first out-of-range access since the last call,
        (0, 0) if none; raises CpbError outside the bounds-checked build."""
        u, ln = _i(), _i()
        self._call("cpb_bounds_status", C.byref(u), C.byref(ln))
        return u.value, ln.value

    def cpb_debug_set(self, wait_limit, inject_row):
        self._call("cpb_debug_set", wait_limit, inject_row)

    def cpb_heat_sum_workspace_bytes(self, nx, ny) -> int:
        return self._lib.cpb_heat_sum_workspace_bytes(nx, ny)

    def cpb_heat_sum(self, u, nx, ny, dtype, d_out, workspace, ws_bytes, stream=None):
        self._call("cpb_heat_sum", ptr(u), nx, ny, dtype, ptr(d_out), ptr(workspace), ws_bytes,
                   stream_handle(stream))

    def cpb_heat_sum_noalloc(self, u, nx, ny, dtype, d_out, stream=None):
        self._call("cpb_heat_sum_noalloc", ptr(u), nx, ny, dtype, ptr(d_out), stream_handle(stream))

    def cpb_bf16_round(self, x, out, n, stream=None):
        self._call("cpb_bf16_round", ptr(x), ptr(out), n, stream_handle(stream))

    def cpb_bf16k_pack(self, u, state, n, stream=None):
        self._call("cpb_bf16k_pack", ptr(u), ptr(state), n, stream_handle(stream))

    def cpb_bf16k_unpack(self, state, u, n, stream=None):
        self._call("cpb_bf16k_unpack", ptr(state), ptr(u), n, stream_handle(stream))

    def cpb_host_workspace_bytes(self, nx, ny, dtype) -> int:
        return self._lib.cpb_host_workspace_bytes(nx, ny, dtype)

    def cpb_stencil_host(self, u0_host, kappa_host, src_host, u_out_host, nx, ny, steps, dt, bc,
                         dtype, d_workspace, ws_bytes, stream=None):
        self._call("cpb_stencil_host", host_ptr(u0_host), host_ptr(kappa_host), host_ptr(src_host),
                   host_ptr(u_out_host), nx, ny, steps, float(dt), bc, dtype, ptr(d_workspace),
                   ws_bytes, stream_handle(stream))

    def cpb_stencil_host_async(self, u0_host, kappa_host, src_host, u_out_host, nx, ny, steps, dt, bc,
                               dtype, d_workspace, ws_bytes, h2d, compute, d2h):
        self._call("cpb_stencil_host_async", host_ptr(u0_host), host_ptr(kappa_host), host_ptr(src_host),
                   host_ptr(u_out_host), nx, ny, steps, float(dt), bc, dtype, ptr(d_workspace), ws_bytes,
                   stream_handle(h2d), stream_handle(compute), stream_handle(d2h))

    def cpb_batch_plan_default(self) -> dict:
        p = cpb_batch_plan()
        self._call("cpb_batch_plan_default", C.byref(p))
        return p.as_dict()

    def cpb_batch_order(self, h_descs, plan=None):
        """h_descs: ctypes array of cpb_grid_desc.  Returns (order list, n_large)."""
        n = len(h_descs)
        order = (C.c_int * max(n, 1))()
        nl = _i()
        pl = C.byref(as_plan(plan)) if plan is not None else None
        self._call("cpb_batch_order", C.addressof(h_descs) if n else None, n, pl, C.addressof(order),
                   C.byref(nl))
        return list(order[:n]), nl.value

    def cpb_batch_work_bytes(self) -> int:
        return self._lib.cpb_batch_work_bytes()

    def cpb_stencil_batched(self, d_descs, d_order, ngrids, n_large, dtype, bc, plan=None,
                            d_work=None, stream=None):
        pl = C.byref(as_plan(plan)) if plan is not None else None
        self._call("cpb_stencil_batched", ptr(d_descs), ptr(d_order), ngrids, n_large, dtype, bc, pl,
                   ptr(d_work), stream_handle(stream))

    def cpb_batch_status(self, d_work, stream=None) -> int:
        st = _i()
        self._call("cpb_batch_status", ptr(d_work), C.byref(st), stream_handle(stream))
        return st.value

    def cpb_batch_autotune(self, d_descs, d_order, ngrids, n_large, dtype, bc, d_work, plan=None,
                           stream=None):
        """Returns (best plan dict, {(depth, grain, threads): ms or None}).
        Overwrites every grid's u_in and u_out (tune on copies)."""
        pl = as_plan(plan if plan is not None else self.cpb_batch_plan_default())
        table = (C.c_float * BATCH_TUNE_CANDIDATES)()
        self._call("cpb_batch_autotune", ptr(d_descs), ptr(d_order), ngrids, n_large, dtype, bc,
                   ptr(d_work), stream_handle(stream), C.byref(pl), table)
        ms = {}
        i = 0
        for d in BATCH_TUNE_DEPTHS:
            for g in BATCH_TUNE_GRAINS:
                for t in BATCH_TUNE_THREADS:
                    ms[(d, g, t)] = float(table[i]) if table[i] > 0 else None
                    i += 1
        return pl.as_dict(), ms

    def cpb_adjoint_workspace_bytes(self, nx, ny, steps, ckpt_every) -> int:
        return self._lib.cpb_adjoint_workspace_bytes(nx, ny, steps, ckpt_every)

    def cpb_adjoint_forward(self, u0, kappa, src, nx, ny, steps, dt, bc, ckpt_every, u_T, workspace,
                            ws_bytes, stream=None):
        self._call("cpb_adjoint_forward", ptr(u0), ptr(kappa), ptr(src), nx, ny, steps, float(dt), bc,
                   ckpt_every, ptr(u_T), ptr(workspace), ws_bytes, stream_handle(stream))

    def cpb_adjoint_backward(self, kappa, src, lambda_T, nx, ny, steps, dt, bc, ckpt_every, grad_u0,
                             grad_kappa, workspace, ws_bytes, stream=None):
        self._call("cpb_adjoint_backward", ptr(kappa), ptr(src), ptr(lambda_T), nx, ny, steps,
                   float(dt), bc, ckpt_every, ptr(grad_u0), ptr(grad_kappa), ptr(workspace), ws_bytes,
                   stream_handle(stream))

    def cpb_stencil_adjoint(self, u0, kappa, src, lambda_T, nx, ny, steps, dt, bc, ckpt_every,
                            grad_u0, grad_kappa, workspace, ws_bytes, stream=None):
        self._call("cpb_stencil_adjoint", ptr(u0), ptr(kappa), ptr(src), ptr(lambda_T), nx, ny, steps,
                   float(dt), bc, ckpt_every, ptr(grad_u0), ptr(grad_kappa), ptr(workspace), ws_bytes,
                   stream_handle(stream))

    def cpb_graph_create(self, u_in, u_out, kappa, src, nx, ny, steps, dt, bc, dtype, tuning=None,
                         scratch=None) -> int:
        g = _vp()
        t = C.byref(as_tuning(tuning)) if tuning is not None else None
        self._call("cpb_graph_create", ptr(u_in), ptr(u_out), ptr(kappa), ptr(src), nx, ny, steps,
                   float(dt), bc, dtype, t, ptr(scratch), C.byref(g))
        return g.value

    def cpb_slab_rows(self, ny, world, rank, depth, bc) -> dict:
        lo, hi, hl, hh = _i(), _i(), _i(), _i()
        self._call("cpb_slab_rows", ny, world, rank, depth, bc, C.byref(lo), C.byref(hi), C.byref(hl),
                   C.byref(hh))
        return {"row_lo": lo.value, "row_hi": hi.value, "halo_lo": hl.value, "halo_hi": hh.value}

    def cpb_slab_exchange(self, slab, nx, n_own, halo_lo, halo_hi, below, below_halo_lo, below_n_own, above,
                          above_halo_lo, above_n_own, dtype, stream=None):
        self._call("cpb_slab_exchange", ptr(slab), nx, n_own, halo_lo, halo_hi, ptr(below), below_halo_lo,
                   below_n_own, ptr(above), above_halo_lo, above_n_own, dtype, stream_handle(stream))

    def cpb_slab_exchange_rows(self, slab, row_bytes, n_own, halo_lo, halo_hi, below, below_halo_lo, below_n_own,
                               above, above_halo_lo, above_n_own, stream=None):
        self._call("cpb_slab_exchange_rows", ptr(slab), row_bytes, n_own, halo_lo, halo_hi, ptr(below),
                   below_halo_lo, below_n_own, ptr(above), above_halo_lo, above_n_own, stream_handle(stream))

    def cpb_slab_step(self, u_in, u_out, kappa, src, nx, rows_total, halo_lo, halo_hi, steps, dt, bc, dtype,
                      tuning=None, stream=None):
        t = C.byref(as_tuning(tuning)) if tuning is not None else None
        self._call("cpb_slab_step", ptr(u_in), ptr(u_out), ptr(kappa), ptr(src), nx, rows_total, halo_lo,
                   halo_hi, steps, float(dt), bc, dtype, t, stream_handle(stream))

    def cpb_graph_launch(self, graph, stream=None):
        self._call("cpb_graph_launch", graph, stream_handle(stream))

    def cpb_graph_destroy(self, graph):
        self._call("cpb_graph_destroy", graph)


def as_tuning(t) -> cpb_tuning:
    if isinstance(t, cpb_tuning):
        return t
    if isinstance(t, dict):
        return cpb_tuning(int(t["k"]), int(t["chunk_rows"]), int(t.get("warps_per_block", 4)),
                          int(t.get("variant", 0)), int(t.get("stages", 8)))
    return cpb_tuning(*[int(v) for v in t])


def as_plan(p) -> cpb_batch_plan:
    if isinstance(p, cpb_batch_plan):
        return p
    d = {"grain": 1, "blocks": 0, "team_cells": 65536, "depth": 4}
    d.update(p)
    d.setdefault("threads", 384 if int(d["depth"]) <= 4 else 256)
    return cpb_batch_plan(int(d["grain"]), int(d["blocks"]), int(d["threads"]), int(d["team_cells"]),
                          int(d.get("depth", 4)), int(d.get("team_warps", 1)))


_LIBS: dict[bool, Library] = {}


def lib(fma: bool = True) -> Library:
    """The default build (fma=True) or the --fmad=false build."""
    if fma not in _LIBS:
        _LIBS[fma] = Library(_build.lib_path("libcpb.so" if fma else "libcpb_nofma.so"))
    return _LIBS[fma]


_CHECKED: list = []


def lib_checked() -> Library:
    """The bounds-checked build (--fmad=false arithmetic, cpb_bounds_status)."""
    if not _CHECKED:
        _CHECKED.append(Library(_build.lib_path("libcpb_check.so")))
    return _CHECKED[0]


def _forward(name):
    def f(*args, library: Library | None = None, **kw):
        return getattr(library or lib(), name)(*args, **kw)
    f.__name__ = name
    f.__doc__ = f"Module-level {name} on the default build (see include/cpb.h)."
    return f


for _n in _SIGS:
    globals()[_n] = _forward(_n)


# ---------------------------------------------------------------------------
# Convenience wrappers built on the C ABI (torch for memory and streams only)
# ---------------------------------------------------------------------------
def stencil(u, kappa, src, steps, dt, bc=CPB_DIRICHLET0, dtype=CPB_F32, tuning=None,
            library: Library | None = None, stream=None):
    """Return a new tensor holding `steps` steps applied to u (u is not modified)."""
    import torch
    out = torch.empty_like(u)
    scratch = torch.empty_like(u) if steps >= 2 else None
    ny, nx = u.shape[0], u.shape[1]
    (library or lib()).cpb_stencil_launch_tuned(u, out, kappa, src, nx, ny, steps, dt, bc, dtype,
                                                tuning=tuning, scratch=scratch, stream=stream)
    return out


def heat_sum(u, dtype=CPB_F32, library: Library | None = None, stream=None):
    """FP64 heat sum of a device field; returns a 0-d float64 CUDA tensor."""
    import torch
    L = library or lib()
    ny, nx = u.shape[0], u.shape[1]
    ws_bytes = L.cpb_heat_sum_workspace_bytes(nx, ny)
    ws = torch.empty(max(ws_bytes, 8) // 8, dtype=torch.float64, device=u.device)
    out = torch.empty((), dtype=torch.float64, device=u.device)
    L.cpb_heat_sum(u, nx, ny, dtype, out, ws, ws_bytes, stream=stream)
    return out


def batch_descriptors(u_in, u_out, kappa, src, offsets, nx, ny, steps, dt):
    """Descriptors of grids packed back to back in flat device tensors.

    u_in/u_out/kappa/src: flat float32 CUDA tensors holding every grid (src may
    be None); offsets/nx/ny/steps/dt: per-grid sequences (element offsets).
    Returns a ctypes array of cpb_grid_desc (host memory)."""
    n = len(nx)
    arr = (cpb_grid_desc * n)()
    bu, bo, bk = ptr(u_in), ptr(u_out), ptr(kappa)
    bs = ptr(src) if src is not None else None
    for g in range(n):
        off = 4 * int(offsets[g])
        arr[g] = cpb_grid_desc(bu + off, bo + off, bk + off, (bs + off) if bs is not None else None,
                               int(nx[g]), int(ny[g]), int(steps[g]), float(dt[g]))
    return arr


def to_device_bytes(carray, device):
    """Copy a ctypes array (descriptors or int order) into a CUDA uint8 tensor."""
    import torch
    raw = bytes(carray) if len(carray) else b"\0"
    return torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(device)


def _stencil_fn():
    import torch

    class StencilFn(torch.autograd.Function):
        """u_T = N steps of the stencil from u0; differentiable w.r.t. u0 and kappa.

        apply(u0, kappa, src, steps, dt, bc=CPB_DIRICHLET0, ckpt_every=20, library=None)
        Forward keeps checkpoints every `ckpt_every` steps in a workspace; backward
        runs the library's adjoint (cpb_adjoint_backward).  FP32 storage."""

        @staticmethod
        def forward(ctx, u0, kappa, src, steps, dt, bc=CPB_DIRICHLET0, ckpt_every=20, library=None):
            L = library or lib()
            ny, nx = u0.shape
            wsb = L.cpb_adjoint_workspace_bytes(nx, ny, steps, ckpt_every)
            ws = torch.empty(wsb, dtype=torch.uint8, device=u0.device)
            u0c, kc = u0.contiguous(), kappa.contiguous()
            sc = src.contiguous() if src is not None else None
            uT = torch.empty_like(u0c)
            L.cpb_adjoint_forward(u0c, kc, sc, nx, ny, steps, dt, bc, ckpt_every, uT, ws, wsb)
            ctx.save_for_backward(kc)
            ctx.extra = (sc, ws, wsb, nx, ny, steps, dt, bc, ckpt_every, L)
            return uT

        @staticmethod
        def backward(ctx, grad_uT):
            (kc,) = ctx.saved_tensors
            sc, ws, wsb, nx, ny, steps, dt, bc, ckpt_every, L = ctx.extra
            g = grad_uT.contiguous()
            gu0 = torch.empty_like(g)
            gk = torch.empty_like(g)
            L.cpb_adjoint_backward(kc, sc, g, nx, ny, steps, dt, bc, ckpt_every, gu0, gk, ws, wsb)
            return gu0, gk, None, None, None, None, None, None

    return StencilFn


def __getattr__(name):
    if name == "StencilFn":
        fn = _stencil_fn()
        globals()["StencilFn"] = fn
        return fn
    raise AttributeError(name)
