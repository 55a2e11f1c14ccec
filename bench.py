"""Benchmark: Gcell-updates/s and fraction of the HBM roofline on one GB300.

Headline workload (one bench step): the plain FP32 stencil at scale -- one
8192 x 8192 grid, lognormal conductivity, periodic boundary, 1000 time steps
at the autotuned temporal-block depth -- followed by the FP64 heat sum of the
result.  Inputs (4 x 256 MiB) are larger than L2 and resident in HBM when the
timed region starts.  The other forms of the path (BF16-Kahan storage at
16384^2, the 4096-grid batch, the adjoint at 2048^2, the 3-D 7-point variant
at 512^3, the multi-barrier kernel at 8192^2, the 512^2 small workload with
the tiled kernel, the tuned path and a CUDA-graph replay) are reported under
"forms" (skipped with --no-forms).

Arms:
  default            the CUDA library (libcpb.so) through its C ABI.
  --impl reference   the CPU oracle (the paper's execution model: tiled kernel
                     run block by block with loop fission on a thread pool),
                     timed on this machine's host cores on a bounded sample.

Multi-GPU: one process per GPU (torchrun); every rank runs its own replica of
the workload (the problems are independent, no collective on the data path);
value = all ranks' cell updates / max-over-ranks time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "Gcell-updates/s and % of HBM roofline (FP32 plain vs BF16/batched/adjoint)"
UNIT = "Gcell-updates/s"
BYTES_PER_CELL_PASS = {"f32": 16, "bf16k": 12}  # read u, kappa, s + write u, once per pass


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


STREAM_SOURCES = ("paper_2206_07896_gb300/csrc/k_stream.cuh", "paper_2206_07896_gb300/csrc/common.cuh",
                  "paper_2206_07896_gb300/csrc/internal.h")


def stream_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in STREAM_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def recorded_traffic(tuning, nx, ny):
    """DRAM bytes per launch of the stream kernel from the committed ncu record
    (profiles/stream_traffic.json: one entry per captured tuning), scaled to
    this grid by cell count; None if the kernel sources changed since the
    counters were taken or no entry has this depth and row-load variant.  The
    CTA shape and chunk height of the entry may differ from the autotuned
    ones: the DRAM bytes per cell do not depend on them (16.13-16.16 over
    every captured shape; halo re-reads come from L2)."""
    p = os.path.join(ROOT, "profiles", "stream_traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p))
    if rec.get("source_sha256") != stream_source_hash():
        return None
    for e in rec.get("entries", []):
        t = e.get("tuning", {})
        if all(int(t.get(key, -1)) == int(tuning.get(key, -2)) for key in ("k", "variant")):
            return float(e["dram_bytes_per_cell"]) * nx * ny
    return None


# FP32 operations per cell-update of the canonical update with the face sums
# (kc + kn) and dt * s held across the steps of a pass: 4 differences, 4
# products, 3 sums, hdt * acc, + dt * s, c + (..): 14.  This is the
# algorithmic figure the roofline reports against.  The flux form shares each
# face flux between its two cells and executes about 10 (FLUX_OPS_PER_UPDATE):
# the implementation's own lane bound, reported beside it.
ALG_OPS_PER_UPDATE = 14
FLUX_OPS_PER_UPDATE = 10


def stream_roofline(cells, k, pass_ms, hbm_gbs, sms, mhz):
    """Roofline of one pass of depth k over `cells` cells taking pass_ms.
    Two lower bounds: HBM (16 B per cell: u, kappa, s read and u written,
    at the measured copy rate) and FP32 lanes (ALG_OPS_PER_UPDATE operations
    per cell-update, one per lane per clock, 128 lanes per SM).  The binding
    bound is the larger time; `achieved` is the algorithmic bytes (hbm) or
    operations (alu) per second of the pass against that bound's peak."""
    alg_bytes = 16.0 * cells
    alg_ops = float(ALG_OPS_PER_UPDATE) * cells * k
    alu_peak = sms * 128 * mhz * 1e6                    # FP32 operations per second
    t_hbm, t_alu = alg_bytes / (hbm_gbs * 1e9), alg_ops / alu_peak
    sec = pass_ms * 1e-3
    hbm = {"achieved": alg_bytes / sec / 1e9, "peak": hbm_gbs, "unit": "GB/s",
           "frac": alg_bytes / sec / 1e9 / hbm_gbs, "time_bound_us": t_hbm * 1e6,
           "algorithmic_bytes_per_launch": alg_bytes}
    alu = {"achieved": alg_ops / sec / 1e12, "peak": alu_peak / 1e12, "unit": "TFLOP/s",
           "frac": alg_ops / sec / alu_peak, "time_bound_us": t_alu * 1e6,
           "algorithmic_ops_per_launch": alg_ops, "ops_per_update": ALG_OPS_PER_UPDATE,
           "peak_derivation": f"{sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz, one operation per lane per clock"}
    main = alu if t_alu > t_hbm else hbm
    return {"bound": "alu" if t_alu > t_hbm else "hbm", "achieved": main["achieved"], "peak": main["peak"],
            "unit": main["unit"], "frac": main["frac"], "hbm": hbm, "alu": alu}


def time_bounds(cells, k, hbm_gbs, clk):
    """Lower bounds on one pass of depth k over `cells` cells: HBM bytes at the
    measured copy rate, and the flux form's FP32 lane operations
    (FLUX_OPS_PER_UPDATE per cell-update) on all SMs at the sampled SM clock
    (or the maximum clock if none was sampled)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
    t_hbm = 16.0 * cells / (hbm_gbs * 1e9) * 1e6
    t_fp32 = float(FLUX_OPS_PER_UPDATE) * cells * k / (sms * 128 * mhz * 1e6) * 1e6
    return {"hbm": t_hbm, "fp32_lanes": t_fp32, "fp32_lanes_ops_per_update": FLUX_OPS_PER_UPDATE,
            "sms": sms, "sm_mhz": mhz}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate(times_ms, updates_per_rank):
    """Whole-job throughput from per-rank times: all ranks' updates / max time."""
    tmax = max(times_ms)
    return sum(updates_per_rank) / (tmax * 1e-3) / 1e9, tmax


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        hi = max(sm)
        loaded = [s for s in sm if s >= 0.5 * hi] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_sample(g, target_s=12.0):
    """Time the fission oracle (FP32, all host cores) on the full grid for as
    many time steps as fit in about target_s seconds.  Returns (Gcell/s, dict)."""
    import oracle
    cores = oracle.host_cores()
    t0 = time.perf_counter()
    oracle.fission(g.u, g.kappa, g.src, 1, g.dt, g.bc, "f32", block=(16, 16), pool=cores)
    t1 = time.perf_counter() - t0
    steps = max(1, int(target_s / max(t1, 1e-3)))
    t0 = time.perf_counter()
    oracle.fission(g.u, g.kappa, g.src, steps, g.dt, g.bc, "f32", block=(16, 16), pool=cores)
    dt = time.perf_counter() - t0
    rate = g.nx * g.ny * steps / dt / 1e9
    return rate, {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                  "sample": f"{steps} time steps of the full {g.nx}x{g.ny} grid, tiled kernel "
                            f"executed with loop fission on a {cores}-thread pool, FP32, "
                            f"{dt:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    g = W.plain_scale(seed=1, n=args.n, steps=args.time_steps)
    cores = oracle.host_cores()
    # Each bench step: a bounded sample of the workload (a few time steps of the
    # full grid) sized so the whole run stays within a few minutes.
    t0 = time.perf_counter()
    oracle.fission(g.u, g.kappa, g.src, 1, g.dt, g.bc, "f32", pool=cores)
    one = time.perf_counter() - t0
    per_step = max(1, int(min(20.0, 150.0 / max(1, args.steps + args.warmup)) / max(one, 1e-3)))
    for _ in range(args.warmup):
        oracle.fission(g.u, g.kappa, g.src, per_step, g.dt, g.bc, "f32", pool=cores)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.fission(g.u, g.kappa, g.src, per_step, g.dt, g.bc, "f32", pool=cores)
        ts.append(time.perf_counter() - t0)
    total = sum(ts)
    value = g.nx * g.ny * per_step * args.steps / total / 1e9
    sample = (f"{per_step} time steps of the full {g.nx}x{g.ny} grid per bench step, tiled kernel "
              f"executed with loop fission on a {cores}-thread pool, FP32")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": g.name, "nx": g.nx, "ny": g.ny, "bc": "periodic",
                       "time_steps_per_bench_step": per_step, "parallelism": "cpu thread pool"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Other forms of the path (reported under "forms", not part of "value")
# ---------------------------------------------------------------------------
def _time(fn, reps, stream):
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def form_precision(L, cpb, dev, stream, n=16384, steps=2000):
    """FP32 vs BF16-Kahan storage on the 16384^2 Dirichlet workload."""
    import torch
    g = W.precision(n=n, steps=steps)
    nx, ny = g.nx, g.ny
    sh = stream.cuda_stream
    u = torch.from_numpy(g.u).to(dev)
    k = torch.from_numpy(g.kappa).to(dev)
    s = torch.from_numpy(g.src).to(dev)
    del g
    a, b, out = torch.empty_like(u), torch.empty_like(u), torch.empty_like(u)
    a.copy_(u)
    t32 = L.cpb_autotune(a, b, k, s, nx, ny, 24, 1e-4, W.DIRICHLET, cpb.CPB_F32, stream=sh)
    dt = float(np.float32(0.2 / float(k.max())))
    ms32 = _time(lambda: L.cpb_stencil_launch_tuned(u, out, k, s, nx, ny, steps, dt, W.DIRICHLET,
                                                    cpb.CPB_F32, tuning=t32, scratch=a, stream=sh),
                 2, stream)
    ref32 = out.clone()
    hs = torch.empty(L.cpb_heat_sum_workspace_bytes(nx, ny) // 8 + 1, dtype=torch.float64, device=dev)
    d_sum = torch.empty((), dtype=torch.float64, device=dev)
    ms_sum = _time(lambda: L.cpb_heat_sum(ref32, nx, ny, cpb.CPB_F32, d_sum, hs, hs.numel() * 8,
                                          stream=sh), 3, stream)
    # BF16-Kahan state and bf16 fields, converted on the device
    N = nx * ny
    st = torch.empty(N, dtype=torch.int32, device=dev)
    kb = torch.empty(N, dtype=torch.int16, device=dev)
    sb = torch.empty(N, dtype=torch.int16, device=dev)
    L.cpb_bf16k_pack(u, st, N, stream=sh)
    L.cpb_bf16_round(k, kb, N, stream=sh)
    L.cpb_bf16_round(s, sb, N, stream=sh)
    del a, b
    sa, sbuf, so = torch.empty_like(st), torch.empty_like(st), torch.empty_like(st)
    sa.copy_(st)
    t16 = L.cpb_autotune(sa, sbuf, kb, sb, nx, ny, 24, dt, W.DIRICHLET, cpb.CPB_BF16_KAHAN, stream=sh)
    ms16 = _time(lambda: L.cpb_stencil_launch_tuned(st, so, kb, sb, nx, ny, steps, dt, W.DIRICHLET,
                                                    cpb.CPB_BF16_KAHAN, tuning=t16, scratch=sa,
                                                    stream=sh), 2, stream)
    un = torch.empty_like(u)
    L.cpb_bf16k_unpack(so, un, N, stream=sh)
    torch.cuda.synchronize()
    diff = float((un - ref32).abs().max() / ref32.abs().max())
    # BF16-Kahan storage rounded once per pass (CPB_BF16_KAHAN_BLOCK)
    sa.copy_(st)
    t16b = L.cpb_autotune(sa, sbuf, kb, sb, nx, ny, 24, dt, W.DIRICHLET, cpb.CPB_BF16_KAHAN_BLOCK, stream=sh)
    ms16b = _time(lambda: L.cpb_stencil_launch_tuned(st, so, kb, sb, nx, ny, steps, dt, W.DIRICHLET,
                                                     cpb.CPB_BF16_KAHAN_BLOCK, tuning=t16b, scratch=sa,
                                                     stream=sh), 2, stream)
    L.cpb_bf16k_unpack(so, un, N, stream=sh)
    torch.cuda.synchronize()
    diff_b = float((un - ref32).abs().max() / ref32.abs().max())
    upd = N * steps
    hbm, _ = peaks()
    # The same comparison at depth 2, where both storages are HBM-bound (the
    # regime in which 12 instead of 16 bytes per cell-update pays).
    k2 = {"k": 2, "chunk_rows": 256, "warps_per_block": 1, "variant": 1, "stages": 2}
    ms32_k2 = _time(lambda: L.cpb_stencil_launch_tuned(u, out, k, s, nx, ny, steps, dt, W.DIRICHLET,
                                                       cpb.CPB_F32, tuning=k2, scratch=sa.view(torch.float32),
                                                       stream=sh), 1, stream)
    ms16_k2 = _time(lambda: L.cpb_stencil_launch_tuned(st, so, kb, sb, nx, ny, steps, dt, W.DIRICHLET,
                                                       cpb.CPB_BF16_KAHAN, tuning=k2, scratch=sa, stream=sh),
                    1, stream)
    return {"workload": f"precision-{n}x{n}-dirichlet-{steps}steps",
            "f32": {"gcells": upd / ms32 / 1e6, "ms": ms32, "tuning": t32,
                    "effective_gbs_16B": upd * 16 / t32["k"] / ms32 / 1e6},
            "bf16_kahan": {"gcells": upd / ms16 / 1e6, "ms": ms16, "tuning": t16,
                           "effective_gbs_12B": upd * 12 / t16["k"] / ms16 / 1e6,
                           "rel_linf_vs_f32_gpu": diff, "rounding": "every step"},
            "bf16_kahan_block": {"gcells": upd / ms16b / 1e6, "ms": ms16b, "tuning": t16b,
                                 "effective_gbs_12B": upd * 12 / t16b["k"] / ms16b / 1e6,
                                 "rel_linf_vs_f32_gpu": diff_b, "rounding": "once per pass (where stored)"},
            "speedup_bf16_vs_f32": ms32 / ms16,
            "speedup_bf16_block_vs_f32": ms32 / ms16b,
            "at_depth_2": {"f32_gcells": upd / ms32_k2 / 1e6, "bf16_kahan_gcells": upd / ms16_k2 / 1e6,
                           "speedup_bf16_vs_f32": ms32_k2 / ms16_k2},
            "heat_sum_fp64": {"ms": ms_sum, "gbs": N * 4 / ms_sum / 1e6, "frac_hbm": N * 4 / ms_sum / 1e6 / hbm},
            "note": "errors vs the FP64 oracle at this size (2000 steps, FP32 and both BF16 forms, also "
                    "against FP64 on the bf16-quantised inputs) are measured by "
                    "tests/test_gpu_precision.py::test_precision_workload_full_size_against_fp64"}


def form_batched(L, cpb, dev, stream, ngrids=4096):
    """4096 uneven grids in one persistent launch vs one tuned launch sequence per grid."""
    import ctypes as C
    import torch
    bt = W.batching(ngrids=ngrids)
    sh = stream.cuda_stream
    # pad each grid to a 16-byte boundary so the 128-bit path applies where nx % 4 == 0
    cells = (bt.nx.astype(np.int64) * bt.ny.astype(np.int64))
    off = np.zeros(bt.ngrids, np.int64)
    off[1:] = np.cumsum((cells + 3) // 4 * 4)[:-1]
    total = int(off[-1] + cells[-1])
    u = torch.empty(total, dtype=torch.float32, device=dev)
    k = torch.ones(total, dtype=torch.float32, device=dev)
    s = torch.zeros(total, dtype=torch.float32, device=dev)
    hu, hk, hs = (torch.from_numpy(x) for x in (bt.u, bt.kappa, bt.src))
    # bulk copy, then scatter to the padded layout on the device
    du, dk, ds = hu.to(dev), hk.to(dev), hs.to(dev)
    src_idx = torch.from_numpy(np.concatenate([np.arange(int(bt.offset[g]), int(bt.offset[g] + cells[g]))
                                               for g in range(bt.ngrids)])).to(dev)
    dst_idx = torch.from_numpy(np.concatenate([np.arange(int(off[g]), int(off[g] + cells[g]))
                                               for g in range(bt.ngrids)])).to(dev)
    u[dst_idx] = du[src_idx]
    k[dst_idx] = dk[src_idx]
    s[dst_idx] = ds[src_idx]
    del du, dk, ds, src_idx, dst_idx
    uin, uo = u.clone(), torch.empty_like(u)
    descs = cpb.batch_descriptors(uin, uo, k, s, off, bt.nx, bt.ny, bt.steps, bt.dt)
    plan = L.cpb_batch_plan_default()
    order, n_large = L.cpb_batch_order(descs, plan)
    d_descs = cpb.to_device_bytes(descs, dev)
    d_order = cpb.to_device_bytes((C.c_int * len(order))(*order), dev)
    work = torch.zeros(4, dtype=torch.int32, device=dev)
    # Grain-size sweep (grids per queue fetch x CTA size), the GPU counterpart
    # of the paper's average vs aggressive coarse-grained fetching; the timed
    # run below uses the fastest plan (each run starts from a fresh copy of u).
    plan, sweep = L.cpb_batch_autotune(d_descs, d_order, bt.ngrids, n_large, cpb.CPB_F32, W.DIRICHLET,
                                       work, plan, stream=sh)
    # Team shapes at the tuned depth, grain and CTA size: grids of at least
    # team_cells cells on a whole CTA, the others on teams of team_warps
    # warps once the CTA's large grids are done.  Each shape re-orders the
    # queue; the fastest (or the tuned plan as it is) is kept.
    ms_copy0 = _time(lambda: uin.copy_(u), 3, stream)

    def time_plan(p, d_ord, nl):
        def run():
            uin.copy_(u)
            L.cpb_stencil_batched(d_descs, d_ord, bt.ngrids, nl, cpb.CPB_F32, W.DIRICHLET, p, work, stream=sh)
        return _time(run, 2, stream) - ms_copy0

    team_ms = {f"team_cells{plan['team_cells']}_team_warps{plan['team_warps']}": time_plan(plan, d_order, n_large)}
    best_ms = next(iter(team_ms.values()))
    for tc in (65536, 131072, 262144, 524288):
        for tw in (2, 3, 4, 6):
            if (plan["threads"] // 32) % tw:
                continue
            p2 = dict(plan, team_cells=tc, team_warps=tw)
            o2, nl2 = L.cpb_batch_order(descs, p2)
            d_o2 = cpb.to_device_bytes((C.c_int * len(o2))(*o2), dev)
            ms2 = time_plan(p2, d_o2, nl2)
            team_ms[f"team_cells{tc}_team_warps{tw}"] = ms2
            if ms2 < best_ms:
                best_ms, plan, d_order, n_large = ms2, p2, d_o2, nl2
    assert L.cpb_batch_status(work, stream=sh) == 0

    def run_batch():
        uin.copy_(u)
        L.cpb_stencil_batched(d_descs, d_order, bt.ngrids, n_large, cpb.CPB_F32, W.DIRICHLET, plan,
                              work, stream=sh)

    def run_copy_only():
        uin.copy_(u)

    ms_total = _time(run_batch, 3, stream)
    ms_copy = _time(run_copy_only, 3, stream)
    ms_b = ms_total - ms_copy
    status = L.cpb_batch_status(work, stream=sh)
    upd = bt.updates
    # The workload as stated: the one persistent launch captured in a CUDA
    # graph and replayed.  Replays run back to back on the buffers the
    # previous replay left (the work does not depend on the values).
    uin.copy_(u)
    torch.cuda.synchronize()
    cap = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=cap):
        L.cpb_stencil_batched(d_descs, d_order, bt.ngrids, n_large, cpb.CPB_F32, W.DIRICHLET, plan, work,
                              stream=cap)
    def replay():
        with torch.cuda.stream(stream):  # on the timed stream, whatever stream is current
            graph.replay()

    ms_graph = _time(replay, 3, stream)
    status_graph = L.cpb_batch_status(work, stream=sh)
    del graph
    hbm, hsrc = peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    roof = batch_roofline(bt, plan["depth"], ms_graph, sms, hbm, hsrc)
    # one-grid-at-a-time baseline (tuned single-grid path, one call per grid)
    scratch = torch.empty(int(cells.max()), dtype=torch.float32, device=dev)

    def run_each():
        for gi in range(bt.ngrids):
            o, c = int(off[gi]), int(cells[gi])
            L.cpb_stencil_launch_tuned(u[o:o + c], uo[o:o + c], k[o:o + c], s[o:o + c], int(bt.nx[gi]),
                                       int(bt.ny[gi]), int(bt.steps[gi]), float(bt.dt[gi]), W.DIRICHLET,
                                       cpb.CPB_F32, tuning=None, scratch=scratch[:c], stream=sh)

    ms_each = _time(run_each, 1, stream)
    # kernel launches of the per-grid baseline: passes of depth 4 (scratch given)
    n_launch_each = int(sum(-(-int(st) // 4) for st in bt.steps))
    return {"workload": f"batch-{bt.ngrids}-grids-32..1024-steps-10..500", "updates": upd,
            "cells": int(cells.sum()), "n_large": n_large, "plan": plan,
            "grain_sweep_ms": {f"depth{d}_grain{g}_threads{t}": v for (d, g, t), v in sweep.items()},
            "team_sweep_ms": team_ms,
            "batched": {"gcells": upd / ms_b / 1e6, "ms": ms_b, "status": status,
                        "timing": "bare launch, u_in restored before each (copy time subtracted)"},
            "batched_cuda_graph": {"gcells": upd / ms_graph / 1e6, "ms": ms_graph, "status": status_graph,
                                   "timing": "the persistent launch captured once in a CUDA graph, "
                                             "replayed back to back"},
            "roofline": roof,
            "one_grid_at_a_time": {"gcells": upd / ms_each / 1e6, "ms": ms_each,
                                   "launches": n_launch_each,
                                   "note": "one cpb_stencil_launch_tuned call per grid from Python at "
                                           "the default depth 4, i.e. launch-bound: the cost the "
                                           "single persistent launch removes"},
            "speedup_batched_vs_per_grid": ms_each / ms_graph}


def batch_roofline(bt, depth, ms, sms, hbm, peak_source="measured", onchip_cells=14336):
    """Lower bound on the batched launch, per class of grid (max of the HBM
    and the FP32-lane time of each class, summed over classes).  Grids whose
    u, kappa, s and ping-pong partner fit in one SM's 227 KB of shared memory
    (16 B per cell: at most 14336 cells) could run all their steps on chip:
    their fields cross HBM once per run.  Every other grid streams its fields
    once per pass of the plan's depth.  FP32 lanes: ALG_OPS_PER_UPDATE
    operations per cell-update (the figure the single-grid roofline uses) on
    all SMs at the maximum SM clock."""
    src = peak_source
    lane_rate = sms * 128 * 2070e6 / float(ALG_OPS_PER_UPDATE)  # cell-updates per second
    cells = bt.nx.astype(np.int64) * bt.ny.astype(np.int64)
    steps = bt.steps.astype(np.int64)
    small = cells <= onchip_cells
    passes = -(-steps // depth)
    bytes_small = float(16 * cells[small].sum())
    bytes_large = float(16 * (cells[~small] * passes[~small]).sum())
    upd_small = float((cells[small] * steps[small]).sum())
    upd_large = float((cells[~small] * steps[~small]).sum())
    t_small = max(bytes_small / (hbm * 1e9), upd_small / lane_rate)
    t_large = max(bytes_large / (hbm * 1e9), upd_large / lane_rate)
    bound_ms = (t_small + t_large) * 1e3
    return {"bound": "hbm" if bytes_large / (hbm * 1e9) >= upd_large / lane_rate else "alu",
            "time_bound_ms": bound_ms, "measured_ms": ms, "frac": bound_ms / ms,
            "classes": {"on_chip": {"grids": int(small.sum()), "hbm_bytes": bytes_small, "updates": upd_small,
                                    "t_hbm_ms": bytes_small / (hbm * 1e9) * 1e3,
                                    "t_fp32_lanes_ms": upd_small / lane_rate * 1e3},
                        "streamed": {"grids": int((~small).sum()), "hbm_bytes": bytes_large,
                                     "updates": upd_large, "t_hbm_ms": bytes_large / (hbm * 1e9) * 1e3,
                                     "t_fp32_lanes_ms": upd_large / lane_rate * 1e3}},
            "peak": f"{hbm} GB/s ({src}); FP32 lanes {sms} SMs x 128 at 2070 MHz, "
                    f"{ALG_OPS_PER_UPDATE} operations per update",
            "depth": depth}


def form_adjoint(L, cpb, dev, stream):
    """Gradient of 0.5||u_T - target||^2 w.r.t. u0 and kappa, 2048^2, 200 steps, ckpt 20."""
    import torch
    g = W.differentiation()
    sh = stream.cuda_stream
    nx, ny, T, ck = g.nx, g.ny, g.steps, g.extras["ckpt"]
    u0 = torch.from_numpy(g.u).to(dev)
    k = torch.from_numpy(g.kappa).to(dev)
    tgt = torch.from_numpy(g.extras["target"]).to(dev)
    wsb = L.cpb_adjoint_workspace_bytes(nx, ny, T, ck)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    uT, gu, gk = torch.empty_like(u0), torch.empty_like(u0), torch.empty_like(u0)
    fwd_out, scr = torch.empty_like(u0), torch.empty_like(u0)
    # The built-in tuning of the grid (depth 4, one wave of items), for the
    # forward and the gradient alike.  An autotuned deeper tuning made the
    # plain forward faster (1.33 vs 1.44 ms) but the gradient slower (6.46 vs
    # 5.94 ms: 20-step segments split into passes of 8, 8, 4).
    tuning = L.cpb_get_tuning(nx, ny, cpb.CPB_F32, g.bc)
    ms_fwd = _time(lambda: L.cpb_stencil_launch_tuned(u0, fwd_out, k, None, nx, ny, T, float(g.dt),
                                                      g.bc, cpb.CPB_F32, scratch=scr, stream=sh),
                   3, stream)

    lam = torch.empty_like(u0)

    def grad(st=stream):
        h = st.cuda_stream
        L.cpb_adjoint_forward(u0, k, None, nx, ny, T, float(g.dt), g.bc, ck, uT, ws, wsb, stream=h)
        with torch.cuda.stream(st):
            torch.sub(uT, tgt, out=lam)
        L.cpb_adjoint_backward(k, None, lam, nx, ny, T, float(g.dt), g.bc, ck, gu, gk, ws, wsb, stream=h)

    ms_grad = _time(grad, 3, stream)
    # The same gradient captured once as a CUDA graph (151 launches: the
    # forward passes, lambda_T, the recompute and adjoint passes) on a side
    # stream (capture needs one that is not the default stream) and replayed
    # on the timed stream.
    grad()
    torch.cuda.synchronize()
    ref = (gu.clone(), gk.clone())
    graph = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    with torch.cuda.graph(graph, stream=cap):
        grad(cap)

    def replay():
        with torch.cuda.stream(stream):
            graph.replay()

    ms_graph = _time(replay, 3, stream)
    same = bool(torch.equal(gu, ref[0]) and torch.equal(gk, ref[1]))
    upd = nx * ny * T
    ndir = 64
    return {"workload": g.name, "tuning": tuning, "forward": {"gcells": upd / ms_fwd / 1e6, "ms": ms_fwd},
            "gradient": {"ms": ms_grad, "gcells_equiv": upd / ms_grad / 1e6,
                         "ratio_to_forward": ms_grad / ms_fwd},
            "gradient_cuda_graph": {"ms": ms_graph, "ratio_to_forward": ms_graph / ms_fwd,
                                    "same_bits_as_eager": same},
            "fd_cost_per_direction_ms": 2 * ms_fwd,
            "fd_64_directions_ms": 2 * ndir * ms_fwd,
            "speedup_gradient_vs_fd_64_directions": 2 * ndir * ms_fwd / ms_grad,
            "note": "one gradient (both dL/du0 and dL/dkappa in full) = forward with checkpoints + recompute + "
                    "adjoint sweep; central differences need 2 forwards per direction, and the workload checks "
                    "64 directions (each for u0 and kappa)"}


def form_volume(L, cpb, dev, stream, n=512, steps=100):
    """The 3-D 7-point variant on the 512^3 volume (one launch per step)."""
    import torch
    g = W.volume(n=n, steps=steps)
    sh = stream.cuda_stream
    u = torch.from_numpy(g.u).to(dev)
    k = torch.from_numpy(g.kappa).to(dev)
    s = torch.from_numpy(g.src).to(dev)
    del g.u, g.kappa, g.src
    out, scr = torch.empty_like(u), torch.empty_like(u)
    ms = _time(lambda: L.cpb_stencil3d_launch(u, out, k, s, n, n, n, steps, float(g.dt), g.bc,
                                              scratch=scr, stream=sh), 2, stream)
    upd = n ** 3 * steps
    hbm, _ = peaks()
    gbs = upd * 16 / ms / 1e6
    return {"workload": g.name, "gcells": upd / ms / 1e6, "ms": ms, "ms_per_step": ms / steps,
            "effective_gbs_16B": gbs, "frac_hbm": gbs / hbm,
            "note": "z-marching tiled kernel, one launch per step, default geometry (32 x 8 threads)"}


def form_tile_blocked(L, cpb, dev, stream, n=8192):
    """The multi-barrier kernel (shared-memory temporal blocking on the
    caller's geometry) on the 8192^2 periodic workload, for a few geometries."""
    import torch
    g = W.plain_scale(seed=1, n=n, steps=1)
    sh = stream.cuda_stream
    u = torch.from_numpy(g.u).to(dev)
    k = torch.from_numpy(g.kappa).to(dev)
    s = torch.from_numpy(g.src).to(dev)
    out, scr = torch.empty_like(u), torch.empty_like(u)
    res = {}
    for bx, by, d in ((32, 8, 1), (32, 16, 4), (64, 16, 8), (32, 32, 16)):
        steps = 4 * d
        geom = (((n + bx - 1) // bx, (n + by - 1) // by, 1), (bx, by, 1), L.cpb_tile_blocked_shared_bytes(bx, by, d))
        ms = _time(lambda: L.cpb_stencil_tile_blocked(u, out, k, s, n, n, steps, d, float(g.dt), g.bc, *geom,
                                                      scratch=scr, stream=sh), 2, stream)
        res[f"block{bx}x{by}_depth{d}"] = {"gcells": n * n * steps / ms / 1e6, "us_per_step": ms / steps * 1e3}
    return {"workload": f"plain-{n}x{n}-periodic", "geometries": res,
            "note": "d steps per launch in shared memory, a __syncthreads after staging and after each step"}


def form_depth1(L, cpb, dev, stream, n=8192):
    """The plain streaming pass at depth 1 (no temporal blocking: 16 B of HBM
    traffic per cell-update) on the 8192^2 periodic workload, over a few
    tunings; the best one against the measured HBM copy rate.  This is the
    bandwidth check of the streaming kernel itself: at depth 1 nothing hides
    HBM."""
    import torch
    g = W.plain_scale(seed=1, n=n, steps=1)
    sh = stream.cuda_stream
    u = torch.from_numpy(g.u).to(dev)
    k = torch.from_numpy(g.kappa).to(dev)
    s = torch.from_numpy(g.src).to(dev)
    out = torch.empty_like(u)
    hbm, src = peaks()
    res = {}
    for c, w, v, st in ((128, 2, 1, 4), (256, 4, 1, 4), (256, 4, 1, 2), (128, 4, 1, 4), (256, 1, 0, 2)):
        t = {"k": 1, "chunk_rows": c, "warps_per_block": w, "variant": v, "stages": st}
        ms = _time(lambda: L.cpb_stencil_launch_tuned(u, out, k, s, n, n, 1, float(g.dt), g.bc, cpb.CPB_F32,
                                                      tuning=t, stream=sh), 10, stream)
        res[f"chunk{c}_wpb{w}_variant{v}_stages{st}"] = {"us_per_pass": ms * 1e3, "gcells": n * n / ms / 1e6,
                                                         "tuning": t}
    best = min(res.values(), key=lambda r: r["us_per_pass"])
    gbs = 16.0 * n * n / (best["us_per_pass"] * 1e-6) / 1e9
    return {"workload": f"plain-{n}x{n}-periodic", "tunings": res, "best": best,
            "algorithmic_gbs": gbs, "frac_hbm": gbs / hbm, "peak": f"{hbm} GB/s ({src})",
            "roofline_gcells": hbm * 1e9 / 16 / 1e9,
            "note": "16 B per cell-update (u, kappa, s read, u written once per pass)"}


def form_small(L, cpb, dev, stream):
    """The small workload (512^2, Dirichlet, 100 steps, 16 x 16 blocks): the
    paper-shaped one-step tiled kernel on the caller's geometry, the tuned
    path, and the tuned path captured once as a CUDA graph and replayed
    (L2-resident, so launch cost matters)."""
    import torch
    g = W.plain_small()
    sh = stream.cuda_stream
    n, T = g.nx, g.steps
    u = torch.from_numpy(g.u).to(dev)
    k = torch.from_numpy(g.kappa).to(dev)
    s = torch.from_numpy(g.src).to(dev)
    out, scr = torch.empty_like(u), torch.empty_like(u)
    grid, block, shm = ((n + 15) // 16, (n + 15) // 16, 1), (16, 16, 1), 2 * 18 * 18 * 4
    ms_tile = _time(lambda: L.cpb_stencil_launch(u, out, k, s, n, n, T, float(g.dt), g.bc, cpb.CPB_F32, grid,
                                                 block, shm, scratch=scr, stream=sh), 5, stream)
    out.copy_(u)
    tuning = L.cpb_autotune(out, scr, k, s, n, n, 24, float(g.dt), g.bc, cpb.CPB_F32, stream=sh)
    ms_tuned = _time(lambda: L.cpb_stencil_launch_tuned(u, out, k, s, n, n, T, float(g.dt), g.bc, cpb.CPB_F32,
                                                        tuning=tuning, scratch=scr, stream=sh), 5, stream)
    graph = L.cpb_graph_create(u, out, k, s, n, n, T, float(g.dt), g.bc, cpb.CPB_F32, tuning=tuning, scratch=scr)
    try:
        ms_graph = _time(lambda: L.cpb_graph_launch(graph, stream=sh), 5, stream)
    finally:
        L.cpb_graph_destroy(graph)
    upd = n * n * T
    passes = -(-T // tuning["k"])
    return {"workload": g.name, "tiled_one_step_16x16": {"gcells": upd / ms_tile / 1e6, "ms": ms_tile,
                                                         "launches": T},
            "tuned": {"gcells": upd / ms_tuned / 1e6, "ms": ms_tuned, "launches": passes, "tuning": tuning},
            "tuned_cuda_graph": {"gcells": upd / ms_graph / 1e6, "ms": ms_graph, "launches": passes},
            "note": "4 MiB working set, L2-resident: HBM roofline not meaningful; the graph removes host "
                    "launch cost"}


def measure_forms(L, cpb, dev, stream):
    out = {}
    for name, fn in (("precision", form_precision), ("batched", form_batched),
                     ("adjoint", form_adjoint), ("volume", form_volume),
                     ("tile_blocked", form_tile_blocked), ("small", form_small), ("depth_1", form_depth1)):
        try:
            out[name] = fn(L, cpb, dev, stream)
        except Exception as e:  # report, never lose the headline line
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        import torch
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    import paper_2206_07896_gb300 as cpb

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device for the GPU arm")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    L = cpb.lib(fma=True)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream

    g = W.plain_scale(seed=1 + rank, n=args.n, steps=args.time_steps)
    nx, ny, T = g.nx, g.ny, g.steps
    u0 = torch.from_numpy(g.u).to(dev)
    kap = torch.from_numpy(g.kappa).to(dev)
    src = torch.from_numpy(g.src).to(dev)
    a, b = torch.empty_like(u0), torch.empty_like(u0)

    tuning_source = "flags"
    if args.k:
        tuning = {"k": args.k, "chunk_rows": args.chunk, "warps_per_block": args.wpb,
                  "variant": args.variant, "stages": args.stages}
    else:
        # CPB_AUTOTUNE_CACHE: a tuning file (cpb_tuning_save format) reused
        # between runs; autotune only when it holds none for this grid.
        cache = os.environ.get("CPB_AUTOTUNE_CACHE")
        tuning = None
        if cache and os.path.exists(cache):
            try:
                L.cpb_tuning_load(cache)
            except cpb.CpbError:
                pass
            tuning = L.cpb_lookup_tuning(nx, ny, cpb.CPB_F32, g.bc)
            tuning_source = "cache"
        if tuning is None:
            a.copy_(u0)
            tuning = L.cpb_autotune(a, b, kap, src, nx, ny, 24, float(g.dt), g.bc, cpb.CPB_F32, stream=sh)
            tuning_source = "autotune"
            if cache and rank == 0:
                L.cpb_tuning_save(cache)
    k = tuning["k"]
    depths = [k] * (T // k) + ([T % k] if T % k else [])
    ws_bytes = L.cpb_heat_sum_workspace_bytes(nx, ny)
    ws = torch.empty(max(8, ws_bytes) // 8, dtype=torch.float64, device=dev)
    hsum = torch.empty((), dtype=torch.float64, device=dev)
    n_pass = len(depths)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(n_pass + 1)]
           for _ in range(args.steps)]

    def one_step(ev=None):
        # One bench step: T time steps in passes of depth k (ping-pong a/b,
        # each pass one launch of the streaming kernel), then the FP64 heat sum
        # of the result.  ev: CUDA events recorded around every pass.
        src_buf, dst = u0, a
        for i, d in enumerate(depths):
            if ev is not None:
                ev[i].record(stream)
            L.cpb_stencil_launch_tuned(src_buf, dst, kap, src, nx, ny, d, float(g.dt), g.bc,
                                       cpb.CPB_F32, tuning=tuning, scratch=None, stream=sh)
            src_buf, dst = dst, (b if dst is a else a)
        if ev is not None:
            ev[n_pass].record(stream)
        L.cpb_heat_sum(src_buf, nx, ny, cpb.CPB_F32, hsum, ws, ws_bytes, stream=sh)
        return src_buf

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    full_pass_ms = []
    with ClockSampler(local) as clocks:
        start.record(stream)
        for st in range(args.steps):
            one_step(evs[st])
        stop.record(stream)
        torch.cuda.synchronize()
    # per-launch durations of the dominant kernel (the full-depth passes)
    for ev in evs:
        for i, d in enumerate(depths):
            if d == k:
                full_pass_ms.append(ev[i].elapsed_time(ev[i + 1]))
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    elapsed = start.elapsed_time(stop)
    per_rank_ms = elapsed / args.steps
    updates = nx * ny * T
    if pg:
        t = torch.tensor([per_rank_ms], device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        tmax = float(t.item())
    else:
        tmax = per_rank_ms
    value = updates * world / (tmax * 1e-3) / 1e9

    clk = clocks.summary()   # reads (and removes) the sample file once
    # Roofline of the dominant kernel (full-depth stream pass): the binding
    # one of its HBM and FP32-lane bounds (at depth 8 the lanes bind).
    hbm, which = peaks()
    avg_pass = sum(full_pass_ms) / len(full_pass_ms)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    roof = stream_roofline(nx * ny, k, avg_pass, hbm, sms, clk.get("sm_mhz") or 2070.0)
    roof.update({"traffic": args.traffic if args.traffic is not None else recorded_traffic(tuning, nx, ny),
                 "peak_source": f"HBM: {which} copy rate; FP32 lanes: the sampled SM clock",
                 "kernel": ("stream_bulk_kernel" if tuning.get("variant") == 1 else "stream_kernel")
                           + f"<K={k},f32>", "avg_launch_ms": avg_pass,
                 # the implementation's own lower bounds (flux form: about 10
                 # FP32 operations per cell-update)
                 "time_bounds_us": time_bounds(nx * ny, k, hbm, clk),
                 "effective_cell_rate_vs_k1_roofline": value / world / (hbm * 1e9 / 16 / 1e9)})

    # End to end through the C ABI on host buffers (pinned), copies timed.
    e2e = None
    if not args.no_e2e:
        hu = torch.from_numpy(g.u).pin_memory()
        hk = torch.from_numpy(g.kappa).pin_memory()
        hs = torch.from_numpy(g.src).pin_memory()
        ho = torch.empty_like(hu).pin_memory()
        L.cpb_set_tuning(nx, ny, cpb.CPB_F32, g.bc, tuning)
        wsb = L.cpb_host_workspace_bytes(nx, ny, cpb.CPB_F32)
        hws = torch.empty(wsb, dtype=torch.uint8, device=dev)
        for _ in range(2):   # warm-up (the first call pays one-time costs)
            L.cpb_stencil_host(hu, hk, hs, ho, nx, ny, T, float(g.dt), g.bc, cpb.CPB_F32, hws, wsb,
                               stream=sh)
        reps = max(1, min(args.steps, 5))
        rep_s = []
        for _ in range(reps):   # each call returns after its device-to-host copy is done
            t0 = time.perf_counter()
            L.cpb_stencil_host(hu, hk, hs, ho, nx, ny, T, float(g.dt), g.bc, cpb.CPB_F32, hws, wsb,
                               stream=sh)
            rep_s.append(time.perf_counter() - t0)
        sync_s = statistics.median(rep_s)
        # The pipelined call: each step copies its inputs in and its result
        # out, on copy streams beside the compute stream, alternating two
        # workspaces, so a step's transfers overlap its neighbours' compute.
        hws2 = [hws, torch.empty(wsb, dtype=torch.uint8, device=dev)]
        ho2 = [ho, torch.empty_like(hu).pin_memory()]
        s_in, s_c, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        done = [None, None]

        def async_step(i):
            w = i % 2
            if done[w] is not None:
                s_in.wait_event(done[w])   # that workspace's previous problem has been copied out
            L.cpb_stencil_host_async(hu, hk, hs, ho2[w], nx, ny, T, float(g.dt), g.bc, cpb.CPB_F32, hws2[w], wsb,
                                     s_in, s_c, s_out)
            ev = torch.cuda.Event()
            ev.record(s_out)
            done[w] = ev

        for i in range(2):
            async_step(i)
        torch.cuda.synchronize()
        n_async = max(args.steps, 5)
        t0 = time.perf_counter()
        for i in range(n_async):
            async_step(i)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / n_async
        if pg:
            t = torch.tensor([e2e_s, sync_s], device=dev)
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            e2e_s, sync_s = float(t[0].item()), float(t[1].item())
        e2e = {"value": updates * world / e2e_s / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": 3 * nx * ny * 4, "d2h_bytes_per_step": nx * ny * 4,
               "ms_per_step": e2e_s * 1e3, "steps": n_async,
               "timing": "cpb_stencil_host_async: consecutive steps on copy-in / compute / copy-out streams and "
                         "two workspaces; wall time of all steps (pinned copies included) / steps",
               "sync_call": {"value": updates * world / sync_s / 1e9, "ms_per_step": sync_s * 1e3, "reps": reps,
                             "ms_min": min(rep_s) * 1e3, "ms_max": max(rep_s) * 1e3,
                             "timing": "cpb_stencil_host (copies in, runs, copies out, synchronises): median "
                                       "of per-call wall times"}}
        del hws, hws2

    forms = measure_forms(L, cpb, dev, stream) if (args.forms and rank == 0) else None

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            _, cpu = oracle_sample(g)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": tmax,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": g.name, "nx": nx, "ny": ny, "time_steps": T,
                           "bc": "periodic", "tuning": tuning, "tuning_source": tuning_source,
                           "l2": "inputs larger than L2 (u, kappa, s, 2 ping-pong buffers: 256 MiB each)",
                           "parallelism": f"replicas x{world}",
                           "step": "1000 time steps + FP64 heat sum"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": args.steps * (n_pass + 2), "clocks": clk}
        if forms is not None:
            line["forms"] = forms
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# Profiling mode: one launch per configuration, for ncu captures
# ---------------------------------------------------------------------------
def _profile_fields(dev, g):
    import torch
    return (torch.from_numpy(g.u).to(dev), torch.from_numpy(g.kappa).to(dev),
            torch.from_numpy(g.src).to(dev))


def profile_stream(L, cpb, dev, args):
    """ONE pass of depth K per --spec K:chunk:wpb:variant:stages on the n x n
    workload (periodic plain_scale fields, or the precision workload's fields
    with --bc dirichlet), FP32 or BF16-Kahan storage (--dtype)."""
    import torch
    n = args.n
    if args.bc == "dirichlet":
        g = W.precision(n=n, steps=16)
    else:
        g = W.plain_scale(seed=1, n=n, steps=16)
    u, k, s = _profile_fields(dev, g)
    dtype = cpb.CPB_F32
    if args.dtype == "bf16k":
        N = n * n
        st = torch.empty(N, dtype=torch.int32, device=dev)
        kb = torch.empty(N, dtype=torch.int16, device=dev)
        sb = torch.empty(N, dtype=torch.int16, device=dev)
        L.cpb_bf16k_pack(u, st, N)
        L.cpb_bf16_round(k, kb, N)
        L.cpb_bf16_round(s, sb, N)
        u, k, s, dtype = st, kb, sb, cpb.CPB_BF16_KAHAN
    out = torch.empty_like(u)
    for sp in args.spec or ["4:256:1:1:2"]:
        K, c, w, v, stg = (int(x) for x in sp.split(":"))
        t = {"k": K, "chunk_rows": c, "warps_per_block": w, "variant": v, "stages": stg}
        L.cpb_stencil_launch_tuned(u, out, k, s, n, n, K, float(g.dt), g.bc, dtype, tuning=t)
    torch.cuda.synchronize()
    return L.cpb_device_status()


def profile_vol(L, cpb, dev, args):
    """ONE step of cpb_stencil3d_launch per --spec by:zchunks on the n^3 volume."""
    import torch
    n = args.n
    if n > 1024:
        raise SystemExit("--profile vol: --n is the cube side, at most 1024")
    g = W.volume(n=n, steps=1)
    u, k, s = _profile_fields(dev, g)
    out = torch.empty_like(u)
    for sp in args.spec or ["8:16"]:
        by, zc = (int(x) for x in sp.split(":"))
        L.cpb_stencil3d_launch(u, out, k, s, n, n, n, 1, float(g.dt), g.bc,
                               ((n + 127) // 128, (n + by - 1) // by, zc), (32, by, 1),
                               L.cpb_stencil3d_shared_bytes(by))
    torch.cuda.synchronize()
    return L.cpb_device_status()


def profile_tileb(L, cpb, dev, args):
    """ONE launch of the multi-barrier kernel per --spec bx:by:depth."""
    import torch
    n = args.n
    g = W.plain_scale(seed=1, n=n, steps=1)
    u, k, s = _profile_fields(dev, g)
    out, scr = torch.empty_like(u), torch.empty_like(u)
    for sp in args.spec or ["64:16:8"]:
        bx, by, d = (int(x) for x in sp.split(":"))
        L.cpb_stencil_tile_blocked(u, out, k, s, n, n, d, d, float(g.dt), g.bc,
                                   ((n + bx - 1) // bx, (n + by - 1) // by, 1), (bx, by, 1),
                                   L.cpb_tile_blocked_shared_bytes(bx, by, d), scratch=scr)
    torch.cuda.synchronize()
    return L.cpb_device_status()


def profile_adjoint(L, cpb, dev, args):
    """ONE gradient of the 2048^2 differentiation workload, as the bench times it."""
    import torch
    g = W.differentiation()
    nx, ny, T, ck = g.nx, g.ny, g.steps, g.extras["ckpt"]
    u0 = torch.from_numpy(g.u).to(dev)
    k = torch.from_numpy(g.kappa).to(dev)
    tgt = torch.from_numpy(g.extras["target"]).to(dev)
    wsb = L.cpb_adjoint_workspace_bytes(nx, ny, T, ck)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    uT, gu, gk = torch.empty_like(u0), torch.empty_like(u0), torch.empty_like(u0)
    L.cpb_adjoint_forward(u0, k, None, nx, ny, T, float(g.dt), g.bc, ck, uT, ws, wsb)
    lam = uT - tgt
    L.cpb_adjoint_backward(k, None, lam, nx, ny, T, float(g.dt), g.bc, ck, gu, gk, ws, wsb)
    torch.cuda.synchronize()
    return L.cpb_device_status()


def profile_batch(L, cpb, dev, args):
    """ONE batched persistent launch over the --n cheapest grids (by
    cell-updates) of the 4096-grid set, default plan: a subset of cheap grids
    keeps every grid far below the per-SM share, so no single grid sets the
    length of the launch."""
    import ctypes as C
    import torch
    n = args.n
    if not 1 <= n <= 4096:
        raise SystemExit("--profile batch: --n is the number of grids, 1..4096")
    bt = W.batching(ngrids=4096)
    sel = np.sort(np.argsort(bt.nx.astype(np.int64) * bt.ny * bt.steps, kind="stable")[:n])
    nx, ny, steps, dt = bt.nx[sel], bt.ny[sel], bt.steps[sel], bt.dt[sel]
    cells = nx.astype(np.int64) * ny.astype(np.int64)
    off = np.zeros(n, np.int64)
    off[1:] = np.cumsum((cells + 3) // 4 * 4)[:-1]  # 16-byte aligned grid starts
    total = int(off[-1] + cells[-1])
    u = torch.zeros(total, dtype=torch.float32, device=dev)
    k = torch.ones(total, dtype=torch.float32, device=dev)
    s = torch.zeros(total, dtype=torch.float32, device=dev)
    for q, gi in enumerate(sel):
        o, c, b = int(off[q]), int(cells[q]), int(bt.offset[gi])
        u[o:o + c] = torch.from_numpy(bt.u[b:b + c])
        k[o:o + c] = torch.from_numpy(bt.kappa[b:b + c])
        s[o:o + c] = torch.from_numpy(bt.src[b:b + c])
    uo = torch.empty_like(u)
    descs = cpb.batch_descriptors(u, uo, k, s, off, nx, ny, steps, dt)
    plan = L.cpb_batch_plan_default()
    order, n_large = L.cpb_batch_order(descs, plan)
    d_descs = cpb.to_device_bytes(descs, dev)
    d_order = cpb.to_device_bytes((C.c_int * len(order))(*order), dev)
    work = torch.zeros(4, dtype=torch.int32, device=dev)
    L.cpb_stencil_batched(d_descs, d_order, n, n_large, cpb.CPB_F32, W.DIRICHLET, plan, work)
    torch.cuda.synchronize()
    return L.cpb_batch_status(work)


PROFILES = {"stream": profile_stream, "vol": profile_vol, "tileb": profile_tileb,
            "adjoint": profile_adjoint, "batch": profile_batch}


def run_profile(args):
    """--profile KIND: a handful of launches of one kernel family and nothing
    else, so that `ncu -k regex:<kernel> -c <count>` captures exactly those
    launches.  Prints one line; exits 1 on a non-zero device status."""
    import torch
    import paper_2206_07896_gb300 as cpb
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    L = cpb.lib(fma=True)
    status = PROFILES[args.profile](L, cpb, dev, args)
    print(f"profile {args.profile} n={args.n} specs={args.spec} dtype={args.dtype} bc={args.bc} "
          f"status {status}", flush=True)
    return 0 if status == 0 else 1


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=8192, help="grid side (default 8192)")
    ap.add_argument("--time-steps", type=int, default=1000)
    ap.add_argument("--k", type=int, default=0, help="force temporal depth (0 = autotune)")
    ap.add_argument("--chunk", type=int, default=256)
    ap.add_argument("--wpb", type=int, default=4)
    ap.add_argument("--variant", type=int, default=1, help="0 register prefetch, 1 TMA bulk ring")
    ap.add_argument("--stages", type=int, default=4)
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu DRAM bytes per launch of the dominant kernel, if measured")
    ap.add_argument("--no-forms", dest="forms", action="store_false",
                    help="skip the BF16 / batched / adjoint forms")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", default=None, choices=sorted(PROFILES),
                    help="profiling mode: one launch per --spec of one kernel family (for ncu)")
    ap.add_argument("--spec", action="append", default=None,
                    help="--profile geometry: stream K:chunk:wpb:variant:stages, vol by:zchunks, "
                         "tileb bx:by:depth (repeatable)")
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16k"], help="--profile stream storage")
    ap.add_argument("--bc", default="periodic", choices=["periodic", "dirichlet"],
                    help="--profile stream boundary (dirichlet: the precision workload's fields)")
    args = ap.parse_args(argv)
    if args.profile:
        return run_profile(args)
    args.warmup = max(3, args.warmup)   # at least 3 untimed warm-up steps
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
