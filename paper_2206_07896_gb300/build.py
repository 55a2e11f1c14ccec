"""Build libcpb for sm_103a, in-tree: paper_2206_07896_gb300/_build/.

Three builds of the same sources:
  libcpb.so        default: the compiler may contract multiply-adds into FMAs.
  libcpb_nofma.so  --fmad=false: every FP32 operation rounds on its own, in
                   the library's defined order (bit-exact against the CPU
                   oracle's FP32 mode).
  libcpb_check.so  the --fmad=false build with a range check on every global
                   element range a kernel reads or writes (a debug build in
                   place of a memory checker; cpb_bounds_status reports).
Translation units compile in parallel; nvcc links each set into a shared
object with the CUDA runtime linked statically.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
          "--expt-relaxed-constexpr"]
VARIANTS = {"libcpb.so": ["--fmad=true"], "libcpb_nofma.so": ["--fmad=false", "-DCPB_EXACT_ARITH"],
            "libcpb_check.so": ["--fmad=false", "-DCPB_EXACT_ARITH", "-DCPB_BOUNDS_CHECK"]}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) \
        + [os.path.join(HERE, "..", "include", "cpb.h"), os.path.abspath(__file__)]


def lib_path(name: str = "libcpb.so") -> str:
    return os.path.join(OUT, name)


def up_to_date() -> bool:
    newest = max(os.path.getmtime(p) for p in _deps())
    return all(os.path.exists(lib_path(v)) and os.path.getmtime(lib_path(v)) >= newest for v in VARIANTS)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False) -> list[str]:
    if not force and up_to_date():
        return [lib_path(v) for v in VARIANTS]
    os.makedirs(OUT, exist_ok=True)
    jobs = []
    for lib, flags in VARIANTS.items():
        tag = os.path.splitext(lib)[0]
        for src in _sources():
            obj = os.path.join(OUT, f"{tag}.{os.path.splitext(os.path.basename(src))[0]}.o")
            cmd = [nvcc()] + ARCH + COMMON + flags + (["-Xptxas", "-v"] if verbose else []) \
                + ["-c", src, "-o", obj]
            jobs.append((lib, obj, cmd))
    workers = max(1, min(len(jobs), os.cpu_count() or 4))
    with ThreadPoolExecutor(workers) as ex:
        logs = list(ex.map(lambda j: _run(j[2]), jobs))
    if verbose:
        for j, log in zip(jobs, logs):
            sys.stdout.write(f"== {os.path.basename(j[1])}\n{log}")
    outs = []
    for lib in VARIANTS:
        objs = [j[1] for j in jobs if j[0] == lib]
        tmp = lib_path(lib) + f".tmp{os.getpid()}"
        _run([nvcc()] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs)
        os.replace(tmp, lib_path(lib))
        outs.append(lib_path(lib))
    return outs


if __name__ == "__main__":
    print("\n".join(build(force="--force" in sys.argv, verbose="-v" in sys.argv)))
