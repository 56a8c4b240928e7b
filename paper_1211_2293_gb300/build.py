"""Build libtc.so (the CUDA treecode library) in-tree with nvcc for sm_103a.

    python -m paper_1211_2293_gb300.build          # incremental
    python -m paper_1211_2293_gb300.build --force  # rebuild everything

Translation units are compiled in parallel, then linked with the static CUDA
runtime into ``paper_1211_2293_gb300/libtc.so``.  No GPU is needed to build.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtc.so")
INCLUDE = os.path.join(ROOT, "include")

# (object, source, defines): the walk kernels, one object per (bodies per
# lane, tile), are the longest compiles and go first
WALK_UNITS = [(f"tc_walk_b{b}_t{t}", "tc_walk_unit.cu", [f"-DTC_WALK_B={b}", f"-DTC_WALK_TILE={t}"])
              for b in (4, 2, 1) for t in (128, 64, 256)]
UNITS = WALK_UNITS + [(s[:-3], s, []) for s in ["tc_api.cu", "tc_walk.cu", "tc_sort.cu", "tc_build.cu", "tc_step.cu",
                                               "tc_noalloc.cu", "tc_mlp.cu", "tc_band.cu", "tc_fmm.cu",
                                               "tc_force_probe.cu"]]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
              "--expt-relaxed-constexpr", f"-I{INCLUDE}"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found (set NVCC or put CUDA on PATH)")


def _headers():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))] + [
        os.path.join(INCLUDE, "tc.h")]


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    hdrs = _headers()
    jobs = []
    for obj, src, defs in UNITS:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, obj + ".o")
        if force or _stale(o, [s, *hdrs]):
            cmd = [nvcc, *ARCH, *NVCC_FLAGS, *defs, "-c", s, "-o", o]
            if ptxas_v:
                cmd += ["-Xptxas", "-v"]
            jobs.append((obj, cmd))
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            futs = {ex.submit(subprocess.run, cmd, capture_output=True, text=True): src for src, cmd in jobs}
            errs = []
            for f in cf.as_completed(futs):
                r = f.result()
                if verbose or ptxas_v:
                    sys.stderr.write(r.stderr)
                if r.returncode != 0:
                    errs.append(f"{futs[f]}:\n{r.stderr}")
            if errs:
                raise RuntimeError("nvcc failed:\n" + "\n".join(errs))
    objs = [os.path.join(BUILD, obj + ".o") for obj, _, _ in UNITS]
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stderr)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--ptxas-v", action="store_true")
    a = ap.parse_args()
    print(build(force=a.force, verbose=True, ptxas_v=a.ptxas_v))
