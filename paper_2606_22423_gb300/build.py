"""Build libgbscan.so in-tree with nvcc for sm_103a.

Translation units compile in parallel (the per-width kernel instantiations
are split into eight ranges of four widths) and link into one shared library that depends
only on the CUDA runtime.  Run ``python -m paper_2606_22423_gb300.build``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgbscan.so")
ROOT = os.path.dirname(HERE)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + [
    "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "--use_fast_math",
    "-I" + os.path.join(ROOT, "include"),
]
RANGES = [(1, 4), (5, 8), (9, 12), (13, 16), (17, 20), (21, 24), (25, 28), (29, 32)]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the scan library needs the CUDA toolkit")


def _units():
    units = []
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hdrs.append(os.path.join(ROOT, "include", "gbscan.h"))
    for lo, hi in RANGES:
        units.append((os.path.join(CSRC, "scan_inst.cu"), f"scan_b{lo:02d}_{hi:02d}.o",
                      [f"-DGB_BLO={lo}", f"-DGB_BHI={hi}"]))
    for flavour in (0, 1):
        for lo, hi in RANGES:
            units.append((os.path.join(CSRC, "batch_inst.cu"), f"batch_k{flavour}_b{lo:02d}_{hi:02d}.o",
                          [f"-DGB_BATCH_BRANCHY={flavour}", f"-DGB_BLO={lo}", f"-DGB_BHI={hi}"]))
    for f in sorted(os.listdir(CSRC)):
        if f.endswith(".cu") and f not in ("scan_inst.cu", "batch_inst.cu"):
            units.append((os.path.join(CSRC, f), f[:-3] + ".o", []))
    return units, hdrs


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> str:
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    units, hdrs = _units()
    flags = NVCC_FLAGS + list(extra_flags or [])
    jobs = []
    for src, obj, defs in units:
        out = os.path.join(BUILD, obj)
        if force or _stale(out, [src] + hdrs + [__file__]):
            jobs.append([nvcc] + flags + defs + ["-c", src, "-o", out])
    workers = max(1, min(len(jobs), os.cpu_count() or 4))
    if jobs:
        with cf.ThreadPoolExecutor(workers) as ex:
            for cmd, res in zip(jobs, ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs)):
                if verbose or res.returncode != 0:
                    sys.stderr.write(" ".join(cmd) + "\n" + res.stdout + res.stderr)
                if res.returncode != 0:
                    raise RuntimeError(f"nvcc failed for {cmd[-3]}")
    objs = [os.path.join(BUILD, obj) for _, obj, _ in units]
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + [
            "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + res.stdout + res.stderr)
            raise RuntimeError("link of libgbscan.so failed")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
