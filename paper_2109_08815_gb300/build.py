"""Build libpds.so (the CUDA library behind include/pds.h) for sm_103a.

Each translation unit is compiled by nvcc in parallel (the rollout kernels
once per chain length), then linked into ``paper_2109_08815_gb300/libpds.so``.
Objects go to ``_build/`` at the repository root (git-ignored).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libpds.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
MAX_LINKS = 8


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _units():
    units = [("pds_api", "pds_api.cu", []), ("reduce", "reduce.cu", []), ("svgd", "svgd.cu", []),
             ("batch", "batch.cu", []), ("server", "server.cu", []), ("armbox", "armbox.cu", []),
             ("metrics", "metrics.cu", []), ("sgld", "sgld.cu", []), ("sobol", "sobol.cu", []), ("rigid2", "rigid2.cu", []),
             ("svgd_tc", "svgd_tc.cu", []), ("median_tc", "median_tc.cu", [])]
    # the rollouts' fused multiply-adds are all explicit (fmaf): no contraction,
    # so the single-problem and batched kernels compute the same bits
    for nl in range(1, MAX_LINKS + 1):
        units.append((f"rollout_nl{nl}", "rollout_nl.cu", [f"-DPDS_NL={nl}", "-fmad=false"]))
    return units


def _sources_mtime() -> float:
    t = 0.0
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            t = max(t, os.path.getmtime(os.path.join(d, f)))
    return t


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int | None = None, defines=(),
          lib_path: str | None = None, build_dir: str | None = None) -> str:
    """Compile and link the library; ``defines`` (e.g. ["PDS_ROLLOUT_MINB=2"])
    and ``lib_path``/``build_dir`` build a variant without touching the
    default library."""
    lib_out = lib_path or LIB
    bdir = build_dir or BUILD
    if not force and os.path.exists(lib_out) and os.path.getmtime(lib_out) >= _sources_mtime():
        return lib_out
    nvcc = _nvcc()
    os.makedirs(bdir, exist_ok=True)
    extra = (["-Xptxas", "-v"] if verbose_ptxas else []) + [f"-D{d}" for d in defines]

    def compile_unit(u):
        name, src, defs = u
        obj = os.path.join(bdir, name + ".o")
        cmd = [nvcc, *NVFLAGS, *extra, *defs, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{r.stderr}")
        return obj, r.stderr

    units = _units()
    with cf.ThreadPoolExecutor(max_workers=jobs or min(len(units), os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_unit, units))
    if verbose_ptxas:
        for (obj, log) in results:
            sys.stderr.write(log)
    tmp = lib_out + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib_out)
    return lib_out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
