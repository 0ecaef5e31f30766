"""Build libgp.so in-tree for sm_103a with nvcc (no cmake, parallel units).

Usage: python -m paper_2503_02259_gb300.build [--force] [--jobs N]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
OBJ = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libgp.so")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I", INCLUDE, "-I", CSRC]

# (object name, source, extra flags)
# The SIMT product is instantiated per (kernel family, grad, dimension template)
# in 24 units, so that a multi-core host compiles them in parallel.
SIMT_UNITS = [(f"kmv_simt_k{k}_g{g}_d{dt}", "kmv_simt_inst.cu",
               [f"-DGP_KIND={k}", f"-DGP_GRAD={g}", f"-DGP_DT={dt}"])
              for k in (0, 1) for g in (0, 1) for dt in (1, 2, 3, 4, 8, 16)]

UNITS = SIMT_UNITS + [
    ("kmv_tc", "kmv_tc.cu", []),
    ("kmv_tc_m1", "kmv_tc_inst.cu", ["-DGP_TC_MODE=1"]),
    ("kmv_tc_m2", "kmv_tc_inst.cu", ["-DGP_TC_MODE=2"]),
    ("kmv_tc_m3", "kmv_tc_inst.cu", ["-DGP_TC_MODE=3"]),
    ("kmv_tc_m4", "kmv_tc_inst.cu", ["-DGP_TC_MODE=4"]),
    ("vec_kernels", "vec_kernels.cu", []),
    ("residual", "residual.cu", []),
    ("residual_pair", "residual_pair.cu", []),
    ("nystrom", "nystrom.cu", []),
    ("grad_ard", "grad_ard.cu", []),
    ("server", "server.cu", []),
    ("static_scratch", "static_scratch.cu", []),
    ("microbench", "microbench.cu", []),
    ("gp_api", "gp_api.cu", []),
]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA 13 toolkit is required to build libgp.so")


def _headers() -> list[str]:
    out = [os.path.join(INCLUDE, "gp.h")]
    for f in os.listdir(CSRC):
        if f.endswith((".cuh", ".h")):
            out.append(os.path.join(CSRC, f))
    return out


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def _compile(unit, force: bool, verbose: bool):
    name, src, extra = unit
    srcp = os.path.join(CSRC, src)
    if not os.path.exists(srcp):
        return None
    obj = os.path.join(OBJ, name + ".o")
    if not force and not _stale(obj, [srcp] + _headers()):
        return obj
    cmd = [nvcc()] + ARCH + FLAGS + extra + ["-c", srcp, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src} ({name}):\n{r.stderr}")
    if verbose and r.stderr:
        with open(os.path.join(OBJ, name + ".ptxas.txt"), "w") as fh:
            fh.write(r.stderr)
    return obj


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    """Compile every unit (in parallel) and link libgp.so; returns its path."""
    os.makedirs(OBJ, exist_ok=True)
    jobs = jobs or min(len(UNITS), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = [o for o in ex.map(lambda u: _compile(u, force, verbose), UNITS) if o]
    if force or _stale(LIB, objs):
        cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "static", "-o", LIB] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
    return LIB


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--jobs", type=int, default=None)
    ap.add_argument("--verbose", action="store_true", help="keep ptxas -v reports in _build/")
    a = ap.parse_args(argv)
    print(build(a.force, a.jobs, a.verbose))
    return 0


if __name__ == "__main__":
    sys.exit(main())
