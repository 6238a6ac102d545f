"""Build the CUDA library ``_lib/libgmq.so`` in-tree with nvcc for sm_103a.

The rule kernel is compiled once per integrand family (-DGMQ_FAM=k) so the
translation units build in parallel; the sweep kernels and the host API are
two more units.  The library links the CUDA runtime statically, so it has no
dependency on a particular libcudart.so.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INC = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libgmq.so")

NUM_FAMILIES = 7
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
CFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                 "-I", INC, "-I", CSRC, "--expt-relaxed-constexpr"]


def _units():
    units = [(os.path.join(CSRC, "gmq_api.cu"), "gmq_api.o", []),
             (os.path.join(CSRC, "sweep_kernels.cu"), "sweep_kernels.o", []),
             (os.path.join(CSRC, "noalloc_sum.cu"), "noalloc_sum.o", []),
             (os.path.join(CSRC, "fma_probe.cu"), "fma_probe.o", []),
             (os.path.join(CSRC, "gm_batch.cu"), "gm_batch.o", [])]
    for fam in range(NUM_FAMILIES):
        units.append((os.path.join(CSRC, "gm_rule_inst.cu"), f"gm_rule_f{fam}.o",
                      [f"-DGMQ_FAM={fam}"]))
    return units


def _deps():
    return (glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
            glob.glob(os.path.join(INC, "*.h")) + [os.path.abspath(__file__)])


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    deps = _deps()
    if not force and not _stale(LIB, deps):
        return LIB
    units = _units()

    def compile_unit(u):
        src, obj, extra = u
        out = os.path.join(BUILD, obj)
        cmd = [NVCC] + CFLAGS + extra + ["-c", src, "-o", out]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {obj}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, flush=True)
        return out

    jobs = jobs or min(len(units), max(1, os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(compile_unit, units))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [NVCC] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
