"""Build libpolydet.so in-tree for sm_103a with nvcc (no cmake).

Each translation unit compiles in its own nvcc process, in parallel; the
objects are linked into ``paper_2010_12117_gb300/_lib/libpolydet.so`` with the
CUDA runtime linked statically.  Objects are rebuilt when a source or header
is newer than them.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libpolydet.so")

SOURCES = ["plan.cu", "ntt.cu", "crt.cu", "probe.cu", "batch.cu", "dispatch.cu", "interp_static.cu", "mlp.cu"]
# condense_inst.cu and fused_inst.cu are compiled once per range of matrix
# orders (must match the ranges in csrc/dispatch.cu)
KERNEL_RANGES = [(1, 6), (7, 10), (11, 12), (13, 16), (17, 20), (21, 24), (25, 28), (29, 32)]
TEMPLATED = ["condense_inst.cu", "fused_inst.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpolydet")


def _headers():
    out = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))]
    out += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return out


def _stale(obj: str, src: str, headers) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(x) > t for x in [src, *headers])


def _compile(src: str, obj: str, verbose_ptxas: bool, defs=()) -> None:
    cmd = [nvcc(), *ARCH, *FLAGS, *defs, "-c", src, "-o", obj]
    if verbose_ptxas:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    if verbose_ptxas:
        sys.stderr.write(r.stderr)


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    headers = _headers()
    todo = []
    objs = []
    units = [(s, s.replace(".cu", ".o"), []) for s in SOURCES]
    for s in TEMPLATED:
        for lo, hi in KERNEL_RANGES:
            units.append((s, s.replace(".cu", f"_{lo}_{hi}.o"), [f"-DPD_N_LO={lo}", f"-DPD_N_HI={hi}"]))
    for s, o, defs in units:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, o)
        objs.append(obj)
        if force or verbose_ptxas or _stale(obj, src, headers):
            todo.append((src, obj, defs))
    # the templated kernel objects dominate the build: start them first
    todo.sort(key=lambda t: 0 if t[2] else 1)
    if todo:
        with ThreadPoolExecutor(max_workers=jobs or min(len(todo), os.cpu_count() or 4)) as ex:
            list(ex.map(lambda u: _compile(u[0], u[1], verbose_ptxas, u[2]), todo))
    if todo or not os.path.exists(LIB):
        tmp = LIB + ".tmp"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import time
    t = time.time()
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
    print(f"built in {time.time() - t:.1f} s")
