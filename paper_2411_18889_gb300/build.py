"""Build libnbody.so (the C-ABI library) in-tree with nvcc for sm_103a.

Each .cu file compiles in parallel to an object under ``_build/``; the objects
link into ``paper_2411_18889_gb300/libnbody.so`` with the CUDA runtime linked
statically, so loading the library needs no GPU.  ``python -m
paper_2411_18889_gb300.build`` runs it from the command line.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libnbody.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["force.cu", "vjp.cu", "batched.cu", "order.cu", "pack.cu", "reduce.cu", "selftest.cu", "capi.cu", "noalloc.cu"]
# The persistent batched kernel: one object per (shape, potential) instantiation.
NUM_BATCHED_SHAPES = 6  # kNumBShapes in csrc/batched_kernel.cuh
INSTANCES = [("batched_inst.cu", f"_{k}{p}", [f"-DNBK_BSHAPE={k}", f"-DNBK_BPOT={p}"])
             for k in range(NUM_BATCHED_SHAPES) for p in range(2)]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libnbody")
    return p


def _flags(extra):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden", "-Xptxas", "-v",
                   "-I", os.path.join(ROOT, "include")] + list(extra)


def _compile(src, obj, extra):
    cmd = [nvcc()] + _flags(extra) + ["-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
    return r.stderr  # ptxas -v report


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, extra=(), lib_path: str = LIB, verbose: bool = False) -> str:
    """Compile and link libnbody.so; returns its path.  Rebuilds only what changed."""
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(ROOT, "include", "nbody.h"))
    tag = "" if not extra else "_" + hashlib.sha1(" ".join(extra).encode()).hexdigest()[:8]
    units = [(src, "", []) for src in SOURCES] + INSTANCES
    objs, jobs = [], []
    with cf.ThreadPoolExecutor(max_workers=min(len(units), os.cpu_count() or 4)) as ex:
        # the slowest units first, so they start while the rest compile
        slow = {"batched_inst.cu": 0, "force.cu": 0, "vjp.cu": 1}
        for src, suffix, defs in sorted(units, key=lambda u: slow.get(u[0], 2)):
            obj = os.path.join(BUILD, src.replace(".cu", f"{suffix}{tag}.o"))
            objs.append(obj)
            if force or _stale(obj, [os.path.join(CSRC, src)] + headers):
                jobs.append((src + suffix, ex.submit(_compile, src, obj, list(defs) + list(extra))))
        reports = [(src, j.result()) for src, j in jobs]
    if reports:
        with open(os.path.join(BUILD, f"ptxas{tag}.log"), "w") as f:
            for src, rep in reports:
                f.write(f"==== {src}\n{rep}\n")
        if verbose:
            for src, rep in reports:
                sys.stderr.write(rep)
    if force or reports or _stale(lib_path, objs):
        tmp = lib_path + f".tmp{os.getpid()}"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static", "-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
