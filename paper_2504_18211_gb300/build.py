"""Build the CUDA library libouro.so in-tree for sm_103a (GB300).

Each translation unit is compiled in parallel with nvcc, then linked into one
shared library next to this file.  The kernel files are compiled once per
queue form (-DOURO_SHARD=<form>) plus once for their host entry points
(-DOURO_SHARD=-1), so the six forms' device code compiles side by side.  No
torch extension machinery: the library exposes a plain C ABI
(include/ouro.h).
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
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libouro.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["ouro_host.cu", "ouro_probe.cu"]
SHARDED = ["ouro_kernels.cu", "ouro_batching.cu", "ouro_serving.cu", "ouro_graph.cu"]
N_FORMS = 6                       # ouro_variant values 0..5
JOBS = [(s, None) for s in SOURCES] + [(s, k) for s in SHARDED for k in range(-1, N_FORMS)]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libouro.so")


def _flags(extra=()):
    return [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
            *extra]


def _compile(job, extra=()) -> str:
    src, shard = job
    stem = os.path.splitext(src)[0]
    if shard is None:
        obj = os.path.join(BUILD, stem + ".o")
    else:
        obj = os.path.join(BUILD, f"{stem}.{'entries' if shard < 0 else f'form{shard}'}.o")
        extra = (f"-DOURO_SHARD={shard}", *extra)
    cmd = [nvcc(), *_flags(extra), "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if "-v" in extra and r.stderr:
        print(r.stderr, file=sys.stderr)     # e.g. -Xptxas -v: registers, spills, shared memory
    return obj


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + \
           [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)] + [os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Compile and link libouro.so unless it is up to date; return its path."""
    if not force and not extra and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    # the long jobs (the probes, then the per-form objects) first
    jobs = sorted(JOBS, key=lambda j: 0 if j[0] == "ouro_probe.cu" else 1 if (j[1] or 0) >= 0 and j[1] is not None else 2)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(lambda j: _compile(j, extra), jobs))
    tmp = f"{LIB}.{os.getpid()}.tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print(f"built {LIB}", file=sys.stderr)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=("-Xptxas", "-v") if "--ptxas-v" in sys.argv else ())
