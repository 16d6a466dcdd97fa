"""Build the test-only library of user kernels (libouro_user.so, sm_103a).

Its kernel files include only the public device header
include/ouro_device.cuh, as an application's kernels would:
ouro_user_plain.cu and ouro_user_staged.cu compile twice each (lane-private
and warp-collective calls), ouro_user_trace.cu once with the device event
ring (-DOURO_TRACE); the five objects compile in parallel.  The GPU tests start this build in
the background when the session collects them (tests/conftest.py), so that
it overlaps the other GPU tests, and wait for it before their first call.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libouro_user.so")
SOURCES = ("ouro_user_plain.cu", "ouro_user_staged.cu", "ouro_user_trace.cu")
# (source, object tag, flags): the two round files for lane-private and
# warp-collective calls, the trace file with the device event ring on
JOBS = [(src, str(coll), [f"-DUT_COLLECTIVE={coll}"]) for src in SOURCES[:2] for coll in (0, 1)] + \
       [("ouro_user_trace.cu", "trace", ["-DOURO_TRACE"])]
DEPS = SOURCES + ("ouro_user_common.cuh", "build_user.py")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(HERE, f) for f in DEPS] + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False) -> str:
    if not force and not stale():
        return LIB
    out_dir = os.path.join(HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)

    def compile_one(job):
        src, tag, flags = job
        obj = os.path.join(out_dir, f"{os.path.splitext(src)[0]}.{tag}.o")
        cmd = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-split-compile", "0", "-Xcompiler", "-fPIC",
               *flags, "-I", INCLUDE, "-I", HERE, "-c", os.path.join(HERE, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(JOBS)) as ex:
        objs = list(ex.map(compile_one, JOBS))
    tmp = f"{LIB}.{os.getpid()}.tmp"
    r = subprocess.run([_nvcc(), *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


_proc = None


def start_background() -> None:
    """Start the build in a child process unless the library is up to date."""
    global _proc
    if _proc is None and stale():
        _proc = subprocess.Popen([sys.executable, os.path.abspath(__file__)], stdout=subprocess.PIPE,
                                 stderr=subprocess.STDOUT, text=True)


def wait() -> str:
    """The library's path, once built (by the background build if one runs)."""
    global _proc
    if _proc is not None:
        out, _ = _proc.communicate()
        rc = _proc.returncode
        _proc = None
        if rc:
            raise RuntimeError(f"background build of {LIB} failed:\n{out}")
    return build()


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
