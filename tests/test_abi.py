"""The C-ABI library loads on the CPU host and exports every declared symbol."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ouro.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ouro_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2504_18211_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ouro_heap_create", "ouro_heap_create_ex", "ouro_heap_destroy", "ouro_batch_malloc",
                     "ouro_batch_free", "ouro_heap_stats", "ouro_heap_trim", "ouro_heap_snapshot",
                     "ouro_round_fused"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (ouro_\w+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_without_gpu(lib_path):
    from paper_2504_18211_gb300 import _binding as B
    lib = B.load(lib_path)
    assert B.ouro_status_string(0) == "ok"
    assert B.ouro_status_string(1) == "invalid argument"
    assert lib.ouro_kernel_launches() == 0


def test_bad_arguments_are_rejected_on_the_host(lib_path):
    import ctypes as C
    from paper_2504_18211_gb300 import _binding as B
    lib = B.load(lib_path)
    h = C.c_void_p()
    # chunk not a power of two, bytes not a multiple, too small, too large
    assert lib.ouro_heap_create(1 << 20, 3000, C.byref(h)) == 1
    assert lib.ouro_heap_create((1 << 20) + 5, 4096, C.byref(h)) == 1
    assert lib.ouro_heap_create(1 << 20, 128, C.byref(h)) == 1
    assert lib.ouro_heap_create(65 << 30, 1 << 20, C.byref(h)) == 1
    assert lib.ouro_heap_create_ex(1 << 20, 4096, 9, None, None, C.byref(h)) == 1
    assert lib.ouro_heap_destroy(None) == 0


def test_every_kernel_source_is_built():
    """Each .cu file of the package is compiled: whole, or once per queue
    form plus once for its entry points (then it includes the shard header
    and keeps its entry points behind OURO_SHARD_ENTRIES)."""
    from paper_2504_18211_gb300 import build
    csrc = os.path.join(ROOT, "paper_2504_18211_gb300", "csrc")
    sources = sorted(f for f in os.listdir(csrc) if f.endswith(".cu"))
    assert sorted(build.SOURCES + build.SHARDED) == sources
    assert not set(build.SOURCES) & set(build.SHARDED)
    for f in build.SHARDED:
        text = open(os.path.join(csrc, f)).read()
        assert '#include "ouro_shard.cuh"' in text, f
        assert "OURO_SHARD_INSTANTIATE(" in text, f
        first_entry = text.find('extern "C"')
        assert first_entry > text.find("#if OURO_SHARD_ENTRIES") >= 0, f
    assert len([j for j in build.JOBS if j[0] == build.SHARDED[0]]) == build.N_FORMS + 1
