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
