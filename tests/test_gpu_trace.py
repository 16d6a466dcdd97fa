"""The compile-time device event ring (OURO_TRACE) in a user's kernels.

tests/cuda/ouro_user_trace.cu includes the public device header with
-DOURO_TRACE; its kernels allocate warp-collectively and free one pointer.
The ring must hold the slow events the oracle implies: a fill of a
64-chunk page-array heap with 64 B requests carves all 64 chunks (the
oracle's carve count) and answers the requests past capacity with null
(the oracle's null count); a virtualized-list heap sets up its queue
segments; a free of a pointer that is no block start records the bad-free
error with its site."""
import ctypes as C
import os
import sys

import numpy as np
import pytest

import oracle
from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu

OURO_TR_CARVE, OURO_TR_CHUNK_CARVE, OURO_TR_EXHAUSTED, OURO_TR_SEGMENT, OURO_TR_GIVEUP, OURO_TR_ERROR = range(1, 7)
SITE_BAD_FREE = 12           # OURO_SITE_BAD_FREE in include/ouro_device.cuh
ERR_BAD_FREE = 1


class Event(C.Structure):
    _fields_ = [("t", C.c_uint64), ("kind", C.c_uint32), ("cls", C.c_uint32), ("a", C.c_uint64), ("b", C.c_uint64)]


@pytest.fixture(scope="module")
def env():
    import paper_2504_18211_gb300 as P
    from paper_2504_18211_gb300 import build
    build.build()
    P.load()
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "cuda"))
    import build_user
    lib = C.CDLL(build_user.wait())
    vp = C.c_void_p
    lib.ut_trace_fill.restype, lib.ut_trace_fill.argtypes = C.c_int, [vp, C.c_uint32, C.c_uint64, vp, vp]
    lib.ut_trace_free.restype, lib.ut_trace_free.argtypes = C.c_int, [vp, vp, vp]
    lib.ut_trace_read.restype = C.c_int
    lib.ut_trace_read.argtypes = [vp, C.c_uint32, C.POINTER(C.c_uint64), C.c_int]
    return P, lib


def read(lib, clear=True):
    buf = (Event * 4096)()
    total = C.c_uint64(0)
    assert lib.ut_trace_read(C.cast(buf, C.c_void_p), 4096, C.byref(total), 1 if clear else 0) == 0
    return [(e.t, e.kind, e.cls, e.a, e.b) for e in buf[:min(total.value, 4096)]], total.value


def test_trace_records_carves_exhaustion_and_errors(env):
    P, lib = env
    torch = torch_cuda()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    heap_bytes, chunk, size, extra = 64 * 4096, 4096, 64, 100
    n = heap_bytes // size + extra
    oh = oracle.OracleHeap(heap_bytes, chunk, "page_array")
    o_nulls = sum(1 for _ in range(n) if oh.malloc(size) < 0)
    ost = oh.stats()
    read(lib)                                                  # start from an empty ring
    ptrs = torch.zeros(n, dtype=torch.int64, device="cuda")
    with P.Heap(heap_bytes, chunk, "page_array") as heap:
        assert lib.ut_trace_fill(C.byref(heap.dev), size, n, ptrs.data_ptr(), stream) == 0
        torch.cuda.synchronize()
        nulls = int((ptrs == 0).sum().item())
        st = heap.stats()
        ev, total = read(lib)
        assert nulls == o_nulls == extra and st["carves"][2] == ost["carves"][2] == 64
        carves = [e for e in ev if e[1] == OURO_TR_CARVE]
        assert carves and all(e[2] == 2 for e in carves) and sum(e[3] for e in carves) == 64
        dead = [e for e in ev if e[1] == OURO_TR_EXHAUSTED]
        assert dead and all(e[2] == 2 for e in dead) and sum(e[3] for e in dead) == extra
        assert all(e[0] > 0 for e in ev) and total == len(ev)
        assert not [e for e in ev if e[1] in (OURO_TR_GIVEUP, OURO_TR_ERROR)]
        # a pointer that is no block start: the error and its site
        assert lib.ut_trace_free(C.byref(heap.dev), C.c_void_p(heap.base + 8), stream) == 0
        torch.cuda.synchronize()
        ev, _ = read(lib)
        assert [(e[1], e[3], e[4]) for e in ev] == [(OURO_TR_ERROR, ERR_BAD_FREE, SITE_BAD_FREE)]
        assert heap.stats()["error_bits"] == ERR_BAD_FREE


def test_trace_records_virtualized_segments(env):
    P, lib = env
    torch = torch_cuda()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    heap_bytes, chunk, size, n = 4 << 20, 4096, 16, 20000
    read(lib)
    ptrs = torch.zeros(n, dtype=torch.int64, device="cuda")
    with P.Heap(heap_bytes, chunk, "page_vlist") as heap:
        assert lib.ut_trace_fill(C.byref(heap.dev), size, n, ptrs.data_ptr(), stream) == 0
        torch.cuda.synchronize()
        assert int((ptrs == 0).sum().item()) == 0
        st = heap.stats()
        ev, _ = read(lib)
        segs = [e for e in ev if e[1] == OURO_TR_SEGMENT]
        # positions 0 .. n-1 of class 0 need ceil(n / ((4096 - 64) / 8)) segments, each a chunk of the
        # heap set up once (recycled segments are set up again without a new chunk)
        want = -(-n // ((chunk - 64) // 8))
        idx = [e[3] for e in segs]
        assert len(set(idx)) == len(idx) and set(range(want)) <= set(idx) and all(e[2] == 0 for e in segs)
        assert all(e[4] < heap_bytes // chunk for e in segs)
        assert st["error_bits"] == 0 and st["seg_chunks"] >= 1
