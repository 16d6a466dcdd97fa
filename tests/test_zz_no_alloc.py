"""ouro_heap_stats_static: statistics for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc when they want the heap's counters:
applications whose device memory is all handed out up front by their own
pool, or latency-bound loops in which a cudaMalloc / cudaFree could stall the
device while other streams work.  ouro_heap_stats_static
gives the same result as ouro_heap_stats with its scratch in a static device
array.  This file is collected last (tests/test_zz_*) so that a failure here
leaves every other test already run; it passes alone and after the others.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _stats_via_abi(lib, h, fn_name, stream):
    from paper_2504_18211_gb300 import _binding as B
    s = B.Stats()
    status = getattr(lib, fn_name)(C.c_void_p(h), C.byref(s), C.c_void_p(stream.cuda_stream))
    assert status in (0, 4), (fn_name, status)     # 4 = device error bits set (reported in the struct)
    return B._stats_dict(s)


@pytest.mark.parametrize("variant", ["page_array", "page_vlist", "page_varray"])
def test_static_stats_match_allocating_stats(variant):
    import torch

    import paper_2504_18211_gb300 as P
    from paper_2504_18211_gb300 import build
    from paper_2504_18211_gb300 import workloads as W
    build.build()
    lib = P.load()
    stream = torch.cuda.current_stream()
    sizes = W.sweep_sizes(30000, seed=W.SEED_BASE + 77)
    d_sizes = torch.from_numpy(sizes.view(np.int32)).cuda()
    with P.Heap(256 << 20, 8192, variant) as heap:
        live = heap.malloc(d_sizes)                       # leave blocks live: non-zero counts everywhere
        done = heap.malloc(d_sizes[:5000])
        heap.free(done)
        zero = heap.malloc(torch.zeros(7, dtype=torch.int32, device="cuda"))
        torch.cuda.synchronize()
        want = _stats_via_abi(lib, heap.h, "ouro_heap_stats", stream)
        assert sum(want["mallocs"]) == 35000 and want["zero_reqs"] == 7
        for call in range(2):                             # two calls in a row share the static scratch
            got = _stats_via_abi(lib, heap.h, "ouro_heap_stats_static", stream)
            assert got == want, (call, got, want)
        heap.free(live)
        torch.cuda.synchronize()
        want2 = _stats_via_abi(lib, heap.h, "ouro_heap_stats", stream)
        got2 = _stats_via_abi(lib, heap.h, "ouro_heap_stats_static", stream)
        assert got2 == want2 and sum(got2["live"]) == 0
        del zero
