"""GPU parity of the public device API, called from a user's own kernels.

The paper's allocator is called from inside kernels on a heap the host
preallocated (Sec. 1).  tests/cuda/ holds a user's kernels that include only
include/ouro_device.cuh and call ouro_malloc / ouro_free on an
ouro_heap_dev from divergent code (a third of the lanes skip phase A, twelve
skip phase B; lanes free while others of their warp already allocate
again), the warp-collective ouro_malloc_warp / ouro_free_warp (every lane
calls, with want = false or a null pointer for the lanes that sit out), and
the staged forms of both after ouro_block_begin(ctx, h) -- all pick the
queue form at run time.  The requests mix every class with zero-byte,
oversize and run requests, and half of phase A's blocks are freed in the
middle of the kernel; a second kernel frees the rest.

Compared with the oracle run on the same requests one at a time: per-class
malloc / free / failure counts, zero-byte and oversize counts, the live
blocks between the two kernels, and the pattern checksums (XOR, sum, word
count) of everything read back; every kept block lies in the heap, aligned
to its class, disjoint from the others; freeing everything and trimming
gives the post-create state.
"""
import ctypes as C
import os
import sys

import numpy as np
import pytest

import oracle
from gpu_helpers import assert_no_overlap, class_of, same_canonical_as_post_create, torch_cuda
from paper_2504_18211_gb300 import workloads as W

HEAP, CHUNK, N, SEED = 256 << 20, 8192, 8192 + 77, 0x0A11CE


@pytest.fixture(scope="module")
def env():
    import paper_2504_18211_gb300 as P
    from paper_2504_18211_gb300 import build
    build.build()
    P.load()
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "cuda"))
    import build_user
    lib = C.CDLL(build_user.wait())
    vp, u64, u32 = C.c_void_p, C.c_uint64, C.c_uint32
    for sfx in ("", "_warp"):
        for name in ("ut_round_plain", "ut_round_staged"):
            f = getattr(lib, name + sfx)
            f.restype, f.argtypes = C.c_int, [vp, vp, vp, u64, u32, vp, vp, vp, vp]
        for name in ("ut_free_plain", "ut_free_staged"):
            f = getattr(lib, name + sfx)
            f.restype, f.argtypes = C.c_int, [vp, vp, u64, vp]
    return P, lib


def expected(a, b, variant):
    """The oracle on the same requests, one at a time, and the round's checksums."""
    t = np.arange(N)
    lane = t % 32
    in_a, in_b = lane % 3 != 2, lane < 20
    valid = lambda s: (s > 0) & (s <= (1 << 20))
    oh = oracle.OracleHeap(HEAP, CHUNK, variant)
    kept = np.zeros(N, np.int64) - 1
    for i in np.flatnonzero(in_a):
        o = oh.malloc(int(a[i]))
        if o >= 0 and i & 1:
            assert oh.free(o) == 0
        elif o >= 0:
            kept[i] = o
    for i in np.flatnonzero(in_b):
        o = oh.malloc(int(b[i]))
        if o >= 0:
            assert oh.free(o) == 0
    mid = oh.stats()
    for o in kept[kept >= 0]:
        assert oh.free(int(o)) == 0
    end = oh.stats()
    ea = oracle.expected_checksums(np.where(in_a & valid(a), a, 0).astype(np.uint32), SEED, 1)
    eb = oracle.expected_checksums(np.where(in_b & valid(b), b, 0).astype(np.uint32), SEED + 1, 1)
    check = [ea["xor64"] ^ eb["xor64"], ea["sum64"] + eb["sum64"], ea["words"] + eb["words"], 0,
             int((in_a & ~valid(a)).sum() + (in_b & ~valid(b)).sum())]
    return mid, end, check, kept >= 0


def describe_mismatches(log, a, b, base):
    """Which requests read back wrong data: phase, size, class, block offset."""
    lg = log.cpu().numpy().view(np.uint64).reshape(-1, 4)
    rows = []
    for ph, sizes in ((0, a), (1, b)):
        for t in np.flatnonzero(lg[:, 2 + ph])[:12]:
            off = int(lg[t, ph]) - base
            rows.append(f"{'AB'[ph]} t={t} size={int(sizes[t])} class={int(class_of(sizes[t:t + 1], CHUNK)[0])} "
                        f"off={off:#x} chunk={off // CHUNK} bad_words={int(lg[t, 2 + ph])}")
    return "; ".join(rows)


CASES = [(v, s, w, False) for v in ("page_array", "chunk_array", "page_vlist", "chunk_vlist", "page_varray",
                                    "chunk_varray") for s in (False, True) for w in (False, True)] + \
        [("page_array", False, True, True), ("page_varray", True, True, True), ("chunk_array", False, False, True)]


@pytest.mark.gpu
@pytest.mark.parametrize("variant,staged,collective,deopt", CASES,
                         ids=[f"{v}-{'staged' if s else 'plain'}-{'warp' if w else 'lane'}{'-deopt' if d else ''}"
                              for v, s, w, d in CASES])
def test_user_kernels_match_oracle(env, variant, staged, collective, deopt):
    P, lib = env
    torch = torch_cuda()
    a = W.mixed_sizes(N, seed=W.SEED_BASE + 61)
    b = W.mixed_sizes(N, seed=W.SEED_BASE + 62)
    mid, end, check, keep_mask = expected(a, b, variant)
    d_a = torch.from_numpy(a.view(np.int32)).cuda()
    d_b = torch.from_numpy(b.view(np.int32)).cuda()
    keep = torch.zeros(N, dtype=torch.int64, device="cuda")
    out = torch.zeros(5, dtype=torch.int64, device="cuda")
    log = torch.zeros(4 * N, dtype=torch.int64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    form = ("staged" if staged else "plain") + ("_warp" if collective else "")
    rnd, fre = getattr(lib, "ut_round_" + form), getattr(lib, "ut_free_" + form)
    with P.Heap(HEAP, CHUNK, variant, deopt=deopt) as heap:
        dev = C.byref(heap.dev)
        assert rnd(dev, d_a.data_ptr(), d_b.data_ptr(), N, SEED, keep.data_ptr(), out.data_ptr(),
                   log.data_ptr(), stream) == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint64).astype(object).tolist()
        assert got == check, (got, check, describe_mismatches(log, a, b, heap.base))
        st = heap.stats()
        assert st["error_bits"] == 0, st["error_bits"]
        for k in ("mallocs", "frees", "failed", "live"):
            assert st[k] == mid[k], (k, st[k], mid[k])
        assert (st["zero_reqs"], st["too_large"]) == (mid["zero_reqs"], mid["too_large"])
        ptrs = keep.cpu().numpy().view(np.uint64)
        assert np.array_equal(ptrs != 0, keep_mask)
        assert_no_overlap(ptrs, np.where(keep_mask, a, 0), heap.base, HEAP, CHUNK)
        assert fre(dev, keep.data_ptr(), N, stream) == 0
        torch.cuda.synchronize()
        st = heap.stats()
        assert st["error_bits"] == 0
        assert st["mallocs"] == end["mallocs"] and st["frees"] == end["frees"] and sum(st["live"]) == 0
        heap.trim()
        same_canonical_as_post_create(heap.snapshot(), HEAP // CHUNK)


def test_mixed_sizes_cover_every_kind():
    """The request mix has every class within a chunk, runs, 0 B, > 1 MiB and tails."""
    a = W.mixed_sizes(N, seed=W.SEED_BASE + 61)
    c = class_of(a, CHUNK)
    assert set(range(10)) <= set(c.tolist()) and (c > 9).any() and (a == 0).any() and (a > (1 << 20)).any()
    assert (a % 4 != 0).any()
