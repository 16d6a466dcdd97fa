"""GPU parity of the allocator (page / chunk queues; plain array, virtualized list, virtualized array) against the oracle.

Every test calls the CUDA library through its C ABI (paper_2504_18211_gb300
binding) and compares with oracle/ on the same seeded inputs:
  - per-class mallocs / frees / live, null answers, read-back checksums: exact;
  - chunks carved in a malloc-only phase: exact for page queues (they carve
    only for debt that exists, in one batch per lock holder); chunk queues
    pack the page needs that waiting groups posted, so their count lies
    between the oracle's and the bound where every group asked for a warp;
  - no overlap, in-heap, aligned (host check of every returned address);
  - free everything + trim: the snapshot equals the post-create state.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import (assert_no_overlap, oracle_round, per_class_counts,
                         same_canonical_as_post_create, to_dev, torch_cuda)
from paper_2504_18211_gb300 import workloads as W

pytestmark = pytest.mark.gpu
PAGE_VARIANTS = ("page_array", "page_vlist", "page_varray")
ALL_VARIANTS = ("page_array", "page_vlist", "chunk_array", "chunk_vlist", "page_varray", "chunk_varray")


def carve_bounds_ok(variant, got, want, sizes, chunk):
    """Chunks carved in a malloc-only phase: exact for page queues; for chunk
    queues at least the oracle's and at most one chunk per 32 pages asked for
    by a full warp group (a group that had not posted its need counts as 32)."""
    n_in_chunk = (chunk.bit_length() - 1) - 3
    if variant.startswith("page"):
        return got == want
    from gpu_helpers import class_of
    cls = class_of(sizes, chunk)
    for c, (g, w) in enumerate(zip(got, want)):
        if c >= n_in_chunk:                  # runs: one per request that found no free run
            if g != w:
                return False
            continue
        n = int((cls == c).sum())
        ppc = chunk // (16 << c)
        groups = sum(len(set(cls[i:i + 32][cls[i:i + 32] == c].tolist())) for i in range(0, cls.size, 32))
        hi = -(-(n + 31 * groups) // ppc) + 1
        if not (w <= g <= hi):
            return False
    return True


@pytest.fixture(scope="module")
def ouro():
    import paper_2504_18211_gb300 as P
    from paper_2504_18211_gb300 import build
    build.build()
    P.load()
    return P


def per_launch_round(P, heap, sizes_np, seed, mode):
    torch = torch_cuda()
    sizes = to_dev(sizes_np)
    ptrs = heap.malloc(sizes)
    torch.cuda.synchronize()
    st_malloc = heap.stats()
    P.pattern_write(ptrs, sizes, seed, mode)
    chk = P.pattern_check(ptrs, sizes, seed, mode)
    torch.cuda.synchronize()
    host_ptrs = ptrs.cpu().numpy().view(np.uint64)
    heap.free(ptrs)
    torch.cuda.synchronize()
    return host_ptrs, P.check_to_dict(chk), st_malloc, heap.stats()


@pytest.mark.parametrize("variant", ALL_VARIANTS)
def test_small_plain_method(ouro, variant):
    """40x256 threads, 16 B each, thread id written and read back."""
    sizes = W.small_sizes()
    bytes_, chunk = 64 << 20, 8192
    oh, ores = oracle_round(bytes_, chunk, variant, sizes, 0, 0, with_memory=True)
    with ouro.Heap(bytes_, chunk, variant) as heap:
        ptrs, chk, st_m, st = per_launch_round(ouro, heap, sizes, 0, 0)
        assert chk == ores, (chk, ores)
        assert_no_overlap(ptrs, sizes, heap.base, bytes_, chunk)
        ost = oh.stats()
        assert st_m["carves"][0] == ost["carves"][0] == 20
        assert st["mallocs"] == ost["mallocs"] and st["frees"] == ost["frees"]
        assert st["failed"] == ost["failed"] and st["live"] == [0] * len(st["live"])
        assert st["error_bits"] == 0
        snap = heap.snapshot()
        q = np.sort(snap["queues"][0])
        if variant.startswith("chunk"):
            # every carved chunk is queued exactly once, with every page free
            owned = np.flatnonzero(snap["chunk_cls"] == 0)
            assert st["queued"][0] == 20 and np.array_equal(q, owned.astype(np.uint32))
            assert np.all(snap["chunk_free"][owned] == 512)
            if variant == "chunk_array":
                assert np.array_equal(q, np.sort(oh.queue_items(0)).astype(np.uint32))
        elif variant == "page_array":
            assert st["queued"][0] == 10240
            # same carve order (bump pointer): the very same page ids
            assert np.array_equal(q, np.sort(oh.queue_items(0)).astype(np.uint32))
        else:
            assert st["queued"][0] == 10240
            # queue segments share the bump pointer, so chunk ids differ from the
            # oracle's: every page of every class-0 chunk is queued exactly once
            owned = np.flatnonzero(snap["chunk_cls"] == 0)
            assert owned.size == 20
            assert np.array_equal(q, (owned[:, None] * 512 + np.arange(512)).ravel().astype(np.uint32))
        heap.trim()
        same_canonical_as_post_create(heap.snapshot(), bytes_ // chunk)


@pytest.mark.parametrize("variant", ALL_VARIANTS)
@pytest.mark.parametrize("threads", [1000, 16384 + 77])
def test_sweep_per_launch(ouro, variant, threads):
    sizes = W.sweep_sizes(threads, seed=W.SEED_BASE + 11)
    seed = 0xC0FFEE
    bytes_, chunk = 256 << 20, 8192
    oh, ores = oracle_round(bytes_, chunk, variant, sizes, seed, 1, with_memory=True)
    with ouro.Heap(bytes_, chunk, variant) as heap:
        ptrs, chk, st_m, st = per_launch_round(ouro, heap, sizes, seed, 1)
        assert chk == ores
        assert chk["mismatches"] == 0 and chk["nulls"] == 0
        assert_no_overlap(ptrs, sizes, heap.base, bytes_, chunk)
        ost = oh.stats()
        want = per_class_counts(sizes, chunk)
        assert st["mallocs"] == ost["mallocs"] == want
        assert st["frees"] == ost["frees"] == want
        assert carve_bounds_ok(variant, st_m["carves"], ost["carves"], sizes, chunk), (st_m["carves"], ost["carves"])
        assert st["error_bits"] == 0
        heap.trim()
        same_canonical_as_post_create(heap.snapshot(), bytes_ // chunk)


@pytest.mark.parametrize("staging", [False, True])
@pytest.mark.parametrize("variant", ALL_VARIANTS)
def test_sweep_fused_rounds(ouro, variant, staging):
    """Fused rounds, with and without shared-memory staging of freed pages
    (every queue form): counts and checksums exact, and every staged page is
    back in its queue (page queues) or its chunk (chunk queues) when the
    kernel ends."""
    torch = torch_cuda()
    threads = 20000
    sizes = W.sweep_sizes(threads, seed=W.SEED_BASE + 12)
    seed = 1234
    bytes_, chunk = 256 << 20, 8192
    expect = oracle.expected_checksums(sizes, seed, 1)
    want = per_class_counts(sizes, chunk)
    with ouro.Heap(bytes_, chunk, variant, staging=staging) as heap:
        d_sizes = to_dev(sizes)
        ptrs = torch.zeros(threads, dtype=torch.int64, device="cuda")
        for r in range(3):
            out = heap.round_fused(d_sizes, seed, 1, ptrs=ptrs)
            chk = ouro.check_to_dict(out)
            assert chk == dict(expect, nulls=0, mismatches=0), (r, chk)
        st = heap.stats()
        assert st["mallocs"] == [3 * w for w in want] and st["frees"] == st["mallocs"]
        assert st["error_bits"] == 0 and sum(st["live"]) == 0
        heap.trim()
        same_canonical_as_post_create(heap.snapshot(), bytes_ // chunk)


@pytest.mark.parametrize("variant", ALL_VARIANTS)
def test_single_class_fill_to_exhaustion(ouro, variant):
    """A full heap answers null exactly as often as the oracle (plain array
    queues); virtualized queues also spend chunks on queue segments."""
    torch = torch_cuda()
    bytes_, chunk, size = 64 * 4096, 4096, 256
    cap = bytes_ // size
    n = cap + 333
    sizes = W.single_size(n, size)
    oh = oracle.OracleHeap(bytes_, chunk, variant)
    o_ok = sum(1 for _ in range(n) if oh.malloc(size) >= 0)
    with ouro.Heap(bytes_, chunk, variant) as heap:
        ptrs = heap.malloc(to_dev(sizes))
        torch.cuda.synchronize()
        p = ptrs.cpu().numpy().view(np.uint64)
        ok = int((p != 0).sum())
        assert_no_overlap(p, sizes, heap.base, bytes_, chunk)
        st = heap.stats()
        if variant in ("page_array", "chunk_array"):
            assert ok == o_ok == cap
        else:
            segs = st["seg_chunks"] + st["spare_chunks"]
            assert ok == (bytes_ // chunk - segs) * (chunk // size)
            assert ok <= o_ok
        assert st["mallocs"][4] == ok and st["failed"][4] == n - ok
        assert st["error_bits"] == 0
        heap.free(ptrs)
        heap.trim()
        same_canonical_as_post_create(heap.snapshot(), bytes_ // chunk)


def test_phase_separated_fills(ouro):
    """Class A then class B to exhaustion: the null count of phase B equals
    the oracle's, which needs exact carving in phase A."""
    torch = torch_cuda()
    bytes_, chunk = 256 * 4096, 4096
    a = W.single_size(5000, 48)      # 64 B class: 64 pages per chunk -> 79 chunks
    b = W.single_size(400, 4000)     # 4 KiB class: one page per chunk
    oh = oracle.OracleHeap(bytes_, chunk, "page_array")
    oa = [oh.malloc(48) for _ in range(a.size)]
    ob_ok = sum(1 for _ in range(b.size) if oh.malloc(4000) >= 0)
    with ouro.Heap(bytes_, chunk, "page_array") as heap:
        pa = heap.malloc(to_dev(a))
        pb = heap.malloc(to_dev(b))
        torch.cuda.synchronize()
        assert int((pa.cpu() != 0).sum()) == sum(o >= 0 for o in oa)
        assert int((pb.cpu() != 0).sum()) == ob_ok == 256 - 79
        st = heap.stats()
        assert st["carves"] == oh.stats()["carves"]


@pytest.mark.parametrize("variant", ALL_VARIANTS)
def test_divergent_and_partial_warps(ouro, variant):
    """Odd lanes only, a single lane, and mixed sizes inside one warp."""
    torch = torch_cuda()
    bytes_, chunk = 16 << 20, 8192
    sizes = W.sweep_sizes(4096, seed=5)
    sizes[1::2] = 0                       # half the lanes ask for nothing
    sizes[100] = 2 << 20                  # above the largest class (1 MiB)
    with ouro.Heap(bytes_, chunk, variant) as heap:
        ptrs = heap.malloc(to_dev(sizes))
        one = heap.malloc(to_dev(np.array([24], np.uint32)))
        torch.cuda.synchronize()
        p = ptrs.cpu().numpy().view(np.uint64)
        assert np.all(p[1::2] == 0) and p[100] == 0
        assert np.all(p[0::2][np.arange(2048) != 50] != 0)
        assert_no_overlap(np.concatenate([p, one.cpu().numpy().view(np.uint64)]),
                          np.concatenate([sizes, np.array([24], np.uint32)]), heap.base, bytes_, chunk)
        st = heap.stats()
        assert st["zero_reqs"] == 2048 and st["too_large"] == 1
        heap.free(ptrs)
        heap.free(one)
        st = heap.stats()
        assert sum(st["live"]) == 0 and st["error_bits"] == 0


@pytest.mark.parametrize("variant", ALL_VARIANTS)
def test_bad_frees_set_error_bits(ouro, variant):
    torch = torch_cuda()
    bytes_, chunk = 4 << 20, 4096
    with ouro.Heap(bytes_, chunk, variant, checked=True) as heap:
        ptrs = heap.malloc(to_dev(W.single_size(64, 32)))
        torch.cuda.synchronize()
        p = ptrs.cpu().numpy().view(np.int64)
        bogus = np.array([p[0] + 8, heap.base + bytes_ + 64, 0, heap.base + 1000 * 4096], np.int64)
        heap.free(torch.from_numpy(bogus).cuda())
        torch.cuda.synchronize()
        st = heap.stats()
        assert st["error_bits"] & ouro.B.ERR_BAD_FREE
        assert sum(st["frees"]) == 0
        heap.free(ptrs)
        heap.free(ptrs[:3].clone())       # double free of three blocks
        st = heap.stats()
        assert st["error_bits"] & ouro.B.ERR_DOUBLE_FREE
        assert st["frees"][1] == 64 and st["live"][1] == 0
        if variant.startswith("chunk"):
            heap.trim()
            same_canonical_as_post_create(heap.snapshot(), bytes_ // chunk)


@pytest.mark.parametrize("variant", ALL_VARIANTS)
def test_stalled_producer_times_out_without_hanging(ouro, variant):
    """A producer slot that is never filled: the waiting consumer gives up
    after its bounded wait, answers null and sets OURO_ERR_TIMEOUT; the heap
    keeps working after a reset."""
    torch = torch_cuda()
    bytes_, chunk = 4 << 20, 4096
    with ouro.Heap(bytes_, chunk, variant, spin_limit=2000, backoff_max_ns=256) as heap:
        ouro.ouro_debug_stall_producer(heap.h, 0, 1)
        ptrs = heap.malloc(to_dev(W.single_size(1, 16)))
        torch.cuda.synchronize()
        assert int(ptrs.cpu()[0]) == 0
        st = heap.stats()
        assert st["error_bits"] & ouro.B.ERR_TIMEOUT and st["failed"][0] == 1
        heap.reset()
        ptrs = heap.malloc(to_dev(W.single_size(1000, 16)))
        torch.cuda.synchronize()
        assert int((ptrs.cpu() != 0).sum()) == 1000
        assert heap.stats()["error_bits"] == 0


@pytest.mark.parametrize("variant", ALL_VARIANTS)
def test_full_scale_sweep(ouro, variant):
    """2^20 threads on the 8 GiB / 8 KiB sweep heap, the bench's launch shape:
    counts and checksums exact against the oracle, carves exact (page) or
    bounded (chunk), free-all + trim back to the post-create state."""
    torch = torch_cuda()
    sizes = W.sweep_sizes()
    seed = 0x5EED
    bytes_, chunk = 8 << 30, 8192
    oh, ores = oracle_round(bytes_, chunk, variant, sizes, seed, 1, with_memory=False)
    with ouro.Heap(bytes_, chunk, variant) as heap:
        ptrs, chk, st_m, st = per_launch_round(ouro, heap, sizes, seed, 1)
        assert chk == ores
        assert_no_overlap(ptrs, sizes, heap.base, bytes_, chunk)
        ost = oh.stats()
        assert carve_bounds_ok(variant, st_m["carves"], ost["carves"], sizes, chunk)
        assert st["mallocs"] == ost["mallocs"] and st["frees"] == ost["frees"]
        out = heap.round_fused(to_dev(sizes), seed, 1)
        assert ouro.check_to_dict(out) == ores
        st2 = heap.stats()
        assert st2["error_bits"] == 0, (st2["error_bits"], st2["error_site"])
        heap.trim()
        same_canonical_as_post_create(heap.snapshot(), bytes_ // chunk)


@pytest.mark.parametrize("variant", ALL_VARIANTS)
def test_deoptimised_form(ouro, variant):
    """The deoptimised form of Sec. 2 (no warp aggregation, a fence in place
    of __nanosleep): per-launch and fused rounds give the oracle's counts and
    checksums, page queues carve exactly, and free-all + trim restores the
    post-create state."""
    torch = torch_cuda()
    threads = 16384 + 77
    sizes = W.sweep_sizes(threads, seed=W.SEED_BASE + 13)
    seed = 0xDE0F7
    bytes_, chunk = 256 << 20, 8192
    oh, ores = oracle_round(bytes_, chunk, variant, sizes, seed, 1, with_memory=True)
    with ouro.Heap(bytes_, chunk, variant, deopt=True) as heap:
        ptrs, chk, st_m, st = per_launch_round(ouro, heap, sizes, seed, 1)
        assert chk == ores
        assert_no_overlap(ptrs, sizes, heap.base, bytes_, chunk)
        ost = oh.stats()
        assert st["mallocs"] == ost["mallocs"] and st["frees"] == ost["frees"]
        assert carve_bounds_ok(variant, st_m["carves"], ost["carves"], sizes, chunk), (st_m["carves"], ost["carves"])
        for _ in range(2):
            out = heap.round_fused(to_dev(sizes), seed, 1)
            assert ouro.check_to_dict(out) == ores
        torch.cuda.synchronize()
        st = heap.stats()
        assert st["error_bits"] == 0 and sum(st["live"]) == 0
        heap.trim()
        same_canonical_as_post_create(heap.snapshot(), bytes_ // chunk)
