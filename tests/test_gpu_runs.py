"""Requests above one chunk on the GPU: runs of contiguous chunks.

The paper is silent on requests larger than a chunk; both implementations
read them as runs of 2^(c - n_classes + 1) chunks for class c, cut at the
bump pointer, reused from the class queue after a free, and returned to the
pool by trim.  Compared with the oracle: successes and nulls of a fill
(exact: a run class carves only for the debt it has), counts and read-back
checksums of rounds that mix pages and runs, reuse without new carving,
double frees and frees inside a run, and the post-create state after
free-all + trim.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import (assert_no_overlap, oracle_round, per_class_counts, same_canonical_as_post_create,
                         to_dev, torch_cuda)
from paper_2504_18211_gb300 import workloads as W

pytestmark = pytest.mark.gpu
ALL_VARIANTS = ("page_array", "page_vlist", "chunk_array", "chunk_vlist", "page_varray", "chunk_varray")


@pytest.fixture(scope="module")
def ouro():
    import paper_2504_18211_gb300 as P
    from paper_2504_18211_gb300 import build
    build.build()
    P.load()
    return P


@pytest.mark.parametrize("variant", ALL_VARIANTS)
def test_run_fill_reuse_and_bad_frees(ouro, variant):
    """64 chunks of 8 KiB; 20000 B is class 11, a run of 4 chunks.  Exactly
    as many of 20 requests succeed as in the oracle (16; 15 with virtualized
    queues, whose first segment takes a chunk); after freeing them all, as
    many requests of the same class reuse the runs without moving the bump."""
    torch = torch_cuda()
    bytes_, chunk, size = 64 * 8192, 8192, 20000
    sizes = W.single_size(20, size)
    oh = oracle.OracleHeap(bytes_, chunk, variant)
    o_ok = sum(1 for _ in range(20) if oh.malloc(size) >= 0)
    assert o_ok == (16 if variant in ("page_array", "chunk_array") else 15)
    ost = oh.stats()
    with ouro.Heap(bytes_, chunk, variant) as heap:
        ptrs = heap.malloc(to_dev(sizes))
        torch.cuda.synchronize()
        p = ptrs.cpu().numpy().view(np.uint64)
        assert int((p != 0).sum()) == o_ok
        assert_no_overlap(p, sizes, heap.base, bytes_, chunk)
        st = heap.stats()
        assert st["n_large"] == 7 and st["mallocs"][11] == o_ok and st["failed"][11] == 20 - o_ok
        assert st["carved_now"][11] == ost["carved_now"][11] == 4 * o_ok and st["bump"] == ost["bump"]
        live = ptrs[p != 0].clone()
        heap.free(live)
        torch.cuda.synchronize()
        assert heap.stats()["queued"][11] == o_ok
        again = heap.malloc(to_dev(W.single_size(o_ok, 16385)))  # same class, smaller size
        torch.cuda.synchronize()
        a = again.cpu().numpy().view(np.uint64)
        assert np.array_equal(np.sort(a), np.sort(p[p != 0]))     # the very same runs
        st = heap.stats()
        assert st["bump"] == ost["bump"] and st["carves"][11] == 4 * o_ok and st["error_bits"] == 0
        heap.free(again[:1].clone())
        heap.free(again[:1].clone())                             # double free of a run
        inner = torch.from_numpy(np.array([int(a[1]) + chunk], np.int64)).cuda()
        heap.free(inner)                                         # inside a run
        torch.cuda.synchronize()
        st = heap.stats()
        assert st["error_bits"] & ouro.B.ERR_DOUBLE_FREE and st["error_bits"] & ouro.B.ERR_BAD_FREE
        assert st["frees"][11] == o_ok + 1
        heap.free(again[1:].clone())
        heap.reset()


@pytest.mark.parametrize("variant", ALL_VARIANTS)
def test_rounds_mixing_pages_and_runs(ouro, variant):
    """Sizes 2^k, k uniform in [4, 16], on 8 KiB chunks: a third of the
    requests are runs of 2 to 8 chunks.  Per-launch and fused rounds match
    the oracle's counts and checksums; free-all + trim gives back the
    post-create state."""
    torch = torch_cuda()
    threads = 12000 + 33
    sizes = W.sweep_sizes(threads, seed=W.SEED_BASE + 15, kmin=4, kmax=16)
    seed = 0xB16
    bytes_, chunk = 512 << 20, 8192
    oh, ores = oracle_round(bytes_, chunk, variant, sizes, seed, 1, with_memory=True)
    want = per_class_counts(sizes, chunk)
    with ouro.Heap(bytes_, chunk, variant) as heap:
        d = to_dev(sizes)
        ptrs = heap.malloc(d)
        ouro.pattern_write(ptrs, d, seed, 1)
        chk = ouro.pattern_check(ptrs, d, seed, 1)
        torch.cuda.synchronize()
        assert ouro.check_to_dict(chk) == ores
        assert_no_overlap(ptrs.cpu().numpy().view(np.uint64), sizes, heap.base, bytes_, chunk)
        st_m = heap.stats()
        assert st_m["mallocs"] == want == oh.stats()["mallocs"]
        assert st_m["carves"][10:] == oh.stats()["carves"][10:]        # one run per request, exact
        heap.free(ptrs)
        for _ in range(2):
            out = heap.round_fused(d, seed, 1)
            assert ouro.check_to_dict(out) == ores
        torch.cuda.synchronize()
        st = heap.stats()
        assert st["mallocs"] == [3 * w for w in want] and st["frees"] == st["mallocs"]
        assert st["error_bits"] == 0 and sum(st["live"]) == 0
        heap.trim()
        same_canonical_as_post_create(heap.snapshot(), bytes_ // chunk)
