"""Edge cases on the GPU, against the oracle: empty and single-request
launches, the largest class (1 MiB) and one byte past it, the smallest and
largest chunk sizes, and the largest heap the library accepts (64 GiB)."""
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
def test_empty_and_single_request(ouro, variant):
    torch = torch_cuda()
    with ouro.Heap(16 << 20, 4096, variant) as heap:
        empty = torch.zeros(0, dtype=torch.int32, device="cuda")
        ptrs = heap.malloc(empty)
        heap.free(ptrs)
        out = heap.round_fused(empty, 1, 1)
        torch.cuda.synchronize()
        assert ptrs.numel() == 0 and ouro.check_to_dict(out) == dict(nulls=0, mismatches=0, xor64=0, sum64=0, words=0)
        st = heap.stats()
        assert sum(st["mallocs"]) == 0 and st["bump"] == 0 and st["error_bits"] == 0
        one = W.single_size(1, 3000)
        want = oracle.expected_checksums(one, 9, 1)
        for _ in range(2):
            out = heap.round_fused(to_dev(one), 9, 1)
            assert ouro.check_to_dict(out) == dict(want, nulls=0, mismatches=0)
        st = heap.stats()
        assert st["mallocs"][8] == 2 and st["frees"][8] == 2 and st["error_bits"] == 0
        heap.trim()
        same_canonical_as_post_create(heap.snapshot(), (16 << 20) // 4096)


@pytest.mark.parametrize("variant", ALL_VARIANTS)
def test_largest_class_and_beyond(ouro, variant):
    """Exactly 1 MiB is the largest class (a run of 128 chunks of 8 KiB);
    1 MiB + 1 is null.  The null counts and checksums match the oracle."""
    torch = torch_cuda()
    bytes_, chunk = 64 << 20, 8192
    sizes = np.array([1 << 20, (1 << 20) + 1, 1 << 20, 16, (1 << 20) - 1] + [1 << 20] * 60, np.uint32)
    oh, ores = oracle_round(bytes_, chunk, variant, sizes, 77, 1, with_memory=True)
    with ouro.Heap(bytes_, chunk, variant) as heap:
        d = to_dev(sizes)
        ptrs = heap.malloc(d)
        ouro.pattern_write(ptrs, d, 77, 1)
        chk = ouro.pattern_check(ptrs, d, 77, 1)
        torch.cuda.synchronize()
        p = ptrs.cpu().numpy().view(np.uint64)
        assert p[1] == 0
        got = ouro.check_to_dict(chk)
        # the heap holds 64 runs of 1 MiB at most (fewer with queue segments):
        # nulls and checksums equal the oracle's
        assert got == ores, (got, ores)
        assert_no_overlap(p, sizes, heap.base, bytes_, chunk)
        st = heap.stats()
        assert st["too_large"] == 1 and st["mallocs"] == oh.stats()["mallocs"]
        heap.free(ptrs)
        torch.cuda.synchronize()
        heap.trim()
        same_canonical_as_post_create(heap.snapshot(), bytes_ // chunk)


@pytest.mark.parametrize("chunk", [256, 1 << 20])
@pytest.mark.parametrize("variant", ["page_array", "chunk_array", "page_varray"])
def test_extreme_chunk_sizes(ouro, variant, chunk):
    """256 B chunks (5 classes within a chunk, 12 run classes) and 1 MiB
    chunks (all 17 classes within a chunk): a size sweep up to 64 KiB in
    per-launch and fused rounds matches the oracle."""
    torch = torch_cuda()
    sizes = W.sweep_sizes(5000 + 17, seed=W.SEED_BASE + 16, kmin=4, kmax=16)
    bytes_ = 512 << 20
    oh, ores = oracle_round(bytes_, chunk, variant, sizes, 5, 1, with_memory=True)
    with ouro.Heap(bytes_, chunk, variant) as heap:
        d = to_dev(sizes)
        ptrs = heap.malloc(d)
        ouro.pattern_write(ptrs, d, 5, 1)
        chk = ouro.pattern_check(ptrs, d, 5, 1)
        torch.cuda.synchronize()
        assert ouro.check_to_dict(chk) == ores
        assert_no_overlap(ptrs.cpu().numpy().view(np.uint64), sizes, heap.base, bytes_, chunk)
        heap.free(ptrs)
        out = heap.round_fused(d, 5, 1)
        assert ouro.check_to_dict(out) == ores
        st = heap.stats()
        assert st["mallocs"] == [2 * w for w in per_class_counts(sizes, chunk)] and st["error_bits"] == 0
        heap.trim()
        same_canonical_as_post_create(heap.snapshot(), bytes_ // chunk)


def test_largest_heap(ouro):
    """The largest heap (64 GiB of 8 KiB chunks, 2^23 chunks): a fill of the
    8 KiB class uses every chunk exactly once, the next request is null, and
    free-all + trim restores the post-create state."""
    torch = torch_cuda()
    bytes_, chunk = 64 << 30, 8192
    n = (bytes_ // chunk) + 1000
    with ouro.Heap(bytes_, chunk, "page_array") as heap:
        ptrs = heap.malloc(to_dev(W.single_size(n, 8192)))
        torch.cuda.synchronize()
        p = ptrs.cpu().numpy().view(np.uint64)
        live = p != 0
        assert int(live.sum()) == bytes_ // chunk
        offs = np.sort(p[live] - np.uint64(heap.base))
        assert np.array_equal(offs, np.arange(bytes_ // chunk, dtype=np.uint64) * np.uint64(chunk))
        st = heap.stats()
        assert st["failed"][9] == 1000 and st["bump"] == bytes_ // chunk and st["error_bits"] == 0
        heap.free(ptrs)
        heap.trim()
        st = heap.stats()
        assert st["bump"] == 0 and st["pool_size"] == 0 and sum(st["live"]) == 0
