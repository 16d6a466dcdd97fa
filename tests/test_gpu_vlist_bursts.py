"""Virtualized-list bursts in one class on the GPU, against the oracle: the
paper's thread-count axis at its largest points (Sec. 4.3), where a malloc
burst retires every list segment it used and relinks it behind the back
(warp-wide front walk, one retiring warp per class at a time) and the next
free burst finds the segments linked.  Checksums, exact per-class counts,
disjoint blocks, no error bit, the list's segment chunks bounded by what
two bursts' positions need, and free-all + trim back to the post-create
state."""
import numpy as np
import pytest

import oracle
from gpu_helpers import assert_no_overlap, same_canonical_as_post_create, to_dev, torch_cuda
from paper_2504_18211_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ouro():
    import paper_2504_18211_gb300 as P
    from paper_2504_18211_gb300 import build
    build.build()
    P.load()
    return P


@pytest.mark.parametrize("threads", [3 << 18, 1 << 20])
@pytest.mark.parametrize("variant", ["page_vlist", "chunk_vlist"])
def test_single_class_bursts(ouro, variant, threads):
    torch = torch_cuda()
    bytes_, chunk, size, seed = 4 << 30, 8192, 1000, 77
    sizes = W.single_size(threads, size)
    want = dict(oracle.expected_checksums(sizes, seed, 1), nulls=0, mismatches=0)
    cls = 6                                                   # 1000 B -> 1 KiB pages
    seg_cap = (chunk - 64) // 8
    with ouro.Heap(bytes_, chunk, variant) as heap:
        d_sizes = to_dev(sizes)
        ptrs = torch.empty(threads, dtype=torch.int64, device="cuda")
        chk = torch.zeros(5, dtype=torch.int64, device="cuda")
        rounds = 4
        for r in range(rounds):
            heap.malloc(d_sizes, ptrs)
            if r == rounds - 1:
                assert_no_overlap(ptrs.cpu().numpy(), sizes, heap.base, bytes_, chunk)
            ouro.pattern_write(ptrs, d_sizes, seed, 1)
            ouro.pattern_check(ptrs, d_sizes, seed, 1, chk)
            heap.free(ptrs)
            torch.cuda.synchronize()
            assert ouro.check_to_dict(chk) == want, (r, ouro.check_to_dict(chk))
        st = heap.stats()
        assert st["error_bits"] == 0, (st["error_bits"], st["error_site"])
        assert st["mallocs"][cls] == rounds * threads and st["frees"][cls] == rounds * threads
        assert sum(st["live"]) == 0 and sum(st["failed"]) == 0
        # page queues: one position per page; chunk queues: one per chunk
        per_burst = threads if variant == "page_vlist" else threads // (chunk // 1024)
        assert st["seg_chunks"] + st["spare_chunks"] <= 2 * (per_burst // seg_cap + 2) + 4, st["seg_chunks"]
        heap.trim()
        same_canonical_as_post_create(heap.snapshot(), bytes_ // chunk)
