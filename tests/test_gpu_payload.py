"""The driver round's written data and the default queue capacity, element by
element against the oracle.

Written data (Sec. 3: the driver writes data into each block and reads it
back): the per-launch form allocates, writes its pattern and stops; every
block is copied back from the heap buffer and compared byte by byte with the
block the oracle's round wrote for the same request (sizes of any byte
count, so tail bytes included; mode 1 and mode 0).  The oracle's written
data is pinned by hand-worked cases (tests/golden/pattern_words.json).

Default capacity: a page-array heap at default options serves at most 2^23
pages of a class (the documented default); a 256 MiB heap has 2^24 pages of
16 B, so a batch of 2^23 + 2^16 requests gets exactly 2^16 nulls, as the
oracle does."""
import numpy as np
import pytest

import oracle
from gpu_helpers import assert_no_overlap, to_dev, torch_cuda
from paper_2504_18211_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ouro():
    import paper_2504_18211_gb300 as P
    from paper_2504_18211_gb300 import build
    build.build()
    P.load()
    return P


@pytest.mark.parametrize("variant", ["page_array", "chunk_array", "page_vlist", "page_varray"])
@pytest.mark.parametrize("mode", [1, 0])
def test_written_blocks_equal_oracle_blocks(ouro, variant, mode):
    torch = torch_cuda()
    bytes_, chunk, seed = 64 << 20, 8192, 0x0BADC0DE
    sizes = W.uniform_sizes(3000 + 5, lo=1, hi=8192, seed=W.SEED_BASE + 71)
    sizes[:5] = (1, 2, 3, 5, 16 << 10)               # tails of 1-3 bytes and a run of two chunks
    oh = oracle.OracleHeap(bytes_, chunk, variant)
    res, offs, mem = oh.round(sizes, seed, mode, return_memory=True)
    assert res["nulls"] == 0 and res["mismatches"] == 0
    buf = torch.zeros(bytes_, dtype=torch.uint8, device="cuda")
    with ouro.Heap(bytes_, chunk, variant, heap_buf=buf) as heap:
        d = to_dev(sizes)
        ptrs = heap.malloc(d)
        ouro.pattern_write(ptrs, d, seed, mode)
        torch.cuda.synchronize()
        p = ptrs.cpu().numpy().view(np.uint64)
        assert np.all(p != 0)
        assert_no_overlap(p, sizes, heap.base, bytes_, chunk)
        host = buf.cpu().numpy()
        goff = (p - np.uint64(heap.base)).astype(np.int64)
        for t in range(sizes.size):
            n = int(sizes[t]) if mode == 1 else 4
            got, want = host[goff[t]:goff[t] + n], mem[offs[t]:offs[t] + n]
            if not np.array_equal(got, want):
                bad = int(np.flatnonzero(got != want)[0])
                raise AssertionError(f"request {t} ({sizes[t]} B): byte {bad} is {got[bad]:#x}, oracle {want[bad]:#x}")
        heap.free(ptrs)
        torch.cuda.synchronize()
        assert heap.stats()["error_bits"] == 0


def test_default_page_array_capacity(ouro):
    torch = torch_cuda()
    n = (1 << 23) + (1 << 16)
    sizes = W.single_size(n, 16)
    oh = oracle.OracleHeap(256 << 20, 8192, "page_array")          # default options on both sides
    ores = oh.round(sizes, 0, 1, with_memory=False)
    ost = oh.stats()
    assert ores["nulls"] == 1 << 16 and ost["mallocs"][0] == 1 << 23
    with ouro.Heap(256 << 20, 8192, "page_array") as heap:
        ptrs = heap.malloc(to_dev(sizes))
        torch.cuda.synchronize()
        nulls = int((ptrs == 0).sum().item())
        st = heap.stats()
        assert nulls == ores["nulls"], nulls
        assert st["mallocs"][0] == ost["mallocs"][0] and st["failed"][0] == ost["failed"][0]
        assert st["carves"][0] == ost["carves"][0] == (1 << 23) // 512
        assert st["error_bits"] == 0
        heap.free(ptrs)
        torch.cuda.synchronize()
        assert sum(heap.stats()["live"]) == 0
