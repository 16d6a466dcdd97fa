"""GPU parity of graph growth: adjacency lists grown inside a kernel.

Checks: every vertex's neighbour multiset equals the host edge list; the
allocator's per-class malloc and free counts equal the closed form of the
growth rule applied to the final degrees (one 16 B list per vertex, one
malloc+free per doubling, one chunk per overflow segment); freeing every
list and trimming gives the post-create state."""
import numpy as np
import pytest

from oracle.patterns import graph_class_counts
from gpu_helpers import same_canonical_as_post_create, torch_cuda
from paper_2504_18211_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2504_18211_gb300 as P
    from paper_2504_18211_gb300 import build
    build.build()
    P.load()
    return P


@pytest.mark.parametrize("variant", ["page_array", "chunk_array", "page_vlist", "page_varray", "chunk_vlist",
                                     "chunk_varray"])
def test_graph_growth_matches_edge_list_and_closed_form(P, variant):
    from paper_2504_18211_gb300.graph import GraphRun
    torch = torch_cuda()
    nv, ne, chunk = 4096, 1 << 17, 8192
    src, dst = W.graph_workload(n_vertices=nv, n_edges=ne, seed=W.SEED_BASE + 51)
    g = GraphRun(src, dst, nv)
    heap_bytes = 256 << 20
    with P.Heap(heap_bytes, chunk, variant) as heap:
        g.init(heap)
        g.insert(heap)
        torch.cuda.synchronize()
        c = g.ctl_dict()
        assert c == {"appended": ne, "failed": 0, "skipped": 0}
        deg, off, out = g.gather(heap)
        want_deg = np.bincount(src, minlength=nv)
        assert np.array_equal(deg, want_deg)
        assert deg.max() > chunk // 4                      # overflow segments are exercised
        got = np.lexsort((out, np.repeat(np.arange(nv), deg)))
        order = np.lexsort((dst, src))
        assert np.array_equal(out[got], dst[order])
        st = heap.stats()
        m, f, _ = graph_class_counts(deg, chunk, heap.n_classes)
        assert st["mallocs"] == m.tolist() and st["frees"] == f.tolist()
        assert st["error_bits"] == 0
        g.free(heap)
        torch.cuda.synchronize()
        assert sum(heap.stats()["live"]) == 0
        heap.trim()
        same_canonical_as_post_create(heap.snapshot(), heap_bytes // chunk)
