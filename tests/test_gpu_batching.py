"""GPU parity of the batching pattern: per-launch, CUDA-graph and persistent forms.

Every request of every batch allocates, writes its pattern (seed + batch,
thread id = index in the batch), reads it back and frees.  Each form's
per-batch check must equal the oracle's driver round on that batch, null
answers included (4 KiB chunks cannot serve requests above 4096 B)."""
import numpy as np
import pytest

import oracle
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


def oracle_checks(sizes, offs, seed, chunk, variant):
    out = []
    for b in range(offs.size - 1):
        s = sizes[int(offs[b]):int(offs[b + 1])]
        h = oracle.OracleHeap(64 << 20, chunk, variant)
        out.append(h.round(s, seed + b, 1, with_memory=True))
    return out


@pytest.mark.parametrize("variant", ["page_array", "page_vlist", "chunk_array", "chunk_vlist", "page_varray",
                                     "chunk_varray"])
@pytest.mark.parametrize("chunk", [8192, 4096])
def test_batching_forms_match_oracle(P, variant, chunk):
    from paper_2504_18211_gb300.batching import FORMS, BatchRun
    torch = torch_cuda()
    sizes, offs = W.batching_workload(n_batches=12, lo=5, hi=12, seed=W.SEED_BASE + 31)
    run = BatchRun(sizes, offs, seed=0xBA7C4)
    want = oracle_checks(sizes, offs, run.seed, chunk, variant)
    with P.Heap(512 << 20, chunk, variant) as heap:
        for form in FORMS:
            run.run(heap, form)
            torch.cuda.synchronize()
            got = run.checks()
            assert got == want, (form, [i for i, (g, w) in enumerate(zip(got, want)) if g != w][:3])
        st = heap.stats()
        assert st["error_bits"] == 0 and sum(st["live"]) == 0
        big = int((sizes > chunk).sum())          # 4 KiB chunks: runs of two chunks
        assert st["too_large"] == 0
        assert sum(st["mallocs"]) == len(FORMS) * sizes.size
        assert sum(st["mallocs"][(chunk.bit_length() - 1) - 3:]) == len(FORMS) * big
        run.close()
        heap.trim()
        same_canonical_as_post_create(heap.snapshot(), (512 << 20) // chunk)


def test_persistent_form_is_one_launch_and_graph_replays(P):
    from paper_2504_18211_gb300.batching import BatchRun
    torch = torch_cuda()
    sizes, offs = W.batching_workload(n_batches=20, lo=4, hi=10, seed=W.SEED_BASE + 32)
    run = BatchRun(sizes, offs)
    with P.Heap(256 << 20, 8192, "page_array") as heap:
        n0 = P.ouro_kernel_launches()
        run.run(heap, "persistent")
        torch.cuda.synchronize()
        assert P.ouro_kernel_launches() - n0 == 1
        first = run.checks()
        run.run(heap, "graph")                   # capture + first replay
        torch.cuda.synchronize()
        n1 = P.ouro_kernel_launches()
        run.run(heap, "graph")                   # replay only
        torch.cuda.synchronize()
        assert P.ouro_kernel_launches() - n1 == 20    # one fused kernel per batch
        assert run.checks() == first
        run.close()


@pytest.mark.parametrize("variant", ["page_array", "page_vlist", "page_varray"])
def test_persistent_form_with_staging(P, variant):
    """Shared-memory staging in the persistent kernel: same per-batch checks
    as the oracle, every page back in its queue at the end."""
    from paper_2504_18211_gb300.batching import BatchRun
    torch = torch_cuda()
    sizes, offs = W.batching_workload(n_batches=16, lo=5, hi=12, seed=W.SEED_BASE + 33)
    run = BatchRun(sizes, offs)
    want = oracle_checks(sizes, offs, run.seed, 8192, variant)
    with P.Heap(512 << 20, 8192, variant, staging=True) as heap:
        for _ in range(2):
            run.run(heap, "persistent")
            torch.cuda.synchronize()
            assert run.checks() == want
        st = heap.stats()
        assert st["error_bits"] == 0 and sum(st["live"]) == 0
        assert sum(st["mallocs"]) == 2 * sizes.size == sum(st["frees"])
        heap.trim()
        same_canonical_as_post_create(heap.snapshot(), (512 << 20) // 8192)
