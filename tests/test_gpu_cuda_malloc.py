"""The comparison allocator: CUDA's built-in device malloc / free running the
same fused driver round (Sec. 1 names it as the baseline that dedicated
allocators improve on).  Its read-back must match the oracle's checksums."""
import pytest

import oracle
from gpu_helpers import to_dev, torch_cuda
from paper_2504_18211_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_cuda_malloc_round_matches_oracle():
    import paper_2504_18211_gb300 as P
    from paper_2504_18211_gb300 import build
    build.build()
    P.load()
    torch = torch_cuda()
    try:
        got = P.ouro_cuda_malloc_heap(512 << 20)
    except P.OuroError:
        pytest.skip("the context's device-malloc heap was fixed before this test ran")
    assert got >= 512 << 20
    sizes = W.sweep_sizes(20000, seed=W.SEED_BASE + 14)
    seed = 0xC0DA
    want = oracle.expected_checksums(sizes, seed, 1)
    d = to_dev(sizes)
    for _ in range(2):
        out = P.ouro_cuda_malloc_round(d, seed, 1)
        torch.cuda.synchronize()
        assert P.check_to_dict(out) == dict(want, nulls=0, mismatches=0)
