"""GPU parity of the serving loop (continuous batching on the device).

Checks against host restatements of the rules: the admission schedule
(admit and completion step of every session) equals the host model; every
completed session's checksum equals the oracle's closed form for its blocks
(seed + session, block index), with no mismatch; the same sessions run
alone give the same checksums as in the mix; allocator counts balance."""
import numpy as np
import pytest

import oracle
from oracle.patterns import serving_schedule
from gpu_helpers import torch_cuda
from paper_2504_18211_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2504_18211_gb300 as P
    from paper_2504_18211_gb300 import build
    build.build()
    P.load()
    return P


def session_checksum(seed, s, nblocks, block_bytes):
    r = oracle.expected_checksums(np.full(nblocks, block_bytes, np.uint32), (seed + s) & 0xFFFFFFFF, 1)
    return r["xor64"], r["sum64"]


@pytest.mark.parametrize("variant", ["page_array", "chunk_array", "page_vlist", "page_varray", "chunk_vlist",
                                     "chunk_varray"])
def test_serving_loop_matches_model_and_oracle(P, variant):
    from paper_2504_18211_gb300.serving import ServeRun
    torch_cuda()
    steps, block = 300, 16384
    arrive, blocks = W.serving_workload(steps=steps, rate=2000.0, dt=0.01, median_bytes=256 << 10, sigma=1.0,
                                        block_bytes=block, max_blocks=256, seed=W.SEED_BASE + 41)
    heap_bytes = 128 << 20
    cap = int(0.95 * heap_bytes // block)
    run = ServeRun(arrive, blocks, n_slots=1024, max_blocks=256, steps=steps, seed=0x5E55, block_bytes=block)
    with P.Heap(heap_bytes, block, variant) as heap:
        run.run(heap, cap)
        r = run.results()
        st = heap.stats()
    assert r["error"] == 0 and r["failed"] == 0 and st["error_bits"] == 0
    admit, done, k = serving_schedule(arrive, blocks, steps, 1024, cap)
    assert np.array_equal(r["admit"], admit)
    assert np.array_equal(r["done"], done)
    assert (done >= 0).sum() > 50 and (admit < 0).sum() > 0          # completions and a binding cap
    assert r["mallocs"] == int(k.sum()) == sum(st["mallocs"])
    fin = np.flatnonzero(done >= 0)
    assert r["frees"] == int(blocks[fin].sum()) == sum(st["frees"])
    assert np.all(r["mism"][fin] == 0)
    for s in fin[:60]:
        x, sm = session_checksum(run.seed, int(s), int(blocks[s]), block)
        assert (int(r["xor"][s]), int(r["sum"][s])) == (x, sm), s
    # the same sessions alone: one at a time, from step 0
    pick = fin[[0, len(fin) // 2, -1]]
    for s in pick:
        solo = ServeRun(np.zeros(1, np.uint32), blocks[s:s + 1], n_slots=4, max_blocks=256,
                        steps=int(blocks[s]) + 1, seed=(run.seed + int(s)) & 0xFFFFFFFF, block_bytes=block)
        with P.Heap(heap_bytes, block, variant) as heap2:
            solo.run(heap2, cap)
            r2 = solo.results()
        assert (int(r2["xor"][0]), int(r2["sum"][0])) == (int(r["xor"][s]), int(r["sum"][s]))


@pytest.mark.parametrize("variant", ["page_array", "chunk_array"])
def test_serving_per_launch_form_equals_loop(P, variant):
    """The per-launch form (four launches per step) gives the loop's results:
    the same admission schedule (the host model's), the same per-session
    checksums and mismatch counts, the same allocator counts."""
    from paper_2504_18211_gb300.serving import ServeRun
    torch_cuda()
    steps, block = 200, 16384
    arrive, blocks = W.serving_workload(steps=steps, rate=2000.0, dt=0.01, median_bytes=256 << 10, sigma=1.0,
                                        block_bytes=block, max_blocks=256, seed=W.SEED_BASE + 43)
    heap_bytes = 128 << 20
    cap = int(0.95 * heap_bytes // block)
    got = {}
    for form in ("persistent", "per_launch"):
        run = ServeRun(arrive, blocks, n_slots=512, max_blocks=256, steps=steps, seed=0x5E57, block_bytes=block)
        with P.Heap(heap_bytes, block, variant) as heap:
            run.run(heap, cap, form=form)
            r = run.results()
            st = heap.stats()
        assert r["error"] == 0 and r["failed"] == 0 and st["error_bits"] == 0, form
        assert sum(st["live"]) == r["mallocs"] - r["frees"], form
        assert np.all(np.diff(run.step_ns.cpu().numpy().reshape(-1, 3)[:, 2]) >= 0), form   # stamps in order
        got[form] = r
    admit, done, k = serving_schedule(arrive, blocks, steps, 512, cap)
    a, b = got["persistent"], got["per_launch"]
    assert (done >= 0).sum() > 30 and (admit < 0).sum() > 0
    for r in (a, b):
        assert np.array_equal(r["admit"], admit) and np.array_equal(r["done"], done)
        assert r["mallocs"] == int(k.sum())
    for key in ("xor", "sum", "mism"):
        assert np.array_equal(a[key], b[key]), key
    assert (a["mallocs"], a["frees"]) == (b["mallocs"], b["frees"])
    fin = np.flatnonzero(done >= 0)
    assert np.all(b["mism"][fin] == 0)
    for s in fin[:: max(1, fin.size // 20)]:
        assert (int(b["xor"][s]), int(b["sum"][s])) == session_checksum(0x5E57, int(s), int(blocks[s]), block), s
