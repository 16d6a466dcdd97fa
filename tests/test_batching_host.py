"""The batching autotuner's host logic, with a fake heap and a fake run (no GPU):
which rows it marks infeasible (warps per SM beyond the kernel's register
limit; any request above 1 MiB), which rows serve requests through runs of
chunks (largest request above the chunk), and that the best row is the
fastest verified one."""
import types

import pytest

from paper_2504_18211_gb300 import batching as BT


class FakeHeap:
    opened = []

    def __init__(self, bytes_, chunk, variant):
        self.chunk, self.variant, self.closed = chunk, variant, False
        FakeHeap.opened.append(self)

    def stats(self):
        return {"error_bits": 1 if (self.chunk, self.variant) == (16384, "page_vlist") else 0}

    def close(self):
        self.closed = True


class FakeRun:
    """ms = a table of (chunk, variant, blocks per SM); checks fail for one row."""

    def __init__(self, ms):
        self.ms, self.n, self.last = ms, 1000, None
        self.torch = types.SimpleNamespace(cuda=types.SimpleNamespace(synchronize=lambda: None))

    def time(self, heap, form, reps, bps):
        assert form == "persistent" and reps == 2
        self.last = (heap.chunk, heap.variant, bps)
        return self.ms[self.last]

    def checks(self):
        bad = self.last == (8192, "chunk_array", 2)
        return [{"mismatches": 1 if bad else 0}]


@pytest.fixture
def limits(monkeypatch):
    # register limit: 4 blocks of 256 (32 warps) per SM for page queues, 2 (16 warps) for chunk queues
    monkeypatch.setattr(BT.B, "persistent_blocks_per_sm", lambda heap: 4 if heap.variant.startswith("page") else 2)
    FakeHeap.opened = []


def test_feasibility_runs_and_best_row(limits):
    chunks, variants, wps = (4096, 8192, 16384), ("page_array", "page_vlist", "chunk_array"), (8, 16, 32, 48)
    ms = {}
    for c in chunks:
        for v in variants:
            for w in wps:
                ms[(c, v, w // 8)] = 10.0 + (c // 4096) + w / 100.0
    ms[(8192, "chunk_array", 2)] = 1.0          # fastest, but its checks fail: not the best
    ms[(16384, "page_vlist", 4)] = 2.0          # fast, but the heap reports an error: not the best
    ms[(4096, "page_array", 2)] = 5.0           # the fastest verified row (runs above 4 KiB)
    best, table = BT.autotune(FakeHeap, FakeRun(ms), 1 << 30, chunks=chunks, variants=variants,
                              warps_per_sm=wps, max_size=8192)
    assert (best["chunk"], best["variant"], best["warps_per_sm"]) == (4096, "page_array", 16)
    assert best["ms"] == 5.0 and best["verified"] and best["runs"]
    for row in table:
        if "status" in row:
            assert row["status"].startswith("infeasible: registers")
            limit = 32 if row["variant"].startswith("page") else 16
            assert row["warps_per_sm"] > limit
        else:
            limit = 32 if row["variant"].startswith("page") else 16
            assert row["warps_per_sm"] <= limit
            assert row["runs"] == (row["chunk"] < 8192)
    bad = [r for r in table if r.get("verified") is False]
    assert {(r["chunk"], r["variant"], r["warps_per_sm"]) for r in bad} >= {(8192, "chunk_array", 16),
                                                                           (16384, "page_vlist", 32)}
    assert all(h.closed for h in FakeHeap.opened) and len(FakeHeap.opened) == len(chunks) * len(variants)


def test_requests_above_largest_class_are_infeasible(limits):
    best, table = BT.autotune(FakeHeap, FakeRun({}), 1 << 30, chunks=(8192,), variants=("page_array",),
                              warps_per_sm=(8,), max_size=(1 << 20) + 1)
    assert best is None and table == [{"chunk": 8192, "variant": "page_array",
                                       "status": "infeasible: requests above 1 MiB"}]
    assert FakeHeap.opened == []
