"""Host-side logic of bench.py that the GPU numbers rest on (no GPU needed):
the class-group counts of the L2-atomic bound, the gate that keeps a
recorded DRAM-traffic figure to the kernel sources it was captured from,
and the workload description of the JSON line."""
import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_classes_per_group_counts_distinct_power_of_two_classes():
    # class = ceil(log2 n) - 4 with a 16-byte floor
    one = np.full(1024, 16, np.uint32)
    g, cls = bench.classes_per_group(one, 32)
    assert g == 1.0 and set(cls.tolist()) == {0}
    # 1..16 bytes share class 0; 17 is class 1; 4096 is class 8; 4097 is class 9
    s = np.array([1, 16, 17, 32, 33, 4096, 4097, 8192] * 4, np.uint32)
    g, cls = bench.classes_per_group(s, 32)
    assert cls[:8].tolist() == [0, 0, 1, 1, 2, 8, 9, 9]
    assert g == 5.0
    # every warp of 32 holds the 10 classes 16 B .. 8 KiB three or more times
    ten = np.tile(np.array([16 << k for k in range(10)], np.uint32), 32 * 10 // 10)
    assert bench.classes_per_group(ten, 32)[0] == 10.0
    assert bench.classes_per_group(ten, 256)[0] == 10.0
    # a ragged tail shorter than one group is left out
    assert bench.classes_per_group(np.full(40, 64, np.uint32), 32)[0] == 1.0


def test_block_groups_never_exceed_warp_groups_per_request():
    from paper_2504_18211_gb300 import workloads as W
    s = W.sweep_sizes(1 << 14, seed=W.SEED_BASE + 1)
    gw, _ = bench.classes_per_group(s, 32)
    gb, _ = bench.classes_per_group(s, 256)
    # groups per request: a block of 256 needs at most the groups of its 8 warps
    assert gb / 256 <= gw / 32
    assert 1 <= gw <= 10 and 1 <= gb <= 10


def _args(**kw):
    a = dict(form="fused", variant="page_array")
    a.update(kw)
    return argparse.Namespace(**a)


def test_recorded_traffic_only_for_the_captured_kernel_and_workload():
    rec = bench.FUSED_TRAFFIC["bytes_per_launch"]
    same = bench.kernel_sources_digest() == bench.FUSED_TRAFFIC["sources_sha256"]
    got = bench.recorded_traffic(_args(), True, bench.THREADS, bench.HEAP_BYTES)
    assert got == (rec if same else None)
    # any other workload or form reports no recorded traffic
    assert bench.recorded_traffic(_args(form="per_launch"), True, bench.THREADS, bench.HEAP_BYTES) is None
    assert bench.recorded_traffic(_args(variant="chunk_array"), True, bench.THREADS, bench.HEAP_BYTES) is None
    assert bench.recorded_traffic(_args(), False, bench.THREADS, bench.HEAP_BYTES) is None
    assert bench.recorded_traffic(_args(), True, bench.THREADS // 2, bench.HEAP_BYTES) is None
    assert bench.recorded_traffic(_args(), True, bench.THREADS, bench.HEAP_BYTES // 2) is None


def test_traffic_gate_follows_the_kernel_sources(monkeypatch):
    monkeypatch.setitem(bench.FUSED_TRAFFIC, "sources_sha256", "0" * 64)
    assert bench.recorded_traffic(_args(), True, bench.THREADS, bench.HEAP_BYTES) is None
    monkeypatch.setitem(bench.FUSED_TRAFFIC, "sources_sha256", bench.kernel_sources_digest())
    assert bench.recorded_traffic(_args(), True, bench.THREADS, bench.HEAP_BYTES) == \
        bench.FUSED_TRAFFIC["bytes_per_launch"]


def test_recorded_traffic_is_below_the_algorithmic_bytes():
    # a write-streaming kernel leaves part of its last writes in L2: the DRAM
    # figure sits a little below payload + metadata, never far above it
    from paper_2504_18211_gb300 import workloads as W
    sizes = W.sweep_sizes(bench.THREADS, seed=bench.replica_seed(0))
    alg = int(sizes.astype(np.int64).sum()) + 37 * bench.THREADS
    rec = bench.FUSED_TRAFFIC["bytes_per_launch"]
    assert 0.85 * alg < rec <= 1.02 * alg


def test_workload_config_names_the_workload():
    c = bench.workload_config(bench.THREADS, "page_array")
    assert c["threads"] == bench.THREADS and c["variant"] == "page_array"
    assert "size sweep" in c["workload"] and "L2" in c["l2"]
    assert not {"model", "global_batch", "seq_len"} & set(c)


def test_l2_note_follows_the_payload():
    """The config's L2 statement is computed from the workload: the
    headline's ~1.7 GB of payload is larger than L2, a small batch is not."""
    from paper_2504_18211_gb300 import workloads as W
    big = bench.l2_note(bench.THREADS)
    assert big.startswith("inputs larger than L2") and "1.72 GB" in big
    mean = float(W.sweep_sizes(1 << 16, seed=5).astype(np.float64).mean())
    assert abs(mean - 1636.8) < 60                       # the note's mean block, k uniform in [4, 13]
    assert "within L2" in bench.l2_note(1 << 16)
