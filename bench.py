#!/usr/bin/env python3
"""Benchmark of the GB300 device-side allocator on the size-sweep workload.

Workload (one step): 2^20 requests on an 8 GiB heap cut into 8 KiB chunks;
request i asks for 2^k bytes, k uniform in [4, 13] (seeded); every request
allocates, writes its pattern, reads it back, checks it and frees -- one
driver round of the paper's method (arXiv 2504.18211, Sec. 3) in one fused
kernel.  value = malloc+free operations per second over the timed steps
(2 x 2^20 ops per step), whole round included.

Printed on one JSON line, besides the contract keys: the per-launch form
(malloc / write / check / free kernels, whose malloc+free share is the
paper's own timing), the other three queue variants, the malloc latency
histogram (p50/p99), the measured L2 atomic rates and the allocator's
fraction of them, the end-to-end figure with host buffers, and the CPU
oracle on a bounded sample.

--impl reference times the sequential CPU oracle (the stand-in for the
paper's comparison system, which cannot run here) on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "malloc+free Mops/s at 2^20 threads vs L2-atomic roofline; p99 alloc latency"
UNIT = "Mops/s"
HEAP_BYTES = 8 << 30
CHUNK = 8192
THREADS = 1 << 20
SEED = 0x5EED
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--variant", default="page_array")
    ap.add_argument("--no-staging", action="store_true",
                    help="headline without shared-memory staging of freed pages")
    ap.add_argument("--threads", type=int, default=THREADS)
    ap.add_argument("--heap-gib", type=int, default=HEAP_BYTES >> 30,
                    help="heap size (smaller only for profiler captures)")
    ap.add_argument("--no-extras", action="store_true", help="headline only (used under a profiler)")
    ap.add_argument("--form", choices=("fused", "per_launch"), default="fused",
                    help="fused: one kernel per round; per_launch: malloc / write / check / free kernels")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--workload", choices=("sweep", "batching", "serving", "graph", "axes"), default="sweep",
                    help="sweep: the headline size sweep; batching: 256 uneven batches, every form + autotuner; "
                         "serving: the device request loop; graph: adjacency-list growth; axes: the paper's "
                         "allocation-size and thread-count axes on all six queue forms")
    ap.add_argument("--batches", type=int, default=256)
    ap.add_argument("--axes-point", default="",
                    help="axes workload: one point THREADS,SIZE only (with --variant; used under a profiler)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one fused
# launch of the default workload, from one ncu capture of the kernel built
# from the sources whose digest is recorded; null once they change.
FUSED_KERNEL_SOURCES = ("include/ouro_device.cuh", "paper_2504_18211_gb300/csrc/ouro_payload.cuh",
                        "paper_2504_18211_gb300/csrc/ouro_kernels.cu", "paper_2504_18211_gb300/csrc/ouro_internal.cuh")
FUSED_TRAFFIC = {"sources_sha256": "ca166ebb2bafe0ca9cfc517fc553e8fb6b8e82b85de8608ef8652ec590515386",
                 "bytes_per_launch": 1643345152}


def kernel_sources_digest() -> str:
    import hashlib
    d = hashlib.sha256()
    for rel in FUSED_KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            d.update(f.read())
    return d.hexdigest()


def recorded_traffic(args, staging, n, heap_bytes):
    default = (args.form == "fused" and args.variant == "page_array" and staging and n == THREADS
               and heap_bytes == HEAP_BYTES)
    if not default or FUSED_TRAFFIC["bytes_per_launch"] is None:
        return None
    return FUSED_TRAFFIC["bytes_per_launch"] if kernel_sources_digest() == FUSED_TRAFFIC["sources_sha256"] else None


def replica_seed(rank: int) -> int:
    """Seed of the size batch replica `rank` draws: every replica runs the
    same workload shape on its own heap with its own requests."""
    from paper_2504_18211_gb300 import workloads as W
    return W.SEED_BASE + 1 + rank


def max_over_ranks(dist, ms: float, device) -> float:
    """The slowest replica's timed region (ms); `dist` None for one process."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(ws: int, steps: int, ops_per_step: int, total_ms: float) -> float:
    """Operations of all replicas over the slowest replica's time, in Mops/s
    (weak scaling: each replica does ops_per_step per step)."""
    return ws * steps * ops_per_step / (total_ms / 1e3) / 1e6


def workload_config(threads, variant, form="fused", heap_bytes=HEAP_BYTES, staging=True):
    return {"workload": f"size sweep: {threads} requests of 2^k B (k uniform in [4,13], seeded), "
                        f"allocate / write pattern / read back + check / free, one round per step",
            "heap_bytes": heap_bytes, "chunk_bytes": CHUNK, "threads": threads, "variant": variant,
            "form": form, "staging": staging,
            "l2": l2_note(threads)}


def l2_note(threads: int) -> str:
    """How the round's payload compares with L2 (mean sweep block: the mean
    of 2^k B over k in [4, 13], 1636.8 B)."""
    gb = threads * 1636.8 / 1e9
    if gb * 1e9 > 129e6:
        return f"inputs larger than L2: ~{gb:.2f} GB of payload per round (L2 129 MB)"
    return f"payload ~{gb * 1e3:.0f} MB per round, within L2 (129 MB): rounds are not HBM-bound"


# ----------------------------------------------------------------- helpers
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


def classes_per_group(sizes, width):
    """Mean number of distinct classes among `width` consecutive requests
    (32: a warp; 256: a block of the batch kernels), and every class."""
    import numpy as np
    s = sizes.astype(np.int64)
    c = np.where(s <= 16, 0, np.ceil(np.log2(s)).astype(np.int64) - 4)
    n = (c.size // width) * width
    w = c[:n].reshape(-1, width)
    return float(np.mean([len(set(r)) for r in w[: min(len(w), 4096)]])), c


# ---------------------------------------------------------------- CPU arm
def host_cpu() -> dict:
    """The host's logical CPU count and CPU model (x86: "model name"; Arm:
    lscpu's model name, else the implementer / part codes of /proc/cpuinfo)."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            info = {}
            for line in open("/proc/cpuinfo"):
                if ":" in line:
                    k, v = (x.strip() for x in line.split(":", 1))
                    info.setdefault(k, v)
            model = info.get("model name") or \
                f"CPU implementer {info.get('CPU implementer', '?')} part {info.get('CPU part', '?')}"
        except OSError:
            model = "unknown"
    return {"host_cpus": os.cpu_count(), "cpu_model": model}


class PinnedCore:
    """Pin this thread to one core (the lowest it may run on) while timing
    the sequential oracle; the previous affinity comes back on exit."""

    def __enter__(self):
        self.old = os.sched_getaffinity(0)
        self.core = min(self.old)
        os.sched_setaffinity(0, {self.core})
        return self

    def __exit__(self, *exc):
        os.sched_setaffinity(0, self.old)


class OracleSweep:
    """The sequential oracle on the headline workload itself: the same 2^20
    request sizes (same seed) and payload seed as the GPU arm, an 8 GiB heap
    of 8 KiB chunks, page-array queues, every payload byte written to and
    read back from host memory (committed lazily: about 1.7 GB is touched)."""

    def __init__(self, threads=THREADS, variant="page_array", seed=SEED):
        import ctypes as C

        import numpy as np

        import oracle
        from paper_2504_18211_gb300 import workloads as W
        self.C, self.n, self.seed = C, threads, seed
        self.sizes = W.sweep_sizes(threads, seed=replica_seed(0))
        self.heap = oracle.OracleHeap(HEAP_BYTES, CHUNK, variant)
        self.mem = np.zeros(HEAP_BYTES, np.uint8)
        self.want = oracle.expected_checksums(self.sizes, seed, 1)
        self.r = oracle.RoundResult()

    def round(self) -> None:
        C, ptr = self.C, (lambda a: a.ctypes.data_as(self.C.c_void_p))
        self.heap.lib.orc_round(self.heap.h, ptr(self.sizes), self.n, self.seed, 1, ptr(self.mem), None,
                                C.byref(self.r))
        res = self.r.as_dict()
        assert res == dict(self.want, nulls=0, mismatches=0), res

    def describe(self) -> str:
        return (f"{self.n} requests of 2^k B (k uniform in [4,13], the GPU arm's sizes and seed), 8 GiB heap, "
                f"8 KiB chunks, page-array; payload written to and read back from host memory")


def cpu_oracle_sample(seconds: float, seed: int = SEED):
    """The sequential oracle on the headline workload (OracleSweep): one
    untimed round, then whole rounds for about `seconds`, one thread pinned
    to one core."""
    sweep = OracleSweep(seed=seed)
    with PinnedCore() as pin:
        sweep.round()
        rounds, t0 = 0, time.perf_counter()
        while True:
            sweep.round()
            rounds += 1
            el = time.perf_counter() - t0
            if el >= seconds:
                break
    return {"value": round(rounds * 2 * sweep.n / el / 1e6, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{rounds} rounds of the headline workload after 1 untimed ({sweep.describe()}), "
                      f"one thread pinned to core {pin.core}, {el:.1f} s", **host_cpu()}


def run_reference(args):
    """The reference arm: the sequential oracle on the headline workload,
    `warmup` untimed rounds then `steps` timed rounds, one thread pinned to
    one core; rank 0 only."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    sweep = OracleSweep(threads=args.threads, variant=args.variant)
    with PinnedCore() as pin:
        for _ in range(args.warmup):
            sweep.round()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sweep.round()
        el = time.perf_counter() - t0
    value = args.steps * 2 * sweep.n / el / 1e6
    sample = f"each step one round of the headline workload ({sweep.describe()}), one thread pinned to core {pin.core}"
    cfg = workload_config(args.threads, args.variant, form="sequential oracle", staging=False)
    cfg["l2"] = "host memory (CPU)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el * 1e3 / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": cfg,
        "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         **host_cpu()},
        "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# ---------------------------------------------------------------- GPU arm
def _ensure_lib():
    import paper_2504_18211_gb300 as P
    from paper_2504_18211_gb300 import build as B
    B.build()
    P.load()
    return P


def measure_batching(variant="page_array", n_batches=256, reps=2, sample_batches=16, tune=False):
    """Batching: n_batches request batches, threads per batch log-uniform in
    [2^10, 2^20], sizes uniform in [4, 8192] B, 16 GiB heap of 8 KiB chunks;
    every form (four launches per batch, one fused launch per batch, a CUDA
    graph of those, one persistent kernel; the persistent kernel also with
    staging).  Verified: no null and no mismatch in any batch of any form,
    every form's per-batch checksums equal, and the oracle's checksums on the
    `sample_batches` smallest batches (the oracle folds every word; all 256
    batches would take it minutes)."""
    import numpy as np

    import oracle
    from paper_2504_18211_gb300 import batching as BT
    from paper_2504_18211_gb300 import workloads as W
    P = _ensure_lib()
    sizes, offs = W.batching_workload(n_batches=n_batches)
    run = BT.BatchRun(sizes, offs)
    heap_bytes = 16 << 30
    res = {"workload": f"batching: {n_batches} batches, {sizes.size} requests (threads per batch log-uniform in "
                       f"[2^10,2^20]), sizes U[4,8192] B, 16 GiB heap, 8 KiB chunks, {variant}",
           "forms": {}}
    checks, errors = {}, 0
    for staged in (False, True):
        with P.Heap(heap_bytes, 8192, variant, staging=staged) as heap:
            for form in (BT.FORMS if not staged else ("persistent",)):
                ms = run.time(heap, form, reps=reps)
                key = form + ("_staged" if staged else "")
                res["forms"][key] = {"ms_per_pass": round(ms, 3), "mops": round(2 * run.n / (ms / 1e3) / 1e6, 1)}
                checks[key] = run.checks()
            errors |= heap.stats()["error_bits"]
            run.close()
    o = offs.astype(np.int64)
    counts = np.diff(o)
    pick = np.argsort(counts, kind="stable")[:sample_batches]
    want = {int(b): oracle.expected_checksums(sizes[o[b]:o[b + 1]], run.seed + int(b), 1) for b in pick}
    first = next(iter(checks.values()))
    ok = errors == 0 and all(c == first for c in checks.values())
    ok = ok and all(c["nulls"] == 0 and c["mismatches"] == 0 for c in first)
    ok = ok and all(first[b] == dict(w, nulls=0, mismatches=0) for b, w in want.items())
    res["verified"] = bool(ok)
    res["verified_by"] = (f"every batch of every form: no null, no mismatch, equal checksums across forms; oracle "
                          f"checksums on the {len(pick)} smallest batches ({int(counts[pick].sum())} requests)")
    base = res["forms"]["per_launch4"]["ms_per_pass"]
    res["speedup_vs_per_launch4"] = {k: round(base / v["ms_per_pass"], 2) for k, v in res["forms"].items()}
    if tune:
        sub_sizes, sub_offs = sizes[: int(offs[16])], offs[:17]
        tune_run = BT.BatchRun(sub_sizes, sub_offs)
        best, table = BT.autotune(P.Heap, tune_run, heap_bytes)
        res["autotune"] = {"best": best, "table": table, "trial": "first 16 batches, persistent form"}
        if best:
            with P.Heap(heap_bytes, best["chunk"], best["variant"]) as heap:
                ms = run.time(heap, "persistent", reps=reps, blocks_per_sm=best["warps_per_sm"] // 8)
                res["tuned_persistent"] = {"ms_per_pass": round(ms, 3), "mops": round(2 * run.n / (ms / 1e3) / 1e6, 1)}
    del run
    return res


def measure_serving(variants=(("page_array", "persistent"), ("page_array", "per_launch")), steps=2000,
                    detail=False):
    """Serving: 64 GiB heap of 16 KiB blocks; Poisson session arrivals
    (2000/s, 10 ms steps); lognormal session sizes (median 4 MiB, sigma 1);
    one block per session per step; admission up to 95 % of the blocks;
    `steps` steps in one cooperative kernel (persistent) or four plain
    launches per step (per_launch).  Verified against the oracle's admission
    schedule and per-session checksums (64 sampled completed sessions)."""
    import numpy as np
    import torch

    import oracle
    from oracle.patterns import serving_schedule
    from paper_2504_18211_gb300 import workloads as W
    from paper_2504_18211_gb300.serving import ServeRun
    P = _ensure_lib()
    block, heap_bytes = 16384, 64 << 30
    arrive, blocks = W.serving_workload(steps=steps)
    cap = int(0.95 * heap_bytes // block)
    admit, done, _ = serving_schedule(arrive, blocks, steps, 16384, cap)
    fin = np.flatnonzero(done >= 0)
    sample = fin[:: max(1, fin.size // 64)]
    res = {"workload": f"serving: {arrive.size} sessions arriving over {steps} steps of 10 ms (2000/s), lognormal "
                       f"sizes median 4 MiB sigma 1 (<= 64 MiB), 16 KiB blocks, 64 GiB heap, admission cap 95 %"}
    for variant, form in variants:
        run = ServeRun(arrive, blocks, n_slots=16384, max_blocks=4096, steps=steps)
        with P.Heap(heap_bytes, block, variant) as heap:
            ms = run.run(heap, cap, form=form)
            r = run.results()
            st = heap.stats()
        ok = all((int(r["xor"][s]), int(r["sum"][s])) == (lambda e: (e["xor64"], e["sum64"]))(
            oracle.expected_checksums(np.full(int(blocks[s]), block, np.uint32), (run.seed + int(s)) & 0xFFFFFFFF, 1))
            for s in sample)
        lat = r["step_us"]
        ops = r["mallocs"] + r["frees"]
        row = {"form": form, "ms": round(ms, 2), "mops": round(ops / (ms / 1e3) / 1e6, 1),
               "step_us_p50": round(float(np.percentile(lat, 50)), 1),
               "step_us_p99": round(float(np.percentile(lat, 99)), 1),
               "mallocs": r["mallocs"], "frees": r["frees"], "failed": r["failed"],
               "admitted": int((r["admit"] >= 0).sum()), "completed": int((r["done"] >= 0).sum()),
               "verified": bool(ok and np.array_equal(r["admit"], admit) and np.array_equal(r["done"], done)
                                and r["error"] == 0 and st["error_bits"] == 0 and np.all(r["mism"][fin] == 0))}
        if detail:
            row["phases"] = {k: {"p50": round(float(np.percentile(v, 50)), 1),
                                 "p99": round(float(np.percentile(v, 99)), 1),
                                 "max": round(float(v.max()), 1), "total_ms": round(float(v.sum()) / 1e3, 1)}
                             for k, v in r["phases"].items()}
            row["slowest_steps"] = [int(i) + 1 for i in np.argsort(lat)[-5:][::-1]]
            row["peak_committed_blocks_cap"] = cap
        res[variant if form == "persistent" else f"{variant}_per_launch"] = row
        del run
        torch.cuda.empty_cache()
    return res


def measure_graph(variants=("page_array", "chunk_array")):
    """Graph growth: 2^20 vertices, 2^24 directed edges with power-law
    endpoints (degree exponent 2.1), lists from 4 entries growing by malloc
    2x / copy / free old, 16 GiB heap of 8 KiB chunks; one insertion kernel
    timed.  Verified: degrees equal the edge list's, per-class malloc / free
    counts equal the oracle's closed form of the growth rule."""
    import numpy as np
    import torch

    from oracle.patterns import graph_class_counts
    from paper_2504_18211_gb300 import workloads as W
    from paper_2504_18211_gb300.graph import GraphRun
    P = _ensure_lib()
    nv, ne, chunk, heap_bytes = 1 << 20, 1 << 24, 8192, 16 << 30
    src, dst = W.graph_workload(nv, ne)
    want_deg = np.bincount(src, minlength=nv)
    m, f, _ = graph_class_counts(want_deg, chunk, 10)
    res = {"workload": "graph growth: 2^20 vertices, 2^24 edges, power-law endpoints (alpha 2.1), "
                       "lists 4 -> doubling -> one chunk -> chained 8 KiB segments, 16 GiB heap"}
    for variant in variants:
        g = GraphRun(src, dst, nv)
        with P.Heap(heap_bytes, chunk, variant) as heap:
            g.init(heap)
            torch.cuda.synchronize()
            st0 = heap.stats()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            g.insert(heap)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            st = heap.stats()
            deg = g.degrees()
            ops = sum(st["mallocs"]) + sum(st["frees"]) - sum(st0["mallocs"])
            ok = (np.array_equal(deg, want_deg) and st["mallocs"] == m.tolist()
                  and st["frees"] == f.tolist() and st["error_bits"] == 0 and g.ctl_dict()["failed"] == 0)
            res[variant] = {"ms": round(ms, 2), "appends_per_s": round(ne / (ms / 1e3), 1),
                            "alloc_ops": ops, "alloc_mops": round(ops / (ms / 1e3) / 1e6, 2),
                            "max_degree": int(deg.max()), "verified": bool(ok)}
            g.free(heap)
        del g
        torch.cuda.empty_cache()
    return res


def run_batching(args):
    print(json.dumps(measure_batching(args.variant, args.batches, tune=True)))


def run_serving(args):
    print(json.dumps(measure_serving(((args.variant, "persistent"), (args.variant, "per_launch"),
                                      ("chunk_array", "persistent")), detail=True)))


def run_graph(args):
    print(json.dumps(measure_graph((args.variant, "chunk_array"))))


def run_axes(args):
    """The paper's experiment axes (Sec. 4.1-4.3): average time of the
    allocation kernel and of the free kernel (a) over allocation sizes
    16 B .. 8 KiB at 1024 threads and (b) over 2^5 .. 2^20 threads at 1000 B,
    each point ten iterations of allocate / write / check / free after one
    untimed iteration (the paper's subsequent-iteration average, Sec. 3), on
    all six queue forms; 4 GiB heap of 8 KiB chunks, reset before every
    point (the largest point holds 1 GiB of blocks).  A device error stops
    the run: an exhausted virtualized queue answers only after its bounded
    waits run out."""
    import numpy as np
    import torch

    import paper_2504_18211_gb300 as P
    from paper_2504_18211_gb300 import build as B
    from paper_2504_18211_gb300 import workloads as W
    B.build()
    P.load()
    stream = torch.cuda.current_stream()
    variants = ("page_array", "chunk_array", "page_varray", "page_vlist", "chunk_varray", "chunk_vlist")
    axes = {"size": [(1024, 16 << k) for k in range(10)],
            "threads": [(1 << k, 1000) for k in range(5, 21)]}
    if args.axes_point:
        t, z = (int(x) for x in args.axes_point.split(","))
        variants, axes = (args.variant,), {"point": [(t, z)]}
    res = {"workload": "paper axes: allocation size x 1024 threads and thread count x 1000 B; 10 timed "
                       "iterations after 1 untimed (median); 4 GiB heap, 8 KiB chunks, reset per point",
           "unit": "us per kernel launch",
           "variants": {}}
    ok_all = True
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for v in variants:
        out_v = {}
        with P.Heap(4 << 30, 8192, v) as heap:
            for axis, points in axes.items():
                rows = []
                for threads, size in points:
                    if not ok_all:
                        break
                    heap.reset()
                    sizes = torch.from_numpy(W.single_size(threads, size).view(np.int32)).cuda()
                    ptrs = torch.empty(threads, dtype=torch.int64, device="cuda")
                    chk = torch.zeros(5, dtype=torch.int64, device="cuda")
                    t_m, t_f = [], []
                    for it in range(11):
                        # keep the GPU busy while the host queues the launches,
                        # so the events time the kernels and not host gaps
                        torch.cuda._sleep(2_000_000)
                        ev[0].record(stream)
                        heap.malloc(sizes, ptrs)
                        ev[1].record(stream)
                        P.pattern_write(ptrs, sizes, it, 1)
                        P.pattern_check(ptrs, sizes, it, 1, chk)
                        ev[2].record(stream)
                        heap.free(ptrs)
                        ev[3].record(stream)
                        torch.cuda.synchronize()
                        c = P.check_to_dict(chk)
                        ok_all &= c["nulls"] == 0 and c["mismatches"] == 0
                        if it:
                            t_m.append(ev[0].elapsed_time(ev[1]) * 1e3)
                            t_f.append(ev[2].elapsed_time(ev[3]) * 1e3)
                    ok_all &= heap.stats()["error_bits"] == 0
                    rows.append({"threads": threads, "size": size, "alloc_us": round(statistics.median(t_m), 2),
                                 "free_us": round(statistics.median(t_f), 2)})
                out_v[axis] = rows
        res["variants"][v] = out_v
    res["verified"] = bool(ok_all)
    print(json.dumps(res))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "axes":
        return run_axes(args)
    if args.workload == "batching":
        return run_batching(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "graph":
        return run_graph(args)
    import numpy as np
    import torch

    import paper_2504_18211_gb300 as P
    from paper_2504_18211_gb300 import build as B
    from paper_2504_18211_gb300 import workloads as W

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        B.build()
    if dist:
        dist.barrier()
    P.load()

    n = args.threads
    sizes_np = W.sweep_sizes(n, seed=replica_seed(rank))          # each replica its own batch
    sizes = torch.from_numpy(sizes_np.view(np.int32)).cuda()
    stream = torch.cuda.current_stream()
    ops_per_step = 2 * n

    heap_bytes = args.heap_gib << 30
    staging = not args.no_staging
    heap = P.Heap(heap_bytes, CHUNK, args.variant, staging=staging)
    out = torch.zeros(5, dtype=torch.int64, device="cuda")
    if args.form == "fused":
        def step():
            heap.round_fused(sizes, SEED, 1, out=out)
    else:
        ptrs = torch.empty(n, dtype=torch.int64, device="cuda")

        def step():
            heap.malloc(sizes, ptrs)
            P.pattern_write(ptrs, sizes, SEED, 1)
            P.pattern_check(ptrs, sizes, SEED, 1, out)
            heap.free(ptrs)
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local).start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = P.ouro_kernel_launches()
    torch.cuda._sleep(1_000_000)        # the GPU is busy while the host queues the first step
    t_start.record(stream)
    for k in range(args.steps):
        ev[2 * k].record(stream)
        step()
        ev[2 * k + 1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    launches = P.ouro_kernel_launches() - launches0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    step_ms = [ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(args.steps)]
    total_ms = max_over_ranks(dist, total_ms, "cuda")
    value = whole_job_value(ws, args.steps, ops_per_step, total_ms)
    chk = P.check_to_dict(out)
    st = heap.stats()

    import oracle
    want = oracle.expected_checksums(sizes_np, SEED, 1)
    verified = chk == dict(want, nulls=0, mismatches=0) and st["error_bits"] == 0

    if rank != 0:
        heap.close()
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    peaks, peak_src = measured_peaks()
    payload = int(sizes_np.astype(np.int64).sum())
    meta_per_req = 37            # sizes 4 + malloc slot read/write 16 + chunk table 1 + free slot CAS 16
    # the fused round writes every payload byte to HBM once; its read-back of
    # each block follows the block's write within the same warp and is served
    # by L2 (ncu: DRAM reads ~1-2 % of DRAM writes), so HBM bytes per request
    # are payload + metadata
    if args.form == "fused":
        alg_bytes = payload + meta_per_req * n
        kernel = f"k_round_fused<{args.variant}{', staged' if staging else ''}>"
        model = "per request: payload written once + 37 B allocator metadata (read-back from L2)"
    else:
        # four kernels: the check reads the payload back from HBM; malloc
        # 28 B, free 25 B, write and check 12 B each of pointer and size
        alg_bytes = 2 * payload + 77 * n
        kernel = "per-launch round (malloc, write, check, free)"
        model = "per request: payload written and read back + 77 B of allocator and kernel metadata"
    mean_kernel_ms = statistics.mean(step_ms)
    achieved = alg_bytes / (mean_kernel_ms / 1e3) / 1e9
    traffic = recorded_traffic(args, staging, n, heap_bytes)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks.get("hbm_gbs", FALLBACK_HBM_GBS),
                "unit": "GB/s", "frac": round(achieved / peaks.get("hbm_gbs", FALLBACK_HBM_GBS), 4),
                "traffic": traffic, "kernel": kernel, "algorithmic_bytes_per_launch": alg_bytes,
                "bytes_model": model, "peak_source": f"{peak_src} hbm_gbs (STREAM-style copy, burst)"}

    line = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": workload_config(n, args.variant, args.form, heap_bytes, staging), "verified": verified,
            "gpu_launches": int(launches), "clocks": clk, "roofline": roofline}

    if not args.no_extras:
        line.update(extras(P, torch, np, heap, sizes, sizes_np, args, n, st, clk))
        heap.close()
        torch.cuda.empty_cache()
        line.update(added_patterns())
        line["cpu_baseline"] = cpu_oracle_sample(args.cpu_seconds)
    heap.close()
    print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def added_patterns() -> dict:
    """The three added usage patterns at their full sizes, each verified:
    batching (every form; fused / graph / persistent against four launches
    per batch), serving (one cooperative loop against four launches per
    step; p50 / p99 step latency) and graph growth."""
    out = {}
    bt = measure_batching("page_array")
    out["batching"] = {"workload": bt["workload"], "mops": {k: v["mops"] for k, v in bt["forms"].items()},
                       "ms_per_pass": {k: v["ms_per_pass"] for k, v in bt["forms"].items()},
                       "speedup_vs_per_launch4": bt["speedup_vs_per_launch4"], "verified": bt["verified"],
                       "verified_by": bt["verified_by"]}
    sv = measure_serving()
    loop, pl = sv["page_array"], sv["page_array_per_launch"]
    out["serving"] = {"workload": sv["workload"], "persistent": loop, "per_launch": pl,
                      "speedup_vs_per_launch": round(pl["ms"] / loop["ms"], 3),
                      "verified": loop["verified"] and pl["verified"]}
    out["graph"] = measure_graph(("page_array",))
    return out


def timed(torch, stream, fn, reps=1, prefill=True):
    """Device time of `reps` calls of fn, per call (ms), from CUDA events on
    the launching stream.  prefill: a sleep kernel keeps the GPU busy while
    the host queues the start event and the launches, so the events bracket
    the kernels and not the host's launch latency (off for end-to-end
    timings, where the host's part counts)."""
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if prefill:
        torch.cuda._sleep(1_000_000)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def extras(P, torch, np, heap, sizes, sizes_np, args, n, st, clk):
    from paper_2504_18211_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    ex = {}

    # ---- end to end through the C ABI with host buffers: every step copies
    # its sizes from pinned host memory and reads its check back; the copy of
    # step k+1's sizes runs on a second stream while step k's round runs
    # (two device buffers), and the read-back follows each round
    h_sizes = torch.from_numpy(sizes_np.view(np.int32)).pin_memory()
    h_out = torch.zeros((args.steps + 3, 5), dtype=torch.int64).pin_memory()
    d_buf = [torch.empty_like(sizes) for _ in range(2)]
    out = torch.zeros(5, dtype=torch.int64, device="cuda")
    copy_stream = torch.cuda.Stream()
    up_done = [torch.cuda.Event() for _ in range(2)]
    used = [torch.cuda.Event() for _ in range(2)]

    def upload(k):
        b = k % 2
        copy_stream.wait_event(used[b])               # the round that read this buffer is done
        with torch.cuda.stream(copy_stream):
            d_buf[b].copy_(h_sizes, non_blocking=True)
        up_done[b].record(copy_stream)

    def e2e_run(steps):
        upload(0)
        for k in range(steps):
            b = k % 2
            if k + 1 < steps:
                upload(k + 1)
            stream.wait_event(up_done[b])
            heap.round_fused(d_buf[b], SEED, 1, out=out)
            used[b].record(stream)
            h_out[k].copy_(out, non_blocking=True)

    e2e_run(3)
    torch.cuda.synchronize()
    t_a, t_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_a.record(stream)
    copy_stream.wait_event(t_a)                       # the first upload starts inside the timed region
    e2e_run(args.steps)
    t_b.record(stream)
    torch.cuda.synchronize()
    ms = t_a.elapsed_time(t_b) / args.steps
    import oracle
    want_e2e = dict(oracle.expected_checksums(sizes_np, SEED, 1), nulls=0, mismatches=0)
    e2e_ok = all(P.check_to_dict(h_out[k]) == want_e2e for k in range(args.steps))
    ex["e2e"] = {"value": round(2 * n / (ms / 1e3) / 1e6, 3), "unit": UNIT,
                 "h2d_bytes_per_step": int(h_sizes.numel() * 4), "d2h_bytes_per_step": 40,
                 "overlap": "step k+1's sizes copied on a second stream during step k's round",
                 "verified": e2e_ok}

    # ---- per-launch form (the paper's protocol: time allocations and frees)
    ptrs = torch.empty(n, dtype=torch.int64, device="cuda")
    chk = torch.zeros(5, dtype=torch.int64, device="cuda")

    def per_launch(variant_heap, reps):
        tm = {"malloc": [], "write": [], "check": [], "free": []}
        for _ in range(reps):
            tm["malloc"].append(timed(torch, stream, lambda: variant_heap.malloc(sizes, ptrs)))
            tm["write"].append(timed(torch, stream, lambda: P.pattern_write(ptrs, sizes, SEED, 1)))
            tm["check"].append(timed(torch, stream, lambda: P.pattern_check(ptrs, sizes, SEED, 1, chk)))
            tm["free"].append(timed(torch, stream, lambda: variant_heap.free(ptrs)))
        return {k: statistics.mean(v[1:]) for k, v in tm.items()}

    pl = per_launch(heap, 6)
    af = pl["malloc"] + pl["free"]
    round_ms = sum(pl.values())
    ex["per_launch"] = {"ms": {k: round(v, 4) for k, v in pl.items()},
                        "alloc_free_mops": round(2 * n / (af / 1e3) / 1e6, 1),
                        "round_mops": round(2 * n / (round_ms / 1e3) / 1e6, 1)}

    # ---- the other five queue forms, fused (unstaged and staged) and per launch
    import oracle
    want_chk = dict(oracle.expected_checksums(sizes_np, SEED, 1), nulls=0, mismatches=0)
    others = {}
    for v in ("page_array", "page_vlist", "chunk_array", "chunk_vlist", "page_varray", "chunk_varray"):
        if v == args.variant:
            continue
        with P.Heap(HEAP_BYTES, CHUNK, v) as h2:
            o2 = torch.zeros(5, dtype=torch.int64, device="cuda")
            for _ in range(3):
                h2.round_fused(sizes, SEED, 1, out=o2)
            fms = timed(torch, stream, lambda: h2.round_fused(sizes, SEED, 1, out=o2), 5)
            pl2 = per_launch(h2, 4)
            ok = P.check_to_dict(o2) == want_chk and h2.stats()["error_bits"] == 0
        with P.Heap(HEAP_BYTES, CHUNK, v, staging=True) as h2s:
            for _ in range(3):
                h2s.round_fused(sizes, SEED, 1, out=o2)
            sms2 = timed(torch, stream, lambda: h2s.round_fused(sizes, SEED, 1, out=o2), 5)
            ok = ok and P.check_to_dict(o2) == want_chk and h2s.stats()["error_bits"] == 0
        others[v] = {"fused_mops": round(2 * n / (fms / 1e3) / 1e6, 1),
                     "fused_staged_mops": round(2 * n / (sms2 / 1e3) / 1e6, 1),
                     "alloc_free_mops": round(2 * n / ((pl2["malloc"] + pl2["free"]) / 1e3) / 1e6, 1),
                     "per_launch_ms": {k: round(x, 4) for k, x in pl2.items()}, "verified": ok}
    ex["variants"] = others

    # ---- the deoptimised form of Sec. 2: no warp aggregation, fences for sleeps
    deopt = {}
    for v in ("page_array", "page_varray", "chunk_array"):
        with P.Heap(HEAP_BYTES, CHUNK, v, deopt=True) as h4:
            o4 = torch.zeros(5, dtype=torch.int64, device="cuda")
            for _ in range(3):
                h4.round_fused(sizes, SEED, 1, out=o4)
            fms = timed(torch, stream, lambda: h4.round_fused(sizes, SEED, 1, out=o4), 5)
            pl4 = per_launch(h4, 4)
            ok = P.check_to_dict(o4)["mismatches"] == 0 and h4.stats()["error_bits"] == 0
            deopt[v] = {"fused_mops": round(2 * n / (fms / 1e3) / 1e6, 1),
                        "alloc_free_mops": round(2 * n / ((pl4["malloc"] + pl4["free"]) / 1e3) / 1e6, 1),
                        "per_launch_ms": {k: round(x, 4) for k, x in pl4.items()}, "verified": ok}
    ex["deoptimised"] = deopt

    # ---- requests above one chunk (runs of chunks) mixed with pages
    n_r = 1 << 18
    sizes_r_np = W.sweep_sizes(n_r, seed=W.SEED_BASE + 5, kmin=4, kmax=16)
    sizes_r = torch.from_numpy(sizes_r_np.view(np.int32)).cuda()
    with P.Heap(16 << 30, CHUNK, args.variant, staging=True) as h6:
        o6 = torch.zeros(5, dtype=torch.int64, device="cuda")
        for _ in range(3):
            h6.round_fused(sizes_r, SEED, 1, out=o6)
        rms = timed(torch, stream, lambda: h6.round_fused(sizes_r, SEED, 1, out=o6), 5)
        import oracle
        ok6 = P.check_to_dict(o6) == dict(oracle.expected_checksums(sizes_r_np, SEED, 1), nulls=0, mismatches=0) \
            and h6.stats()["error_bits"] == 0
        pay = int(sizes_r_np.astype(np.int64).sum())
        ex["runs"] = {"workload": f"{n_r} requests of 2^k B, k uniform in [4,16] (runs of 2-8 chunks above 8 KiB), "
                                  f"16 GiB heap, fused round, staged", "fused_mops": round(2 * n_r / (rms / 1e3) / 1e6, 1),
                      "ms": round(rms, 4), "payload_gbs": round(pay / (rms / 1e3) / 1e9, 1),
                      "run_requests": int((sizes_r_np > CHUNK).sum()), "verified": ok6}

    # ---- CUDA's built-in device malloc on the same round (the baseline of Sec. 1)
    try:
        got = P.ouro_cuda_malloc_heap(HEAP_BYTES)
        o5 = torch.zeros(5, dtype=torch.int64, device="cuda")
        t0 = time.perf_counter()
        P.ouro_cuda_malloc_round(sizes, SEED, 1, out=o5)
        torch.cuda.synchronize()
        first_s = time.perf_counter() - t0
        reps = 3 if first_s < 2.0 else 0
        cms = timed(torch, stream, lambda: P.ouro_cuda_malloc_round(sizes, SEED, 1, out=o5), reps) if reps else first_s * 1e3
        c5 = P.check_to_dict(o5)
        ex["cuda_device_malloc"] = {"fused_mops": round(2 * n / (cms / 1e3) / 1e6, 1), "ms": round(cms, 3),
                                    "first_round_s": round(first_s, 3), "nulls": c5["nulls"],
                                    "mismatches": c5["mismatches"], "heap_bytes": got,
                                    "timed_rounds": reps}
    except P.OuroError as e:
        ex["cuda_device_malloc"] = {"unavailable": str(e)}

    # ---- the first round on a fresh heap (it carves every chunk) against warm rounds
    with P.Heap(HEAP_BYTES, CHUNK, args.variant, staging=not args.no_staging) as hc:
        oc = torch.zeros(5, dtype=torch.int64, device="cuda")
        cold = timed(torch, stream, lambda: hc.round_fused(sizes, SEED, 1, out=oc))
        okc = P.check_to_dict(oc) == want_chk
        warm = timed(torch, stream, lambda: hc.round_fused(sizes, SEED, 1, out=oc), 5)
        okc = okc and P.check_to_dict(oc) == want_chk and hc.stats()["error_bits"] == 0
        ex["cold_round"] = {"first_round_ms": round(cold, 4), "warm_round_ms": round(warm, 4),
                            "ratio": round(cold / warm, 2), "chunks_carved": int(sum(hc.stats()["carves"])),
                            "verified": okc}

    # ---- the headline round with the other staging setting
    with P.Heap(HEAP_BYTES, CHUNK, args.variant, staging=args.no_staging) as h3:
        o3 = torch.zeros(5, dtype=torch.int64, device="cuda")
        for _ in range(3):
            h3.round_fused(sizes, SEED, 1, out=o3)
        sms = timed(torch, stream, lambda: h3.round_fused(sizes, SEED, 1, out=o3), 5)
        ok3 = P.check_to_dict(o3)["mismatches"] == 0 and h3.stats()["error_bits"] == 0
        ex["staging_off" if not args.no_staging else "staging_on"] = {
            "fused_mops": round(2 * n / (sms / 1e3) / 1e6, 1), "ms": round(sms, 4), "verified": ok3}

    # ---- malloc latency histogram (warm heap, malloc-only batch)
    hist = torch.zeros(256, dtype=torch.int64, device="cuda")
    P.ouro_malloc_latency(heap.h, sizes, ptrs, hist)
    heap.free(ptrs)
    torch.cuda.synchronize()
    hc = hist.cpu().numpy()
    cum = np.cumsum(hc) / max(hc.sum(), 1)

    def q(p):
        b = int(np.searchsorted(cum, p))
        lo, hi = P.B.latency_bin_bounds(b)
        return (lo + hi) / 2

    mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
    ex["alloc_latency"] = {"p50_cycles": q(0.50), "p99_cycles": q(0.99),
                           "p50_ns": round(q(0.50) / mhz * 1e3, 1), "p99_ns": round(q(0.99) / mhz * 1e3, 1),
                           "clock_mhz_for_ns": mhz, "clock_source": "median SM clock sampled in the timed region",
                           "resolution": "log2 bins, 4 per octave (bin width 25% of its lower edge)",
                           "load": f"{n} concurrent mallocs on a warm heap"}

    # ---- L2 atomic rates and the allocator's share of them
    words = 1 << 24
    buf = torch.zeros(words, dtype=torch.int64, device="cuda")
    blocks = 8 * torch.cuda.get_device_properties(0).multi_processor_count
    rates = {}
    for pat, iters in ((0, 16), (1, 64), (2, 64)):
        P.ouro_probe_atomics(buf, pat, iters, blocks)
        ms = timed(torch, stream, lambda: P.ouro_probe_atomics(buf, pat, iters, blocks), 3)
        per = 256 if pat == 2 else 256 // 32          # patterns 0 and 1: one atomic per warp
        rates[pat] = blocks * per * iters / (ms / 1e3)
    def roof_pairs_for(width):
        g, cls = classes_per_group(sizes_np, width)
        groups = n / width * g
        max_class_groups = groups * max(np.bincount(cls, minlength=10)) / n
        t_same = 2 * max_class_groups / rates[0]       # head (malloc) + tail (free) of the busiest class
        t_dist = n / rates[2]                           # one slot CAS per free
        return n / (t_same + t_dist), g

    # the batch kernels on page queues aggregate per block: 256 threads, four
    # requests each on plain arrays once a batch fills every SM that way (as
    # the library does); chunk queues aggregate per warp
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    if args.variant.startswith("page_"):
        span = 256 * (4 if args.variant == "page_array" and n >= 4 * 256 * sms else 1)
    else:
        span = 32
    roof_pairs, g_blk = roof_pairs_for(span)
    warp_pairs, g_warp = roof_pairs_for(32)
    ach_pairs = n / (af / 1e3)
    ex["atomic_roofline"] = {
        "rates_gops": {"same_address": round(rates[0] / 1e9, 3), "32_addresses": round(rates[1] / 1e9, 3),
                       "distinct_cas": round(rates[2] / 1e9, 3)},
        "block_span": span, "classes_per_block": round(g_blk, 2), "classes_per_warp": round(g_warp, 2),
        "roofline_mops": round(2 * roof_pairs / 1e6, 1),
        "achieved_mops": round(2 * ach_pairs / 1e6, 1), "frac": round(ach_pairs / roof_pairs, 4),
        "warp_aggregated_roofline_mops": round(2 * warp_pairs / 1e6, 1),
        "model": "per malloc+free pair: one same-address atomic per block class group (block_span requests) "
                 "on head and on tail (busiest class serialises), one distinct-address slot CAS per free; "
                 "per-launch timings. warp_aggregated_roofline_mops: the same bound with one atomic per warp "
                 "class group"}
    return ex


if __name__ == "__main__":
    main()
