"""Host side of the batching pattern: task tables, the four forms, the autotuner.

Forms (all run the same work: every request of every batch allocates,
writes its pattern, reads it back and frees):
  per_launch4  four library launches per batch (malloc, write, check, free)
  per_launch1  one fused-round launch per batch
  graph        the per-batch fused launches captured once as a CUDA graph
  persistent   one kernel for all batches, 256-request tasks from a device counter
Only marshalling and timing happen here; every step runs in libouro.so.
"""
from __future__ import annotations

import itertools
import time

import numpy as np

from . import _binding as B

TASK_REQ = 256
FORMS = ("per_launch4", "per_launch1", "graph", "persistent")


def task_offsets(offs: np.ndarray) -> np.ndarray:
    counts = np.diff(offs.astype(np.int64))
    tasks = (counts + TASK_REQ - 1) // TASK_REQ
    return np.concatenate([[0], np.cumsum(tasks)]).astype(np.uint64)


class BatchRun:
    """Device copies of one batching workload, reusable across forms and heaps."""

    def __init__(self, sizes: np.ndarray, offs: np.ndarray, seed: int = 0xBA7C4, mode: int = 1):
        import torch
        self.torch = torch
        self.sizes_np, self.offs_np = sizes, offs.astype(np.uint64)
        self.nb = offs.size - 1
        self.seed, self.mode = seed, mode
        self.n = int(sizes.size)
        self.d_sizes = torch.from_numpy(sizes.view(np.int32)).cuda()
        self.d_offs = torch.from_numpy(self.offs_np.view(np.int64)).cuda()
        to = task_offsets(self.offs_np)
        self.n_tasks = int(to[-1])
        self.d_task = torch.from_numpy(to.view(np.int64)).cuda()
        self.out = torch.zeros((self.nb, 5), dtype=torch.int64, device="cuda")
        self.work = torch.zeros(1, dtype=torch.int64, device="cuda")
        self.max_batch = int(np.diff(self.offs_np.astype(np.int64)).max())
        self.ptrs = torch.empty(self.max_batch, dtype=torch.int64, device="cuda")
        self.graphs = {}

    def checks(self) -> list:
        v = self.out.cpu().numpy().view(np.uint64)
        return [dict(nulls=int(r[0]), mismatches=int(r[1]), xor64=int(r[2]), sum64=int(r[3]), words=int(r[4]))
                for r in v]

    def run(self, heap, form: str, blocks_per_sm: int = 0):
        torch = self.torch
        if form == "persistent":
            B.ouro_batches_persistent(heap.h, self.d_sizes, self.d_offs, self.d_task, self.n_tasks, self.seed,
                                      self.mode, self.out, self.work, blocks_per_sm)
        elif form == "graph":
            key = (heap.h, 0)
            if key not in self.graphs:
                self.graphs[key] = B.ouro_batch_graph_create(heap.h, self.d_sizes, self.offs_np, self.seed,
                                                             self.mode, self.out, None, 0)
            B.ouro_batch_graph_launch(self.graphs[key])
        else:
            o = self.offs_np.astype(np.int64)
            for b in range(self.nb):
                sz = self.d_sizes[o[b]:o[b + 1]]
                ob = self.out[b]
                if form == "per_launch1":
                    B.ouro_round_fused(heap.h, sz, self.seed + b, self.mode, ob)
                else:
                    p = self.ptrs[:sz.numel()]
                    B.ouro_batch_malloc(heap.h, sz, p)
                    B.ouro_pattern_write(p, sz, self.seed + b, self.mode)
                    B.ouro_pattern_check(p, sz, self.seed + b, self.mode, ob)
                    B.ouro_batch_free(heap.h, p)
        return torch

    def time(self, heap, form: str, reps: int = 3, blocks_per_sm: int = 0) -> float:
        """Mean ms per pass over all batches (one warm-up pass first)."""
        torch = self.torch
        self.run(heap, form, blocks_per_sm)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            self.run(heap, form, blocks_per_sm)
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    def close(self):
        for g in self.graphs.values():
            B.ouro_batch_graph_destroy(g)
        self.graphs = {}


def autotune(Heap, run: BatchRun, heap_bytes: int, chunks=(4096, 8192, 16384, 65536),
             variants=("page_array", "page_vlist", "chunk_array", "chunk_vlist", "page_varray", "chunk_varray"),
             warps_per_sm=(8, 16, 32, 48, 64), reps: int = 2, max_size: int = 8192):
    """Time the persistent form over chunk size x queue variant x warps per SM.

    A chunk smaller than the largest request serves those requests as runs
    of chunks (row "runs": true); requests above 1 MiB cannot be served at
    all, so max_size above it marks every row infeasible.  A warps-per-SM
    value above what the kernel's registers allow is marked infeasible too.
    Returns (best, table)."""
    torch = run.torch
    table = []
    best = None
    for chunk, variant in itertools.product(chunks, variants):
        if max_size > (1 << 20):
            table.append({"chunk": chunk, "variant": variant, "status": "infeasible: requests above 1 MiB"})
            continue
        heap = Heap(heap_bytes, chunk, variant)
        try:
            limit = B.persistent_blocks_per_sm(heap)
            for wps in warps_per_sm:
                bps = wps // 8
                if bps > limit:
                    table.append({"chunk": chunk, "variant": variant, "warps_per_sm": wps,
                                  "status": f"infeasible: registers allow {8 * limit} warps/SM"})
                    continue
                ms = run.time(heap, "persistent", reps, bps)
                ok = all(c["mismatches"] == 0 for c in run.checks()) and heap.stats()["error_bits"] == 0
                row = {"chunk": chunk, "variant": variant, "warps_per_sm": wps, "ms": round(ms, 3),
                       "mops": round(2 * run.n / (ms / 1e3) / 1e6, 1), "verified": ok,
                       "runs": max_size > chunk}
                table.append(row)
                if ok and (best is None or ms < best["ms"]):
                    best = row
        finally:
            heap.close()
        torch.cuda.synchronize()
    return best, table
