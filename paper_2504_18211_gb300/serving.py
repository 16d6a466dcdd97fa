"""Host side of the serving pattern: buffers, one call of the device loop, summary.

The whole request loop (admission, per-step growth, completion) runs on the
GPU inside ouro_serve; this module owns the device buffers (torch) and turns
the per-step timestamps into latency percentiles.
"""
from __future__ import annotations

import numpy as np

from . import _binding as B
import ctypes as C


class ServeRun:
    def __init__(self, arrive: np.ndarray, blocks: np.ndarray, n_slots: int = 16384, max_blocks: int = 4096,
                 steps: int = 2000, seed: int = 0x5E55, block_bytes: int = 16384):
        import torch
        self.torch = torch
        self.arrive, self.blocks = arrive.astype(np.uint32), blocks.astype(np.uint32)
        assert int(self.blocks.max(initial=1)) <= max_blocks
        self.n = int(arrive.size)
        self.n_slots, self.max_blocks, self.steps, self.seed, self.block_bytes = \
            n_slots, max_blocks, steps, seed, block_bytes
        dev = "cuda"
        self.d_arrive = torch.from_numpy(self.arrive.view(np.int32)).to(dev)
        self.d_blocks = torch.from_numpy(self.blocks.view(np.int32)).to(dev)
        self.slot_session = torch.empty(n_slots, dtype=torch.int32, device=dev)
        self.slot_k = torch.empty(n_slots, dtype=torch.int32, device=dev)
        self.slot_acc = torch.empty(3 * n_slots, dtype=torch.int64, device=dev)
        self.tables = torch.empty(n_slots * max_blocks, dtype=torch.int64, device=dev)
        self.sess_out = torch.empty(5 * max(self.n, 1), dtype=torch.int64, device=dev)
        self.step_ns = torch.zeros(3 * steps, dtype=torch.int64, device=dev)
        self.ctl = torch.zeros(11, dtype=torch.int64, device=dev)
        self.free_stack = torch.empty(2 * n_slots, dtype=torch.int32, device=dev)   # stack, then done list

    def run(self, heap, cap_blocks: int, blocks_per_sm: int = 0, form: str = "persistent") -> float:
        """One call of the loop; returns its duration in ms (CUDA events).
        form "persistent": ouro_serve, every step in one cooperative kernel;
        "per_launch": ouro_serve_per_launch, four launches per step."""
        torch = self.torch
        if form not in ("persistent", "per_launch"):
            raise ValueError(f"unknown serving form {form!r}")
        fn = B.load().ouro_serve if form == "persistent" else B.load().ouro_serve_per_launch
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s = torch.cuda.current_stream()
        a.record(s)
        st = fn(
            C.c_void_p(heap.h), B._ptr(self.d_arrive), B._ptr(self.d_blocks), self.n, self.n_slots,
            self.max_blocks, B._ptr(self.slot_session), B._ptr(self.slot_k), B._ptr(self.slot_acc),
            B._ptr(self.tables), B._ptr(self.sess_out), B._ptr(self.step_ns), B._ptr(self.ctl),
            B._ptr(self.free_stack), self.steps,
            self.seed, cap_blocks, self.block_bytes, blocks_per_sm, B._stream(None))
        B._check("ouro_serve" if form == "persistent" else "ouro_serve_per_launch", st)
        b.record(s)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    def results(self) -> dict:
        so = self.sess_out.cpu().numpy().view(np.uint64).reshape(-1, 5)[: self.n]
        ctl = self.ctl.cpu().numpy().view(np.uint64)
        ns = self.step_ns.cpu().numpy().view(np.uint64).astype(np.int64).reshape(-1, 3)
        ends = ns[:, 2]
        lat = np.diff(ends) / 1e3 if ends.size > 1 else np.zeros(0)
        phases = {"admit_us": (ns[1:, 0] - ends[:-1]) / 1e3, "grow_us": (ns[1:, 1] - ns[1:, 0]) / 1e3,
                  "complete_us": (ns[1:, 2] - ns[1:, 1]) / 1e3}
        never = np.uint64(0xFFFFFFFFFFFFFFFF)
        return {"xor": so[:, 0], "sum": so[:, 1], "mism": so[:, 2],
                "admit": np.where(so[:, 3] == never, -1, so[:, 3].astype(np.int64)),
                "done": np.where(so[:, 4] == never, -1, so[:, 4].astype(np.int64)),
                "mallocs": int(ctl[5]), "frees": int(ctl[6]), "failed": int(ctl[7]), "error": int(ctl[4]),
                "step_us": lat, "phases": phases}

