"""Host side of the graph-growth pattern: device buffers and one insertion pass.

The lists grow inside ouro_graph_insert (libouro.so); this module only owns
the vertex table and the edge arrays (torch) and reads results back.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _binding as B


class GraphRun:
    def __init__(self, src: np.ndarray, dst: np.ndarray, n_vertices: int):
        import torch
        self.torch = torch
        self.nv, self.ne = n_vertices, int(src.size)
        vb = int(B.load().ouro_graph_vertex_bytes())
        self.vt = torch.empty((n_vertices * vb + 7) // 8, dtype=torch.int64, device="cuda")
        self.d_src = torch.from_numpy(src.view(np.int32)).cuda()
        self.d_dst = torch.from_numpy(dst.view(np.int32)).cuda()
        self.ctl = torch.zeros(4, dtype=torch.int64, device="cuda")
        self.vbytes = vb

    def init(self, heap):
        B._check("ouro_graph_init", B.load().ouro_graph_init(C.c_void_p(heap.h), B._ptr(self.vt), self.nv,
                                                              B._ptr(self.ctl), B._stream(None)))

    def insert(self, heap):
        B._check("ouro_graph_insert", B.load().ouro_graph_insert(C.c_void_p(heap.h), B._ptr(self.vt),
                                                                  B._ptr(self.d_src), B._ptr(self.d_dst), self.ne,
                                                                  B._ptr(self.ctl), B._stream(None)))

    def free(self, heap):
        B._check("ouro_graph_free", B.load().ouro_graph_free(C.c_void_p(heap.h), B._ptr(self.vt), self.nv,
                                                              B._stream(None)))

    def degrees(self) -> np.ndarray:
        """deg field of every vertex record (uint32 at byte 32 of the 40-byte record)."""
        raw = self.vt.cpu().numpy().view(np.uint8)[: self.nv * self.vbytes].reshape(self.nv, self.vbytes)
        return raw[:, 32:36].copy().view(np.uint32).ravel()

    def gather(self, heap) -> tuple:
        torch = self.torch
        deg = self.degrees()
        off = np.concatenate([[0], np.cumsum(deg.astype(np.int64))]).astype(np.int64)
        d_off = torch.from_numpy(off[:-1].copy()).cuda()
        out = torch.empty(max(int(off[-1]), 1), dtype=torch.int32, device="cuda")
        B._check("ouro_graph_gather", B.load().ouro_graph_gather(C.c_void_p(heap.h), B._ptr(self.vt), self.nv,
                                                                  B._ptr(d_off), B._ptr(out), B._stream(None)))
        torch.cuda.synchronize()
        return deg, off, out.cpu().numpy().view(np.uint32)[: int(off[-1])]

    def ctl_dict(self) -> dict:
        c = self.ctl.cpu().numpy()
        return {"appended": int(c[0]), "failed": int(c[1]), "skipped": int(c[2])}

