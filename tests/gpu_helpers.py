"""Shared helpers of the GPU parity tests (CUDA path through the C ABI vs the oracle)."""
from __future__ import annotations

import numpy as np

import oracle


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU test run without a GPU"
    return torch


def to_dev(a: np.ndarray):
    torch = torch_cuda()
    return torch.from_numpy(a.astype(np.int32, copy=False).view(np.int32)).cuda()


ALL_CLASSES = 17            # 16 B .. 1 MiB: classes within a chunk, then runs of chunks


def class_of(sizes: np.ndarray, chunk: int) -> np.ndarray:
    """Closed-form class per request (-1: no class); independent of both implementations."""
    s = sizes.astype(np.int64)
    c = np.where(s <= 16, 0, np.ceil(np.log2(np.maximum(s, 1))).astype(np.int64) - 4)
    return np.where((s == 0) | (s > (1 << 20)), -1, c)


def per_class_counts(sizes: np.ndarray, chunk: int, n_classes: int = ALL_CLASSES) -> list:
    c = class_of(sizes, chunk)
    return [int((c == k).sum()) for k in range(n_classes)]


def assert_no_overlap(ptrs: np.ndarray, sizes: np.ndarray, base: int, heap_bytes: int, chunk: int):
    """Every non-null block lies in the heap, is aligned to its class and
    overlaps no other block."""
    p = ptrs.astype(np.uint64)
    live = p != 0
    cls = class_of(sizes, chunk)
    assert np.all(cls[live] >= 0)
    page = (np.uint64(16) << cls[live].astype(np.uint64)).astype(np.uint64)
    off = p[live] - np.uint64(base)
    assert np.all(off < np.uint64(heap_bytes)), "block outside the heap"
    align = np.minimum(page, np.uint64(chunk))           # runs of chunks start on a chunk
    assert np.all(off % align == 0), "block not aligned to its class"
    assert np.all(off + page <= np.uint64(heap_bytes)), "block runs past the heap"
    order = np.argsort(off, kind="stable")
    o, pg = off[order], page[order]
    if o.size > 1:
        assert np.all(o[:-1] + pg[:-1] <= o[1:]), "live blocks overlap"


def oracle_round(bytes_, chunk, variant, sizes, seed, mode, with_memory=False):
    h = oracle.OracleHeap(bytes_, chunk, variant)
    res = h.round(sizes, seed, mode, with_memory=with_memory)
    return h, res


def same_canonical_as_post_create(snap: dict, n_chunks: int):
    assert snap["bump"] == 0, snap["bump"]
    assert snap["pool"].size == 0, snap["pool"][:10]
    assert np.all(snap["chunk_cls"] == 0xFF)
    assert all(q.size == 0 for q in snap["queues"])
