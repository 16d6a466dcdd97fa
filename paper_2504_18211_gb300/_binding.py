"""ctypes binding of libouro.so (include/ouro.h) -- argument marshalling only.

Every function named ``ouro_*`` here calls the C entry point of the same
name; all allocator work happens in the library's CUDA kernels.  PyTorch is
used only to own device buffers and to name the CUDA stream.  If the library
cannot be loaded the import fails: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libouro.so")
MAX_CLASSES = 17

PAGE_ARRAY, CHUNK_ARRAY, PAGE_VLIST, CHUNK_VLIST, PAGE_VARRAY, CHUNK_VARRAY = 0, 1, 2, 3, 4, 5
VARIANTS = {"page_array": PAGE_ARRAY, "chunk_array": CHUNK_ARRAY,
            "page_vlist": PAGE_VLIST, "chunk_vlist": CHUNK_VLIST,
            "page_varray": PAGE_VARRAY, "chunk_varray": CHUNK_VARRAY}
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EDEVICE", 5: "ENOTSUP"}
ERR_BAD_FREE, ERR_DOUBLE_FREE, ERR_QUEUE_FULL, ERR_TIMEOUT, ERR_QUEUE_OVERFLOW = 1, 2, 4, 8, 16


class OuroError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__(f"{fn} returned {STATUS.get(status, status)} ({status})")
        self.status = status


class Options(C.Structure):
    _fields_ = [("spin_limit", C.c_uint32), ("backoff_min_ns", C.c_uint32),
                ("backoff_max_ns", C.c_uint32), ("max_carve", C.c_uint32),
                ("array_queue_capacity", C.c_uint64), ("checked", C.c_uint32),
                ("staging", C.c_uint32), ("deopt", C.c_uint32), ("reserved", C.c_uint32)]


class HeapDev(C.Structure):
    _fields_ = [("base", C.c_void_p), ("bytes", C.c_ulonglong), ("n_chunks", C.c_ulonglong),
                ("chunk_bytes", C.c_uint), ("log2_chunk", C.c_uint), ("n_classes", C.c_uint),
                ("variant", C.c_uint), ("seg_cap", C.c_uint), ("words_per_chunk", C.c_uint),
                ("spin_limit", C.c_uint), ("backoff_min_ns", C.c_uint), ("backoff_max_ns", C.c_uint),
                ("max_carve", C.c_uint), ("checked", C.c_uint), ("staging", C.c_uint),
                ("deopt", C.c_uint), ("pad", C.c_uint),
                ("qhdr", C.c_void_p), ("cells", C.c_void_p),
                ("ring_off", C.c_ulonglong * MAX_CLASSES), ("ring_mask", C.c_ulonglong * MAX_CLASSES),
                ("qcap", C.c_ulonglong * MAX_CLASSES), ("chunk_cls", C.c_void_p),
                ("chunk_free", C.c_void_p), ("bits", C.c_void_p), ("pool", C.c_void_p),
                ("glob", C.c_void_p), ("stats", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [(k, C.c_uint64 * MAX_CLASSES) for k in
                ("mallocs", "frees", "failed", "carves", "carved_now", "queued", "live",
                 "repushes", "dead")] + \
               [("zero_reqs", C.c_uint64), ("too_large", C.c_uint64), ("bump", C.c_uint64),
                ("pool_size", C.c_uint64), ("seg_chunks", C.c_uint64), ("spare_chunks", C.c_uint64),
                ("error_bits", C.c_uint32), ("n_classes", C.c_uint32),
                ("error_site", C.c_uint32), ("n_large", C.c_uint32)]


class Snapshot(C.Structure):
    _fields_ = [("n_classes", C.c_uint32), ("n_chunks", C.c_uint64), ("bump", C.c_uint64),
                ("pool_n", C.c_uint64), ("pool", C.POINTER(C.c_uint32)),
                ("chunk_cls", C.POINTER(C.c_uint8)), ("chunk_free", C.POINTER(C.c_int32)),
                ("queue_n", C.c_uint64 * MAX_CLASSES),
                ("queue", C.POINTER(C.c_uint32) * MAX_CLASSES)]


class Check(C.Structure):
    _fields_ = [("nulls", C.c_ulonglong), ("mismatches", C.c_ulonglong), ("xor64", C.c_ulonglong),
                ("sum64", C.c_ulonglong), ("words", C.c_ulonglong)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libouro.so (raises OSError when it is missing: no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(path)
    vp, sz, st, u32, i32, u64 = C.c_void_p, C.c_size_t, C.c_int, C.c_uint32, C.c_int, C.c_uint64
    sigs = {
        "ouro_heap_create": (st, [sz, sz, C.POINTER(vp)]),
        "ouro_heap_create_ex": (st, [sz, sz, i32, C.POINTER(Options), vp, C.POINTER(vp)]),
        "ouro_heap_destroy": (st, [vp]),
        "ouro_heap_reset": (st, [vp, vp]),
        "ouro_heap_trim": (st, [vp, vp]),
        "ouro_heap_device": (st, [vp, C.POINTER(HeapDev)]),
        "ouro_heap_stats": (st, [vp, C.POINTER(Stats), vp]),
        "ouro_heap_snapshot": (st, [vp, C.POINTER(Snapshot), vp]),
        "ouro_snapshot_free": (None, [C.POINTER(Snapshot)]),
        "ouro_batch_malloc": (st, [vp, vp, vp, sz, vp]),
        "ouro_batch_free": (st, [vp, vp, sz, vp]),
        "ouro_pattern_write": (st, [vp, vp, sz, u32, i32, vp]),
        "ouro_pattern_check": (st, [vp, vp, sz, u32, i32, vp, vp]),
        "ouro_round_fused": (st, [vp, vp, sz, u32, i32, vp, vp, vp]),
        "ouro_status_string": (C.c_char_p, [st]),
        "ouro_last_cuda_error": (i32, []),
        "ouro_kernel_launches": (u64, []),
        "ouro_debug_stall_producer": (st, [vp, i32, u32, vp]),
        "ouro_probe_atomics": (st, [vp, sz, i32, u32, i32, vp]),
        "ouro_malloc_latency": (st, [vp, vp, vp, sz, vp, vp]),
        "ouro_cuda_malloc_heap": (st, [sz, C.POINTER(sz)]),
        "ouro_cuda_malloc_round": (st, [vp, sz, u32, i32, vp, vp]),
        "ouro_heap_stats_static": (st, [vp, C.POINTER(Stats), vp]),
        "ouro_batches_persistent": (st, [vp, vp, vp, vp, u32, u64, u32, i32, vp, vp, i32, vp]),
        "ouro_batch_graph_create": (st, [vp, vp, vp, u32, u32, i32, vp, vp, i32, C.POINTER(vp)]),
        "ouro_batch_graph_launch": (st, [vp, vp]),
        "ouro_batch_graph_nodes": (u64, [vp]),
        "ouro_batch_graph_destroy": (st, [vp]),
        "ouro_batches_max_blocks_per_sm": (i32, [vp]),
        "ouro_serve": (st, [vp, vp, vp, u32, u32, u32, vp, vp, vp, vp, vp, vp, vp, vp, u32, u32, u64, u32, i32, vp]),
        "ouro_serve_per_launch": (st, [vp, vp, vp, u32, u32, u32, vp, vp, vp, vp, vp, vp, vp, vp, u32, u32, u64, u32,
                                       i32, vp]),
        "ouro_graph_vertex_bytes": (sz, []),
        "ouro_graph_init": (st, [vp, vp, u32, vp, vp]),
        "ouro_graph_insert": (st, [vp, vp, vp, vp, u64, vp, vp]),
        "ouro_graph_gather": (st, [vp, vp, u32, vp, vp, vp]),
        "ouro_graph_free": (st, [vp, vp, u32, vp]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    _lib = lib
    return lib


def _check(fn: str, status: int, ok=(0,)):
    if status not in ok:
        raise OuroError(fn, status)
    return status


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


# ---- same-named thin wrappers ------------------------------------------------
def ouro_heap_create_ex(bytes_: int, chunk_bytes: int, variant: int = PAGE_ARRAY,
                        options: Options | None = None, heap_buf_ptr: int = 0) -> int:
    h = C.c_void_p()
    _check("ouro_heap_create_ex", load().ouro_heap_create_ex(
        bytes_, chunk_bytes, variant, C.byref(options) if options else None,
        C.c_void_p(heap_buf_ptr) if heap_buf_ptr else None, C.byref(h)))
    return h.value


def ouro_heap_destroy(h: int) -> None:
    _check("ouro_heap_destroy", load().ouro_heap_destroy(C.c_void_p(h)))


def ouro_heap_reset(h: int, stream=None) -> None:
    _check("ouro_heap_reset", load().ouro_heap_reset(C.c_void_p(h), _stream(stream)))


def ouro_heap_trim(h: int, stream=None) -> None:
    _check("ouro_heap_trim", load().ouro_heap_trim(C.c_void_p(h), _stream(stream)))


def ouro_heap_device(h: int) -> HeapDev:
    d = HeapDev()
    _check("ouro_heap_device", load().ouro_heap_device(C.c_void_p(h), C.byref(d)))
    return d


def _stats_dict(s: Stats) -> dict:
    """Per-class lists cover every class: those within one chunk (n_classes),
    then the runs above one chunk (n_large)."""
    nc = s.n_classes + s.n_large
    out = {k: [int(x) for x in getattr(s, k)[:nc]] for k in
           ("mallocs", "frees", "failed", "carves", "carved_now", "queued", "live", "repushes", "dead")}
    for k in ("zero_reqs", "too_large", "bump", "pool_size", "seg_chunks", "spare_chunks",
              "error_bits", "n_classes", "n_large", "error_site"):
        out[k] = int(getattr(s, k))
    return out


def ouro_heap_stats_static(h: int, stream=None) -> dict:
    """ouro_heap_stats without any device allocation (scratch in a static device array)."""
    s = Stats()
    _check("ouro_heap_stats_static", load().ouro_heap_stats_static(C.c_void_p(h), C.byref(s), _stream(stream)),
           ok=(0, 4))
    return _stats_dict(s)


def ouro_heap_stats(h: int, stream=None) -> dict:
    s = Stats()
    load().ouro_heap_stats(C.c_void_p(h), C.byref(s), _stream(stream))
    return _stats_dict(s)


def ouro_heap_snapshot(h: int, stream=None) -> dict:
    import numpy as np
    sn = Snapshot()
    lib = load()
    _check("ouro_heap_snapshot", lib.ouro_heap_snapshot(C.c_void_p(h), C.byref(sn), _stream(stream)))
    try:
        nc, nch = sn.n_classes, sn.n_chunks
        out = {"bump": int(sn.bump),
               "pool": np.ctypeslib.as_array(sn.pool, (max(sn.pool_n, 1),))[:sn.pool_n].copy(),
               "chunk_cls": np.ctypeslib.as_array(sn.chunk_cls, (nch,)).copy(),
               "chunk_free": (np.ctypeslib.as_array(sn.chunk_free, (nch,)).copy()
                              if sn.chunk_free else None),
               "queues": [np.ctypeslib.as_array(sn.queue[c], (max(sn.queue_n[c], 1),))[:sn.queue_n[c]].copy()
                          for c in range(MAX_CLASSES)]}
    finally:
        lib.ouro_snapshot_free(C.byref(sn))
    return out


def ouro_batch_malloc(h: int, sizes, ptrs, stream=None) -> None:
    _check("ouro_batch_malloc", load().ouro_batch_malloc(C.c_void_p(h), _ptr(sizes), _ptr(ptrs),
                                                          sizes.numel(), _stream(stream)))


def ouro_batch_free(h: int, ptrs, stream=None) -> None:
    _check("ouro_batch_free", load().ouro_batch_free(C.c_void_p(h), _ptr(ptrs), ptrs.numel(),
                                                      _stream(stream)))


def ouro_pattern_write(ptrs, sizes, seed: int, mode: int = 1, stream=None) -> None:
    _check("ouro_pattern_write", load().ouro_pattern_write(_ptr(ptrs), _ptr(sizes), sizes.numel(),
                                                            seed & 0xFFFFFFFF, mode, _stream(stream)))


def ouro_pattern_check(ptrs, sizes, seed: int, mode: int, out, stream=None) -> None:
    _check("ouro_pattern_check", load().ouro_pattern_check(_ptr(ptrs), _ptr(sizes), sizes.numel(),
                                                            seed & 0xFFFFFFFF, mode, _ptr(out),
                                                            _stream(stream)))


def ouro_round_fused(h: int, sizes, seed: int, mode: int, out, ptrs=None, stream=None) -> None:
    _check("ouro_round_fused", load().ouro_round_fused(C.c_void_p(h), _ptr(sizes), sizes.numel(),
                                                        seed & 0xFFFFFFFF, mode, _ptr(out), _ptr(ptrs),
                                                        _stream(stream)))


def ouro_debug_stall_producer(h: int, cls: int, n: int, stream=None) -> None:
    _check("ouro_debug_stall_producer",
           load().ouro_debug_stall_producer(C.c_void_p(h), cls, n, _stream(stream)))


def ouro_kernel_launches() -> int:
    return int(load().ouro_kernel_launches())


def ouro_status_string(s: int) -> str:
    return load().ouro_status_string(s).decode()


def check_to_dict(t) -> dict:
    """Read an ouro_check written to a device tensor of 5 int64 words."""
    v = t.cpu().view(-1).tolist()
    m = (1 << 64) - 1
    return {"nulls": v[0] & m, "mismatches": v[1] & m, "xor64": v[2] & m, "sum64": v[3] & m,
            "words": v[4] & m}


def ouro_probe_atomics(buf, pattern: int, iters: int, blocks: int, stream=None) -> None:
    _check("ouro_probe_atomics", load().ouro_probe_atomics(_ptr(buf), buf.numel(), pattern, iters, blocks,
                                                            _stream(stream)))


def ouro_malloc_latency(h: int, sizes, ptrs, hist, stream=None) -> None:
    _check("ouro_malloc_latency", load().ouro_malloc_latency(C.c_void_p(h), _ptr(sizes), _ptr(ptrs),
                                                              sizes.numel(), _ptr(hist), _stream(stream)))


def ouro_cuda_malloc_heap(nbytes: int) -> int:
    """Size CUDA's device-malloc heap of this context; returns the size CUDA reports."""
    got = C.c_size_t(0)
    _check("ouro_cuda_malloc_heap", load().ouro_cuda_malloc_heap(nbytes, C.byref(got)))
    return got.value


def ouro_cuda_malloc_round(sizes, seed: int, mode: int = 1, out=None, stream=None):
    """The fused driver round on CUDA's device malloc / free; returns the check tensor."""
    import torch
    if out is None:
        out = torch.zeros(5, dtype=torch.int64, device=sizes.device)
    _check("ouro_cuda_malloc_round", load().ouro_cuda_malloc_round(_ptr(sizes), sizes.numel(), seed & 0xFFFFFFFF,
                                                                    mode, _ptr(out), _stream(stream)))
    return out


def latency_bin_bounds(b: int):
    """[lo, hi) cycles of histogram bin b of ouro_malloc_latency."""
    if b < 4:
        return b, b + 1
    l, q = b >> 2, b & 3
    return (1 << l) + q * (1 << (l - 2)), (1 << l) + (q + 1) * (1 << (l - 2))


def ouro_batches_persistent(h: int, sizes, offs, task_offs, n_tasks: int, seed: int, mode: int, out, work,
                            blocks_per_sm: int = 0, stream=None) -> None:
    _check("ouro_batches_persistent", load().ouro_batches_persistent(
        C.c_void_p(h), _ptr(sizes), _ptr(offs), _ptr(task_offs), offs.numel() - 1, n_tasks, seed & 0xFFFFFFFF,
        mode, _ptr(out), _ptr(work), blocks_per_sm, _stream(stream)))


def ouro_batch_graph_create(h: int, sizes, h_offs, seed: int, mode: int, out, ptrs=None, form: int = 0) -> int:
    import numpy as np
    offs = np.ascontiguousarray(h_offs, dtype=np.uint64)
    g = C.c_void_p()
    _check("ouro_batch_graph_create", load().ouro_batch_graph_create(
        C.c_void_p(h), _ptr(sizes), offs.ctypes.data_as(C.c_void_p), offs.size - 1, seed & 0xFFFFFFFF, mode,
        _ptr(out), _ptr(ptrs), form, C.byref(g)))
    return g.value


def ouro_batch_graph_launch(g: int, stream=None) -> None:
    _check("ouro_batch_graph_launch", load().ouro_batch_graph_launch(C.c_void_p(g), _stream(stream)))


def ouro_batch_graph_destroy(g: int) -> None:
    _check("ouro_batch_graph_destroy", load().ouro_batch_graph_destroy(C.c_void_p(g)))


def persistent_blocks_per_sm(heap) -> int:
    """ouro_batches_max_blocks_per_sm for a Heap (or raw handle)."""
    return int(load().ouro_batches_max_blocks_per_sm(C.c_void_p(getattr(heap, "h", heap))))
