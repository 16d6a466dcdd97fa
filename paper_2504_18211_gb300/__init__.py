"""GB300-native device-side dynamic memory allocator (arXiv 2504.18211, Ouroboros method).

The allocator runs inside CUDA kernels (libouro.so, built for sm_103a from
csrc/ and include/); this package only loads it and marshals arguments.
``Heap`` is a convenience owner of one heap; the ``ouro_*`` functions are the
C entry points under the same names.
"""
from __future__ import annotations

from . import _binding as B
from ._binding import (CHUNK_ARRAY, CHUNK_VARRAY, CHUNK_VLIST, PAGE_ARRAY, PAGE_VARRAY, PAGE_VLIST, VARIANTS, Options,  # noqa: F401
                       OuroError, check_to_dict, load, ouro_batch_free, ouro_batch_malloc,
                       ouro_debug_stall_producer, ouro_heap_create_ex, ouro_heap_destroy,
                       ouro_heap_device, ouro_heap_reset, ouro_heap_snapshot, ouro_heap_stats,
                       ouro_cuda_malloc_heap, ouro_cuda_malloc_round,
                       ouro_heap_trim, ouro_kernel_launches, ouro_malloc_latency, ouro_pattern_check,
                       ouro_pattern_write, ouro_probe_atomics, ouro_round_fused, ouro_status_string)


class Heap:
    """Owns one device heap (ouro_heap_create_ex / ouro_heap_destroy)."""

    def __init__(self, bytes_: int, chunk_bytes: int, variant="page_array", *, spin_limit: int = 0,
                 backoff_min_ns: int = 0, backoff_max_ns: int = 0, max_carve: int = 0,
                 array_queue_capacity: int = 0, checked: bool = False, staging: bool = False,
                 deopt: bool = False, heap_buf=None):
        if isinstance(variant, str):
            variant = VARIANTS[variant]
        opt = Options(spin_limit, backoff_min_ns, backoff_max_ns, max_carve, array_queue_capacity,
                      1 if checked else 0, 1 if staging else 0, 1 if deopt else 0, 0)
        self._buf = heap_buf       # keep a caller buffer alive as long as the heap
        self.h = ouro_heap_create_ex(bytes_, chunk_bytes, variant, opt,
                                     heap_buf.data_ptr() if heap_buf is not None else 0)
        self.bytes, self.chunk_bytes, self.variant = bytes_, chunk_bytes, variant
        self.dev = ouro_heap_device(self.h)
        self.base = int(self.dev.base)
        self.n_classes = int(self.dev.n_classes)

    def close(self):
        if getattr(self, "h", None):
            ouro_heap_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # batch API
    def malloc(self, sizes, ptrs=None, stream=None):
        import torch
        if ptrs is None:
            ptrs = torch.empty(sizes.numel(), dtype=torch.int64, device=sizes.device)
        ouro_batch_malloc(self.h, sizes, ptrs, stream)
        return ptrs

    def free(self, ptrs, stream=None):
        ouro_batch_free(self.h, ptrs, stream)

    def round_fused(self, sizes, seed: int, mode: int = 1, out=None, ptrs=None, stream=None):
        import torch
        if out is None:
            out = torch.zeros(5, dtype=torch.int64, device=sizes.device)
        ouro_round_fused(self.h, sizes, seed, mode, out, ptrs, stream)
        return out

    def stats(self, stream=None) -> dict:
        return ouro_heap_stats(self.h, stream)

    def snapshot(self, stream=None) -> dict:
        return ouro_heap_snapshot(self.h, stream)

    def trim(self, stream=None):
        ouro_heap_trim(self.h, stream)

    def reset(self, stream=None):
        ouro_heap_reset(self.h, stream)


def pattern_write(ptrs, sizes, seed: int, mode: int = 1, stream=None):
    ouro_pattern_write(ptrs, sizes, seed, mode, stream)


def pattern_check(ptrs, sizes, seed: int, mode: int = 1, out=None, stream=None):
    import torch
    if out is None:
        out = torch.zeros(5, dtype=torch.int64, device=sizes.device)
    ouro_pattern_check(ptrs, sizes, seed, mode, out, stream)
    return out
