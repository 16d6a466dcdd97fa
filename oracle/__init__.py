"""Sequential CPU oracle of the device-side allocator (arXiv 2504.18211).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  It
shares no code with the CUDA library and never imports it.

The C source (``ouro_oracle.c``) runs the method one request at a time:
host-preallocated heap (Sec. 1), chunks and pages with one queue per
power-of-two size (Sec. 1; Sec. 4 preamble; Sec. 4.2), page queues (Sec. 4.1),
chunk queues with a free-page scan (Sec. 4.2), virtualized list queues whose
storage lives in heap chunks (Sec. 4.3), and the allocate / write / check /
free driver round (Sec. 3).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ouro_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

PAGE_ARRAY, CHUNK_ARRAY, PAGE_VLIST, CHUNK_VLIST, PAGE_VARRAY, CHUNK_VARRAY = 0, 1, 2, 3, 4, 5
VARIANTS = {"page_array": PAGE_ARRAY, "chunk_array": CHUNK_ARRAY,
            "page_vlist": PAGE_VLIST, "chunk_vlist": CHUNK_VLIST,
            "page_varray": PAGE_VARRAY, "chunk_varray": CHUNK_VARRAY}
MAX_CLASSES = 17
ERR_BAD_FREE, ERR_DOUBLE_FREE, ERR_QUEUE_FULL = 1, 2, 4


def build(out: str = _LIB, cflags: tuple = ("-O2",), defines: tuple = ()) -> str:
    """Compile the oracle with gcc into a shared library and return its path."""
    tmp = f"{out}.{os.getpid()}.tmp"
    cmd = ["gcc", *cflags, "-std=c11", "-Wall", "-shared", "-fPIC",
           *[f"-D{d}" for d in defines], "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)     # atomic: concurrent loaders see the old or the new file
    return out


def ensure_built() -> str:
    """Build the oracle library unless an up-to-date one exists."""
    if not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        build(_LIB)
    return _LIB


class _Stats(C.Structure):
    _fields_ = [("mallocs", C.c_uint64 * MAX_CLASSES), ("frees", C.c_uint64 * MAX_CLASSES),
                ("failed", C.c_uint64 * MAX_CLASSES), ("carves", C.c_uint64 * MAX_CLASSES),
                ("carved_now", C.c_uint64 * MAX_CLASSES), ("queued", C.c_uint64 * MAX_CLASSES),
                ("live", C.c_uint64 * MAX_CLASSES),
                ("zero_reqs", C.c_uint64), ("too_large", C.c_uint64),
                ("bump", C.c_uint64), ("pool_size", C.c_uint64),
                ("seg_chunks", C.c_uint64), ("spare_chunks", C.c_uint64),
                ("error_bits", C.c_uint32), ("n_classes", C.c_uint32),
                ("n_large", C.c_uint32), ("pad", C.c_uint32)]


class RoundResult(C.Structure):
    _fields_ = [("nulls", C.c_uint64), ("mismatches", C.c_uint64), ("xor64", C.c_uint64),
                ("sum64", C.c_uint64), ("words", C.c_uint64)]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


_libs: dict = {}


def load(path: str = _LIB):
    """Load (building if needed) the oracle library at ``path``."""
    if path in _libs:
        return _libs[path]
    if path == _LIB:
        ensure_built()
    lib = C.CDLL(path)
    u64, i64, u32, i32, vp = C.c_uint64, C.c_int64, C.c_uint32, C.c_int, C.c_void_p
    sig = {
        "orc_create": (vp, [u64, u64, i32, u64]),
        "orc_destroy": (None, [vp]),
        "orc_reset": (None, [vp]),
        "orc_num_classes": (i32, [u64]),
        "orc_size_class": (i32, [u64, u64]),
        "orc_page_bytes": (u64, [i32]),
        "orc_malloc": (i64, [vp, u64]),
        "orc_free": (u32, [vp, i64]),
        "orc_trim": (None, [vp]),
        "orc_get_stats": (None, [vp, C.POINTER(_Stats)]),
        "orc_queue_items": (u64, [vp, i32, vp, u64]),
        "orc_pool_items": (u64, [vp, vp, u64]),
        "orc_chunk_classes": (u64, [vp, vp, u64]),
        "orc_chunk_free_pages": (u64, [vp, vp, u64]),
        "orc_seg_chunks": (u64, [vp, i32, vp, u64]),
        "orc_error_bits": (u32, [vp]),
        "orc_fmix32": (u32, [u32]),
        "orc_pattern_word": (u32, [u32, u32, u32, i32]),
        "orc_round": (None, [vp, vp, u64, u32, i32, vp, vp, C.POINTER(RoundResult)]),
        "orc_expected_checksums": (None, [vp, u64, u32, i32, C.POINTER(RoundResult)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    _libs[path] = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class OracleHeap:
    """One sequential heap: the same size classes, chunk/page layout and queue
    semantics as the device allocator, executed one request at a time."""

    def __init__(self, bytes_: int, chunk_bytes: int, variant: int | str = PAGE_ARRAY,
                 queue_cap: int = 0, lib_path: str = _LIB):
        self.lib = load(lib_path)
        if isinstance(variant, str):
            variant = VARIANTS[variant]
        self.bytes, self.chunk_bytes, self.variant = bytes_, chunk_bytes, variant
        self.n_chunks = bytes_ // chunk_bytes
        self.h = self.lib.orc_create(bytes_, chunk_bytes, variant, queue_cap)
        if not self.h:
            raise ValueError("orc_create rejected the arguments")
        self.n_classes = self.lib.orc_num_classes(chunk_bytes)

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.orc_destroy(self.h)
            self.h = None

    # --- single requests -------------------------------------------------
    def malloc(self, n: int) -> int:
        return int(self.lib.orc_malloc(self.h, n))

    def free(self, off: int) -> int:
        return int(self.lib.orc_free(self.h, off))

    def trim(self) -> None:
        self.lib.orc_trim(self.h)

    def reset(self) -> None:
        self.lib.orc_reset(self.h)

    def size_class(self, n: int) -> int:
        return int(self.lib.orc_size_class(self.chunk_bytes, n))

    def page_bytes(self, c: int) -> int:
        return int(self.lib.orc_page_bytes(c))

    # --- inspection ------------------------------------------------------
    def stats(self) -> dict:
        s = _Stats()
        self.lib.orc_get_stats(self.h, C.byref(s))
        nc = s.n_classes + s.n_large            # classes within one chunk, then runs of chunks
        out = {k: [int(x) for x in getattr(s, k)[:nc]]
               for k in ("mallocs", "frees", "failed", "carves", "carved_now", "queued", "live")}
        for k in ("zero_reqs", "too_large", "bump", "pool_size", "seg_chunks",
                  "spare_chunks", "error_bits"):
            out[k] = int(getattr(s, k))
        return out

    def queue_items(self, c: int) -> np.ndarray:
        n = self.lib.orc_queue_items(self.h, c, None, 0)
        out = np.zeros(max(n, 1), np.uint64)
        self.lib.orc_queue_items(self.h, c, _ptr(out), n)
        return out[:n]

    def pool_items(self) -> np.ndarray:
        n = self.lib.orc_pool_items(self.h, None, 0)
        out = np.zeros(max(n, 1), np.uint64)
        self.lib.orc_pool_items(self.h, _ptr(out), n)
        return out[:n]

    def chunk_classes(self) -> np.ndarray:
        out = np.zeros(self.n_chunks, np.int16)
        self.lib.orc_chunk_classes(self.h, _ptr(out), self.n_chunks)
        return out

    def chunk_free_pages(self) -> np.ndarray:
        out = np.zeros(self.n_chunks, np.uint32)
        self.lib.orc_chunk_free_pages(self.h, _ptr(out), self.n_chunks)
        return out

    def seg_chunks(self, c: int) -> np.ndarray:
        n = self.lib.orc_seg_chunks(self.h, c, None, 0)
        out = np.zeros(max(n, 1), np.uint64)
        self.lib.orc_seg_chunks(self.h, c, _ptr(out), n)
        return out[:n]

    def canonical_state(self) -> dict:
        """Schedule-independent view of the queues: sorted items per class,
        sorted pool, bump pointer and the chunk class table."""
        return {"queues": [np.sort(self.queue_items(c)) for c in range(MAX_CLASSES)],
                "pool": np.sort(self.pool_items()), "bump": self.stats()["bump"],
                "chunk_cls": self.chunk_classes()}

    # --- driver round ----------------------------------------------------
    def round(self, sizes: np.ndarray, seed: int, mode: int = 1, with_memory: bool = True,
              return_offsets: bool = False, return_memory: bool = False):
        """One driver round (Sec. 3) over `sizes`: allocate all, write, read
        back and check, free all.  Returns the checksum dict; with
        return_offsets / return_memory also the block offsets and the heap
        bytes as the round left them (host memory, zero where never written)."""
        sizes = np.ascontiguousarray(sizes, dtype=np.uint32)
        n = sizes.size
        mem = np.zeros(self.bytes, np.uint8) if (with_memory or return_memory) else None
        offs = np.zeros(max(n, 1), np.int64) if (return_offsets or return_memory) else None
        r = RoundResult()
        self.lib.orc_round(self.h, _ptr(sizes), n, seed, mode,
                           _ptr(mem) if mem is not None else None,
                           _ptr(offs) if offs is not None else None, C.byref(r))
        out = [r.as_dict()]
        if return_offsets or return_memory:
            out.append(offs[:n])
        if return_memory:
            out.append(mem)
        return tuple(out) if len(out) > 1 else out[0]


def expected_checksums(sizes: np.ndarray, seed: int, mode: int = 1) -> dict:
    lib = load()
    sizes = np.ascontiguousarray(sizes, dtype=np.uint32)
    r = RoundResult()
    lib.orc_expected_checksums(_ptr(sizes), sizes.size, seed, mode, C.byref(r))
    return r.as_dict()


def fmix32(x: int) -> int:
    return int(load().orc_fmix32(x & 0xFFFFFFFF))


def pattern_word(seed: int, tid: int, i: int, mode: int = 1) -> int:
    return int(load().orc_pattern_word(seed & 0xFFFFFFFF, tid & 0xFFFFFFFF, i, mode))
