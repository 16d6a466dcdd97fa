"""A trivially correct set-allocator used to pin the oracle by brute force.

It knows nothing about queues: it keeps the set of live blocks and, per chunk,
the size class the chunk was given.  A request of class c can be served iff
some chunk of class c still has a page that is not live, or a chunk that no
class owns is left (and, for page-array queues, the class still has room
under its queue capacity).  The allocator must take a new chunk only when the
first condition fails.  Nothing here is shared with the oracle.
"""
from __future__ import annotations


def ceil_log2(n: int) -> int:
    return (n - 1).bit_length()


class SetModel:
    def __init__(self, bytes_: int, chunk_bytes: int, page_array_cap: int | None = None):
        self.bytes, self.chunk = bytes_, chunk_bytes
        self.n_chunks = bytes_ // chunk_bytes
        self.owner = [-1] * self.n_chunks
        self.live: dict[int, int] = {}
        self.page_array_cap = page_array_cap
        nc = ceil_log2(chunk_bytes) - 4 + 1
        self.mallocs = [0] * nc
        self.frees = [0] * nc
        self.failed = [0] * nc

    def cls(self, n: int):
        if n == 0 or n > self.chunk:
            return None
        return max(0, ceil_log2(n) - 4)

    def page(self, c: int) -> int:
        return 16 * 2 ** c

    def chunk_has_free_page(self, x: int) -> bool:
        c = self.owner[x]
        base = x * self.chunk
        return any((base + p) not in self.live for p in range(0, self.chunk, self.page(c)))

    def class_has_free_page(self, c: int) -> bool:
        return any(self.owner[x] == c and self.chunk_has_free_page(x) for x in range(self.n_chunks))

    def can_take_chunk(self, c: int) -> bool:
        if -1 not in self.owner:
            return False
        if self.page_array_cap is not None:
            ppc = self.chunk // self.page(c)
            qc = min(self.bytes // self.page(c), self.page_array_cap)
            if (self.owner.count(c) + 1) * ppc > qc:
                return False
        return True

    def check_malloc(self, n: int, off: int) -> None:
        """Validate the allocator's answer `off` (-1 = null) to malloc(n)."""
        c = self.cls(n)
        if c is None:
            assert off == -1, f"malloc({n}) must be null"
            return
        if off == -1:
            assert not self.class_has_free_page(c), f"null for class {c} with a free page"
            assert not self.can_take_chunk(c), f"null for class {c} with a chunk left"
            self.failed[c] += 1
            return
        assert 0 <= off < self.bytes, "block outside the heap"
        assert off % self.page(c) == 0, "block not aligned to its class"
        assert off not in self.live, "block handed out twice"
        x = off // self.chunk
        if self.owner[x] == -1:
            assert not self.class_has_free_page(c), "new chunk taken while the class had a free page"
            assert self.can_take_chunk(c), "chunk taken beyond the queue capacity"
            self.owner[x] = c
        assert self.owner[x] == c, "block in a chunk of another class"
        end = off + self.page(c)
        for o, oc in self.live.items():
            assert end <= o or o + self.page(oc) <= off, "live blocks overlap"
        self.live[off] = c
        self.mallocs[c] += 1

    def expected_free_error(self, off: int) -> int:
        """0, 1 (bad free) or 2 (double free) for free(off)."""
        if off < 0 or off >= self.bytes:
            return 1
        x = off // self.chunk
        if self.owner[x] < 0 or off % self.page(self.owner[x]):
            return 1
        if off not in self.live:
            return 2
        return 0

    def free(self, off: int) -> None:
        c = self.live.pop(off)
        self.frees[c] += 1

    def trim(self) -> None:
        for x in range(self.n_chunks):
            if self.owner[x] >= 0 and not any(o // self.chunk == x for o in self.live):
                self.owner[x] = -1
