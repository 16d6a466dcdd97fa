"""A trivially correct set-allocator used to pin the oracle by brute force.

It knows nothing about queues: it keeps the set of live blocks and, per chunk,
the size class the chunk was given.  A request of class c can be served iff
some chunk of class c still has a page that is not live, or a chunk that no
class owns is left (and, for page-array queues, the class still has room
under its queue capacity).  The allocator must take a new chunk only when the
first condition fails.

Classes above one chunk are runs of 2^(c - C + 1) contiguous chunks (C =
classes within a chunk): a run that is owned but not live must be reused
before a new one is cut, and a new run starts at the frontier -- one past the
highest owned chunk -- where contiguous free chunks are certain.  Nothing here
is shared with the oracle.
"""
from __future__ import annotations


def ceil_log2(n: int) -> int:
    return (n - 1).bit_length()


MAX_REQUEST = 1 << 20
ALL_CLASSES = 17


class SetModel:
    def __init__(self, bytes_: int, chunk_bytes: int, page_array_cap: int | None = None,
                 strict_frontier: bool = True):
        self.bytes, self.chunk = bytes_, chunk_bytes
        self.n_chunks = bytes_ // chunk_bytes
        self.owner = [-1] * self.n_chunks
        self.live: dict[int, int] = {}
        self.run_start: dict[int, int] = {}      # first chunk of each owned run -> class
        self.page_array_cap = page_array_cap
        # strict_frontier=False: the allocator may own chunks this model does
        # not see (queue segments), so a new run may start above the frontier
        self.strict_frontier = strict_frontier
        self.C = ceil_log2(chunk_bytes) - 4 + 1
        self.mallocs = [0] * ALL_CLASSES
        self.frees = [0] * ALL_CLASSES
        self.failed = [0] * ALL_CLASSES

    def cls(self, n: int):
        if n == 0 or n > MAX_REQUEST:
            return None
        return max(0, ceil_log2(n) - 4)

    def run_chunks(self, c: int) -> int:
        return self.page(c) // self.chunk

    def frontier(self) -> int:
        owned = [x for x in range(self.n_chunks) if self.owner[x] >= 0]
        return max(owned) + 1 if owned else 0

    def free_run_of(self, c: int) -> bool:
        return any(rc == c and x * self.chunk not in self.live for x, rc in self.run_start.items())

    def check_run_malloc(self, c: int, off: int) -> None:
        k = self.run_chunks(c)
        if off == -1:
            assert not self.free_run_of(c), f"null for class {c} with a free run"
            if self.strict_frontier:
                assert self.frontier() + k > self.n_chunks, f"null for class {c} with room at the frontier"
            self.failed[c] += 1
            return
        assert 0 <= off < self.bytes and off % self.chunk == 0, "run not at a chunk start"
        assert off not in self.live, "run handed out twice"
        x = off // self.chunk
        if x in self.run_start:
            assert self.run_start[x] == c, "run of another class"
        else:
            assert not self.free_run_of(c), "new run cut while the class had a free run"
            if self.strict_frontier:
                assert x == self.frontier(), "new run not at the frontier"
            assert x + k <= self.n_chunks, "run past the heap"
            assert all(self.owner[x + i] == -1 for i in range(k)), "run over owned chunks"
            for i in range(k):
                self.owner[x + i] = c
            self.run_start[x] = c
        end = off + self.page(c)
        for o, oc in self.live.items():
            assert end <= o or o + self.page(oc) <= off, "live blocks overlap"
        self.live[off] = c
        self.mallocs[c] += 1

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
        if c >= self.C:
            self.check_run_malloc(c, off)
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
        if self.owner[x] >= self.C:
            if x not in self.run_start or off % self.chunk:
                return 1
            return 0 if off in self.live else 2
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
            if 0 <= self.owner[x] < self.C and not any(o // self.chunk == x for o in self.live):
                self.owner[x] = -1
        for x, c in list(self.run_start.items()):
            if x * self.chunk not in self.live:
                for i in range(self.run_chunks(c)):
                    self.owner[x + i] = -1
                del self.run_start[x]
