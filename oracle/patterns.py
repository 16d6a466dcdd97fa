"""Oracle of the two added usage patterns: serving admission and graph growth.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may import it.
The product package never does.

Neither pattern is in the paper (arXiv 2504.18211); both are workloads built
on its allocator (an in-kernel malloc/free from a host-preallocated heap,
Sec. 1).  What each function computes is the stated rule of the workload,
run one step or one request at a time:

  serving_schedule      admission and completion step of every session
                        (arrival order, a free slot, committed blocks within
                        the cap; one block per active session per step)
  graph_class_counts    per-class malloc / free totals of the list-growth
                        rule, in closed form from the final degrees
  graph_growth_run      the same rule applied edge by edge to an oracle heap
                        (sequential malloc / copy / free), whose own counters
                        then give the totals
"""
from __future__ import annotations

import numpy as np


def serving_schedule(arrive: np.ndarray, blocks: np.ndarray, steps: int, n_slots: int, cap_blocks: int):
    """Admission rule of the serving loop, one step at a time.

    At the start of step t, sessions are admitted in arrival order while the
    next one has arrived (arrive <= t), a session slot is free and the
    committed blocks plus the newcomer's whole size stay within cap_blocks;
    the first session that does not fit stops admission for the step (no
    overtaking).  Then every active session grows by one block; a session
    that reaches its size completes in that step, frees its blocks and its
    slot, which count from the next step on.  Since an active session grows
    one block in every step, a session of b blocks admitted at step a
    completes at step a + b - 1.

    Returns (admit step, completion step, blocks grown) per session; -1 for
    a session never admitted / never completed."""
    n = int(arrive.size)
    admit = np.full(n, -1, np.int64)
    done = np.full(n, -1, np.int64)
    grown = np.zeros(n, np.int64)
    completing = {}          # step -> sessions that complete in it
    active = 0
    nxt = 0
    committed = 0
    for step in range(steps):
        while nxt < n:
            need = int(blocks[nxt])
            if int(arrive[nxt]) > step or committed + need > cap_blocks or active >= n_slots:
                break
            admit[nxt] = step
            committed += need
            active += 1
            completing.setdefault(step + need - 1, []).append(nxt)
            nxt += 1
        for s in completing.pop(step, []):
            done[s] = step
            committed -= int(blocks[s])
            active -= 1
    on = admit >= 0
    grown[on] = np.minimum(blocks[on].astype(np.int64), steps - admit[on])
    return admit, done, grown


def _class_of_entries(entries: int) -> int:
    """Class of a list of `entries` 4-byte entries (a power of two >= 4)."""
    c = 0
    while (16 << c) < 4 * entries:
        c += 1
    return c


def graph_class_counts(deg: np.ndarray, chunk_bytes: int, n_classes: int, max_classes: int = 17):
    """Allocator traffic of the list-growth rule, from the final degrees.

    Every vertex starts with a list of 4 entries (16 B, class 0).  While a
    list is below one chunk (chunk_bytes / 4 entries) and full, an append
    allocates a list of twice the entries and frees the old one.  Entries
    past one chunk go to overflow segments of one chunk each, holding
    (chunk_bytes - 8) / 4 entries behind an 8-byte link; a segment is
    allocated when the previous one is full.  Lists are not freed.

    Returns (mallocs per class, frees per class, final list entries), the
    per-class arrays padded to max_classes."""
    max_plain = chunk_bytes // 4
    seg_cap = (chunk_bytes - 8) // 4
    mallocs = np.zeros(max_classes, np.int64)
    frees = np.zeros(max_classes, np.int64)
    caps = np.zeros(deg.size, np.int64)
    for v, d in enumerate(deg.astype(np.int64).tolist()):
        cap = 4
        mallocs[0] += 1
        while cap < min(d, max_plain):
            frees[_class_of_entries(cap)] += 1
            cap *= 2
            mallocs[_class_of_entries(cap)] += 1
        over = max(d - max_plain, 0)
        mallocs[n_classes - 1] += (over + seg_cap - 1) // seg_cap
        caps[v] = cap
    return mallocs, frees, caps


def graph_growth_run(heap, src: np.ndarray, n_vertices: int, chunk_bytes: int):
    """The growth rule run edge by edge on an oracle heap (oracle.OracleHeap):
    a 16 B list per vertex, then for each edge in order an append to its
    source's list -- allocate twice the entries and free the old list when a
    list below one chunk is full, allocate a one-chunk overflow segment when
    the list and its last segment are full.  Returns the heap's stats after
    the last edge (lists stay live) and the degree of every vertex."""
    max_plain = chunk_bytes // 4
    seg_cap = (chunk_bytes - 8) // 4
    lists = [heap.malloc(16) for _ in range(n_vertices)]
    cap = [4] * n_vertices
    deg = [0] * n_vertices
    seg_fill = [seg_cap] * n_vertices      # entries in the newest overflow segment (full: none open)
    for s in src.tolist():
        if deg[s] < max_plain:
            if deg[s] == cap[s]:
                new = heap.malloc(8 * cap[s])
                assert new >= 0 and heap.free(lists[s]) == 0
                lists[s] = new
                cap[s] *= 2
        else:
            if seg_fill[s] == seg_cap:
                assert heap.malloc(chunk_bytes) >= 0
                seg_fill[s] = 0
            seg_fill[s] += 1
        deg[s] += 1
    return heap.stats(), np.array(deg, np.int64)
