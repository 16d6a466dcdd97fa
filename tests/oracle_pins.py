"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Each pin takes the path of an oracle build so that the mutation test can run
the same pins against deliberately broken builds (tests/test_oracle_mutants.py).

What pins what:
  class map          closed form ceil(log2 n) - 4 over every n in [0, chunk+1] and
                     past it up to 1 MiB (runs of chunks), null above
  layout / address   a single-class fill of a tiny heap returns exactly the
                     multiples of the page size in [0, bytes)
  capacity           closed form n_chunks * chunk / page; page-array limit
                     floor(min(bytes/page, cap) / ppc) * ppc; runs: floor(n_chunks / k)
                     and freed runs reused before the bump pointer moves
  queue semantics    brute force against a set allocator (tests/setmodel.py)
  small workload     closed form of the 10,240 x 16 B run (tests/golden/c0_small.json)
  restore            free everything, trim: the state equals the post-create state
  queue segments     closed form of segment use for a fill that ends on a segment edge
  fmix32             MurmurHash3 reference vectors (tests/golden/murmur3_fmix32.json)
  written data       hand-worked words, tail bytes and checksums of the driver round
                     (tests/golden/pattern_words.json)
  default capacity   the page-array limit at default options is the documented 2^23
  serving admission  hand-worked schedules (binding cap, full slot table, late arrival)
  graph growth       hand-worked per-class counts, and the rule run request by request
                     on the oracle heap
"""
from __future__ import annotations

import ctypes
import itertools
import json
import os

import numpy as np

import oracle
from setmodel import SetModel, ceil_log2

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
ALL_VARIANTS = ("page_array", "chunk_array", "page_vlist", "chunk_vlist", "page_varray", "chunk_varray")


def plain_array(variant):
    """Plain array queues hold their storage outside the heap."""
    return variant in ("page_array", "chunk_array")


def heap(lib_path, bytes_, chunk, variant, cap=0):
    return oracle.OracleHeap(bytes_, chunk, variant, cap, lib_path=lib_path)


def pin_class_map(lib_path):
    lib = oracle.load(lib_path)
    for chunk in (256, 1024, 8192, 65536, 1 << 20):
        assert lib.orc_num_classes(chunk) == ceil_log2(chunk) - 3
        assert lib.orc_num_large(chunk) == 17 - (ceil_log2(chunk) - 3)
        ns = list(range(0, chunk + 2)) if chunk <= 65536 else list(range(0, 4097))
        ns += [chunk - 1, chunk, chunk + 1] + [2 ** k + d for k in range(5, 21) for d in (-1, 0, 1)]
        for n in ns:
            c = lib.orc_size_class(chunk, n)
            if n == 0 or n > (1 << 20):
                assert c == -1, (chunk, n, c)
            else:
                assert c == max(0, ceil_log2(n) - 4), (chunk, n, c)
                pb = lib.orc_page_bytes(c)
                assert pb >= n and (pb == 16 or pb // 2 < n)


def pin_layout(lib_path):
    """Every class of every variant: filling a tiny heap with one class hands
    out each page-aligned block exactly once and then returns null."""
    for variant in ALL_VARIANTS:
        for chunk in (256, 512):
            bytes_ = 8 * chunk
            for c in range(ceil_log2(chunk) - 3):
                page = 16 << c
                h = heap(lib_path, bytes_, chunk, variant)
                offs = []
                while True:
                    o = h.malloc(page)
                    if o < 0:
                        break
                    offs.append(o)
                    assert len(offs) <= bytes_ // page
                st = h.stats()
                if plain_array(variant):
                    assert sorted(offs) == list(range(0, bytes_, page)), (variant, chunk, c)
                else:
                    # queue segments take whole chunks out of the same heap
                    segs = st["seg_chunks"] + st["spare_chunks"]
                    assert segs >= 1
                    assert len(offs) == (bytes_ // chunk - segs) * (chunk // page), (variant, c)
                    assert len(set(offs)) == len(offs)
                    assert all(o % page == 0 for o in offs)
                assert st["mallocs"][c] == len(offs) and st["failed"][c] == 1
                assert st["carved_now"][c] * (chunk // page) == len(offs)


def pin_capacity(lib_path):
    # plain capacity: n_chunks * pages per chunk
    for variant in ("page_array", "chunk_array"):
        h = heap(lib_path, 64 * 1024, 1024, variant)
        got = sum(1 for _ in range(5000) if h.malloc(48) >= 0)
        assert got == (64 * 1024) // 64, (variant, got)
    # page-array queue capacity min(bytes/page, cap), rounded down to whole chunks
    for cap in (100, 512, 1000, 4096):
        h = heap(lib_path, 64 * 1024, 1024, "page_array", cap)
        got = sum(1 for _ in range(5000) if h.malloc(16) >= 0)
        qc = min(64 * 1024 // 16, cap)
        assert got == (qc // 64) * 64, (cap, got)
    # runs above one chunk: 3000 B on 1 KiB chunks is a 4 KiB run of 4 chunks
    # (class 8); 64 chunks hold floor(64 / 4) = 16 runs, each at the next bump
    # position; freed runs are reused in the order they were freed, without
    # moving the bump (plain array queues: the heap holds no queue segments)
    for variant in ("page_array", "chunk_array"):
        h = heap(lib_path, 64 * 1024, 1024, variant)
        offs = [h.malloc(3000) for _ in range(20)]
        assert offs[:16] == [4096 * i for i in range(16)] and offs[16:] == [-1] * 4, (variant, offs)
        st = h.stats()
        assert st["mallocs"][8] == 16 and st["failed"][8] == 4 and st["carved_now"][8] == 64, (variant, st)
        for o in offs[15::-1]:
            assert h.free(o) == 0
        assert h.free(offs[3]) == oracle.ERR_DOUBLE_FREE and h.free(offs[3] + 1024) == oracle.ERR_BAD_FREE
        again = [h.malloc(2049) for _ in range(16)]         # 2049 B: the same class
        assert again == offs[15::-1], (variant, again)
        assert h.stats()["bump"] == 64 and h.malloc(16) == -1
    # the page-array limit at default options is the library's documented
    # default, 2^23 items per class (include/ouro.h): a 256 MiB heap holds
    # 2^24 pages of 16 B, of which exactly 2^23 are served
    h = heap(lib_path, 256 << 20, 8192, "page_array")
    res = h.round(np.full((1 << 23) + 1000, 16, np.uint32), seed=0, mode=1, with_memory=False)
    assert res["nulls"] == 1000, res
    st = h.stats()
    assert st["mallocs"][0] == 1 << 23 and st["failed"][0] == 1000 and st["carves"][0] == (1 << 23) // 512, st


def _run_sequence(lib_path, variant, bytes_, chunk, ops, model_nulls=True):
    """Apply ops to the oracle and the set model; compare after every op.
    model_nulls=False (virtualized queues, whose segments hold chunks of the
    same heap): blocks and counts are checked, null answers only counted."""
    h = heap(lib_path, bytes_, chunk, variant)
    m = SetModel(bytes_, chunk, strict_frontier=model_nulls)
    order = []   # live offsets in allocation order
    freed = []   # offsets freed at least once
    for op, arg in ops:
        if op == "m":
            o = h.malloc(arg)
            c = m.cls(arg)
            if o >= 0 or model_nulls or c is None:
                m.check_malloc(arg, o)
            else:
                m.failed[c] += 1
            if o >= 0:
                order.append(o)
        elif op == "f":
            if not order:
                continue
            o = order.pop(arg % len(order))
            assert h.free(o) == 0
            m.free(o)
            freed.append(o)
        elif op == "d":     # free a block a second time (unless it was handed out again)
            if not freed:
                continue
            o = freed[arg % len(freed)]
            want = m.expected_free_error(o)
            if want:
                assert h.free(o) == want, (o, want)
        elif op == "x":     # a pointer that is not a block start
            want = m.expected_free_error(arg)
            assert h.free(arg) == want, (arg, want)
        elif op == "t":
            h.trim()
            m.trim()
        st = h.stats()
        if st["error_bits"] & oracle.ERR_QUEUE_FULL:
            # a virtualized queue found no chunk for a segment and dropped the
            # freed page: the set model no longer applies from here on
            assert not model_nulls
            return h, m
        for c in range(len(m.mallocs)):
            assert st["mallocs"][c] == m.mallocs[c]
            assert st["frees"][c] == m.frees[c]
            assert st["failed"][c] == m.failed[c]
            assert st["live"][c] == m.mallocs[c] - m.frees[c]
            assert st["carved_now"][c] == m.owner.count(c)
    return h, m


def pin_brute_force(lib_path, max_len=4, random_runs=60, random_len=250):
    sizes = (0, 1, 16, 17, 33, 100, 256, 257)
    alphabet = [("m", s) for s in sizes] + [("f", 0), ("f", 1), ("d", 0), ("x", 8), ("x", 1 << 20),
                                            ("t", 0)]
    for variant in ("page_array", "chunk_array"):
        for L in range(1, max_len + 1):
            for ops in itertools.product(alphabet, repeat=L):
                _run_sequence(lib_path, variant, 2 * 256, 256, ops)
    rng = np.random.default_rng(20250424)
    for variant in ALL_VARIANTS:
        nulls = plain_array(variant)
        for _ in range(random_runs):
            ops = []
            for _ in range(random_len):
                r = rng.random()
                if r < 0.55:
                    ops.append(("m", int(rng.choice([1, 16, 20, 32, 50, 64, 120, 128, 200, 256, 300, 700, 1100]))))
                elif r < 0.90:
                    ops.append(("f", int(rng.integers(0, 1000))))
                elif r < 0.93:
                    ops.append(("d", int(rng.integers(0, 1000))))
                elif r < 0.97:
                    ops.append(("x", int(rng.integers(0, 4 * 256)) | 1))
                else:
                    ops.append(("t", 0))
            chunk, nch = (256, 6) if nulls else (512, 12)
            _run_sequence(lib_path, variant, nch * chunk, chunk, ops, model_nulls=nulls)


def pin_small_workload(lib_path):
    g = json.load(open(os.path.join(GOLDEN, "c0_small.json")))
    h = heap(lib_path, g["heap_bytes"], g["chunk_bytes"], "page_array")
    sizes = np.full(g["threads"], g["request_bytes"], np.uint32)
    res, offs = h.round(sizes, seed=0, mode=0, return_offsets=True)
    st = h.stats()
    assert res["nulls"] == 0 and res["mismatches"] == 0
    assert res["xor64"] == g["xor_of_thread_ids"] and res["sum64"] == g["sum_of_thread_ids"]
    assert st["carves"][g["class"]] == g["chunks_carved"]
    assert st["queued"][g["class"]] == g["queued_after_free_all"]
    assert sorted(offs.tolist()) == list(range(0, g["threads"] * 16, 16))
    assert st["mallocs"][0] == st["frees"][0] == g["threads"] and st["live"][0] == 0


def _post_create(lib_path, variant, bytes_, chunk):
    return heap(lib_path, bytes_, chunk, variant).canonical_state()


def _same_state(a, b):
    assert a["bump"] == b["bump"], (a["bump"], b["bump"])
    assert np.array_equal(a["pool"], b["pool"])
    assert np.array_equal(a["chunk_cls"], b["chunk_cls"])
    for qa, qb in zip(a["queues"], b["queues"]):
        assert np.array_equal(qa, qb)


def pin_restore(lib_path):
    rng = np.random.default_rng(7)
    for variant in ALL_VARIANTS:
        bytes_, chunk = 8 << 20, 4096        # roomy: no request fails, no segment is refused
        h = heap(lib_path, bytes_, chunk, variant)
        live = []
        for _ in range(3000):
            if rng.random() < 0.6 or not live:
                n = int(rng.integers(1, chunk + 1)) if rng.random() < 0.9 else int(rng.integers(chunk + 1, 4 * chunk))
                o = h.malloc(n)
                assert o >= 0
                if o >= 0:
                    live.append(o)
            else:
                assert h.free(live.pop(int(rng.integers(0, len(live))))) == 0
        rng.shuffle(live)
        for o in live:
            assert h.free(o) == 0
        h.trim()
        st = h.stats()
        assert sum(st["live"]) == 0 and st["error_bits"] == 0
        _same_state(h.canonical_state(), _post_create(lib_path, variant, bytes_, chunk))
    # a partial trim keeps live chunks and returns only the all-free ones
    h = heap(lib_path, 64 * 4096, 4096, "page_array")
    a = [h.malloc(16) for _ in range(256 * 3)]          # three chunks of class 0
    for o in a[256:]:
        h.free(o)
    h.trim()
    st = h.stats()
    assert st["carved_now"][0] == 1 and st["queued"][0] == 0 and st["bump"] == 1


def pin_segments(lib_path):
    """Virtualized queue storage (Sec. 4.3) under the stated rule: a segment is
    one chunk holding (chunk - 64) / 8 cells, and it retires once every
    position in it was consumed -- in the list form only when a successor
    exists too.  Closed form with 512 B chunks (56 cells) and 64 B requests
    (8 pages per chunk): 56 requests use 7 data chunks and exactly fill
    segment 0; the 57th needs segment 1.
      list:  segment 0 stays (no successor) -> (1 live, 0 spare, bump 8);
             the 57th links segment 1 (chunk 8), carves chunk 9, then
             segment 0 retires -> (1, 1, 10).
      array: segment 0 retires with its last consumer -> (0, 1, 8); the 57th
             reuses it as segment 1 and carves chunk 8 -> (1, 0, 9)."""
    for variant, after56, after57 in (("page_vlist", (1, 0, 8), (1, 1, 10)),
                                      ("page_varray", (0, 1, 8), (1, 0, 9))):
        h = heap(lib_path, 64 * 512, 512, variant)
        for _ in range(55):
            assert h.malloc(64) >= 0
        st = h.stats()      # one position of segment 0 is still unconsumed: it stays
        assert (st["seg_chunks"], st["spare_chunks"], st["bump"]) == (1, 0, 8), (variant, st)
        assert h.malloc(64) >= 0
        st = h.stats()
        assert (st["seg_chunks"], st["spare_chunks"], st["bump"]) == after56, (variant, st)
        assert h.malloc(64) >= 0
        st = h.stats()
        assert (st["seg_chunks"], st["spare_chunks"], st["bump"]) == after57, (variant, st)
    # chunk queues hold one position per carved chunk: 56 chunks of one class
    # fill segment 0 exactly (heap of 64 chunks of 512 B, requests of 512 B)
    for variant, after56 in (("chunk_vlist", (1, 0, 57)), ("chunk_varray", (0, 1, 57))):
        h = heap(lib_path, 64 * 512, 512, variant)
        for _ in range(56):
            assert h.malloc(512) >= 0
        st = h.stats()
        assert (st["seg_chunks"], st["spare_chunks"], st["bump"]) == after56, (variant, st)


def pin_pattern(lib_path):
    """The written data of the driver round against the hand-worked cases of
    tests/golden/pattern_words.json (keys from the MurmurHash3 vectors):
    the words of mode 1, the tail bytes of sizes that are not a multiple of
    4 (the low bytes of the next word, little-endian), the XOR / sum folds
    of the checksum, the bytes the round leaves in memory, and mode 0's
    thread id in word 0."""
    lib = oracle.load(lib_path)
    g = json.load(open(os.path.join(GOLDEN, "pattern_words.json")))
    gold = int(g["gold"], 16)
    for c in g["mode1"]:
        seed, tid, key, size = int(c["seed"], 16), c["tid"], int(c["key"], 16), c["size"]
        want = bytes.fromhex(c["bytes"])
        assert len(want) == size
        for i in range(size // 4):
            assert lib.orc_pattern_word(seed, tid, i, 1) == int.from_bytes(want[4 * i:4 * i + 4], "little"), c
        assert lib.orc_pattern_word(seed, tid, 0, 1) == key, c
        assert lib.orc_pattern_word(seed, tid, 5, 1) == (key + 5 * gold) & 0xFFFFFFFF, c
        sizes = np.array([size] if tid == 0 else [0] * tid + [size], np.uint32)
        exp = {"xor64": c["xor64"], "sum64": c["sum64"], "words": c["words"]}
        r = oracle.RoundResult()
        lib.orc_expected_checksums(sizes.ctypes.data_as(ctypes.c_void_p), sizes.size, seed, 1, ctypes.byref(r))
        assert {k: v for k, v in r.as_dict().items() if k in exp} == exp, (c, r.as_dict())
        h = heap(lib_path, 1 << 16, 1024, "page_array")
        res, offs, mem = h.round(sizes, seed=seed, mode=1, return_memory=True)
        assert res["mismatches"] == 0 and res["nulls"] == tid, (c, res)
        assert {k: v for k, v in res.items() if k in exp} == exp, (c, res)
        o = int(offs[tid])
        assert bytes(mem[o:o + size]) == want, (c, bytes(mem[o:o + size]).hex())
        assert not mem[o + size:o + 16 * ((size + 15) // 16)].any()     # nothing past the request
    m0 = g["mode0"]
    sizes = np.array(m0["sizes"], np.uint32)
    h = heap(lib_path, 1 << 16, 1024, "page_array")
    res, offs, mem = h.round(sizes, seed=int(m0["seed"], 16), mode=0, return_memory=True)
    assert (res["xor64"], res["sum64"], res["words"], res["mismatches"]) == (m0["xor64"], m0["sum64"], m0["words"], 0)
    for t, o in enumerate(offs):
        assert int.from_bytes(bytes(mem[o:o + 4]), "little") == m0["word0"][t] and not mem[o + 4:o + 16].any()


def _patterns(mod):
    if mod is None:
        from oracle import patterns as mod
    return mod


def pin_serving_schedule(lib_path, mod=None):
    """The serving admission rule against hand-worked schedules.
    (a) 2 slots, cap 10 blocks; sessions (arrive, blocks) = (0,3) (0,4)
        (0,5) (1,2).  Step 0 admits s0, s1 (7 committed); s2 would make 12
        and blocks s3 behind it.  s0 completes at step 2 (4 committed); at
        step 3 s2 fits (9) and s1 completes (5); at step 4 s3 fits (7);
        s3 completes at step 5, s2 at step 7.
    (b) 1 slot, cap 100: (0,2) (0,1): s1 waits for the slot; s0 completes
        at step 1, s1 is admitted at step 2 and completes there.
    (c) a late arrival (5,1) is admitted at step 5; a session larger than
        the cap is never admitted and blocks every later one.
    (d) (0,4) (0,6) under cap 10 fill it exactly: both are admitted at 0.
    (e) sessions still growing at the last step have no completion."""
    m = _patterns(mod)
    a, d, k = m.serving_schedule(np.array([0, 0, 0, 1]), np.array([3, 4, 5, 2]), 10, 2, 10)
    assert a.tolist() == [0, 0, 3, 4] and d.tolist() == [2, 3, 7, 5] and k.tolist() == [3, 4, 5, 2], (a, d, k)
    a, d, k = m.serving_schedule(np.array([0, 0]), np.array([2, 1]), 4, 1, 100)
    assert a.tolist() == [0, 2] and d.tolist() == [1, 2], (a, d)
    a, d, k = m.serving_schedule(np.array([5, 5, 6]), np.array([1, 11, 1]), 9, 4, 10)
    assert a.tolist() == [5, -1, -1] and d.tolist() == [5, -1, -1] and k.tolist() == [1, 0, 0], (a, d, k)
    a, d, k = m.serving_schedule(np.array([0, 0]), np.array([4, 6]), 8, 4, 10)     # exactly at the cap
    assert a.tolist() == [0, 0] and d.tolist() == [3, 5], (a, d)
    a, d, k = m.serving_schedule(np.array([0, 0]), np.array([3, 3]), 2, 4, 10)
    assert a.tolist() == [0, 0] and d.tolist() == [-1, -1] and k.tolist() == [2, 2], (a, d, k)


def pin_graph_counts(lib_path, mod=None):
    """The list-growth rule's allocator traffic against a hand-worked case
    and against the same rule run request by request on an oracle heap.
    Hand-worked, 256 B chunks (lists up to 64 entries, overflow segments of
    (256 - 8) / 4 = 62 entries, 5 classes 16..256 B), final degrees 0, 4, 5,
    9, 64, 65, 200: seven 16 B lists; doublings 4->8 for degrees 5, 9, 64,
    65, 200, 8->16 for 9 and up, 16->32 and 32->64 for 64 and up; overflow
    segments 0 + 1 + ceil(136 / 62) = 4 more 256 B blocks."""
    m = _patterns(mod)
    deg = np.array([0, 4, 5, 9, 64, 65, 200])
    mal, fre, cap = m.graph_class_counts(deg, 256, 5)
    assert mal[:5].tolist() == [7, 5, 4, 3, 3 + 4] and not mal[5:].any(), mal
    assert fre[:5].tolist() == [5, 4, 3, 3, 0] and not fre[5:].any(), fre
    assert cap.tolist() == [4, 4, 8, 16, 64, 64, 64], cap
    # the rule run edge by edge on the oracle heap (its own counters)
    rng = np.random.default_rng(11)
    for chunk, nv, ne in ((256, 40, 3000), (1024, 64, 6000)):
        src = (rng.zipf(1.6, ne) - 1) % nv
        h = heap(lib_path, 4 << 20, chunk, "page_array")
        st, d = m.graph_growth_run(h, src, nv, chunk)
        assert d.max() > chunk // 4 + (chunk - 8) // 4          # several overflow segments
        mal, fre, _ = m.graph_class_counts(d, chunk, h.n_classes)
        assert st["mallocs"] == mal[:len(st["mallocs"])].tolist(), (chunk, st["mallocs"], mal)
        assert st["frees"] == fre[:len(st["frees"])].tolist(), (chunk, st["frees"], fre)


def pin_fmix32(lib_path):
    lib = oracle.load(lib_path)
    g = json.load(open(os.path.join(GOLDEN, "murmur3_fmix32.json")))
    for v in g["vectors"]:
        assert lib.orc_fmix32(int(v["seed"], 16)) == int(v["hash"], 16)


ALL_PINS = (pin_class_map, pin_layout, pin_capacity, pin_brute_force, pin_small_workload,
            pin_restore, pin_segments, pin_fmix32, pin_pattern, pin_serving_schedule, pin_graph_counts)
