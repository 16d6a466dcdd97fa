"""Planted mistakes in the oracle must be caught by its pins.

Each mutant is a one-line change to a copy of oracle/ouro_oracle.c (a dropped
term, a wrong index, an off-by-one, a swapped operand), compiled on the CPU
into a temporary library.  The pins of tests/oracle_pins.py run against it and
at least one of them must fail.  The real oracle is never modified.
"""
import os
import subprocess
import sys
import tempfile

import pytest

import oracle
import oracle_pins as P

SRC = os.path.join(os.path.dirname(oracle.__file__), "ouro_oracle.c")
PY_SRC = os.path.join(os.path.dirname(oracle.__file__), "patterns.py")

MUTANTS = {
    "class_off_by_one": ("while (orc_page_bytes(c) < n) c++;", "while (orc_page_bytes(c) <= n) c++;"),
    "pages_per_chunk_halved": ("return h->chunk_bytes / orc_page_bytes(c);",
                               "return h->chunk_bytes / orc_page_bytes(c) / 2;"),
    "page_address_scale": ("off = id * pb;", "off = id * 16;"),
    "free_pushes_wrong_id": ("q_push(h, c, off / pb);", "q_push(h, c, off / 16);"),
    "chunk_not_requeued": ("if (h->free_pages[x] == 1) q_push(h, c, x);",
                           "if (h->free_pages[x] == 0) q_push(h, c, x);"),
    "trim_keeps_bump": ("while (np && pv[np - 1] == h->bump - 1) { np--; h->bump--; }", ""),
    "chunk_claims_wrong_bit": ("w[p >> 6] &= ~(1ull << (p & 63));", "w[p >> 6] &= ~(1ull << ((p + 1) & 63));"),
    "no_double_free_check": ("if (!live_get(h, off))", "if (0)"),
    "bump_past_end": ("if (h->bump < h->n_chunks) return", "if (h->bump <= h->n_chunks) return"),
    "page_array_cap_ignored": ("if ((h->carved_now[c] + 1) * ppc > qc) return -1;", ""),
    "segment_retired_early": ("const uint64_t keep = varray(h) ? 1 : 2;", "const uint64_t keep = 1;"),
    "varray_waits_for_successor": ("const uint64_t keep = varray(h) ? 1 : 2;", "const uint64_t keep = 2;"),
    "segment_retired_unconsumed": ("h->qhead[c] >= (h->seg_first[c] + 1) * h->seg_cap",
                                   "h->qhead[c] + 1 >= (h->seg_first[c] + 1) * h->seg_cap"),
    "trim_reclaims_partial": ("if (fr == ppc) reclaim[x] = 1;", "if (fr + 1 >= ppc) reclaim[x] = 1;"),
    "chunk_full_not_popped": ("if (h->free_pages[x] == 0) q_pop(h, c);", ""),
    "fmix_shift": ("x ^= x >> 13;", "x ^= x >> 12;"),
    "free_run_not_reused": ("  if (h->q[c].n == 0 && run_carve(h, c)) { h->failed[c]++; return -1; }",
                            "  if (run_carve(h, c)) { h->failed[c]++; return -1; }"),
    "run_overlaps_next": ("  h->bump += k;", "  h->bump += 1;"),
    "trim_keeps_free_runs": ("        h->chunk_cls[x + j] = CLS_NONE;", ""),
    "run_double_free_missed": ("    if (c >= CLS_RUN_FREE) { h->err |= ORC_ERR_DOUBLE_FREE; return ORC_ERR_DOUBLE_FREE; }", ""),
    "default_cap_2_24": ("h->queue_cap = queue_cap ? queue_cap : (1ull << 23);",
                         "h->queue_cap = queue_cap ? queue_cap : (1ull << 24);"),
    "pattern_key_without_gold": ("uint32_t key = orc_fmix32(seed ^ (tid * 0x9E3779B9u));",
                                 "uint32_t key = orc_fmix32(seed ^ tid);"),
    "pattern_step_dropped": ("return key + i * 0x9E3779B9u;", "return key + i;"),
    "pattern_mode0_off": ("if (mode == 0) return tid;", "if (mode == 0) return tid + 1;"),
    "tail_written_from_high_end": ("for (uint64_t j = 0; j < tail; j++) b[4 * nw + j] = (uint8_t)(v >> (8 * j));",
                                   "for (uint64_t j = 0; j < tail; j++) b[4 * nw + j] = (uint8_t)(v >> (24 - 8 * j));"),
    "tail_checked_from_high_end": ("uint8_t wb = (uint8_t)(v >> (8 * j));", "uint8_t wb = (uint8_t)(v >> (24 - 8 * j));"),
    "tail_folded_from_high_end": ("fold(res, v & (uint32_t)((1ull << (8 * tail)) - 1));",
                                  "fold(res, v >> (8 * (4 - tail)));"),
    "tail_word_index": ("uint32_t v = orc_pattern_word(seed, (uint32_t)t, (uint32_t)nw, 1);\n      fold(",
                        "uint32_t v = orc_pattern_word(seed, (uint32_t)t, (uint32_t)nw - 1, 1);\n      fold("),
}


def _build_mutant(name, old, new, tmpdir):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site of {name} not unique"
    path = os.path.join(tmpdir, f"ouro_oracle_{name}.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    # the mutant compiles beside a copy of the header
    with open(os.path.join(tmpdir, "ouro_oracle.h"), "w") as f:
        f.write(open(SRC.replace(".c", ".h")).read())
    lib = os.path.join(tmpdir, f"lib_{name}.so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-w", "-shared", "-fPIC", "-o", lib, path], check=True)
    return lib


_RUNNER = """
import sys
sys.path[:0] = [{root!r}, {tests!r}]
import oracle_pins as P
pin = getattr(P, {pin!r})
if {pin!r} == "pin_brute_force":
    pin({lib!r}, max_len=3, random_runs=25, random_len=200)
else:
    pin({lib!r})
"""


def _pin_fails(pin_name, lib):
    """Run one pin in a child process: a planted mistake may crash or loop."""
    tests = os.path.dirname(os.path.abspath(__file__))
    code = _RUNNER.format(root=os.path.dirname(tests), tests=tests, pin=pin_name, lib=lib)
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, timeout=120)
    except subprocess.TimeoutExpired:
        return True
    return r.returncode != 0


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    old, new = MUTANTS[name]
    with tempfile.TemporaryDirectory() as d:
        lib = _build_mutant(name, old, new, d)
        caught = next((p.__name__ for p in P.ALL_PINS if _pin_fails(p.__name__, lib)), None)
        assert caught, f"mutant {name} passed every pin"


# planted mistakes in the oracle of the added patterns (oracle/patterns.py);
# each must fail its pin (run in a child process against the mutated module)
PY_MUTANTS = {
    "admit_overtakes": ("                break\n            admit[nxt] = step",
                        "                nxt += 1\n                continue\n            admit[nxt] = step", "pin_serving_schedule"),
    "admit_ignores_slots": (" or active >= n_slots:", ":", "pin_serving_schedule"),
    "admit_cap_strict": ("committed + need > cap_blocks", "committed + need >= cap_blocks", "pin_serving_schedule"),
    "complete_one_late": ("completing.setdefault(step + need - 1, [])", "completing.setdefault(step + need, [])",
                          "pin_serving_schedule"),
    "complete_keeps_blocks": ("            committed -= int(blocks[s])\n", "", "pin_serving_schedule"),
    "complete_keeps_slot": ("            active -= 1\n", "", "pin_serving_schedule"),
    "grown_past_size": ("np.minimum(blocks[on].astype(np.int64), steps - admit[on])", "steps - admit[on]",
                        "pin_serving_schedule"),
    "growth_stops_early": ("while cap < min(d, max_plain):", "while cap < min(d, max_plain // 2):", "pin_graph_counts"),
    "growth_frees_new_class": ("frees[_class_of_entries(cap)] += 1\n            cap *= 2",
                               "cap *= 2\n            frees[_class_of_entries(cap)] += 1", "pin_graph_counts"),
    "segment_without_link": ("    seg_cap = (chunk_bytes - 8) // 4\n    mallocs =", "    seg_cap = chunk_bytes // 4\n    mallocs =",
                             "pin_graph_counts"),
    "segments_floor": ("(over + seg_cap - 1) // seg_cap", "over // seg_cap", "pin_graph_counts"),
}

_PY_RUNNER = """
import importlib.util, sys
sys.path[:0] = [{root!r}, {tests!r}]
import oracle, oracle_pins as P
spec = importlib.util.spec_from_file_location("mutant_patterns", {path!r})
mod = importlib.util.module_from_spec(spec)
spec.loader.exec_module(mod)
getattr(P, {pin!r})(oracle.ensure_built(), mod)
"""


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_pattern_mutant_is_caught(name):
    old, new, pin = PY_MUTANTS[name]
    src = open(PY_SRC).read()
    assert src.count(old) == 1, f"mutation site of {name} not unique"
    tests = os.path.dirname(os.path.abspath(__file__))
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "patterns_mutant.py")
        with open(path, "w") as f:
            f.write(src.replace(old, new))
        code = _PY_RUNNER.format(root=os.path.dirname(tests), tests=tests, path=path, pin=pin)
        try:
            r = subprocess.run([sys.executable, "-c", code], capture_output=True, timeout=120)
        except subprocess.TimeoutExpired:
            return
        assert r.returncode != 0, f"mutant {name} passed {pin}"
