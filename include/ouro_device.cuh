/*
 * ouro_device.cuh -- device-side ouro_malloc / ouro_free (sm_103a).
 *
 * Include from any kernel; pass the heap's ouro_heap_dev (ouro_heap_device())
 * by value.  Any subset of a warp may call in divergent code.  Results are
 * aligned to their power-of-two class (at least 16 B).  No call traps or
 * waits without bound: a wait that runs out answers null and sets
 * OURO_ERR_TIMEOUT in the heap's error word.
 *
 * Method (arXiv 2504.18211, which ports Ouroboros):
 *   - one preallocated heap cut into chunks; requests are served as pages
 *     of a chunk, through one lock-free queue per power-of-two size
 *     (Sec. 1; Sec. 4 preamble; Sec. 4.2);
 *   - page queues hand out fixed-size pages (Sec. 4.1);
 *   - virtualized queues keep their slots inside heap chunks (Sec. 4.3);
 *   - lanes of a warp that ask for the same size are served together by one
 *     queue operation, with the active mask deciding who takes part
 *     (Sec. 2, warp votes masked by the active mask);
 *   - waiting threads are throttled with nanosleep (Sec. 2).
 *
 * GB300 design (not in the paper):
 *   - a queue slot is one 64-bit word {sequence, item}; positions come from
 *     two monotone 64-bit counters (head for consumers, tail for producers),
 *     so a warp group needs ONE atomic on head (malloc) or tail (free) and its
 *     lanes then touch consecutive slots (coalesced);
 *   - a consumer whose position is beyond the producers is "in debt": the
 *     one lane per class that takes the class carve lock carves the chunks
 *     the current debt needs, at most 4096 pages' worth, releases the lock
 *     and its whole warp writes the new page ids into the slots, so that
 *     other warps in debt carve and fill the rest at the same time;
 *   - when the heap has no chunk left, the remaining debt positions are
 *     answered with a null marker, so a full heap returns null exactly as
 *     often as a sequential allocator would in a malloc-only phase.
 */
#ifndef OURO_DEVICE_CUH
#define OURO_DEVICE_CUH

#include <cuda_runtime.h>
#include <stdint.h>

#include "ouro.h"

#define OURO_NIL 0xFFFFFFFFu
#define OURO_BUSY 0xFFFFFFFEu   /* successor segment being created by one thread */
#define OURO_CLS_NONE 0xFFu
#define OURO_CLS_SEG 0xFEu
#define OURO_CLS_RUN_FREE 0x40u   /* | class: first chunk of a free run (on its class stack) */
#define OURO_CLS_RUN_BODY 0x80u   /* | class: second or later chunk of a run */
#define OURO_MAX_REQUEST (16ull << (OURO_MAX_CLASSES - 1))   /* 1 MiB */
#define OURO_ROW_NONE OURO_MAX_CLASSES   /* counter row of requests without a class */
#define OURO_VL_HINTS 4096   /* lookaside hints per class: segments live at once in a burst of 2^22 positions */
#define OURO_NSTAT 8
#define OURO_SHARDS 32
#define OURO_SEG_HDR 64
#define OURO_AHEAD_POS (1ull << 20)   /* recycled segments go at most this many positions past the tail */
#define OURO_CARVE_SLOTS 4096u        /* slots one page carve fills at most (one chunk at least) */

/* queue storage forms */
#define OURO_QF_RING 0     /* plain array: a ring of slots outside the heap */
#define OURO_QF_LIST 1     /* virtualized list: segments linked in position order */
#define OURO_QF_VARRAY 2   /* virtualized array: segments found through a directory */
__host__ __device__ constexpr int ouro_qform(int v) {
  return (v == OURO_PAGE_VLIST || v == OURO_CHUNK_VLIST)     ? OURO_QF_LIST
         : (v == OURO_PAGE_VARRAY || v == OURO_CHUNK_VARRAY) ? OURO_QF_VARRAY
                                                            : OURO_QF_RING;
}
__host__ __device__ constexpr bool ouro_page_queues(int v) {
  return v == OURO_PAGE_ARRAY || v == OURO_PAGE_VLIST || v == OURO_PAGE_VARRAY;
}

enum {
  OURO_ST_MALLOC = 0, OURO_ST_FREE = 1, OURO_ST_FAILED = 2, OURO_ST_CARVE = 3,
  OURO_ST_REPUSH = 4, OURO_ST_CANCEL = 5, OURO_ST_DEAD = 6, OURO_ST_SEG = 7
};
/* stats row n_classes holds requests without a class */
enum { OURO_ST_ZERO = 0, OURO_ST_TOO_LARGE = 1 };

/* one hot counter per 128-byte line */
struct __align__(128) ouro_line {
  unsigned long long v;
  unsigned long long pad[15];
};

struct ouro_qhdr {
  ouro_line head;    /* next consumer position */
  ouro_line tail;    /* next producer position */
  ouro_line lock;    /* carve lock: 0 free, 1 held */
  ouro_line carved;  /* chunks owned by the class (page-array capacity) */
  ouro_line front;   /* virtualized list: oldest live segment (idx << 32 | chunk) */
  ouro_line back;    /* virtualized list: newest segment (hint) */
  ouro_line spare;   /* virtualized list: retired segments (tag << 32 | chunk) */
  ouro_line adv;     /* virtualized list: 1 while one thread or warp retires front segments */
  unsigned long long hint[OURO_VL_HINTS];  /* virtualized list: segment lookaside */
};

struct ouro_glob {
  ouro_line bump;        /* next never-carved chunk (may overshoot n_chunks) */
  ouro_line pool_taken;  /* pool entries handed out (may overshoot pool_size) */
  unsigned long long pool_size;
  unsigned int error_bits;
  unsigned int error_site;   /* OURO_SITE_* of the first error */
};

/* header of a virtualized-list segment (first 64 bytes of its chunk) */
struct ouro_seg {
  unsigned long long link;   /* (segment index << 32) | next chunk */
  unsigned int done;         /* position events seen (2 per slot: produced, consumed) */
  unsigned int spare_next;   /* next retired segment on the class spare stack */
  unsigned long long pad[6];
};

namespace ouro {
namespace detail {

/* ------------------------------------------------------------ PTX helpers */
__device__ __forceinline__ unsigned laneid() {
  unsigned r;
  asm volatile("mov.u32 %0, %%laneid;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned r;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned smid() {
  unsigned r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned long long ld_acq(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_rlx(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_acq32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_rlx32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rlx(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_rel(unsigned long long *p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long cas_rel(unsigned long long *p, unsigned long long c,
                                                      unsigned long long v) {
  unsigned long long o;
  asm volatile("atom.release.gpu.global.cas.b64 %0, [%1], %2, %3;"
               : "=l"(o) : "l"(p), "l"(c), "l"(v) : "memory");
  return o;
}
__device__ __forceinline__ unsigned long long exch_rel(unsigned long long *p, unsigned long long v) {
  unsigned long long o;
  asm volatile("atom.release.gpu.global.exch.b64 %0, [%1], %2;" : "=l"(o) : "l"(p), "l"(v) : "memory");
  return o;
}
__device__ __forceinline__ unsigned long long cas_rlx(unsigned long long *p, unsigned long long c,
                                                      unsigned long long v) {
  unsigned long long o;
  asm volatile("atom.relaxed.gpu.global.cas.b64 %0, [%1], %2, %3;"
               : "=l"(o) : "l"(p), "l"(c), "l"(v) : "memory");
  return o;
}
/* with a relaxed load before it, an acquire; with a relaxed write after it, a release */
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ unsigned long long cas_ar(unsigned long long *p, unsigned long long c,
                                                     unsigned long long v) {
  unsigned long long o;
  asm volatile("atom.acq_rel.gpu.global.cas.b64 %0, [%1], %2, %3;"
               : "=l"(o) : "l"(p), "l"(c), "l"(v) : "memory");
  return o;
}

/* ------------------------------------------------------------------ basics */
__host__ __device__ __forceinline__ ouro_qhdr *qh(const ouro_heap_dev &h, int c) {
  return reinterpret_cast<ouro_qhdr *>(h.qhdr) + c;
}
__device__ __forceinline__ ouro_glob *gl(const ouro_heap_dev &h) {
  return reinterpret_cast<ouro_glob *>(h.glob);
}
/* statistics counter, sharded by SM; a reduction (no value returned), so the
 * thread never waits for it */
__device__ __forceinline__ void stat_add(const ouro_heap_dev &h, int row, int kind,
                                         unsigned long long v) {
  if (v) {
    unsigned long long *a = &h.stats[((size_t)row * OURO_NSTAT + kind) * OURO_SHARDS + (smid() & (OURO_SHARDS - 1))];
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(a), "l"(v) : "memory");
  }
}
/* error sites: where the first recorded error of a heap came from */
enum {
  OURO_SITE_SPARE = 1, OURO_SITE_VL_FIRST, OURO_SITE_VL_NEXT, OURO_SITE_VL_WALK, OURO_SITE_PUT,
  OURO_SITE_PUSH_ONE, OURO_SITE_PAGE_GIVEUP, OURO_SITE_PAGE_CHECKED, OURO_SITE_CLAIM,
  OURO_SITE_CHUNK_GIVEUP, OURO_SITE_CHUNK_DOUBLE, OURO_SITE_BAD_FREE, OURO_SITE_PAGE_DOUBLE,
  OURO_SITE_TRIM, OURO_SITE_GRAPH_LOCK, OURO_SITE_VA_NEW, OURO_SITE_VA_WAIT, OURO_SITE_RUN_FREE
};
}  // namespace detail
}  // namespace ouro

/* ---------------------------------------------------- debug event ring */
/* Compile a kernel's translation unit with -DOURO_TRACE to record the slow
 * events of the allocator it calls -- carves, null answers of an exhausted
 * heap, new queue segments, bounded waits that ran out, errors -- in a ring
 * of OURO_TRACE_CAP events kept in that translation unit's device memory.
 * ouro_trace_copy (host) reads the newest events back.  Without
 * OURO_TRACE the calls compile to nothing.  Debug aid only: every event
 * takes one global atomic. */
enum {
  OURO_TR_CARVE = 1,       /* page or run carve: a = chunks taken, b = first producer position */
  OURO_TR_CHUNK_CARVE,     /* chunk-queue carve batch: a = chunks taken, b = positions answered */
  OURO_TR_EXHAUSTED,       /* positions answered null (no chunk left): a = count, b = first position */
  OURO_TR_SEGMENT,         /* a queue segment set up: a = segment index, b = chunk */
  OURO_TR_GIVEUP,          /* a bounded wait ran out: a = position, b = OURO_SITE_* */
  OURO_TR_ERROR            /* an error bit was set: a = bits, b = OURO_SITE_* */
};
typedef struct {
  unsigned long long t;    /* %globaltimer, ns */
  unsigned kind, cls;      /* OURO_TR_*, size class (or ~0u) */
  unsigned long long a, b;
} ouro_trace_event;
#ifdef OURO_TRACE
#ifndef OURO_TRACE_CAP
#define OURO_TRACE_CAP 4096   /* a power of two */
#endif
static __device__ ouro_trace_event ouro_trace_ring[OURO_TRACE_CAP];
static __device__ unsigned long long ouro_trace_next;
__device__ __forceinline__ void ouro_trace_event_put(unsigned kind, int cls, unsigned long long a,
                                                     unsigned long long b) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  const unsigned long long i = atomicAdd(&ouro_trace_next, 1ull);
  ouro_trace_event *e = &ouro_trace_ring[i & (OURO_TRACE_CAP - 1)];
  e->t = t;
  e->kind = kind;
  e->cls = (unsigned)cls;
  e->a = a;
  e->b = b;
}
#define OURO_TRACE_EVENT(kind, cls, a, b) ouro_trace_event_put((kind), (cls), (a), (b))
/* Host: the newest min(total, OURO_TRACE_CAP, cap) events of this
 * translation unit's ring, oldest first, into out; *total = events ever
 * recorded.  Synchronous (cudaMemcpyFromSymbol); call when the kernels that
 * record are done.  Clears the ring when clear != 0. */
static inline __host__ cudaError_t ouro_trace_copy(ouro_trace_event *out, unsigned cap, unsigned long long *total,
                                                   int clear) {
  unsigned long long n = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&n, ouro_trace_next, sizeof(n));
  if (e != cudaSuccess) return e;
  if (total) *total = n;
  const unsigned long long keep = n < OURO_TRACE_CAP ? n : OURO_TRACE_CAP;
  const unsigned long long want = keep < cap ? keep : cap;
  for (unsigned long long k = 0; k < want; ++k) {
    const unsigned long long i = (n - want + k) & (OURO_TRACE_CAP - 1);
    e = cudaMemcpyFromSymbol(out + k, ouro_trace_ring, sizeof(ouro_trace_event), i * sizeof(ouro_trace_event));
    if (e != cudaSuccess) return e;
  }
  if (clear) {
    const unsigned long long zero = 0;
    e = cudaMemcpyToSymbol(ouro_trace_next, &zero, sizeof(zero));
  }
  return e;
}
#else
#define OURO_TRACE_EVENT(kind, cls, a, b) ((void)0)
#endif

namespace ouro {
namespace detail {
__device__ __forceinline__ void set_error(const ouro_heap_dev &h, unsigned bits, unsigned site) {
  atomicOr(&gl(h)->error_bits, bits);
  atomicCAS(&gl(h)->error_site, 0u, site);
  OURO_TRACE_EVENT(OURO_TR_ERROR, -1, bits, site);
}

/* power-of-two class: ceil(log2 n) - 4, floor 16 B; -1 for 0 or above
 * 1 MiB.  Classes from h.n_classes up are runs of chunks. */
__device__ __forceinline__ int size_class(const ouro_heap_dev &h, unsigned long long n) {
  (void)h;
  if (n == 0 || n > OURO_MAX_REQUEST) return -1;
  if (n <= 16) return 0;
  return 64 - __clzll(n - 1) - 4;
}

/* slot word: high 32 bits = sequence, low 32 bits = item.  For the slot of
 * position p: seq p = empty, p+1 = item, p+2 = null answer (heap exhausted),
 * >= p+3 = position retired (consumed; or given up by its consumer). */
__device__ __forceinline__ unsigned long long slot(unsigned long long seq, unsigned item) {
  return ((unsigned long long)(unsigned)seq << 32) | item;
}
__device__ __forceinline__ int slot_d(unsigned long long v, unsigned long long pos) {
  return (int)((unsigned)(v >> 32) - (unsigned)pos);
}

/* Lanes of mask that share key: one warp group takes one queue atomic for
 * all its lanes (warp aggregation).  The deoptimised form (option deopt,
 * Sec. 2) makes every lane its own group. */
template <typename T>
__device__ __forceinline__ unsigned warp_group(const ouro_heap_dev &h, unsigned mask, T key) {
  if (h.deopt) return 1u << laneid();
  return __match_any_sync(mask, key);
}

/* One step of a bounded wait: __nanosleep with the caller's backoff, or in
 * the deoptimised form a memory fence in its place (Sec. 2). */
__device__ __forceinline__ void backoff_wait(const ouro_heap_dev &h, unsigned ns) {
  if (h.deopt) __threadfence();
  else __nanosleep(ns);
}

__device__ __forceinline__ bool try_lock(unsigned long long *l) {
  if (ld_rlx(l) != 0) return false;
  return cas_ar(l, 0ull, 1ull) == 0ull;
}
__device__ __forceinline__ void unlock(unsigned long long *l) { st_rel(l, 0ull); }

/* ------------------------------------------------------------ chunk supply */
struct chunk_range {
  unsigned long long p0, b0;
  unsigned k1, k2;
};
/* Up to m chunks: pool entries first (in pool order), then never-carved
 * chunks from the bump pointer. */
__device__ inline chunk_range take_chunks(const ouro_heap_dev &h, unsigned m) {
  chunk_range r{0, 0, 0, 0};
  ouro_glob *g = gl(h);
  const unsigned long long ps = ld_rlx(&g->pool_size);
  if (m && ld_rlx(&g->pool_taken.v) < ps) {
    unsigned long long pt = atomicAdd(&g->pool_taken.v, (unsigned long long)m);
    if (pt < ps) {
      r.p0 = pt;
      r.k1 = (unsigned)min((unsigned long long)m, ps - pt);
    }
  }
  unsigned rest = m - r.k1;
  if (rest && ld_rlx(&g->bump.v) < h.n_chunks) {
    unsigned long long b = atomicAdd(&g->bump.v, (unsigned long long)rest);
    if (b < h.n_chunks) {
      r.b0 = b;
      r.k2 = (unsigned)min((unsigned long long)rest, h.n_chunks - b);
    }
  }
  return r;
}
__device__ __forceinline__ unsigned range_chunk(const ouro_heap_dev &h, const chunk_range &r,
                                                unsigned j) {
  return j < r.k1 ? h.pool[r.p0 + j] : (unsigned)(r.b0 + (j - r.k1));
}

/* ------------------------------------------------------- array slot rings */
__device__ __forceinline__ unsigned long long *ring_slot(const ouro_heap_dev &h, int c,
                                                         unsigned long long pos) {
  return h.cells + h.ring_off[c] + (pos & h.ring_mask[c]);
}

/* --------------------------------------------- virtualized-list segments */
__device__ __forceinline__ ouro_seg *seg_of(const ouro_heap_dev &h, unsigned x) {
  return reinterpret_cast<ouro_seg *>(h.base + ((size_t)x << h.log2_chunk));
}
__device__ __forceinline__ unsigned long long *seg_cells(const ouro_heap_dev &h, unsigned x) {
  return reinterpret_cast<unsigned long long *>(h.base + ((size_t)x << h.log2_chunk) + OURO_SEG_HDR);
}
__device__ __forceinline__ unsigned hi32(unsigned long long v) { return (unsigned)(v >> 32); }
__device__ __forceinline__ unsigned lo32(unsigned long long v) { return (unsigned)v; }
__device__ __forceinline__ unsigned long long pack(unsigned a, unsigned b) {
  return ((unsigned long long)a << 32) | b;
}

__device__ inline void spare_push(const ouro_heap_dev &h, int c, unsigned x) {
  unsigned long long *top = &qh(h, c)->spare.v;
  for (unsigned it = 0; it < h.spin_limit; ++it) {
    unsigned long long old = ld_acq(top);
    seg_of(h, x)->spare_next = lo32(old);
    __threadfence();
    if (cas_ar(top, old, pack(hi32(old) + 1, x)) == old) return;
  }
  set_error(h, OURO_ERR_TIMEOUT, OURO_SITE_SPARE);
}
__device__ inline unsigned spare_pop(const ouro_heap_dev &h, int c) {
  unsigned long long *top = &qh(h, c)->spare.v;
  for (unsigned it = 0; it < h.spin_limit; ++it) {
    unsigned long long old = ld_acq(top);
    if (lo32(old) == OURO_NIL) return OURO_NIL;
    unsigned nxt = *(volatile unsigned *)&seg_of(h, lo32(old))->spare_next;
    if (cas_ar(top, old, pack(hi32(old) + 1, nxt)) == old) return lo32(old);
  }
  return OURO_NIL;
}

/* Set chunk x up as segment idx, linked to next (OURO_NIL: none yet): every
 * slot reads empty for its own position.  No fence: the caller publishes. */
__device__ inline void seg_setup(const ouro_heap_dev &h, unsigned x, unsigned idx, bool fresh, unsigned next) {
  ouro_seg *s = seg_of(h, x);
  s->done = 0;
  /* A segment recycled from the spare stack always serves a higher index, so
   * its stale slots hold sequences below every new position: single-use list
   * slots read "sequence behind position" as empty, and the slots need no
   * rewrite -- unless the index jumped so far that 32-bit sequences could
   * wrap.  A chunk fresh from the heap is initialised. */
  bool init = fresh;
  if (!fresh) {
    const unsigned old_idx = hi32(s->link);
    const int ahead = (int)(idx - old_idx);
    init = ahead <= 0 || (unsigned long long)ahead * h.seg_cap >= (1ull << 30);
  }
  if (init) {
    unsigned long long *cells = seg_cells(h, x);
    const unsigned long long p0 = (unsigned long long)idx * h.seg_cap;
    for (unsigned i = 0; i < h.seg_cap; i += 2) {
      ulonglong2 v = make_ulonglong2(slot(p0 + i, 0), slot(p0 + i + 1, 0));
      *reinterpret_cast<ulonglong2 *>(cells + i) = v;   /* seg_cap is even, cells 16-B aligned */
    }
  }
  s->link = pack(idx, next);
}

/* Set chunk x up as segment idx with no successor, and fence. */
__device__ inline void seg_init(const ouro_heap_dev &h, unsigned x, unsigned idx, bool fresh) {
  seg_setup(h, x, idx, fresh, OURO_NIL);
  __threadfence();
}

/* A fresh segment with index idx: spare of the class first, else a chunk of
 * the heap. */
__device__ inline unsigned seg_new(const ouro_heap_dev &h, int c, unsigned idx) {
  unsigned x = spare_pop(h, c);
  const bool fresh = x == OURO_NIL;
  if (fresh) {
    chunk_range r = take_chunks(h, 1);
    if (r.k1 + r.k2 == 0) return OURO_NIL;
    x = range_chunk(h, r, 0);
    h.chunk_cls[x] = OURO_CLS_SEG;
    stat_add(h, c, OURO_ST_SEG, 1);
  }
  seg_init(h, x, idx, fresh);
  OURO_TRACE_EVENT(OURO_TR_SEGMENT, c, idx, x);
  return x;
}

/* Retired list segments xs[0..k), in list order, are appended behind the
 * back segment as one chain -- indices back + 1 .. back + k, each linked to
 * the next, published by one store of the back's link -- at most up to
 * OURO_AHEAD_POS positions past the tail, so that producers find their
 * segments linked; what does not fit joins the spare stack.  A burst that
 * retires many segments thus re-links them in runs rather than one append
 * (a claim, a set-up and a publish of the back's link) per segment. */
__device__ inline void vl_append_run(const ouro_heap_dev &h, int c, const unsigned *xs, unsigned k) {
  ouro_qhdr *q = qh(h, c);
  unsigned placed = 0, ns = h.backoff_min_ns;
  for (int tries = 0; tries < 16 && placed < k; ++tries) {
    const unsigned long long b = ld_acq(&q->back.v);
    const unsigned bx = lo32(b);
    if (bx >= OURO_BUSY) break;
    ouro_seg *sg = seg_of(h, bx);
    const unsigned long long link = ld_acq(&sg->link);
    if (hi32(link) != hi32(b)) continue;                 /* stale back hint */
    if (lo32(link) < OURO_BUSY) {                        /* a successor exists: move the hint on */
      cas_ar(&q->back.v, b, pack(hi32(b) + 1, lo32(link)));
      continue;
    }
    if (lo32(link) == OURO_BUSY) {                       /* another thread is appending: its run is short */
      backoff_wait(h, ns);
      ns = min(ns * 2, h.backoff_max_ns);
      continue;
    }
    const unsigned long long lim = ld_rlx(&q->tail.v) + OURO_AHEAD_POS;
    const unsigned long long at = (unsigned long long)(hi32(b) + 1) * h.seg_cap;   /* first position appended */
    if (at > lim) break;
    const unsigned m = (unsigned)min((unsigned long long)(k - placed), (lim - at) / h.seg_cap + 1);
    if (cas_ar(&sg->link, link, pack(hi32(b), OURO_BUSY)) != link) continue;
    for (unsigned j = 0; j < m; ++j)
      seg_setup(h, xs[placed + j], hi32(b) + 1 + j, false, j + 1 < m ? xs[placed + j + 1] : OURO_NIL);
    __threadfence();
    st_rel(&sg->link, pack(hi32(b), xs[placed]));
    atomicMax(&q->back.v, pack(hi32(b) + m, xs[placed + m - 1]));   /* indices only grow */
    for (unsigned j = 0; j < m; ++j)
      st_rlx(&q->hint[(hi32(b) + 1 + j) & (OURO_VL_HINTS - 1)], pack(hi32(b) + 1 + j, xs[placed + j]));
    placed += m;
  }
  for (unsigned j = placed; j < k; ++j) spare_push(h, c, xs[j]);
}

#define OURO_VL_RUN 16   /* front segments one retire takes off the list at once */

/* Retire fully used front segments (all slots produced and consumed, and a
 * successor linked): up to OURO_VL_RUN consecutive ones leave the list with
 * one move of the front and are appended behind the back as a chain (or
 * spared).  The single-lane form, for callers that are not a whole warp;
 * several may race, the front moves by compare-and-swap.  Out of line: it
 * runs once per segment's worth of positions. */
static __device__ __noinline__ void vl_advance(const ouro_heap_dev &h, int c) {
  ouro_qhdr *q = qh(h, c);
  unsigned xs[OURO_VL_RUN];
  for (int i = 0; i < 64; ++i) {
    const unsigned long long f = ld_acq(&q->front.v);
    if (lo32(f) >= OURO_BUSY) return;
    unsigned k = 0;
    bool stale = false;
    unsigned long long cur = f;
    while (k < OURO_VL_RUN) {
      const unsigned cx = lo32(cur);
      const unsigned long long link = ld_acq(&seg_of(h, cx)->link);
      if (hi32(link) != hi32(cur)) {                     /* the front moved on meanwhile */
        stale = k == 0;
        break;
      }
      if (lo32(link) >= OURO_BUSY) break;
      if (ld_acq32(&seg_of(h, cx)->done) != 2u * h.seg_cap) break;
      xs[k++] = cx;
      cur = pack(hi32(cur) + 1, lo32(link));
    }
    if (stale) continue;
    if (!k) return;
    const unsigned long long b = ld_acq(&q->back.v);   /* never leave the back hint on a retired segment */
    if (lo32(b) < OURO_BUSY && hi32(b) < hi32(cur)) cas_ar(&q->back.v, b, cur);
    if (cas_ar(&q->front.v, f, cur) != f) continue;
    vl_append_run(h, c, xs, k);
    if (k < OURO_VL_RUN) return;
  }
}

/* Is the front segment of the list fully used (its own index in its link,
 * a successor linked, every position produced and consumed)? */
__device__ inline bool vl_front_ready(const ouro_heap_dev &h, ouro_qhdr *q) {
  const unsigned long long f = ld_acq(&q->front.v);
  if (lo32(f) >= OURO_BUSY) return false;
  const unsigned long long link = ld_acq(&seg_of(h, lo32(f))->link);
  return hi32(link) == hi32(f) && lo32(link) < OURO_BUSY && ld_acq32(&seg_of(h, lo32(f))->done) == 2u * h.seg_cap;
}

/* Front segments per lane in one round of the warp-wide retire (W below):
 * two for most callers; four for the block-aggregated batch kernels,
 * which run long single-class bursts (more registers in the walk, which
 * other kernels would carry too). */
#define OURO_VL_WIDE 2
#define OURO_VL_WIDE_BATCH 4

/* Value v[j / 32] of lane j % 32 (0 <= j < 32 * W); every lane
 * of the warp calls. */
template <int W>
__device__ __forceinline__ unsigned vl_pick(const unsigned (&v)[W], unsigned j) {
  unsigned r = 0;
#pragma unroll
  for (int p = 0; p < W; ++p) {
    const unsigned t = __shfl_sync(0xffffffffu, v[p], j & 31);
    if ((j >> 5) == (unsigned)p) r = t;
  }
  return r;
}

/* The back hint of class c trails the list (segments were linked behind
 * it by producers): every lane of the warp reads the segments of indices
 * back + 1 .. back + 32 * W at once (lookaside hints, then
 * links), and the hint moves to the last one of the leading run that is
 * linked in order.  succ: the successor the back segment links to. */
template <int W>
static __device__ __noinline__ void vl_back_chase_warp(const ouro_heap_dev &h, ouro_qhdr *q, unsigned long long b,
                                                       unsigned succ) {
  const unsigned lane = laneid(), bi = hi32(b);
  unsigned xc[W], nxt[W];
  unsigned long long lk[W];
#pragma unroll
  for (int p = 0; p < W; ++p) {
    const unsigned j = 32u * p + lane;
    if (j == 0) {
      xc[p] = succ;
    } else {
      const unsigned long long e = ld_rlx(&q->hint[(bi + 1 + j) & (OURO_VL_HINTS - 1)]);
      xc[p] = hi32(e) == bi + 1 + j && lo32(e) < OURO_BUSY ? lo32(e) : OURO_NIL;
    }
  }
#pragma unroll
  for (int p = 0; p < W; ++p) lk[p] = xc[p] != OURO_NIL ? ld_rlx(&seg_of(h, xc[p])->link) : 0ull;
  fence_acq_rel();
  unsigned run = 0;
  bool stop = false;
#pragma unroll
  for (int p = 0; p < W; ++p) {
    nxt[p] = lo32(lk[p]);
    if (stop) continue;
    const unsigned j = 32u * p + lane;
    const unsigned carry = p ? __shfl_sync(0xffffffffu, nxt[p ? p - 1 : 0], 31) : succ;
    const unsigned upn = __shfl_up_sync(0xffffffffu, nxt[p], 1);
    const unsigned prev = lane == 0 ? carry : upn;
    const bool linked = xc[p] != OURO_NIL && prev == xc[p] && hi32(lk[p]) == bi + 1 + j;
    const unsigned vm = __ballot_sync(0xffffffffu, linked);
    if (vm == 0xffffffffu) {
      run += 32;
      continue;
    }
    run += __ffs(~vm) - 1;
    stop = true;
  }
  if (!run) return;   /* the successor is still being set up */
  const unsigned xl = vl_pick(xc, run - 1);
  if (lane == 0) atomicMax(&q->back.v, pack(bi + run, xl));   /* indices only grow */
}

/* vl_append_run for a whole warp: the run's chunks are held as x[p] by lane
 * j % 32 for run offset j = 32 p + lane (j < k).  Lane 0 claims the back
 * segment's empty link; every lane sets its own segments up; lane 0
 * publishes the chain with one store; every lane then writes its segments'
 * lookaside hints.  A back hint that trails the list is moved up to 128
 * segments at a time; what finds no room goes to the spare stack as one
 * chain (one push). */
template <int W>
static __device__ __noinline__ void vl_append_run_warp(const ouro_heap_dev &h, int c,
                                                       const unsigned (&x)[W], unsigned k,
                                                       unsigned long long &bk) {
  ouro_qhdr *q = qh(h, c);
  const unsigned lane = laneid();
  unsigned nx[W];   /* chunk at run offset j + 1 */
#pragma unroll
  for (int p = 0; p < W; ++p) {
    const unsigned dn = __shfl_down_sync(0xffffffffu, x[p], 1);
    const unsigned up = p + 1 < W ? __shfl_sync(0xffffffffu, x[p + 1 < W ? p + 1 : p], 0)
                                             : OURO_NIL;
    nx[p] = lane == 31 ? up : dn;
  }
  unsigned placed = 0, ns = h.backoff_min_ns;
  for (int tries = 0; tries < 16 && placed < k; ++tries) {
    unsigned long long b = 0, link = 0;
    unsigned m = 0;
    int act = 0;   /* 0: look again, 1: link claimed for m segments, 2: no room behind the back, 3: chase the back */
    if (lane == 0) {
      /* the first try starts from the back this warp published last (a
       * segment whose link still has no successor is the list's last) */
      b = tries == 0 && bk ? bk : ld_acq(&q->back.v);
      const unsigned bx = lo32(b);
      if (bx >= OURO_BUSY) {
        act = 2;
      } else {
        ouro_seg *sg = seg_of(h, bx);
        const unsigned long long tail = ld_rlx(&q->tail.v);
        const unsigned long long empty = pack(hi32(b), OURO_NIL);
        link = cas_ar(&sg->link, empty, pack(hi32(b), OURO_BUSY));   /* claim the empty link */
        if (link == empty) {
          const unsigned long long lim = tail + OURO_AHEAD_POS;
          const unsigned long long at = (unsigned long long)(hi32(b) + 1) * h.seg_cap;
          if (at > lim) {
            st_rel(&sg->link, empty);
            act = 2;
          } else {
            m = (unsigned)min((unsigned long long)(k - placed), (lim - at) / h.seg_cap + 1);
            act = 1;
          }
        } else if (hi32(link) != hi32(b)) {                  /* stale back hint */
        } else if (lo32(link) < OURO_BUSY) {                 /* a successor exists: the hint trails */
          act = 3;
        } else {                                             /* another thread is appending */
          backoff_wait(h, ns);
          ns = min(ns * 2, h.backoff_max_ns);
        }
      }
    }
    act = __shfl_sync(0xffffffffu, act, 0);
    if (act == 2) break;
    if (act == 3) {
      vl_back_chase_warp<W>(h, q, __shfl_sync(0xffffffffu, b, 0), lo32(__shfl_sync(0xffffffffu, link, 0)));
      continue;
    }
    if (act == 0) continue;
    b = __shfl_sync(0xffffffffu, b, 0);
    m = __shfl_sync(0xffffffffu, m, 0);
    const unsigned bi = hi32(b);
#pragma unroll
    for (int p = 0; p < W; ++p) {
      const unsigned j = 32u * p + lane;
      if (j >= placed && j < placed + m)
        seg_setup(h, x[p], bi + 1 + (j - placed), false, j + 1 < placed + m ? nx[p] : OURO_NIL);
    }
    __threadfence();
    const unsigned first = vl_pick(x, placed), last = vl_pick(x, placed + m - 1);
    __syncwarp();
    if (lane == 0) {
      st_rel(&seg_of(h, lo32(b))->link, pack(bi, first));
      atomicMax(&q->back.v, pack(bi + m, last));   /* indices only grow */
    }
    bk = pack(bi + m, last);
    __syncwarp();
#pragma unroll
    for (int p = 0; p < W; ++p) {
      const unsigned j = 32u * p + lane;
      if (j >= placed && j < placed + m)
        st_rlx(&q->hint[(bi + 1 + (j - placed)) & (OURO_VL_HINTS - 1)], pack(bi + 1 + (j - placed), x[p]));
    }
    placed += m;
  }
  if (placed < k) {   /* the rest onto the spare stack, as one chain */
#pragma unroll
    for (int p = 0; p < W; ++p) {
      const unsigned j = 32u * p + lane;
      if (j >= placed && j + 1 < k) seg_of(h, x[p])->spare_next = nx[p];
    }
    __threadfence();
    const unsigned first = vl_pick(x, placed), last = vl_pick(x, k - 1);
    __syncwarp();
    if (lane == 0) {
      unsigned long long *top = &q->spare.v;
      unsigned it = 0;
      for (; it < h.spin_limit; ++it) {
        const unsigned long long old = ld_acq(top);
        seg_of(h, last)->spare_next = lo32(old);
        __threadfence();
        if (cas_ar(top, old, pack(hi32(old) + 1, first)) == old) break;
      }
      if (it == h.spin_limit) set_error(h, OURO_ERR_TIMEOUT, OURO_SITE_SPARE);
    }
    __syncwarp();
  }
}

/* vl_advance for a whole warp (every lane calls).  One warp at a time
 * retires (the class's adv lock): a warp that finds the lock taken returns,
 * and the holder, once it let go, looks at the front once more, so that no
 * retire is lost; retires thus gather into long runs and few appends
 * instead of one short run (and one append behind the back) per caller.
 * Lane j % 32 looks at the
 * segment of index front + j for j < 32 * W: its chunk from the
 * lookaside hint, its link and its done count, all loaded at once behind one
 * fence, instead of following the links one dependent load at a time; the
 * leading run of fully used segments leaves the list with one move of the
 * front and is appended behind the back.  A segment whose hint is missing
 * or stale ends the round; the next round starts at it (then the front). */
template <int W>
static __device__ __noinline__ void vl_advance_warp_runs(const ouro_heap_dev &h, int c);
template <int W>
static __device__ __noinline__ void vl_advance_warp(const ouro_heap_dev &h, int c) {
  ouro_qhdr *q = qh(h, c);
  __syncwarp();   /* the lanes' done counts are ordered before the lock attempt */
  for (int a = 0; a < 8; ++a) {
    unsigned got = 0;
    if (laneid() == 0) got = try_lock(&q->adv.v);
    if (!__shfl_sync(0xffffffffu, got, 0)) return;
    vl_advance_warp_runs<W>(h, c);
    unsigned again = 0;
    if (laneid() == 0) {
      unlock(&q->adv.v);
      __threadfence();
      again = vl_front_ready(h, q);
    }
    if (!__shfl_sync(0xffffffffu, again, 0)) return;
  }
}
template <int W>
static __device__ __noinline__ void vl_advance_warp_runs(const ouro_heap_dev &h, int c) {
  ouro_qhdr *q = qh(h, c);
  const unsigned lane = laneid(), used = 2u * h.seg_cap;
  unsigned long long f = 0, bk = 0;   /* bk: the back this warp published last, 0 none */
  bool known = false;
  for (int i = 0; i < 64; ++i) {
    if (!known) {
      if (lane == 0) f = ld_acq(&q->front.v);
      f = __shfl_sync(0xffffffffu, f, 0);
    }
    known = false;
    if (lo32(f) >= OURO_BUSY) return;
    const unsigned fi = hi32(f);
    unsigned x[W], nxt[W], dn[W];
    unsigned long long lk[W];
#pragma unroll
    for (int p = 0; p < W; ++p) {
      const unsigned j = 32u * p + lane;
      if (j == 0) {
        x[p] = lo32(f);
      } else {
        const unsigned long long e = ld_rlx(&q->hint[(fi + j) & (OURO_VL_HINTS - 1)]);
        x[p] = hi32(e) == fi + j && lo32(e) < OURO_BUSY ? lo32(e) : OURO_NIL;
      }
    }
#pragma unroll
    for (int p = 0; p < W; ++p) {
      lk[p] = 0;
      dn[p] = 0;
      if (x[p] != OURO_NIL) {
        lk[p] = ld_rlx(&seg_of(h, x[p])->link);
        dn[p] = ld_rlx32(&seg_of(h, x[p])->done);
      }
    }
    fence_acq_rel();
    /* offset j leaves if its chunk is the successor that offset j - 1 links
     * to (offset 0: the front), its link carries index front + j and a
     * successor, and all its positions were produced and consumed */
    unsigned k = 0;
    int stop = 0;   /* 1: a known segment is not done yet; 2: a segment not known from its hint */
#pragma unroll
    for (int p = 0; p < W; ++p) {
      nxt[p] = lo32(lk[p]);
      if (stop) continue;
      const unsigned j = 32u * p + lane;
      const unsigned carry = p ? __shfl_sync(0xffffffffu, nxt[p ? p - 1 : 0], 31) : lo32(f);
      const unsigned upn = __shfl_up_sync(0xffffffffu, nxt[p], 1);
      const unsigned prev = lane == 0 ? carry : upn;
      const bool known_j = x[p] != OURO_NIL && prev == x[p] && hi32(lk[p]) == fi + j;
      const bool ready = known_j && nxt[p] < OURO_BUSY && dn[p] == used;
      const unsigned rm = __ballot_sync(0xffffffffu, ready);
      if (rm == 0xffffffffu) {
        k += 32;
        continue;
      }
      const unsigned jj = __ffs(~rm) - 1;
      k += jj;
      stop = (__ballot_sync(0xffffffffu, known_j) >> jj) & 1 ? 1 : 2;
    }
    if (k == 0) {
      /* the front itself is not done, or it moved on meanwhile (its link
       * holds another index): look again */
      if (__shfl_sync(0xffffffffu, (unsigned)(hi32(lk[0]) != fi), 0)) continue;
      return;
    }
    const unsigned long long cur = pack(fi + k, vl_pick(nxt, k - 1));
    unsigned moved = 0;
    if (lane == 0) {
      /* never leave the back hint on a retired segment (the hint only
       * grows: a back this warp published at or past cur needs no look) */
      if (!bk || hi32(bk) < hi32(cur)) {
        const unsigned long long b = ld_acq(&q->back.v);
        if (lo32(b) < OURO_BUSY && hi32(b) < hi32(cur)) cas_ar(&q->back.v, b, cur);
      }
      moved = cas_ar(&q->front.v, f, cur) == f;
    }
    if (!__shfl_sync(0xffffffffu, moved, 0)) continue;
    vl_append_run_warp<W>(h, c, x, k, bk);
    if (stop == 1) return;
    f = cur;   /* the next round starts at the new front */
    known = true;
  }
}

/* ------------------------------------------ virtualized-array directory */
/* Entry of segment index s in the directory of class c: (index << 32) |
 * chunk, with chunk OURO_NIL while segment s does not exist yet and
 * OURO_BUSY while its one creator sets it up.  The directory has D = 2^k
 * entries; segment s uses entry s mod D, whose index field runs ahead by D
 * each time a segment in it retires. */
__device__ __forceinline__ unsigned long long *va_entry(const ouro_heap_dev &h, int c, unsigned long long s) {
  return h.cells + h.ring_off[c] + (s & h.ring_mask[c]);
}

/* Segment x has seen all its position events: its entry is emptied for the
 * next lap (index + D), and the chunk is set up again as a missing segment
 * ahead of the producers, so that a burst of producers finds its segments in
 * place.  The class front line counts out those indices, (next index << 32)
 * | NIL: every retiring segment takes its own, starting past the tail's
 * segment.  An index whose entry a producer has made meanwhile is skipped;
 * past D/2 segments, or OURO_AHEAD_POS positions, ahead of the tail the
 * chunk joins the spare stack instead. */
__device__ inline void va_retire(const ouro_heap_dev &h, int c, unsigned x) {
  ouro_qhdr *q = qh(h, c);
  const unsigned idx = hi32(ld_acq(&seg_of(h, x)->link));
  const unsigned long long D = h.ring_mask[c] + 1;
  st_rel(va_entry(h, c, idx), pack(idx + (unsigned)D, OURO_NIL));
  const unsigned long long tail = ld_rlx(&q->tail.v), ts = tail / h.seg_cap;
  const unsigned long long lim = ts + min(D >> 1, OURO_AHEAD_POS / h.seg_cap + 1);
  for (int k = 0; k < 8; ++k) {
    const unsigned long long sn = hi32(atomicAdd(&q->front.v, 1ull << 32));
    if (sn < ts + 1) {                     /* the count fell behind the tail: jump past it */
      atomicMax(&q->front.v, pack((unsigned)(ts + 1), OURO_NIL));
      continue;
    }
    if (sn >= lim) break;
    unsigned long long *e = va_entry(h, c, sn);
    const unsigned long long v = pack((unsigned)sn, OURO_NIL);
    if (ld_rlx(e) != v) continue;
    if (cas_ar(e, v, pack((unsigned)sn, OURO_BUSY)) != v) continue;
    seg_init(h, x, (unsigned)sn, false);
    st_rel(e, pack((unsigned)sn, x));
    return;
  }
  spare_push(h, c, x);
}

/* Look-ahead for producers early in segment s - 1: set up
 * segment s from the class spare stack (never from the heap, so exhaustion
 * is unchanged) if nobody has, so that the producers reaching it do not wait
 * for its creation. */
__device__ inline void va_prefetch(const ouro_heap_dev &h, int c, unsigned s32) {
  unsigned long long *e = va_entry(h, c, s32);
  const unsigned long long v = pack(s32, OURO_NIL);
  if (ld_rlx(e) != v || lo32(ld_rlx(&qh(h, c)->spare.v)) == OURO_NIL) return;
  if (cas_ar(e, v, pack(s32, OURO_BUSY)) != v) return;
  const unsigned x = spare_pop(h, c);
  if (x == OURO_NIL) {
    st_rel(e, v);
    return;
  }
  seg_init(h, x, s32, false);
  st_rel(e, pack(s32, x));
}

/* Slot of position pos in the virtualized array of class c.  create: make
 * the segment if it does not exist (one creator, the others wait);
 * otherwise null while it does not exist.  Null too for a segment that has
 * retired already (only a look-ahead can ask for one: a thread holding an
 * unfinished position keeps its segment alive). */
__device__ inline unsigned long long *va_slot(const ouro_heap_dev &h, int c, unsigned long long pos,
                                              bool create) {
  const unsigned long long s = pos / h.seg_cap;
  const unsigned s32 = (unsigned)s;
  const unsigned off = (unsigned)(pos - s * h.seg_cap);
  unsigned long long *e = va_entry(h, c, s);
  unsigned ns = h.backoff_min_ns;
  for (unsigned it = 0; it < h.spin_limit; ++it) {
    const unsigned long long v = ld_acq(e);
    const int d = (int)(hi32(v) - s32);
    const unsigned x = lo32(v);
    if (d > 0) return nullptr;
    if (d == 0 && x < OURO_BUSY) {
      if (create && off - (h.seg_cap >> 3) < 32u) va_prefetch(h, c, s32 + 1);
      return seg_cells(h, x) + off;
    }
    if (!create) return nullptr;
    if (d == 0 && x == OURO_NIL) {
      if (cas_ar(e, v, pack(s32, OURO_BUSY)) == v) {
        const unsigned nx = seg_new(h, c, s32);
        if (nx == OURO_NIL) {
          st_rel(e, v);
          set_error(h, OURO_ERR_QUEUE_FULL, OURO_SITE_VA_NEW);
          return nullptr;
        }
        st_rel(e, pack(s32, nx));
        return seg_cells(h, nx) + off;
      }
      continue;
    }
    /* being created, or the entry still serves segment s - D (wait for it to retire) */
    backoff_wait(h, ns);
    ns = min(ns * 2, h.backoff_max_ns);
  }
  set_error(h, OURO_ERR_TIMEOUT, OURO_SITE_VA_WAIT);
  return nullptr;
}

/* n position events on the segment holding `cell` */
template <int QF>
__device__ inline void seg_event(const ouro_heap_dev &h, int c, const unsigned long long *cell, unsigned n) {
  unsigned x = (unsigned)(((const unsigned char *)cell - h.base) >> h.log2_chunk);
  unsigned r = atomicAdd(&seg_of(h, x)->done, n) + n;
  if (r == 2u * h.seg_cap) {
    __threadfence();
    if (QF == OURO_QF_LIST) vl_advance(h, c);
    else va_retire(h, c, x);
  }
}

/* Position events of the lanes of mask (every lane of mask calls): lanes
 * with `active` and a slot count one event on the segment of their slot;
 * lanes on the same segment are summed into one atomic. */
template <int QF, int W = OURO_VL_WIDE>
__device__ inline void seg_event_warp(const ouro_heap_dev &h, int c, const unsigned long long *cell, bool active,
                                      unsigned mask) {
  const bool on = active && cell;
  const unsigned x = on ? (unsigned)(((const unsigned char *)cell - h.base) >> h.log2_chunk) : OURO_NIL;
  const unsigned g = warp_group(h, mask, x) & __ballot_sync(mask, on);
  bool retire = false;
  if (on && laneid() == (unsigned)(__ffs(g) - 1)) {
    const unsigned n = __popc(g);
    const unsigned r = atomicAdd(&seg_of(h, x)->done, n) + n;
    if (r == 2u * h.seg_cap) {
      __threadfence();
      if (QF != OURO_QF_LIST) va_retire(h, c, x);
      else if (mask != 0xffffffffu) vl_advance(h, c);
      else retire = true;
    }
  }
  if (QF == OURO_QF_LIST && mask == 0xffffffffu) {
    /* a whole warp: the front advance runs warp-wide, once per class that
     * retired a segment */
    unsigned rm = __ballot_sync(mask, retire);
    while (rm) {
      const int cj = __shfl_sync(mask, c, __ffs(rm) - 1);
      rm &= ~__ballot_sync(mask, retire && c == cj);
      vl_advance_warp<W>(h, cj);
    }
  }
}

/* Look-ahead for producers early in segment cur = (idx, x):
 * link its successor from the class spare stack (never from the heap) if it
 * has none yet, so that the producers reaching it find it linked. */
__device__ inline void vl_prefetch(const ouro_heap_dev &h, int c, unsigned long long cur) {
  ouro_qhdr *q = qh(h, c);
  ouro_seg *sg = seg_of(h, lo32(cur));
  const unsigned long long link = pack(hi32(cur), OURO_NIL);
  if (ld_rlx(&sg->link) != link || lo32(ld_rlx(&q->spare.v)) == OURO_NIL) return;
  if (cas_ar(&sg->link, link, pack(hi32(cur), OURO_BUSY)) != link) return;
  const unsigned x = spare_pop(h, c);
  if (x == OURO_NIL) {
    st_rel(&sg->link, link);
    return;
  }
  seg_init(h, x, hi32(cur) + 1, false);
  st_rel(&sg->link, pack(hi32(cur), x));
  cas_ar(&q->back.v, cur, pack(hi32(cur) + 1, x));
  st_rlx(&q->hint[(hi32(cur) + 1) & (OURO_VL_HINTS - 1)], pack(hi32(cur) + 1, x));
  __threadfence();
  vl_advance(h, c);
}

/* Slot of position pos in the virtualized list of class c.  create: link
 * missing segments (producers); otherwise null while the segment is not
 * linked yet.  One thread creates each segment: it first claims the empty
 * link (next = OURO_BUSY); others wait for the link instead of creating. */
static __device__ __noinline__ unsigned long long *vl_slot_walk(const ouro_heap_dev &h, int c, unsigned long long pos,
                                                        bool create);

__device__ __forceinline__ unsigned long long *vl_slot(const ouro_heap_dev &h, int c, unsigned long long pos,
                                                       bool create) {
  ouro_qhdr *q = qh(h, c);
  const unsigned long long s = pos / h.seg_cap;
  const unsigned s32 = (unsigned)s;
  const unsigned off = (unsigned)(pos - s * h.seg_cap);
  unsigned long long e = ld_rlx(&q->hint[s32 & (OURO_VL_HINTS - 1)]);
  if (hi32(e) == s32 && lo32(e) < OURO_BUSY && hi32(ld_acq(&seg_of(h, lo32(e))->link)) == s32) {
    if (create && off - (h.seg_cap >> 3) < 32u) vl_prefetch(h, c, e);
    return seg_cells(h, lo32(e)) + off;
  }
  return vl_slot_walk(h, c, pos, create);
}

/* the lookup past a missed hint: out of line, it is the slow path */
static __device__ __noinline__ unsigned long long *vl_slot_walk(const ouro_heap_dev &h, int c, unsigned long long pos,
                                                        bool create) {
  ouro_qhdr *q = qh(h, c);
  const unsigned long long s = pos / h.seg_cap;
  const unsigned s32 = (unsigned)s;
  const unsigned off = (unsigned)(pos - s * h.seg_cap);
  unsigned ns = h.backoff_min_ns;
  unsigned long long cur = 0;
  bool walking = false;
  /* a missed hint: start from the nearest valid hint a few segments back */
  for (unsigned k = 1; k <= 8 && k <= s32; ++k) {
    const unsigned long long e2 = ld_rlx(&q->hint[(s32 - k) & (OURO_VL_HINTS - 1)]);
    if (hi32(e2) == s32 - k && lo32(e2) < OURO_BUSY && hi32(ld_acq(&seg_of(h, lo32(e2))->link)) == s32 - k) {
      cur = e2;
      walking = true;
      break;
    }
  }
  for (unsigned it = 0; it < h.spin_limit; ++it) {
    if (!walking) {
      cur = ld_acq(&q->back.v);
      if (lo32(cur) == OURO_NIL) {                   /* no segment yet: claim the first */
        if (!create) return nullptr;
        const unsigned long long busy = pack(hi32(cur), OURO_BUSY);
        if (cas_ar(&q->back.v, cur, busy) == cur) {
          unsigned x = seg_new(h, c, hi32(cur));
          if (x == OURO_NIL) {
            st_rel(&q->back.v, cur);
            set_error(h, OURO_ERR_QUEUE_FULL, OURO_SITE_VL_FIRST);
            return nullptr;
          }
          st_rel(&q->front.v, pack(hi32(cur), x));
          st_rel(&q->back.v, pack(hi32(cur), x));
        }
        continue;
      }
      if (lo32(cur) == OURO_BUSY) {                  /* first segment being created */
        backoff_wait(h, ns);
        ns = min(ns * 2, h.backoff_max_ns);
        continue;
      }
      if ((int)(s32 - hi32(cur)) < 0) {
        cur = ld_acq(&q->front.v);
        if (lo32(cur) >= OURO_BUSY || (int)(s32 - hi32(cur)) < 0) continue;
      }
      walking = true;
    }
    if (hi32(cur) == s32) {
      st_rlx(&q->hint[s32 & (OURO_VL_HINTS - 1)], cur);
      if (create && off - (h.seg_cap >> 3) < 32u) vl_prefetch(h, c, cur);
      return seg_cells(h, lo32(cur)) + off;
    }
    ouro_seg *sg = seg_of(h, lo32(cur));
    const unsigned long long link = ld_acq(&sg->link);
    if (hi32(link) != hi32(cur)) { walking = false; continue; }   /* segment was recycled */
    const unsigned nxt = lo32(link);
    if (nxt == OURO_NIL) {
      if (!create) return nullptr;
      if (cas_ar(&sg->link, link, pack(hi32(cur), OURO_BUSY)) == link) {
        unsigned x = seg_new(h, c, hi32(cur) + 1);
        if (x == OURO_NIL) {
          st_rel(&sg->link, link);
          set_error(h, OURO_ERR_QUEUE_FULL, OURO_SITE_VL_NEXT);
          return nullptr;
        }
        st_rel(&sg->link, pack(hi32(cur), x));
        const unsigned long long nb = pack(hi32(cur) + 1, x);
        cas_ar(&q->back.v, cur, nb);
        __threadfence();
        vl_advance(h, c);
        cur = nb;
      }
      continue;
    }
    if (nxt == OURO_BUSY) {                          /* someone is creating the successor */
      backoff_wait(h, ns);
      ns = min(ns * 2, h.backoff_max_ns);
      continue;
    }
    cur = pack(hi32(cur) + 1, nxt);
  }
  set_error(h, OURO_ERR_TIMEOUT, OURO_SITE_VL_WALK);
  return nullptr;
}

/* slot of position pos for storage form QF (template-resolved) */
template <int QF>
__device__ __forceinline__ unsigned long long *slot_at(const ouro_heap_dev &h, int c,
                                                       unsigned long long pos, bool create) {
  if (QF == OURO_QF_LIST) return vl_slot(h, c, pos, create);
  if (QF == OURO_QF_VARRAY) return va_slot(h, c, pos, create);
  return ring_slot(h, c, pos);
}

/* slot of position pos, storage form chosen at run time (host-side kernels) */
__device__ inline unsigned long long *slot_any(const ouro_heap_dev &h, int c, unsigned long long pos) {
  switch (ouro_qform((int)h.variant)) {
    case OURO_QF_LIST: return vl_slot(h, c, pos, false);
    case OURO_QF_VARRAY: return va_slot(h, c, pos, false);
    default: return ring_slot(h, c, pos);
  }
}

/* Queue storage first: make sure the segments for positions [first, last]
 * exist before a carve takes data chunks (virtualized forms). */
template <int QF>
__device__ inline void seg_prepare(const ouro_heap_dev &h, int c, unsigned long long first,
                                   unsigned long long last) {
  if (QF == OURO_QF_LIST) vl_slot(h, c, last, true);
  if (QF == OURO_QF_VARRAY)
    for (unsigned long long s = first / h.seg_cap; s <= last / h.seg_cap; ++s)
      va_slot(h, c, s * h.seg_cap, true);
}

/* ------------------------------------------------------- slot operations */
/* Producer of position pos puts item (or the null marker).  0: placed;
 * 1: the consumer gave the position up (caller re-queues the item);
 * -1: an earlier lap never drained (timeout). */
__device__ inline int put_at(const ouro_heap_dev &h, unsigned long long *cell, unsigned long long pos,
                             unsigned item, bool null_marker, bool single_use = false) {
  const unsigned long long want = null_marker ? slot(pos + 2, 0) : slot(pos + 1, item);
  if (single_use) {
    /* a single-use slot only ever holds: a stale sequence or a posted need
     * (empty), or the retired mark of a consumer that gave the position up;
     * one exchange publishes the answer, and the old value tells which */
    return slot_d(exch_rel(cell, want), pos) >= 3 ? 1 : 0;
  }
  unsigned long long expect = slot(pos, 0);
  unsigned ns = h.backoff_min_ns;
  for (unsigned it = 0; it < h.spin_limit; ++it) {
    unsigned long long old = cas_rel(cell, expect, want);
    if (old == expect) return 0;
    int d = slot_d(old, pos);
    if (d == 0 || (single_use && d < 0)) { expect = old; continue; }   /* empty (posted value / stale lap) */
    if (d >= 3) return 1;
    backoff_wait(h, ns);
    ns = min(ns * 2, h.backoff_max_ns);
    expect = slot(pos, 0);
  }
  set_error(h, OURO_ERR_QUEUE_OVERFLOW, OURO_SITE_PUT);
  return -1;
}

/* Consumer of position pos: 1 item, 2 null marker, 0 not there yet.
 * retired_seq: what the slot becomes (array rings: pos + ring size, ready
 * for the producer of the next lap; lists leave single-use slots alone). */
template <bool VL>
__device__ __forceinline__ int try_take(const ouro_heap_dev &h, int c, unsigned long long *cell,
                                        unsigned long long pos, unsigned *item) {
  unsigned long long v = ld_acq(cell);
  int d = slot_d(v, pos);
  if (d == 1 || d == 2) {
    *item = lo32(v);
    if (!VL) st_rlx(cell, slot(pos + h.ring_mask[c] + 1, 0));
    return d;
  }
  return 0;
}

/* Consumer gives up position pos: 3 given up, 1/2 the answer arrived
 * meanwhile, 0 not possible now (an earlier lap still holds the slot). */
template <bool VL>
__device__ inline int give_up(const ouro_heap_dev &h, int c, unsigned long long *cell,
                              unsigned long long pos, unsigned *item) {
  const unsigned long long retired = VL ? slot(pos + 3, 0) : slot(pos + h.ring_mask[c] + 1, 0);
  for (int it = 0; it < 8; ++it) {
    unsigned long long v = ld_acq(cell);
    int d = slot_d(v, pos);
    if (d == 1 || d == 2) {
      *item = lo32(v);
      if (!VL) st_rlx(cell, retired);
      return d;
    }
    if (d > 0 || (!VL && d != 0)) return 0;     /* list slots: behind the position is empty too */
    if (cas_ar(cell, v, retired) == v) return 3;
  }
  return 0;
}

/* Queue one item at a fresh producer position (re-queue after a give-up). */
template <int QF>
__device__ inline void push_one(const ouro_heap_dev &h, int c, unsigned item) {
  constexpr bool VL = QF != OURO_QF_RING;
  ouro_qhdr *q = qh(h, c);
  for (int tries = 0; tries < 64; ++tries) {
    unsigned long long t = atomicAdd(&q->tail.v, 1ull);
    unsigned long long *cell = slot_at<QF>(h, c, t, true);
    if (!cell) return;   /* error already recorded */
    int rc = put_at(h, cell, t, item, false, VL);
    if (VL) seg_event<QF>(h, c, cell, 1);
    if (rc == 0) return;
    if (rc < 0) return;
    stat_add(h, c, OURO_ST_REPUSH, 1);
  }
  set_error(h, OURO_ERR_TIMEOUT, OURO_SITE_PUSH_ONE);
}

/* ---------------------------------------------- page queues: carve batch */
/* Called by every lane of vmask; lane `owner` holds the carve lock of class
 * c and releases it.  Carves the chunks the class's current debt needs, up
 * to OURO_CARVE_SLOTS pages (one batch), then the warp writes the new page
 * ids into the debt slots.  If the heap (or the page-array capacity) is
 * exhausted, the remaining debt slots get the null marker.  The lock covers
 * only the reservation (chunks taken, tail advanced, or the tail moved to
 * the head with null answers): it is released before the slots are
 * written, so that the next warp in debt carves the next batch of the class
 * while this one fills, and a large debt is filled by many warps at once. */
template <int V, int FILL = 1>
__device__ void page_carve(const ouro_heap_dev &h, int c, unsigned vmask, int owner) {
  constexpr int QF = ouro_qform(V);
  constexpr bool VL = QF != OURO_QF_RING;
  ouro_qhdr *q = qh(h, c);
  const unsigned lane = laneid();
  const unsigned ppc_log = h.log2_chunk - 4 - c;
  const unsigned long long ppc = 1ull << ppc_log;
  unsigned m = 0;
  int exhausted = 0;
  unsigned long long t0 = 0;
  chunk_range r{0, 0, 0, 0};
  if ((int)lane == owner) {
    unsigned long long t = ld_acq(&q->tail.v), hd = ld_acq(&q->head.v);
    if (hd > t) {
      unsigned long long want = (hd - t + ppc - 1) >> ppc_log;
      unsigned long long ask = min(want, (unsigned long long)h.max_carve);
      ask = min(ask, max(1ull, (unsigned long long)(OURO_CARVE_SLOTS >> ppc_log)));
      if (V == OURO_PAGE_ARRAY) {
        unsigned long long limit = h.qcap[c] >> ppc_log, have = ld_rlx(&q->carved.v);
        ask = have >= limit ? 0 : min(ask, limit - have);
      }
      if (VL) {
        /* queue storage first: segments for every slot this carve (or its
         * null answers) will write, before the data chunks are taken */
        unsigned long long last = max(hd, t + (ask << ppc_log)) - 1;
        seg_prepare<QF>(h, c, t, last);
      }
      if (ask) r = take_chunks(h, (unsigned)ask);
      m = r.k1 + r.k2;
      exhausted = m < ask || ask == 0;
      if (m) {
        t0 = atomicAdd(&q->tail.v, (unsigned long long)m << ppc_log);
        atomicAdd(&q->carved.v, (unsigned long long)m);
        stat_add(h, c, OURO_ST_CARVE, m);
        OURO_TRACE_EVENT(OURO_TR_CARVE, c, m, t0);
      }
    }
  }
  unsigned long long dt = 0, dn = 0;
  if ((int)lane == owner) {
    if (exhausted) {   /* every position still in debt gets the null answer */
      for (unsigned it = 0; it < h.spin_limit; ++it) {
        unsigned long long t = ld_acq(&q->tail.v), hd = ld_acq(&q->head.v);
        if (hd <= t) break;
        if (atomicCAS(&q->tail.v, t, hd) == t) { dt = t; dn = hd - t; break; }
      }
      stat_add(h, c, OURO_ST_DEAD, dn);
      if (dn) OURO_TRACE_EVENT(OURO_TR_EXHAUSTED, c, dn, dt);
    }
    unlock(&q->lock.v);
  }
  m = __shfl_sync(vmask, m, owner);
  dt = __shfl_sync(vmask, dt, owner);
  dn = __shfl_sync(vmask, dn, owner);
  t0 = __shfl_sync(vmask, t0, owner);
  r.p0 = __shfl_sync(vmask, r.p0, owner);
  r.b0 = __shfl_sync(vmask, r.b0, owner);
  r.k1 = __shfl_sync(vmask, r.k1, owner);
  r.k2 = __shfl_sync(vmask, r.k2, owner);
  const unsigned nl = __popc(vmask), rk = __popc(vmask & lanemask_lt());
  if (m) {
    for (unsigned i = rk; i < m; i += nl) h.chunk_cls[range_chunk(h, r, i)] = (unsigned char)c;
    if (h.checked)
      for (unsigned long long i = rk; i < ((unsigned long long)m << ppc_log); i += nl) {
        unsigned x = range_chunk(h, r, (unsigned)(i >> ppc_log));
        unsigned pg = (unsigned)(i & (ppc - 1));
        atomicOr(&h.bits[(size_t)x * h.words_per_chunk + (pg >> 5)], 1u << (pg & 31));
      }
    __threadfence();
    __syncwarp(vmask);
    const unsigned long long total = (unsigned long long)m << ppc_log;
    /* FILL positions per lane per round: their first compare-and-swaps are
     * issued back to back (independent), then checked; a slot that was not
     * plainly empty falls back to put_at.  FILL = 1 keeps the callers'
     * registers free; latency-bound callers take more in flight. */
    for (unsigned long long i0 = 0; i0 < total; i0 += (unsigned long long)nl * FILL) {
      unsigned long long *cell[FILL];
      unsigned item[FILL];
      unsigned long long got[FILL];
#pragma unroll
      for (int f = 0; f < FILL; ++f) {
        const unsigned long long i = i0 + (unsigned long long)f * nl + rk;
        cell[f] = nullptr;
        item[f] = 0;
        if (i < total) {
          const unsigned x = range_chunk(h, r, (unsigned)(i >> ppc_log));
          item[f] = (x << ppc_log) | (unsigned)(i & (ppc - 1));
          cell[f] = slot_at<QF>(h, c, t0 + i, true);      /* null: queue storage exhausted (recorded) */
        }
      }
#pragma unroll
      for (int f = 0; f < FILL; ++f) {
        const unsigned long long p = t0 + i0 + (unsigned long long)f * nl + rk;
        got[f] = cell[f] ? cas_rel(cell[f], slot(p, 0), slot(p + 1, item[f])) : 0;
      }
#pragma unroll
      for (int f = 0; f < FILL; ++f) {
        const unsigned long long i = i0 + (unsigned long long)f * nl + rk;
        const unsigned long long p = t0 + i;
        int rc = 0;
        if (cell[f] && got[f] != slot(p, 0)) rc = put_at(h, cell[f], p, item[f], false, VL);
        if (VL) seg_event_warp<QF>(h, c, cell[f], i < total, vmask);
        if (cell[f] && rc == 1) push_one<QF>(h, c, item[f]);
      }
    }
  }
  for (unsigned long long i0 = 0; i0 < dn; i0 += nl) {
    const unsigned long long i = i0 + rk;
    const bool act = i < dn;
    unsigned long long *cell = act ? slot_at<QF>(h, c, dt + i, true) : nullptr;
    if (cell) put_at(h, cell, dt + i, 0, true, VL);
    if (VL) seg_event_warp<QF>(h, c, cell, act, vmask);
  }
  __syncwarp(vmask);
}

/* ------------------------------------------- run queues: carve batch */
/* Carve for a class above one chunk; called like page_carve (lane `owner`
 * holds the carve lock of class c).  The lock holder cuts every run the
 * class's debt needs -- m runs of k contiguous chunks -- with one
 * compare-and-swap at the bump pointer (pooled chunks are never gathered
 * into runs), and the warp writes the runs' first chunks into the debt
 * slots; the rest of the debt gets null markers once the heap is exhausted. */
template <int V>
__device__ __noinline__ void run_carve(const ouro_heap_dev &h, int c, unsigned vmask, int owner) {
  constexpr int QF = ouro_qform(V);
  constexpr bool VL = QF != OURO_QF_RING;
  ouro_qhdr *q = qh(h, c);
  ouro_glob *g = gl(h);
  const unsigned lane = laneid();
  const unsigned k_log = (unsigned)c - h.n_classes + 1;
  unsigned long long m = 0, b = 0, t0 = 0;
  int exhausted = 0;
  if ((int)lane == owner) {
    const unsigned long long t = ld_acq(&q->tail.v), hd = ld_acq(&q->head.v);
    if (hd > t) {
      const unsigned long long want = min(hd - t, (unsigned long long)h.max_carve);
      seg_prepare<QF>(h, c, t, t + want - 1);       /* queue storage first */
      b = ld_rlx(&g->bump.v);
      for (unsigned it = 0; it < h.spin_limit; ++it) {
        const unsigned long long avail = b < h.n_chunks ? (h.n_chunks - b) >> k_log : 0;
        const unsigned long long mm = min(want, avail);
        if (!mm) break;
        const unsigned long long seen = atomicCAS(&g->bump.v, b, b + (mm << k_log));
        if (seen == b) {
          m = mm;
          break;
        }
        b = seen;
      }
      exhausted = m < want;
      if (m) {
        t0 = atomicAdd(&q->tail.v, m);
        stat_add(h, c, OURO_ST_CARVE, m << k_log);
        OURO_TRACE_EVENT(OURO_TR_CARVE, c, m << k_log, t0);
      }
    }
  }
  m = __shfl_sync(vmask, m, owner);
  b = __shfl_sync(vmask, b, owner);
  t0 = __shfl_sync(vmask, t0, owner);
  exhausted = __shfl_sync(vmask, exhausted, owner);
  const unsigned nl = __popc(vmask), rk = __popc(vmask & lanemask_lt());
  if (m) {
    const unsigned long long nch = m << k_log;
    for (unsigned long long i = rk; i < nch; i += nl)
      h.chunk_cls[b + i] = (unsigned char)((i & ((1ull << k_log) - 1)) ? (OURO_CLS_RUN_BODY | c)
                                                                        : (OURO_CLS_RUN_FREE | c));
    __threadfence();
    __syncwarp(vmask);
    for (unsigned long long i0 = 0; i0 < m; i0 += nl) {
      const unsigned long long i = i0 + rk;
      const bool act = i < m;
      unsigned long long *cell = act ? slot_at<QF>(h, c, t0 + i, true) : nullptr;
      int rc = 0;
      if (cell) rc = put_at(h, cell, t0 + i, (unsigned)(b + (i << k_log)), false, VL);
      if (VL) seg_event_warp<QF>(h, c, cell, act, vmask);
      if (cell && rc == 1) push_one<QF>(h, c, (unsigned)(b + (i << k_log)));
    }
  }
  if (exhausted) {
    unsigned long long dt = 0, dn = 0;
    if ((int)lane == owner) {
      for (unsigned it = 0; it < h.spin_limit; ++it) {
        const unsigned long long t = ld_acq(&q->tail.v), hd = ld_acq(&q->head.v);
        if (hd <= t) break;
        seg_prepare<QF>(h, c, t, hd - 1);
        if (atomicCAS(&q->tail.v, t, hd) == t) { dt = t; dn = hd - t; break; }
      }
      stat_add(h, c, OURO_ST_DEAD, dn);
      if (dn) OURO_TRACE_EVENT(OURO_TR_EXHAUSTED, c, dn, dt);
    }
    dt = __shfl_sync(vmask, dt, owner);
    dn = __shfl_sync(vmask, dn, owner);
    for (unsigned long long i0 = 0; i0 < dn; i0 += nl) {
      const unsigned long long i = i0 + rk;
      const bool act = i < dn;
      unsigned long long *cell = act ? slot_at<QF>(h, c, dt + i, true) : nullptr;
      if (cell) put_at(h, cell, dt + i, 0, true, VL);
      if (VL) seg_event_warp<QF>(h, c, cell, act, vmask);
    }
  }
  __syncwarp(vmask);
  if ((int)lane == owner) unlock(&q->lock.v);
}

/* --------------------------------------------------------- page queues */
/* Every lane of vmask calls.  A lane with cls >= 0 asks for a page of that
 * class (any mix of classes); a lane with cls < 0 asks for nothing and only
 * helps: it takes part in the warp's carves, so that a warp in which one
 * lane allocates still fills new slots 32 lanes wide. */
template <int V, int FILL = 1, bool RESERVED = false>
__device__ void *page_malloc(const ouro_heap_dev &h, int cls, unsigned vmask, unsigned long long p_reserved = 0) {
  constexpr int QF = ouro_qform(V);
  constexpr bool VL = QF != OURO_QF_RING;
  const bool req = cls >= 0;
  ouro_qhdr *q = qh(h, req ? cls : 0);
  const unsigned lane = laneid();
  const unsigned grp = warp_group(h, vmask, cls);
  const unsigned leader = __ffs(grp) - 1;
  const unsigned rank = __popc(grp & lanemask_lt());
  unsigned long long pos = 0;
  if (RESERVED) pos = p_reserved;    /* the caller took this lane's head position (block aggregation) */
  else if (req && lane == leader) pos = atomicAdd(&q->head.v, (unsigned long long)__popc(grp));
  const unsigned long long p0 = __shfl_sync(vmask, pos, leader);   /* the group leader's position */
  if (!RESERVED) pos = p0 + rank;

  unsigned item = 0;
  int st = req ? 0 : 3;   /* 0 waiting, 1 item, 2 null answer, 3 gave up (helpers: nothing asked) */
  unsigned long long *cell = nullptr;
  if (VL) {   /* the leader finds its segment; lanes in the same segment reuse it */
    unsigned long long *c0 = (req && lane == leader) ? slot_at<QF>(h, cls, p0, false) : nullptr;
    c0 = reinterpret_cast<unsigned long long *>(
        __shfl_sync(vmask, reinterpret_cast<unsigned long long>(c0), leader));
    if (req)
      cell = (c0 && pos / h.seg_cap == p0 / h.seg_cap) ? c0 + (long long)(pos - p0) : slot_at<QF>(h, cls, pos, false);
  } else if (req) {
    cell = ring_slot(h, cls, pos);
  }
  if (req && cell) st = try_take<VL>(h, cls, cell, pos, &item);

  bool gave_up = false;
  if (__ballot_sync(vmask, st == 0)) {
    unsigned ns = h.backoff_min_ns;
    for (unsigned it = 0;; ++it) {
      bool debt = false, progressed = false;
      if (st == 0) {
        if (VL && !cell) cell = slot_at<QF>(h, cls, pos, false);
        if (cell) st = try_take<VL>(h, cls, cell, pos, &item);
        if (st) progressed = true;
        else debt = pos >= ld_acq(&q->tail.v);
      }
      const unsigned dmask = __ballot_sync(vmask, debt);
      if (dmask) {
        /* one lock attempt per warp, for the class of its lowest lane in
         * debt: a warp carves one class at a time, and the lock holder
         * carves the whole debt of its class, so the classes of a cold heap
         * are carved by different warps at once (a warp that took the locks
         * of several classes carved them in turn while the others waited) */
        const bool trier = debt && lane == (unsigned)(__ffs(dmask) - 1);
        const bool got = trier && try_lock(&q->lock.v);
        unsigned lockers = __ballot_sync(vmask, got);
        while (lockers) {
          const int j = __ffs(lockers) - 1;
          lockers &= lockers - 1;
          const int cj = __shfl_sync(vmask, cls, j);
          if (cj >= (int)h.n_classes) run_carve<V>(h, cj, vmask, j);
          else page_carve<V, FILL>(h, cj, vmask, j);
        }
      }
      const unsigned waiting = __ballot_sync(vmask, st == 0);
      if (!waiting) break;
      if (it >= h.spin_limit) {
        if (st == 0) {   /* give the position up so its producer re-queues the item */
          if (!cell) cell = slot_at<QF>(h, cls, pos, true);
          int g = cell ? give_up<VL>(h, cls, cell, pos, &item) : 0;
          st = g ? g : 3;
          gave_up = g == 3;
          if (st == 3) {
            set_error(h, OURO_ERR_TIMEOUT, OURO_SITE_PAGE_GIVEUP);
            stat_add(h, cls, OURO_ST_CANCEL, 1);
            OURO_TRACE_EVENT(OURO_TR_GIVEUP, cls, pos, OURO_SITE_PAGE_GIVEUP);
          }
        }
        break;
      }
      if (!__any_sync(vmask, progressed)) {
        backoff_wait(h, ns);
        ns = min(ns * 2, h.backoff_max_ns);
      } else {
        ns = h.backoff_min_ns;
      }
    }
  }
  if (VL) seg_event_warp<QF, RESERVED ? OURO_VL_WIDE_BATCH : OURO_VL_WIDE>(h, cls, cell, st != 0 && (st != 3 || gave_up), vmask);

  void *res = nullptr;
  if (st == 1) {
    if (cls >= (int)h.n_classes) {          /* a run: item is its first chunk, live again */
      h.chunk_cls[item] = (unsigned char)cls;
      res = h.base + ((size_t)item << h.log2_chunk);
    } else {
      if (h.checked) {
        unsigned pg = item & ((1u << (h.log2_chunk - 4 - cls)) - 1);
        unsigned x = item >> (h.log2_chunk - 4 - cls);
        unsigned bit = 1u << (pg & 31);
        unsigned old = atomicAnd(&h.bits[(size_t)x * h.words_per_chunk + (pg >> 5)], ~bit);
        if (!(old & bit)) set_error(h, OURO_ERR_DOUBLE_FREE, OURO_SITE_PAGE_CHECKED);
      }
      res = h.base + ((size_t)item << (4 + cls));
    }
  }
  /* per-class counters, one update per class group of the warp (a caller
   * with reserved positions counts for its whole block) */
  if (!RESERVED) {
    const unsigned g2 = warp_group(h, vmask, cls);
    const unsigned okm = __ballot_sync(vmask, st == 1) & g2;
    if (req && lane == (unsigned)(__ffs(g2) - 1)) {
      stat_add(h, cls, OURO_ST_MALLOC, __popc(okm));
      stat_add(h, cls, OURO_ST_FAILED, __popc(g2) - __popc(okm));
    }
  }
  return res;
}

template <int V, bool RESERVED = false>
__device__ void page_free(const ouro_heap_dev &h, int cls, unsigned item, unsigned vmask,
                          unsigned long long t_reserved = 0) {
  constexpr int QF = ouro_qform(V);
  constexpr bool VL = QF != OURO_QF_RING;
  ouro_qhdr *q = qh(h, cls);
  const unsigned lane = laneid();
  const unsigned grp = warp_group(h, vmask, cls);
  const unsigned leader = __ffs(grp) - 1;
  const unsigned rank = __popc(grp & lanemask_lt());
  unsigned long long t = 0;
  if (RESERVED) {
    t = t_reserved;    /* the caller took this lane's tail position and counted the frees */
  } else if (lane == leader) {
    t = atomicAdd(&q->tail.v, (unsigned long long)__popc(grp));
    stat_add(h, cls, OURO_ST_FREE, __popc(grp));
  }
  const unsigned long long t0 = __shfl_sync(vmask, t, leader);   /* the group leader's position */
  if (!RESERVED) t = t0 + rank;
  unsigned long long *cell;
  if (VL) {   /* the leader finds (or links) its segment; lanes in the same segment reuse it */
    unsigned long long *c0 = lane == leader ? slot_at<QF>(h, cls, t0, true) : nullptr;
    c0 = reinterpret_cast<unsigned long long *>(
        __shfl_sync(vmask, reinterpret_cast<unsigned long long>(c0), leader));
    cell = (c0 && t / h.seg_cap == t0 / h.seg_cap) ? c0 + (long long)(t - t0) : slot_at<QF>(h, cls, t, true);
  } else {
    cell = ring_slot(h, cls, t);
  }
  int rc = cell ? put_at(h, cell, t, item, false, VL) : 0;   /* no slot: queue storage exhausted, page lost (recorded) */
  if (VL) seg_event_warp<QF>(h, cls, cell, true, vmask);
  if (rc == 1) {
    stat_add(h, cls, OURO_ST_REPUSH, 1);
    push_one<QF>(h, cls, item);
  }
}

/* Locate a block: class and page id (a class of one chunk or less), or
 * class and first chunk (a run); -1 when p is no block start. */
__device__ __forceinline__ int locate(const ouro_heap_dev &h, const void *p, unsigned *item) {
  const unsigned char *b = static_cast<const unsigned char *>(p);
  if (b < h.base || b >= h.base + h.bytes) return -1;
  const unsigned long long off = (unsigned long long)(b - h.base);
  unsigned c = h.chunk_cls[off >> h.log2_chunk];
  if (c < h.n_classes) {
    if (off & ((16ull << c) - 1)) return -1;
    *item = (unsigned)(off >> (4 + c));
    return (int)c;
  }
  if ((c & 0xC0u) == OURO_CLS_RUN_FREE) c &= 0x3Fu;   /* a free run: run_free reports the double free */
  if (c >= OURO_MAX_CLASSES || (off & (h.chunk_bytes - 1))) return -1;
  *item = (unsigned)(off >> h.log2_chunk);
  return (int)c;
}

/* ------------------------------------------------ runs above one chunk */
/* Requests above one chunk (the paper is silent on them): class c >=
 * n_classes is a run of 2^(c - n_classes + 1) contiguous chunks.  Its class
 * queue, in the heap's queue form like every other class, holds the first
 * chunks of free runs; a debt is carved by cutting runs at the bump pointer
 * (run_carve).  The class byte of a run's first chunk tells a live run (c)
 * from a free one (RUN_FREE | c), so that a second free is seen. */

/* Mark run x of class c free: its class byte turns from c to RUN_FREE | c
 * in one compare-and-swap of the word holding it.  False (error recorded)
 * when the run is already free or x is no run start. */
__device__ inline bool run_mark_free(const ouro_heap_dev &h, int c, unsigned x) {
  unsigned *w = reinterpret_cast<unsigned *>(h.chunk_cls + (x & ~3u));
  const unsigned sh = (x & 3u) * 8u;
  for (unsigned it = 0; it < h.spin_limit; ++it) {
    const unsigned v = *(volatile unsigned *)w;
    const unsigned byte = (v >> sh) & 0xFFu;
    if (byte != (unsigned)c) {
      set_error(h, byte == (OURO_CLS_RUN_FREE | (unsigned)c) ? OURO_ERR_DOUBLE_FREE : OURO_ERR_BAD_FREE,
                OURO_SITE_RUN_FREE);
      return false;
    }
    if (atomicCAS(w, v, (v & ~(0xFFu << sh)) | ((OURO_CLS_RUN_FREE | (unsigned)c) << sh)) == v) return true;
  }
  set_error(h, OURO_ERR_TIMEOUT, OURO_SITE_RUN_FREE);
  return false;
}

/* ------------------------------------------------------- chunk queues */
/* Chunk queues (Sec. 4.2): a class queue holds ids of chunks that have free
 * pages; a malloc obtains a chunk id, then claims free pages of that chunk
 * from its bitmap.  GB300 form: a warp group POPS a chunk id (one position,
 * like a page queue), reserves pages with one atomicSub on the chunk's free
 * count, claims the bits, and pushes the chunk back while it still has free
 * pages; a chunk is in its queue at most once.  A free sets the bit, adds to
 * the count, and the increment that lifts the count from <= 0 to >= 1 queues
 * the chunk again.  Carving packs the page needs that waiting groups posted
 * in their empty slots into fresh chunks, with those pages reserved, so the
 * number of chunks carved for a malloc-only burst follows the demand. */

/* slot item of a chunk queue: chunk id, or a reserved fill
 * (bit 31 | (reserved pages - 1) << 26 | chunk id) */
#define OURO_CQ_RES 0x80000000u
#define OURO_CQ_ID(it) ((it) & ((1u << 26) - 1))
#define OURO_CQ_CNT(it) ((((it) >> 26) & 31u) + 1)

template <int QF>
__device__ inline void chunk_push(const ouro_heap_dev &h, int c, unsigned x) {
  push_one<QF>(h, c, x);
}

/* Queue item x in class c's queue for every lane of mask with `want` (any
 * mix of classes): one tail atomic per class group of the warp, then every
 * such lane publishes its own slot.  Every lane of mask calls. */
template <int QF>
__device__ inline void push_group(const ouro_heap_dev &h, int c, unsigned x, bool want, unsigned mask) {
  constexpr bool VL = QF != OURO_QF_RING;
  const unsigned pm = __ballot_sync(mask, want);
  if (!pm) return;
  const unsigned g = warp_group(h, mask, want ? c : -1) & pm;
  const unsigned leader = want ? (unsigned)(__ffs(g) - 1) : laneid();
  unsigned long long t = 0;
  if (want && laneid() == leader) t = atomicAdd(&qh(h, c)->tail.v, (unsigned long long)__popc(g));
  t = __shfl_sync(mask, t, leader);
  if (!want) return;
  t += __popc(g & lanemask_lt());
  unsigned long long *cell = slot_at<QF>(h, c, t, true);
  if (!cell) return;                            /* queue storage exhausted (recorded) */
  const int rc = put_at(h, cell, t, x, false, VL);
  if (VL) seg_event<QF>(h, c, cell, 1);
  if (rc == 1) push_one<QF>(h, c, x);            /* the consumer gave the position up */
}

/* Called by every lane of vmask; lane `owner` holds the carve lock of class c. */
template <int V>
__device__ __noinline__ void chunk_carve(const ouro_heap_dev &h, int c, unsigned vmask, int owner) {
  constexpr int QF = ouro_qform(V);
  constexpr bool VL = QF != OURO_QF_RING;
  ouro_qhdr *q = qh(h, c);
  const unsigned lane = laneid();
  const unsigned ppc_log = h.log2_chunk - 4 - c;
  const unsigned ppc = 1u << ppc_log;
  const unsigned words_c = (ppc + 31) >> 5;
  const unsigned nl = __popc(vmask), rk = __popc(vmask & lanemask_lt());
  const bool full_warp = vmask == 0xffffffffu;
  for (int batch = 0; batch < 64; ++batch) {
    /* 1. the debt positions of this batch, claimed as producer */
    unsigned long long t = 0, hd = 0;
    unsigned D = 0;
    if ((int)lane == owner) {
      for (unsigned it = 0; it < 64; ++it) {
        t = ld_acq(&q->tail.v);
        hd = ld_acq(&q->head.v);
        if (hd <= t) break;
        unsigned d = (unsigned)min(hd - t, 8ull * nl);   /* each lane plans up to 8 positions */
        seg_prepare<QF>(h, c, t, t + d - 1);              /* segments before chunks */
        if (atomicCAS(&q->tail.v, t, t + d) == t) { D = d; break; }
      }
    }
    D = __shfl_sync(vmask, D, owner);
    if (!D) break;
    t = __shfl_sync(vmask, t, owner);
    /* 2. posted needs (an unposted slot counts as a full warp) and their prefix sum */
    unsigned need[8];
    unsigned long long *cell[8];
    unsigned excl[8];
    unsigned running = 0;
    for (int r = 0; r < 8; ++r) {
      const unsigned i = rk + (unsigned)r * nl;
      need[r] = 0;
      cell[r] = nullptr;
      if (i < D) {
        cell[r] = slot_at<QF>(h, c, t + i, true);
        unsigned long long v = cell[r] ? ld_acq(cell[r]) : 0;
        unsigned posted = (cell[r] && slot_d(v, t + i) == 0) ? lo32(v) : 0;
        need[r] = posted ? min(posted, 32u) : 32u;
      }
      /* inclusive scan over the lanes of vmask (positions rk + r*nl are in lane order) */
      unsigned x = need[r];
      if (full_warp) {
        for (int o = 1; o < 32; o <<= 1) {
          unsigned y = __shfl_up_sync(0xffffffffu, x, o);
          if ((int)lane >= o) x += y;
        }
      } else {
        /* sparse warp: gather through the lanes in order */
        unsigned acc = 0, mm = vmask;
        while (mm) {
          int l = __ffs(mm) - 1;
          mm &= mm - 1;
          unsigned v = __shfl_sync(vmask, need[r], l);
          if ((unsigned)l <= lane) acc += v;
        }
        x = acc;
      }
      excl[r] = running + x - need[r];
      unsigned last = 31 - __clz(vmask);
      running += __shfl_sync(vmask, x, last);
    }
    const unsigned total = running;
    const unsigned m = (total + ppc - 1) >> ppc_log;
    /* 3. chunks for the batch */
    chunk_range cr{0, 0, 0, 0};
    if ((int)lane == owner) {
      cr = take_chunks(h, m);
      if (cr.k1 + cr.k2) stat_add(h, c, OURO_ST_CARVE, cr.k1 + cr.k2);
      OURO_TRACE_EVENT(OURO_TR_CHUNK_CARVE, c, cr.k1 + cr.k2, D);
    }
    cr.p0 = __shfl_sync(vmask, cr.p0, owner);
    cr.b0 = __shfl_sync(vmask, cr.b0, owner);
    cr.k1 = __shfl_sync(vmask, cr.k1, owner);
    cr.k2 = __shfl_sync(vmask, cr.k2, owner);
    const unsigned g = cr.k1 + cr.k2;
    for (unsigned k = rk; k < g; k += nl) {
      const unsigned x = range_chunk(h, cr, k);
      h.chunk_cls[x] = (unsigned char)c;
      h.chunk_free[x] = 0;                 /* reservations below, then +ppc once published */
      unsigned *w = h.bits + (size_t)x * h.words_per_chunk;
      for (unsigned j = 0; j < words_c; ++j) w[j] = ppc >= 32 ? 0xffffffffu : ((1u << ppc) - 1);
    }
    __threadfence();
    __syncwarp(vmask);
    /* 4. reservations: position i takes min(need, room left in its chunk) */
    unsigned item[8];
    for (int r = 0; r < 8; ++r) {
      item[r] = 0xffffffffu;
      const unsigned i = rk + (unsigned)r * nl;
      if (i >= D) continue;
      const unsigned k = excl[r] >> ppc_log;
      if (k >= g) continue;                                /* heap exhausted: null answer */
      const unsigned x = range_chunk(h, cr, k);
      const unsigned res = min(need[r], ppc - (excl[r] & (ppc - 1)));
      atomicSub(&h.chunk_free[x], (int)res);
      item[r] = OURO_CQ_RES | ((res - 1) << 26) | x;
    }
    __threadfence();
    __syncwarp(vmask);
    /* 5. publish; then queue every new chunk that still has free pages */
    for (int r = 0; r < 8; ++r) {
      const unsigned i = rk + (unsigned)r * nl;
      if (i >= D || !cell[r]) continue;
      const bool isnull = item[r] == 0xffffffffu;
      int rc = put_at(h, cell[r], t + i, isnull ? 0 : item[r], isnull, VL);
      if (VL) seg_event<QF>(h, c, cell[r], 1);   /* planned positions: at most 8 per lane */
      if (rc == 1 && !isnull) {   /* its group gave up: hand the reserved pages back */
        const unsigned x = OURO_CQ_ID(item[r]);
        int before = atomicAdd(&h.chunk_free[x], (int)OURO_CQ_CNT(item[r]));
        if (before <= 0 && before + (int)OURO_CQ_CNT(item[r]) >= 1) chunk_push<QF>(h, c, x);
      }
      if (isnull) stat_add(h, c, OURO_ST_DEAD, 1);
    }
    __syncwarp(vmask);
    /* the count stays <= 0 until now (frees of reserved pages only return
     * what was reserved), so adding the pages here lifts it above zero
     * exactly once: the chunk is queued once iff it has a free page */
    for (unsigned k0 = 0; k0 < g; k0 += nl) {
      const unsigned k = k0 + rk;
      const unsigned x = k < g ? range_chunk(h, cr, k) : 0;
      bool lift = false;
      if (k < g) {
        const int b = atomicAdd(&h.chunk_free[x], (int)ppc);
        lift = b <= 0 && b + (int)ppc >= 1;
      }
      push_group<QF>(h, c, x, lift, vmask);
    }
    __syncwarp(vmask);
    if (g < m) {
      /* exhausted: every remaining waiting position gets the null answer */
      unsigned long long dt = 0, dn = 0;
      if ((int)lane == owner) {
        for (unsigned it = 0; it < h.spin_limit; ++it) {
          unsigned long long t2 = ld_acq(&q->tail.v), h2 = ld_acq(&q->head.v);
          if (h2 <= t2) break;
          seg_prepare<QF>(h, c, t2, h2 - 1);
          if (atomicCAS(&q->tail.v, t2, h2) == t2) { dt = t2; dn = h2 - t2; break; }
        }
        stat_add(h, c, OURO_ST_DEAD, dn);
        if (dn) OURO_TRACE_EVENT(OURO_TR_EXHAUSTED, c, dn, dt);
      }
      dt = __shfl_sync(vmask, dt, owner);
      dn = __shfl_sync(vmask, dn, owner);
      for (unsigned long long i = rk; i < dn; i += nl) {
        unsigned long long *cl = slot_at<QF>(h, c, dt + i, true);
        if (!cl) continue;
        put_at(h, cl, dt + i, 0, true, VL);
        if (VL) seg_event<QF>(h, c, cl, 1);
      }
      break;
    }
  }
  __syncwarp(vmask);
  if ((int)lane == owner) unlock(&q->lock.v);
}

/* Claim `got` free pages of chunk x for the lanes of group gmask whose rank
 * is below got; lanes receive their page index.  The reservation on the
 * chunk's count guarantees that enough bits are set, so the claim keeps
 * scanning (bounded by spin_limit) until it has them all.  The leader
 * claims several bits per atomicAnd and reuses the word value the atomic
 * returned; every lane of gmask calls. */
__device__ inline unsigned claim_pages(const ouro_heap_dev &h, unsigned x, unsigned ppc, unsigned got,
                                       unsigned gmask, unsigned leader, unsigned rank, unsigned seed) {
  const unsigned lane = laneid();
  const unsigned words_c = (ppc + 31) >> 5;
  unsigned *bw = h.bits + (size_t)x * h.words_per_chunk;
  unsigned need = got, base = 0, mine = OURO_NIL;
  unsigned w = words_c > 1 ? seed % words_c : 0;
  unsigned v = 0, empty = 0, ns = h.backoff_min_ns;
  if (lane == leader) v = *(volatile unsigned *)&bw[w];
  for (unsigned it = 0; need && it < h.spin_limit; ++it) {
    unsigned claimed = 0, cword = 0;
    if (lane == leader) {
      if (v) {
        cword = w;
        unsigned m = 0, tmp = v;
        for (unsigned k = 0; k < need && tmp; ++k) {
          const unsigned b = tmp & (0u - tmp);
          m |= b;
          tmp ^= b;
        }
        const unsigned old = atomicAnd(&bw[w], ~m);
        claimed = old & m;
        v = old & ~m;                       /* bits still free in this word */
        empty = 0;
      }
      if (!v) {
        w = (w + 1 == words_c) ? 0 : w + 1;
        if (++empty > words_c) {            /* a whole pass found nothing: bits still being freed */
          backoff_wait(h, ns);
          ns = min(ns * 2, h.backoff_max_ns);
          empty = 0;
        }
        v = *(volatile unsigned *)&bw[w];
      }
    }
    const unsigned cw = __shfl_sync(gmask, claimed ? cword : 0u, leader);
    claimed = __shfl_sync(gmask, claimed, leader);
    const unsigned n = __popc(claimed);
    if (rank >= base && rank < base + n && rank < got) {
      unsigned tmp = claimed;
      for (unsigned k = base; k < rank; ++k) tmp &= tmp - 1;
      mine = (cw << 5) + (__ffs(tmp) - 1);
    }
    base += n;
    need -= n;
  }
  if (need && lane == leader) set_error(h, OURO_ERR_TIMEOUT, OURO_SITE_CLAIM);
  return mine;
}

/* Every lane of vmask calls; lanes with cls < 0 only help (see page_malloc). */
template <int V>
__device__ void *chunk_malloc(const ouro_heap_dev &h, int cls, unsigned vmask) {
  constexpr int QF = ouro_qform(V);
  constexpr bool VL = QF != OURO_QF_RING;
  const bool req = cls >= 0;
  ouro_qhdr *q = qh(h, req ? cls : 0);
  const unsigned lane = laneid();
  const unsigned ppc_log = req ? h.log2_chunk - 4 - cls : 0;
  const unsigned ppc = 1u << ppc_log;
  int st = req ? 0 : 2;          /* 0 waiting, 1 page, 2 null (helpers: nothing asked) */
  unsigned page = 0, chunk = 0;
  /* group-leader state: one queue position at a time */
  bool have = false, posted = false;
  unsigned long long pos = 0;
  unsigned long long *cell = nullptr;
  unsigned ns = h.backoff_min_ns;
  for (unsigned it = 0;; ++it) {
    const unsigned pend = __ballot_sync(vmask, st == 0);
    if (!pend) break;
    const unsigned gmask = warp_group(h, vmask, st == 0 ? cls : -1) & pend;
    const bool mine = st == 0;
    const unsigned leader = mine ? __ffs(gmask) - 1 : 0;
    const unsigned rank = mine ? __popc(gmask & lanemask_lt()) : 0;
    const unsigned need = __popc(gmask);
    unsigned got_item = 0, res = 0;    /* res: 0 none, 1 chunk, 2 null marker */
    bool debt = false;
    if (mine && lane == leader) {
      if (!have) {
        pos = atomicAdd(&q->head.v, 1ull);
        have = true;
        posted = false;
        cell = nullptr;
      }
      if (!cell) cell = slot_at<QF>(h, cls, pos, false);
      unsigned item = 0;
      int r = cell ? try_take<VL>(h, cls, cell, pos, &item) : 0;
      if (r) {
        if (VL) seg_event<QF>(h, cls, cell, 1);
        have = false;
        res = (unsigned)r;
        got_item = item;
      } else if (pos >= ld_acq(&q->tail.v)) {
        debt = true;
        if (!posted) {
          if (!cell && VL) cell = slot_at<QF>(h, cls, pos, true);
          if (cell) {
            const unsigned long long e = ld_acq(cell);
            const int d = slot_d(e, pos);
            posted = true;
            if (d == 0 || (VL && d < 0)) cas_ar(cell, e, slot(pos, need));
          }
        }
      }
      if (it >= h.spin_limit && !res) {                 /* bounded wait ran out */
        if (!cell) cell = slot_at<QF>(h, cls, pos, true);
        unsigned item2 = 0;
        int g = cell ? give_up<VL>(h, cls, cell, pos, &item2) : 0;
        if (g == 1 || g == 2) {
          res = (unsigned)g;
          got_item = item2;
        } else {
          res = 2;
          set_error(h, OURO_ERR_TIMEOUT, OURO_SITE_CHUNK_GIVEUP);
          stat_add(h, cls, OURO_ST_CANCEL, 1);
        }
        if (VL && cell && g) seg_event<QF>(h, cls, cell, 1);
        have = false;
      }
    }
    /* carve: one lock taker per class among the debtors of the warp */
    const unsigned dmask = __ballot_sync(vmask, debt);
    if (dmask) {
      const bool got = debt && lane == (unsigned)(__ffs(dmask) - 1) && try_lock(&q->lock.v);   /* see page_malloc */
      unsigned lockers = __ballot_sync(vmask, got);
      while (lockers) {
        const int j = __ffs(lockers) - 1;
        lockers &= lockers - 1;
        chunk_carve<V>(h, __shfl_sync(vmask, cls, j), vmask, j);
      }
    }
    /* every group learns its leader's answer */
    const unsigned gl_leader = mine ? leader : lane;
    res = __shfl_sync(vmask, res, gl_leader);
    got_item = __shfl_sync(vmask, got_item, gl_leader);
    const unsigned any = __ballot_sync(vmask, mine && res != 0);
    if (mine && res == 2) st = 2;
    /* groups holding a chunk reserve and claim pages, every group at once:
     * the leaders' count atomics (and pushes) are issued together, then each
     * group claims from its own chunk with collectives over its own lanes */
    const bool holder = mine && res == 1;            /* uniform within a group */
    unsigned granted = 0, x = 0;
    if (holder && lane == leader) {
      x = OURO_CQ_ID(got_item);
      if (got_item & OURO_CQ_RES) {
        const unsigned cnt = OURO_CQ_CNT(got_item);
        granted = min(cnt, need);
        if (cnt > need) {   /* reserved for a warp-sized need that was not posted: hand back the rest */
          const int ex = (int)(cnt - need);
          const int b = atomicAdd(&h.chunk_free[x], ex);
          if (b <= 0 && b + ex >= 1) chunk_push<QF>(h, cls, x);
        }
      } else {
        const int old = atomicSub(&h.chunk_free[x], (int)need);
        granted = old <= 0 ? 0 : min((unsigned)old, need);
        const int left = old - (int)need;
        if (left >= 1) chunk_push<QF>(h, cls, x);
        if (granted < need) {
          const int ex = (int)(need - granted);
          const int b = atomicAdd(&h.chunk_free[x], ex);
          if (b <= 0 && b + ex >= 1) chunk_push<QF>(h, cls, x);
        }
      }
    }
    granted = __shfl_sync(vmask, granted, gl_leader);
    x = __shfl_sync(vmask, x, gl_leader);
    if (holder) {
      /* start word: spread groups of different warps over the chunk's words */
      const unsigned seed = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 0x9E3779B1u ^ (x * 0x85EBCA6Bu) ^ it;
      const unsigned pg = claim_pages(h, x, ppc, granted, gmask, leader, rank, seed >> 7);
      if (pg != OURO_NIL) {
        st = 1;
        page = pg;
        chunk = x;
      }
    }
    if (__ballot_sync(vmask, st == 0) == 0) break;
    if (!any) {
      backoff_wait(h, ns);
      ns = min(ns * 2, h.backoff_max_ns);
    } else {
      ns = h.backoff_min_ns;
    }
  }
  void *ret = nullptr;
  if (st == 1) ret = h.base + ((size_t)chunk << h.log2_chunk) + ((size_t)page << (4 + cls));
  const unsigned g2 = warp_group(h, vmask, cls);
  const unsigned okm = __ballot_sync(vmask, st == 1) & g2;
  if (req && lane == (unsigned)(__ffs(g2) - 1)) {
    stat_add(h, cls, OURO_ST_MALLOC, __popc(okm));
    stat_add(h, cls, OURO_ST_FAILED, __popc(g2) - __popc(okm));
  }
  (void)ppc;
  return ret;
}

/* The release half of a chunk-queue free: every lane of mask calls; lanes
 * with cls < 0 only take part.  Sets the page's bit and counts it back on
 * its chunk; true for the lane whose count increment lifted the chunk from
 * <= 0 to >= 1 (that lane queues chunk x).  cls turns to -1 on a double
 * free (recorded).  FENCE = false: the caller's blocks were written before
 * the kernel began and no malloc runs in the same kernel (the batch free
 * kernels), so no release is needed */
template <bool FENCE = true>
__device__ bool chunk_release(const ouro_heap_dev &h, int &cls, const void *p, unsigned mask, unsigned &x) {
  const unsigned lane = laneid();
  unsigned pg = 0;
  x = 0;
  if (cls >= 0) {
    const unsigned long long off = (unsigned long long)((const unsigned char *)p - h.base);
    x = (unsigned)(off >> h.log2_chunk);
    pg = (unsigned)((off & (h.chunk_bytes - 1)) >> (4 + cls));
  }
  /* 1. set the page bits, one atomicOr per (chunk, word) group; the fence
   * releases the block's data (and, after a warp barrier, the data other
   * lanes wrote into it) before the page can be claimed again */
  if (FENCE) fence_acq_rel();
  const unsigned long long wkey = cls >= 0 ? (((unsigned long long)x << 32) | (pg >> 5)) : ~0ull;
  const unsigned wg = warp_group(h, mask, wkey);
  const unsigned bit = cls >= 0 ? 1u << (pg & 31) : 0u;
  const unsigned bits = __reduce_or_sync(wg, bit);
  unsigned old = 0;
  if (cls >= 0 && lane == (unsigned)(__ffs(wg) - 1))
    old = atomicOr(&h.bits[(size_t)x * h.words_per_chunk + (pg >> 5)], bits);
  old = __shfl_sync(mask, old, __ffs(wg) - 1);
  if (cls >= 0 && (old & bit)) {
    set_error(h, OURO_ERR_DOUBLE_FREE, OURO_SITE_CHUNK_DOUBLE);
    cls = -1;
  }
  /* 2. count the pages back per chunk; lifting the count from <= 0 queues it */
  const unsigned cg = warp_group(h, mask, cls >= 0 ? x : OURO_NIL) & __ballot_sync(mask, cls >= 0);
  bool lift = false;
  if (cls >= 0 && lane == (unsigned)(__ffs(cg) - 1)) {
    /* the count goes up after the bits are set (a reserving malloc that
     * sees the count finds the bits, or waits for them in its claim) */
    const int k = __popc(cg);
    if (FENCE) fence_acq_rel();
    const int b = atomicAdd(&h.chunk_free[x], k);
    lift = b <= 0 && b + k >= 1;
  }
  return lift;
}

/* free into a chunk queue: every lane of mask calls; lanes with cls < 0 only
 * take part (FENCE as for chunk_release) */
template <int V, bool FENCE = true>
__device__ void chunk_free_impl(const ouro_heap_dev &h, int cls, const void *p, unsigned mask) {
  constexpr int QF = ouro_qform(V);
  const unsigned lane = laneid();
  unsigned x;
  const bool lift = chunk_release<FENCE>(h, cls, p, mask, x);
  push_group<QF>(h, cls, x, lift, mask);   /* the lifted chunks, one tail atomic per class */
  const unsigned sg = warp_group(h, mask, cls);
  if (cls >= 0 && lane == (unsigned)(__ffs(sg) - 1)) stat_add(h, cls, OURO_ST_FREE, __popc(sg));
}

/* One lane claims `want` free pages of chunk x (its reservation on the
 * chunk's count guarantees them) from the chunk's bitmap, starting at a
 * spread word, and writes their page ids (x << ppc_log | page) to dst; a
 * wait that runs out fills the rest with OURO_NIL and records a timeout. */
__device__ inline void claim_into(const ouro_heap_dev &h, unsigned x, unsigned ppc_log, unsigned want, unsigned *dst,
                                  unsigned seed) {
  const unsigned words_c = ((1u << ppc_log) + 31) >> 5;
  unsigned *bw = h.bits + (size_t)x * h.words_per_chunk;
  unsigned w = words_c > 1 ? seed % words_c : 0;
  unsigned done = 0, empty = 0, ns = h.backoff_min_ns;
  unsigned v = *(volatile unsigned *)&bw[w];
  for (unsigned it = 0; done < want && it < h.spin_limit; ++it) {
    if (v) {
      unsigned m = 0, tmp = v;
      for (unsigned k = done; k < want && tmp; ++k) {
        const unsigned b = tmp & (0u - tmp);
        m |= b;
        tmp ^= b;
      }
      const unsigned old = atomicAnd(&bw[w], ~m);
      unsigned cl = old & m;
      while (cl) {
        dst[done++] = (x << ppc_log) | (w * 32 + __ffs(cl) - 1);
        cl &= cl - 1;
      }
      v = old & ~m;
      empty = 0;
    }
    if (!v && done < want) {
      w = (w + 1 == words_c) ? 0 : w + 1;
      if (++empty > words_c) {          /* a whole pass found nothing: bits still being freed */
        backoff_wait(h, ns);
        ns = min(ns * 2, h.backoff_max_ns);
        empty = 0;
      }
      v = *(volatile unsigned *)&bw[w];
    }
  }
  if (done < want) {
    set_error(h, OURO_ERR_TIMEOUT, OURO_SITE_CLAIM);
    for (; done < want; ++done) dst[done] = OURO_NIL;
  }
}

/* The whole warp (all 32 lanes call) obtains up to `need` pages of class c
 * from a chunk queue for its block, and writes their page ids to out[0, got).
 * Each round pops m positions at once -- the chunks the rest needs at one
 * full chunk each (32 pages each while the queue looks empty), at most 32
 * -- one per lane: a lane reserves its share on
 * its chunk's count (or takes its part of a carve's reservation), the
 * chunks that keep free pages are queued again with one tail atomic, and
 * every lane claims its pages from its chunk's bitmap.  A position in debt
 * posts its share (at most 32 pages) for the carve, as chunk_malloc does.
 * Returns got: fewer than need only when the heap is exhausted (a round
 * of null answers only ends the acquisition) or a bounded wait ran out. */
template <int V>
__device__ unsigned chunk_acquire(const ouro_heap_dev &h, int c, unsigned need, unsigned *out) {
  constexpr int QF = ouro_qform(V);
  constexpr bool VL = QF != OURO_QF_RING;
  constexpr unsigned FULL = 0xffffffffu;
  ouro_qhdr *q = qh(h, c);
  const unsigned lane = laneid();
  const unsigned ppc_log = h.log2_chunk - 4 - c, ppc = 1u << ppc_log;
  unsigned got = 0;
  for (unsigned round = 0; got < need && round < h.spin_limit; ++round) {
    const unsigned rem = need - got;
    /* share per position: a whole chunk while the queue holds chunks; 32
     * pages (what a carve reserves for one position) when it looks empty,
     * so that a carve packs the block's need as the per-warp path does */
    unsigned gran_log = ppc_log;
    if (lane == 0 && ld_rlx(&q->tail.v) <= ld_rlx(&q->head.v)) gran_log = min(ppc_log, 5u);
    gran_log = __shfl_sync(FULL, gran_log, 0);
    const unsigned gran = 1u << gran_log;
    const unsigned m = min(32u, (rem + gran - 1) >> gran_log);
    unsigned long long p0 = 0;
    if (lane == 0) p0 = atomicAdd(&q->head.v, (unsigned long long)m);
    p0 = __shfl_sync(FULL, p0, 0);
    const bool mine = lane < m;
    const unsigned share = mine ? min(gran, rem - lane * gran) : 0;
    const unsigned long long pos = p0 + lane;
    int st = mine ? 0 : 3;              /* 0 waiting, 1 item, 2 null answer, 3 no position */
    unsigned item = 0;
    bool posted = false;
    unsigned long long *cell = nullptr;
    unsigned ns = h.backoff_min_ns;
    for (unsigned it = 0;; ++it) {
      bool debt = false, progressed = false;
      if (st == 0) {
        if (!cell) cell = slot_at<QF>(h, c, pos, false);
        if (cell) {
          st = try_take<VL>(h, c, cell, pos, &item);
          if (st) {
            progressed = true;
            if (VL) seg_event<QF>(h, c, cell, 1);
          }
        }
        if (!st && pos >= ld_acq(&q->tail.v)) {
          debt = true;
          if (!posted) {
            if (!cell && VL) cell = slot_at<QF>(h, c, pos, true);
            if (cell) {
              const unsigned long long e = ld_acq(cell);
              const int d = slot_d(e, pos);
              posted = true;
              if (d == 0 || (VL && d < 0)) cas_ar(cell, e, slot(pos, min(share, 32u)));
            }
          }
        }
      }
      const unsigned dmask = __ballot_sync(FULL, debt);
      if (dmask) {   /* one lock taker: its whole warp carves */
        const bool lk = lane == (unsigned)(__ffs(dmask) - 1) && try_lock(&q->lock.v);
        const unsigned lockers = __ballot_sync(FULL, lk);
        if (lockers) chunk_carve<V>(h, c, FULL, __ffs(lockers) - 1);
      }
      if (!__ballot_sync(FULL, st == 0)) break;
      if (it >= h.spin_limit) {          /* the bounded wait ran out: give the position up */
        if (st == 0) {
          if (!cell) cell = slot_at<QF>(h, c, pos, true);
          unsigned item2 = 0;
          const int g = cell ? give_up<VL>(h, c, cell, pos, &item2) : 0;
          if (g == 1 || g == 2) {
            st = g;
            item = item2;
          } else {
            st = 2;
            set_error(h, OURO_ERR_TIMEOUT, OURO_SITE_CHUNK_GIVEUP);
            stat_add(h, c, OURO_ST_CANCEL, 1);
          }
          if (VL && cell && g) seg_event<QF>(h, c, cell, 1);
        }
        break;
      }
      if (!__any_sync(FULL, progressed)) {
        backoff_wait(h, ns);
        ns = min(ns * 2, h.backoff_max_ns);
      } else {
        ns = h.backoff_min_ns;
      }
    }
    /* reserve the shares on the chunks; chunks that keep free pages go back */
    unsigned granted = 0, x = 0;
    bool push = false;
    if (st == 1) {
      x = OURO_CQ_ID(item);
      if (item & OURO_CQ_RES) {
        const unsigned cnt = OURO_CQ_CNT(item);
        granted = min(cnt, share);
        if (cnt > share) {   /* reserved for more than this share: hand back the rest */
          const int ex = (int)(cnt - share);
          const int b = atomicAdd(&h.chunk_free[x], ex);
          push = b <= 0 && b + ex >= 1;
        }
      } else {
        const int old = atomicSub(&h.chunk_free[x], (int)share);
        granted = old <= 0 ? 0 : min((unsigned)old, share);
        if (old - (int)share >= 1) {
          push = true;
        } else if (granted < share) {
          const int ex = (int)(share - granted);
          const int b = atomicAdd(&h.chunk_free[x], ex);
          push = b <= 0 && b + ex >= 1;
        }
      }
    }
    push_group<QF>(h, c, x, push, FULL);
    /* every lane claims its pages into its part of out */
    unsigned off = granted;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(FULL, off, o);
      if ((int)lane >= o) off += y;
    }
    const unsigned total = __shfl_sync(FULL, off, 31);
    off -= granted;
    if (granted)
      claim_into(h, x, ppc_log, granted, out + got + off,
                 (((blockIdx.x * blockDim.x + threadIdx.x) * 0x9E3779B1u) ^ (x * 0x85EBCA6Bu) ^ round) >> 7);
    got += total;
    /* a round whose every position was answered null finds the heap
     * exhausted: the rest of the need is answered null (a round with some
     * chunks goes on, so pages queued meanwhile are still handed out) */
    if (!__any_sync(FULL, st == 1)) break;
  }
  __syncwarp();
  return got;
}

/* Chunk-queue heaps: classes within a chunk go to the chunk queues, runs
 * above one chunk to their page-style run queues.  Every lane of mask calls. */
template <int V>
__device__ void *chunk_or_run_malloc(const ouro_heap_dev &h, int cls, unsigned mask) {
  const int pc = cls < (int)h.n_classes ? cls : -1;
  const int rc = cls >= (int)h.n_classes ? cls : -1;
  void *a = nullptr, *b = nullptr;
  if (__any_sync(mask, pc >= 0)) a = chunk_malloc<V>(h, pc, mask);
  if (__any_sync(mask, rc >= 0)) b = page_malloc<V>(h, rc, mask);
  return rc >= 0 ? b : a;
}

/* cls: the block's class, its run already marked free (runs), or -1 */
template <int V, bool FENCE = true>
__device__ void chunk_or_run_free(const ouro_heap_dev &h, int cls, unsigned item, const void *p, unsigned mask) {
  chunk_free_impl<V, FENCE>(h, cls < (int)h.n_classes ? cls : -1, p, mask);
  const unsigned rm = __ballot_sync(mask, cls >= (int)h.n_classes);
  if (rm && ((rm >> laneid()) & 1)) page_free<V>(h, cls, item, rm);
}

}  // namespace detail
}  // namespace ouro

/* ------------------------------------------------------------ block staging */
/* Shared-memory staging of freed pages: every warp of a block owns, per size
 * class, a stack of up to OURO_STAGE_CAP page ids.  A staged free pushes the
 * page id there instead of into the class queue; a later staged malloc of
 * the same class in the same warp pops it, with no global atomic and no
 * queue slot traffic.  Stacks are warp-private, so no synchronisation beyond
 * __syncwarp is needed.  ouro_block_end pushes what is left back to the
 * class queues (page queues) or to their chunks (chunk queues); a kernel must
 * call it before it exits.  Runs above one chunk are not staged.  On chunk
 * queues a staged page keeps its bitmap bit clear (it is still taken from
 * its chunk's point of view) until the flush. */
#define OURO_STAGE_CAP 16
template <int WARPS>
struct ouro_block_ctx {
  unsigned char cnt[WARPS][OURO_MAX_CLASSES];
  unsigned ids[WARPS][OURO_MAX_CLASSES][OURO_STAGE_CAP];
  unsigned busy[WARPS];   /* bit c: a lane group of the warp holds class c's stack (public staged calls) */
  ouro_heap_dev heap;     /* the heap of the staged public calls (ouro_block_begin(ctx, h)) */
};

namespace ouro {
namespace detail {

/* LOCKED: callers whose warps may call in lane subsets that run at the same
 * time (divergent code in user kernels).  A group leader then takes its
 * class's stack with a try-lock bit of the warp (ctx.busy) and holds it
 * until its lanes have read or written their ids; a stack that another
 * subset holds is skipped (the requests go to the queues). */
template <bool LOCKED, int WARPS>
__device__ __forceinline__ bool stack_try_take(ouro_block_ctx<WARPS> &ctx, unsigned w, int cls) {
  if (!LOCKED) return true;
  const unsigned bit = 1u << cls;
  if (atomicOr(&ctx.busy[w], bit) & bit) return false;
  __threadfence_block();
  return true;
}
template <bool LOCKED, int WARPS>
__device__ __forceinline__ void stack_release(ouro_block_ctx<WARPS> &ctx, unsigned w, int cls) {
  if (!LOCKED) return;
  __threadfence_block();
  atomicAnd(&ctx.busy[w], ~(1u << cls));
}

/* staged malloc; every lane of mask calls (mask: the calling
 * lanes, or only the calling lane for callers in arbitrary divergent code) */
template <int V, int WARPS, bool LOCKED = false, int FILL = 1>
__device__ void *stage_malloc(ouro_block_ctx<WARPS> &ctx, const ouro_heap_dev &h, unsigned long long n, bool want,
                              unsigned mask) {
  const unsigned lane = laneid(), w = threadIdx.x >> 5;
  int cls = want ? size_class(h, n) : -1;
  if (want && cls < 0) stat_add(h, OURO_ROW_NONE, n == 0 ? OURO_ST_ZERO : OURO_ST_TOO_LARGE, 1);
  const unsigned g = __match_any_sync(mask, cls);
  const unsigned leader = __ffs(g) - 1, rank = __popc(g & lanemask_lt()), k = __popc(g);
  unsigned have = 0, take = 0;
  bool held = false;
  if (cls >= 0 && cls < (int)h.n_classes && lane == leader && stack_try_take<LOCKED>(ctx, w, cls)) {
    held = true;
    have = ctx.cnt[w][cls];
    take = min(have, k);
    ctx.cnt[w][cls] = (unsigned char)(have - take);
  }
  have = __shfl_sync(mask, have, leader);
  take = __shfl_sync(mask, take, leader);
  void *res = nullptr;
  if (cls >= 0 && rank < take) {
    const unsigned item = ctx.ids[w][cls][have - 1 - rank];
    if (ouro_page_queues(V) && h.checked) {
      const unsigned sh = h.log2_chunk - 4 - cls, pg = item & ((1u << sh) - 1), x = item >> sh;
      const unsigned bit = 1u << (pg & 31);
      const unsigned old = atomicAnd(&h.bits[(size_t)x * h.words_per_chunk + (pg >> 5)], ~bit);
      if (!(old & bit)) set_error(h, OURO_ERR_DOUBLE_FREE, OURO_SITE_PAGE_CHECKED);
    }
    res = h.base + ((size_t)item << (4 + cls));
  }
  if (cls >= 0 && lane == leader && take) stat_add(h, cls, OURO_ST_MALLOC, take);
  __syncwarp(mask);
  if (held) stack_release<LOCKED>(ctx, w, cls);
  const int rest = (cls >= 0 && rank >= take) ? cls : -1;   /* served lanes help the rest */
  if (__any_sync(mask, rest >= 0)) {
    void *p;
    if constexpr (ouro_page_queues(V)) p = page_malloc<V, FILL>(h, rest, mask);
    else p = chunk_or_run_malloc<V>(h, rest, mask);
    if (rest >= 0) res = p;
  }
  return res;
}
template <int V, int WARPS>
__device__ __forceinline__ void *stage_malloc(ouro_block_ctx<WARPS> &ctx, const ouro_heap_dev &h,
                                              unsigned long long n, bool want) {
  return stage_malloc<V, WARPS>(ctx, h, n, want, __activemask());
}

/* staged free; every lane of mask calls (as stage_malloc).  known_cls >= 0:
 * the caller allocated p itself with that page class (the library's fused
 * kernels), so the chunk table is not read and p is not checked; only for
 * page queues outside checked mode. */
template <int V, int WARPS, bool LOCKED = false>
__device__ void stage_free(ouro_block_ctx<WARPS> &ctx, const ouro_heap_dev &h, void *p, unsigned mask,
                           int known_cls = -1) {
  const unsigned lane = laneid(), w = threadIdx.x >> 5;
  unsigned item = 0;
  int cls = -1;
  if (p && known_cls >= 0 && known_cls < (int)h.n_classes && ouro_page_queues(V) && !h.checked) {
    cls = known_cls;
    item = (unsigned)(((const unsigned char *)p - h.base) >> (4 + cls));
  } else if (p) {
    cls = locate(h, p, &item);
    if (cls < 0) set_error(h, OURO_ERR_BAD_FREE, OURO_SITE_BAD_FREE);
    else if (cls >= (int)h.n_classes) {
      if (!run_mark_free(h, cls, item)) cls = -1;
    } else if (ouro_page_queues(V) && h.checked) {
      const unsigned sh = h.log2_chunk - 4 - cls, pg = item & ((1u << sh) - 1), x = item >> sh;
      const unsigned bit = 1u << (pg & 31);
      __threadfence();
      const unsigned old = atomicOr(&h.bits[(size_t)x * h.words_per_chunk + (pg >> 5)], bit);
      if (old & bit) {
        set_error(h, OURO_ERR_DOUBLE_FREE, OURO_SITE_PAGE_DOUBLE);
        cls = -1;
      }
    } else if (!ouro_page_queues(V)) {
      /* chunk queues: a page back in its chunk has its bit set; a staged
       * page keeps it clear until the block flushes it */
      const unsigned sh = h.log2_chunk - 4 - cls, pg = item & ((1u << sh) - 1), x = item >> sh;
      if (*(volatile unsigned *)&h.bits[(size_t)x * h.words_per_chunk + (pg >> 5)] & (1u << (pg & 31))) {
        set_error(h, OURO_ERR_DOUBLE_FREE, OURO_SITE_CHUNK_DOUBLE);
        cls = -1;
      }
    }
  }
  const unsigned g = __match_any_sync(mask, cls);
  const unsigned leader = __ffs(g) - 1, rank = __popc(g & lanemask_lt()), k = __popc(g);
  unsigned have = 0, take = 0;
  bool held = false;
  if (cls >= 0 && cls < (int)h.n_classes && lane == leader && stack_try_take<LOCKED>(ctx, w, cls)) {
    held = true;                                                /* runs are not staged */
    have = ctx.cnt[w][cls];
    take = min(OURO_STAGE_CAP - have, k);
    ctx.cnt[w][cls] = (unsigned char)(have + take);
    if (take) stat_add(h, cls, OURO_ST_FREE, take);
  }
  have = __shfl_sync(mask, have, leader);
  take = __shfl_sync(mask, take, leader);
  if (cls >= 0 && rank < take) ctx.ids[w][cls][have + rank] = item;
  __syncwarp(mask);
  if (held) stack_release<LOCKED>(ctx, w, cls);
  const unsigned rest = __ballot_sync(mask, cls >= 0 && rank >= take);
  if constexpr (ouro_page_queues(V)) {
    if (rest && ((rest >> lane) & 1)) page_free<V>(h, cls, item, rest);
  } else {
    if (rest) chunk_or_run_free<V>(h, ((rest >> lane) & 1) ? cls : -1, item, p, mask);
  }
}
template <int V, int WARPS>
__device__ __forceinline__ void stage_free(ouro_block_ctx<WARPS> &ctx, const ouro_heap_dev &h, void *p) {
  stage_free<V, WARPS>(ctx, h, p, __activemask());
}

}  // namespace detail
}  // namespace ouro

/* Every thread of the block calls (clears the stacks, then __syncthreads). */
template <int WARPS>
__device__ void ouro_block_begin(ouro_block_ctx<WARPS> &ctx) {
  for (unsigned i = threadIdx.x; i < WARPS * OURO_MAX_CLASSES; i += blockDim.x)
    (&ctx.cnt[0][0])[i] = 0;
  for (unsigned i = threadIdx.x; i < WARPS; i += blockDim.x) ctx.busy[i] = 0;
  __syncthreads();
}

/* Every thread of the block calls: each warp returns its staged pages to
 * the class queues (page queues) or to their chunks (chunk queues), then
 * __syncthreads.  The staged ids of all classes go back 32 at a time, lane j
 * of a round taking the j-th id of the round in class order, so that one
 * call serves the lanes of several classes at once (the classes' queue
 * atomics in flight together) instead of one call per class. */
template <int V, int WARPS>
__device__ void ouro_block_end_v(ouro_block_ctx<WARPS> &ctx, const ouro_heap_dev &h) {
  using namespace ouro::detail;
  const unsigned lane = laneid(), w = threadIdx.x >> 5;
  __syncwarp();
  unsigned total = 0;
  for (unsigned c = 0; c < h.n_classes; ++c) total += ctx.cnt[w][c];
  for (unsigned j0 = 0; j0 < total; j0 += 32) {
    const unsigned j = j0 + lane;
    int cj = -1;
    unsigned item = 0;
    if (j < total) {
      unsigned acc = 0;
      for (unsigned c = 0; c < h.n_classes; ++c) {
        const unsigned k = ctx.cnt[w][c];
        if (j < acc + k) {
          cj = (int)c;
          item = ctx.ids[w][c][j - acc];
          break;
        }
        acc += k;
      }
    }
    if constexpr (ouro_page_queues(V)) {
      const unsigned m = __ballot_sync(0xffffffffu, cj >= 0);
      if (cj >= 0) page_free<V>(h, cj, item, m);
    } else {
      void *p = cj >= 0 ? h.base + ((size_t)item << (4 + cj)) : nullptr;
      chunk_free_impl<V>(h, cj, p, 0xffffffffu);
    }
    __syncwarp();
  }
  if (lane < h.n_classes && ctx.cnt[w][lane]) {
    /* these pages were counted as freed when they were staged */
    stat_add(h, lane, OURO_ST_FREE, 0ull - (unsigned long long)ctx.cnt[w][lane]);
    ctx.cnt[w][lane] = 0;
  }
  __syncthreads();
}

/* ------------------------------------------------------------- public API */
/* Two ways to call, both on an ouro_heap_dev passed by value to the kernel:
 *
 *   ouro_malloc(h, n) / ouro_free(h, p)
 *     from anywhere: any lane, in any divergent code, alone or with others.
 *     Each calling lane runs the queue steps on its own (its warp-level
 *     steps name only itself), so no assumption is made about which lanes
 *     of the warp call at the same time.
 *
 *   ouro_malloc_warp(h, n, want) / ouro_free_warp(h, p)
 *     warp-collective: all 32 lanes of the warp call at the same point of the
 *     program (a lane without a request passes want = false, or p = null).
 *     Lanes that ask for the same class are served by one queue operation
 *     (warp aggregation with __match_any_sync), and a carve fills the new
 *     slots 32 lanes wide.  This is the form the library's own kernels use.
 *
 * The lane-private form exists because warp aggregation over the lanes that
 * __activemask() reports is not safe when several lane subsets of one warp
 * are inside the allocator at the same time (some lanes freeing while the
 * others already allocate again): GPU tests of such kernels found queue
 * slots produced twice, runs handed out twice and blocks overwritten by
 * another request.  With one lane per call, or the whole warp per call,
 * the same tests pass. */
namespace ouro {
namespace detail {
/* One queue form each, out of line: the run-time dispatch of the public
 * calls below picks one of these (and each compiles as its own function).
 * FILL: slot writes in flight per lane when a carve fills new slots (a lane
 * on its own fills a carve alone). */
template <int V, int FILL>
__device__ __noinline__ void *public_malloc_v(const ouro_heap_dev &h, int cls, unsigned mask) {
  if constexpr (ouro_page_queues(V)) return page_malloc<V, FILL>(h, cls, mask);   /* pages and runs */
  else return chunk_or_run_malloc<V>(h, cls, mask);
}

/* cls, item: from locate (a run already marked free), or -1 */
template <int V>
__device__ __noinline__ void public_free_v(const ouro_heap_dev &h, int cls, unsigned item, void *p, unsigned mask) {
  if constexpr (ouro_page_queues(V)) {
    const unsigned vmask = __ballot_sync(mask, cls >= 0);
    if (cls >= 0) page_free<V>(h, cls, item, vmask);
  } else {
    chunk_or_run_free<V>(h, cls, item, p, mask);
  }
}

template <int FILL>
__device__ __forceinline__ void *public_malloc(const ouro_heap_dev &h, size_t n, bool want, unsigned mask) {
  const int cls = want ? size_class(h, n) : -1;
  if (want && cls < 0) stat_add(h, OURO_ROW_NONE, n == 0 ? OURO_ST_ZERO : OURO_ST_TOO_LARGE, 1);
  if (!__any_sync(mask, cls >= 0)) return nullptr;
  /* lanes without a class stay in as helpers of the warp's carves */
  switch (h.variant) {
    case OURO_PAGE_ARRAY: return public_malloc_v<OURO_PAGE_ARRAY, FILL>(h, cls, mask);
    case OURO_PAGE_VLIST: return public_malloc_v<OURO_PAGE_VLIST, FILL>(h, cls, mask);
    case OURO_PAGE_VARRAY: return public_malloc_v<OURO_PAGE_VARRAY, FILL>(h, cls, mask);
    case OURO_CHUNK_ARRAY: return public_malloc_v<OURO_CHUNK_ARRAY, FILL>(h, cls, mask);
    case OURO_CHUNK_VLIST: return public_malloc_v<OURO_CHUNK_VLIST, FILL>(h, cls, mask);
    case OURO_CHUNK_VARRAY: return public_malloc_v<OURO_CHUNK_VARRAY, FILL>(h, cls, mask);
    default: return nullptr;
  }
}

__device__ __forceinline__ void public_free(const ouro_heap_dev &h, void *p, unsigned mask) {
  unsigned item = 0;
  int cls = -1;
  if (p) {
    cls = locate(h, p, &item);
    if (cls < 0) set_error(h, OURO_ERR_BAD_FREE, OURO_SITE_BAD_FREE);
    else if (cls >= (int)h.n_classes) {   /* a run */
      if (!run_mark_free(h, cls, item)) cls = -1;
    } else if (h.checked && ouro_page_queues((int)h.variant)) {
      unsigned ppcm = (1u << (h.log2_chunk - 4 - cls)) - 1;
      unsigned pg = item & ppcm, x = item >> (h.log2_chunk - 4 - cls);
      unsigned bit = 1u << (pg & 31);
      __threadfence();
      unsigned old = atomicOr(&h.bits[(size_t)x * h.words_per_chunk + (pg >> 5)], bit);
      if (old & bit) { set_error(h, OURO_ERR_DOUBLE_FREE, OURO_SITE_PAGE_DOUBLE); cls = -1; }
    }
  }
  switch (h.variant) {
    case OURO_PAGE_ARRAY: public_free_v<OURO_PAGE_ARRAY>(h, cls, item, p, mask); break;
    case OURO_PAGE_VLIST: public_free_v<OURO_PAGE_VLIST>(h, cls, item, p, mask); break;
    case OURO_PAGE_VARRAY: public_free_v<OURO_PAGE_VARRAY>(h, cls, item, p, mask); break;
    case OURO_CHUNK_ARRAY: public_free_v<OURO_CHUNK_ARRAY>(h, cls, item, p, mask); break;
    case OURO_CHUNK_VLIST: public_free_v<OURO_CHUNK_VLIST>(h, cls, item, p, mask); break;
    case OURO_CHUNK_VARRAY: public_free_v<OURO_CHUNK_VARRAY>(h, cls, item, p, mask); break;
    default: break;
  }
}
}  // namespace detail
}  // namespace ouro

/* Allocate n bytes from the heap; null when n is 0 or above 1 MiB, when
 * the heap is exhausted, or when a bounded wait ran out.  Any lane, any
 * divergent code. */
static __device__ __noinline__ void *ouro_malloc(const ouro_heap_dev &h, size_t n) {
  return ouro::detail::public_malloc<8>(h, n, true, 1u << ouro::detail::laneid());
}

/* Return a block to the heap; null is ignored; a pointer that is not a live
 * block start sets OURO_ERR_BAD_FREE (or OURO_ERR_DOUBLE_FREE) and is
 * ignored.  Any lane, any divergent code. */
static __device__ __noinline__ void ouro_free(const ouro_heap_dev &h, void *p) {
  ouro::detail::public_free(h, p, 1u << ouro::detail::laneid());
}

/* Warp-collective malloc: every lane of the warp calls at the same point;
 * want = false: the lane asks for nothing (and returns null).  Same answers
 * as ouro_malloc, with one queue operation per class among the lanes. */
static __device__ __noinline__ void *ouro_malloc_warp(const ouro_heap_dev &h, size_t n, bool want) {
  __syncwarp();
  return ouro::detail::public_malloc<1>(h, n, want, 0xffffffffu);
}

/* Warp-collective free: every lane of the warp calls at the same point
 * (p = null for a lane with nothing to free). */
static __device__ __noinline__ void ouro_free_warp(const ouro_heap_dev &h, void *p) {
  __syncwarp();
  ouro::detail::public_free(h, p, 0xffffffffu);
}

/* ------------------------------------------------- public API, staged form */
/* Block staging for user kernels: the heap is named once per block.
 *
 *   __shared__ ouro_block_ctx<8> ctx;      // WARPS >= warps of the block
 *   ouro_block_begin(ctx, h);              // every thread of the block
 *   void *p = ouro_malloc(ctx, n);         // any lane, divergent code
 *   ouro_free(ctx, p);
 *   void *q = ouro_malloc_warp(ctx, n, want);   // or warp-collective
 *   ouro_free_warp(ctx, q);
 *   ouro_block_end(ctx);                   // every thread, before the kernel exits
 *
 * On page queues a freed page stays on its warp's shared-memory stack (up to
 * OURO_STAGE_CAP per class) and serves that warp's next malloc of the class
 * without a queue operation; ouro_block_end returns what is left to the class
 * queues.  A lane-private call takes the warp's class stack with a try-lock
 * bit (another lane holding it sends the request to the queues).  Chunk
 * queues stage the same way (the page stays taken in its chunk's bitmap
 * until ouro_block_end returns it).  The block is one-dimensional
 * with at most 32 * WARPS threads; a page freed through the staged form
 * must not be used by another block before ouro_block_end. */
template <int WARPS>
__device__ void ouro_block_begin(ouro_block_ctx<WARPS> &ctx, const ouro_heap_dev &h) {
  if (threadIdx.x == 0) ctx.heap = h;
  ouro_block_begin(ctx);
}

template <int WARPS>
__device__ void ouro_block_end(ouro_block_ctx<WARPS> &ctx) {
  switch (ctx.heap.variant) {
    case OURO_PAGE_ARRAY: ouro_block_end_v<OURO_PAGE_ARRAY, WARPS>(ctx, ctx.heap); break;
    case OURO_PAGE_VLIST: ouro_block_end_v<OURO_PAGE_VLIST, WARPS>(ctx, ctx.heap); break;
    case OURO_PAGE_VARRAY: ouro_block_end_v<OURO_PAGE_VARRAY, WARPS>(ctx, ctx.heap); break;
    case OURO_CHUNK_ARRAY: ouro_block_end_v<OURO_CHUNK_ARRAY, WARPS>(ctx, ctx.heap); break;
    case OURO_CHUNK_VLIST: ouro_block_end_v<OURO_CHUNK_VLIST, WARPS>(ctx, ctx.heap); break;
    case OURO_CHUNK_VARRAY: ouro_block_end_v<OURO_CHUNK_VARRAY, WARPS>(ctx, ctx.heap); break;
    default: __syncthreads(); break;
  }
}

namespace ouro {
namespace detail {
template <int V, int WARPS, int FILL>
__device__ __noinline__ void *public_stage_malloc_v(ouro_block_ctx<WARPS> &ctx, size_t n, bool want, unsigned mask) {
  return stage_malloc<V, WARPS, true, FILL>(ctx, ctx.heap, n, want, mask);
}
template <int V, int WARPS>
__device__ __noinline__ void public_stage_free_v(ouro_block_ctx<WARPS> &ctx, void *p, unsigned mask) {
  stage_free<V, WARPS, true>(ctx, ctx.heap, p, mask);
}
template <int WARPS, int FILL>
__device__ __forceinline__ void *public_stage_malloc(ouro_block_ctx<WARPS> &ctx, size_t n, bool want, unsigned mask) {
  switch (ctx.heap.variant) {
    case OURO_PAGE_ARRAY: return public_stage_malloc_v<OURO_PAGE_ARRAY, WARPS, FILL>(ctx, n, want, mask);
    case OURO_PAGE_VLIST: return public_stage_malloc_v<OURO_PAGE_VLIST, WARPS, FILL>(ctx, n, want, mask);
    case OURO_PAGE_VARRAY: return public_stage_malloc_v<OURO_PAGE_VARRAY, WARPS, FILL>(ctx, n, want, mask);
    case OURO_CHUNK_ARRAY: return public_stage_malloc_v<OURO_CHUNK_ARRAY, WARPS, FILL>(ctx, n, want, mask);
    case OURO_CHUNK_VLIST: return public_stage_malloc_v<OURO_CHUNK_VLIST, WARPS, FILL>(ctx, n, want, mask);
    case OURO_CHUNK_VARRAY: return public_stage_malloc_v<OURO_CHUNK_VARRAY, WARPS, FILL>(ctx, n, want, mask);
    default: return nullptr;
  }
}
template <int WARPS>
__device__ __forceinline__ void public_stage_free(ouro_block_ctx<WARPS> &ctx, void *p, unsigned mask) {
  switch (ctx.heap.variant) {
    case OURO_PAGE_ARRAY: public_stage_free_v<OURO_PAGE_ARRAY, WARPS>(ctx, p, mask); break;
    case OURO_PAGE_VLIST: public_stage_free_v<OURO_PAGE_VLIST, WARPS>(ctx, p, mask); break;
    case OURO_PAGE_VARRAY: public_stage_free_v<OURO_PAGE_VARRAY, WARPS>(ctx, p, mask); break;
    case OURO_CHUNK_ARRAY: public_stage_free_v<OURO_CHUNK_ARRAY, WARPS>(ctx, p, mask); break;
    case OURO_CHUNK_VLIST: public_stage_free_v<OURO_CHUNK_VLIST, WARPS>(ctx, p, mask); break;
    case OURO_CHUNK_VARRAY: public_stage_free_v<OURO_CHUNK_VARRAY, WARPS>(ctx, p, mask); break;
    default: break;
  }
}
}  // namespace detail
}  // namespace ouro

/* staged malloc, any lane, any divergent code */
template <int WARPS>
__device__ void *ouro_malloc(ouro_block_ctx<WARPS> &ctx, size_t n) {
  return ouro::detail::public_stage_malloc<WARPS, 8>(ctx, n, true, 1u << ouro::detail::laneid());
}

/* staged free, any lane, any divergent code */
template <int WARPS>
__device__ void ouro_free(ouro_block_ctx<WARPS> &ctx, void *p) {
  ouro::detail::public_stage_free<WARPS>(ctx, p, 1u << ouro::detail::laneid());
}

/* staged malloc, warp-collective (every lane of the warp calls) */
template <int WARPS>
__device__ void *ouro_malloc_warp(ouro_block_ctx<WARPS> &ctx, size_t n, bool want) {
  __syncwarp();
  return ouro::detail::public_stage_malloc<WARPS, 1>(ctx, n, want, 0xffffffffu);
}

/* staged free, warp-collective (every lane of the warp calls) */
template <int WARPS>
__device__ void ouro_free_warp(ouro_block_ctx<WARPS> &ctx, void *p) {
  __syncwarp();
  ouro::detail::public_stage_free<WARPS>(ctx, p, 0xffffffffu);
}

#endif
