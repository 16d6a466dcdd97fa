/*
 * Sequential CPU oracle of the device-side allocator (arXiv 2504.18211).
 * TEST INFRASTRUCTURE ONLY -- see ouro_oracle.h for who may use it and for
 * the passages of the paper each part follows.
 *
 * Plain, slow and sequential on purpose: one request at a time, FIFO queues
 * held as growable rings, no concurrency, no blocking, no fusion.
 */
#include "ouro_oracle.h"

#include <stdlib.h>
#include <string.h>

#define CLS_NONE (-1)   /* chunk never carved, or back in the pool */
#define CLS_SEG  (-2)   /* chunk holds a segment of a virtualized queue */
#define CLS_RUN_FREE 64   /* + class: first chunk of a free run (in its class queue) */
#define CLS_RUN_BODY 128  /* + class: second or later chunk of a run */
#define MAX_REQUEST (16ull << (ORC_MAX_CLASSES - 1))   /* 1 MiB */

/* ------------------------------------------------------------------ FIFO */
typedef struct { uint64_t *v; uint64_t cap, lo, n; } fifo;

static int fifo_grow(fifo *f) {
  uint64_t nc = f->cap ? 2 * f->cap : 16;
  uint64_t *nv = (uint64_t *)malloc(nc * sizeof(uint64_t));
  if (!nv) return -1;
  for (uint64_t i = 0; i < f->n; i++) nv[i] = f->v[(f->lo + i) % f->cap];
  free(f->v);
  f->v = nv; f->cap = nc; f->lo = 0;
  return 0;
}
static int fifo_push(fifo *f, uint64_t x) {
  if (f->n == f->cap && fifo_grow(f)) return -1;
  f->v[(f->lo + f->n) % f->cap] = x;
  f->n++;
  return 0;
}
static uint64_t fifo_at(const fifo *f, uint64_t i) { return f->v[(f->lo + i) % f->cap]; }
static uint64_t fifo_pop_front(fifo *f) {
  uint64_t x = f->v[f->lo];
  f->lo = (f->lo + 1) % f->cap;
  f->n--;
  return x;
}
static uint64_t fifo_pop_back(fifo *f) { f->n--; return f->v[(f->lo + f->n) % f->cap]; }
static void fifo_clear(fifo *f) { f->lo = 0; f->n = 0; }
static void fifo_free(fifo *f) { free(f->v); f->v = NULL; f->cap = f->lo = f->n = 0; }

/* ------------------------------------------------------------------ heap */
struct orc_heap {
  uint64_t bytes, chunk_bytes, n_chunks, queue_cap, seg_cap, words_per_chunk;
  int variant, n_classes;
  int16_t *chunk_cls;
  uint8_t *live;          /* one bit per 16-byte unit: a live block starts here */
  uint32_t *free_pages;   /* chunk variants: free pages of each chunk */
  uint64_t *bits;         /* chunk variants: bit set = page free */
  fifo q[ORC_MAX_CLASSES];
  fifo pool;
  uint64_t bump;
  /* virtualized queues: positions and the chain of segment chunks */
  uint64_t qhead[ORC_MAX_CLASSES], qtail[ORC_MAX_CLASSES];
  fifo segs[ORC_MAX_CLASSES];
  uint64_t seg_first[ORC_MAX_CLASSES];
  fifo spare[ORC_MAX_CLASSES];
  uint64_t carved_now[ORC_MAX_CLASSES];
  uint64_t mallocs[ORC_MAX_CLASSES], frees[ORC_MAX_CLASSES], failed[ORC_MAX_CLASSES],
           carves[ORC_MAX_CLASSES];
  uint64_t zero_reqs, too_large;
  uint32_t err;
};

static int is_pow2(uint64_t x) { return x && !(x & (x - 1)); }
static int log2u(uint64_t x) { int l = 0; while ((1ull << l) < x) l++; return l; }
static int page_variant(const orc_heap *h) {
  return h->variant == ORC_PAGE_ARRAY || h->variant == ORC_PAGE_VLIST || h->variant == ORC_PAGE_VARRAY;
}
/* virtualized queues, list or array form: storage in segments of the heap */
static int virt(const orc_heap *h) {
  return h->variant == ORC_PAGE_VLIST || h->variant == ORC_CHUNK_VLIST ||
         h->variant == ORC_PAGE_VARRAY || h->variant == ORC_CHUNK_VARRAY;
}
static int varray(const orc_heap *h) {
  return h->variant == ORC_PAGE_VARRAY || h->variant == ORC_CHUNK_VARRAY;
}

/* Classes are the powers of two from 16 B up to the chunk size
 * (Sec. 4.2: queues manage sizes that are powers of two).  The 16 B floor
 * is a reading: the paper does not name a smallest size. */
int orc_num_classes(uint64_t chunk_bytes) { return log2u(chunk_bytes) - 4 + 1; }
uint64_t orc_page_bytes(int cls) { return 16ull << cls; }

int orc_num_large(uint64_t chunk_bytes) { return ORC_MAX_CLASSES - orc_num_classes(chunk_bytes); }

/* Smallest power of two >= max(n, 16); requests of 0 bytes or above 1 MiB
 * have no class and are answered with null (reading: the paper is silent).
 * Classes above the chunk size are runs of contiguous chunks (reading). */
int orc_size_class(uint64_t chunk_bytes, uint64_t n) {
  (void)chunk_bytes;
  if (n == 0 || n > MAX_REQUEST) return -1;
  int c = 0;
  while (orc_page_bytes(c) < n) c++;
  return c;
}

/* chunks in one run of class c (c >= n_classes): the class size / chunk */
static uint64_t run_chunks(const orc_heap *h, int c) { return orc_page_bytes(c) / h->chunk_bytes; }

static uint64_t pages_per_chunk(const orc_heap *h, int c) {
  return h->chunk_bytes / orc_page_bytes(c);
}

static void live_set(orc_heap *h, uint64_t off, int on) {
  uint64_t u = off >> 4;
  if (on) h->live[u >> 3] |= (uint8_t)(1u << (u & 7));
  else    h->live[u >> 3] &= (uint8_t)~(1u << (u & 7));
}
static int live_get(const orc_heap *h, uint64_t off) {
  uint64_t u = off >> 4;
  return (h->live[u >> 3] >> (u & 7)) & 1;
}

orc_heap *orc_create(uint64_t bytes, uint64_t chunk_bytes, int variant, uint64_t queue_cap) {
  if (!is_pow2(chunk_bytes) || chunk_bytes < 256 || chunk_bytes > (1u << 20)) return NULL;
  if (bytes == 0 || bytes % chunk_bytes) return NULL;
  if (variant < ORC_PAGE_ARRAY || variant > ORC_CHUNK_VARRAY) return NULL;
  orc_heap *h = (orc_heap *)calloc(1, sizeof(orc_heap));
  if (!h) return NULL;
  h->bytes = bytes;
  h->chunk_bytes = chunk_bytes;
  h->n_chunks = bytes / chunk_bytes;
  h->variant = variant;
  h->n_classes = orc_num_classes(chunk_bytes);
  h->queue_cap = queue_cap ? queue_cap : (1ull << 23);
  /* a segment is one chunk: a 64-byte header, then 8-byte cells */
  h->seg_cap = (chunk_bytes - 64) / 8;
  h->words_per_chunk = (chunk_bytes / 16 + 63) / 64;
  h->chunk_cls = (int16_t *)malloc(h->n_chunks * sizeof(int16_t));
  h->live = (uint8_t *)calloc((bytes / 16 + 7) / 8, 1);
  if (!page_variant(h)) {
    h->free_pages = (uint32_t *)calloc(h->n_chunks, sizeof(uint32_t));
    h->bits = (uint64_t *)calloc(h->n_chunks * h->words_per_chunk, sizeof(uint64_t));
  }
  if (!h->chunk_cls || !h->live || (!page_variant(h) && (!h->free_pages || !h->bits))) {
    orc_destroy(h);
    return NULL;
  }
  orc_reset(h);
  return h;
}

void orc_destroy(orc_heap *h) {
  if (!h) return;
  for (int c = 0; c < ORC_MAX_CLASSES; c++) {
    fifo_free(&h->q[c]); fifo_free(&h->segs[c]); fifo_free(&h->spare[c]);
  }
  fifo_free(&h->pool);
  free(h->chunk_cls); free(h->live); free(h->free_pages); free(h->bits);
  free(h);
}

/* post-create state: every chunk uncarved, pool empty, bump at 0, queues empty */
void orc_reset(orc_heap *h) {
  for (uint64_t i = 0; i < h->n_chunks; i++) h->chunk_cls[i] = CLS_NONE;
  memset(h->live, 0, (h->bytes / 16 + 7) / 8);
  if (h->free_pages) memset(h->free_pages, 0, h->n_chunks * sizeof(uint32_t));
  if (h->bits) memset(h->bits, 0, h->n_chunks * h->words_per_chunk * sizeof(uint64_t));
  for (int c = 0; c < ORC_MAX_CLASSES; c++) {
    fifo_clear(&h->q[c]); fifo_clear(&h->segs[c]); fifo_clear(&h->spare[c]);
    h->qhead[c] = h->qtail[c] = h->seg_first[c] = 0;
    h->carved_now[c] = h->mallocs[c] = h->frees[c] = h->failed[c] = h->carves[c] = 0;
  }
  fifo_clear(&h->pool);
  h->bump = 0;
  h->zero_reqs = h->too_large = 0;
  h->err = 0;
}

/* A free chunk comes from the pool front first, else from the bump pointer
 * (reading: the heap is divided among the queues on demand). */
static int64_t take_chunk(orc_heap *h) {
  if (h->pool.n) return (int64_t)fifo_pop_front(&h->pool);
  if (h->bump < h->n_chunks) return (int64_t)h->bump++;
  return -1;
}

/* ---------------------------------------- virtualized queue storage (Sec. 4.3) */
/* Make sure the segment holding position pos exists: retired segments of the
 * same queue are reused first, then the pool, then the bump pointer. */
static int seg_ensure(orc_heap *h, int c, uint64_t pos) {
  uint64_t s = pos / h->seg_cap;
  while (s >= h->seg_first[c] + h->segs[c].n) {
    int64_t x;
    if (h->spare[c].n) x = (int64_t)fifo_pop_back(&h->spare[c]);
    else {
      x = take_chunk(h);
      if (x < 0) return -1;
      h->chunk_cls[x] = CLS_SEG;
    }
    if (h->segs[c].n == 0) h->seg_first[c] = h->qhead[c] / h->seg_cap;
    fifo_push(&h->segs[c], (uint64_t)x);
  }
  return 0;
}
/* A segment retires once all its positions were consumed.  The list form
 * also needs a successor, because the list is entered through its oldest
 * segment; the array form finds every segment through its index, so its
 * last segment retires too. */
static void seg_retire(orc_heap *h, int c) {
  const uint64_t keep = varray(h) ? 1 : 2;
  while (h->segs[c].n >= keep && h->qhead[c] >= (h->seg_first[c] + 1) * h->seg_cap) {
    fifo_push(&h->spare[c], fifo_pop_front(&h->segs[c]));
    h->seg_first[c]++;
  }
}

static int q_push(orc_heap *h, int c, uint64_t item) {
  if (virt(h)) {
    if (seg_ensure(h, c, h->qtail[c])) { h->err |= ORC_ERR_QUEUE_FULL; return -1; }
    h->qtail[c]++;
    seg_retire(h, c);
  }
  fifo_push(&h->q[c], item);
  return 0;
}
static uint64_t q_pop(orc_heap *h, int c) {
  if (virt(h)) { h->qhead[c]++; seg_retire(h, c); }
  return fifo_pop_front(&h->q[c]);
}

/* -------------------------------------------------------------- carving */
/* Carve one chunk for class c and enqueue what it offers: every page id in
 * ascending order (page queues, Sec. 4.1) or the chunk id with all pages
 * free (chunk queues, Sec. 4.2).  Page-array queues hold at most
 * min(bytes / page, queue_cap) ids; a carve beyond that is refused. */
static int carve(orc_heap *h, int c) {
  uint64_t ppc = pages_per_chunk(h, c);
  if (h->variant == ORC_PAGE_ARRAY) {
    uint64_t qc = h->bytes / orc_page_bytes(c);
    if (qc > h->queue_cap) qc = h->queue_cap;
    if ((h->carved_now[c] + 1) * ppc > qc) return -1;
  }
  if (virt(h)) {
    /* queue storage first: segments for every position the carve will fill */
    uint64_t need = page_variant(h) ? ppc : 1;
    if (seg_ensure(h, c, h->qtail[c] + need - 1)) return -1;
  }
  int64_t x = take_chunk(h);
  if (x < 0) return -1;
  h->chunk_cls[x] = (int16_t)c;
  h->carved_now[c]++;
  h->carves[c]++;
  if (page_variant(h)) {
    for (uint64_t p = 0; p < ppc; p++) q_push(h, c, (uint64_t)x * ppc + p);
  } else {
    uint64_t *w = h->bits + (uint64_t)x * h->words_per_chunk;
    memset(w, 0, h->words_per_chunk * sizeof(uint64_t));
    for (uint64_t p = 0; p < ppc; p++) w[p >> 6] |= 1ull << (p & 63);
    h->free_pages[x] = (uint32_t)ppc;
    q_push(h, c, (uint64_t)x);
  }
  return 0;
}

/* ---------------------------------------------- runs above one chunk */
/* A request above one chunk takes a run of run_chunks(c) contiguous chunks
 * from its class queue, which holds the first chunks of free runs in the
 * order they were freed.  An empty queue is refilled with a run cut at the
 * bump pointer, the only place where contiguous chunks are sure to be free
 * (pooled chunks are not gathered into runs).  Reading: the paper is silent
 * on requests larger than a chunk. */
static int run_carve(orc_heap *h, int c) {
  uint64_t k = run_chunks(h, c);
  if (virt(h) && seg_ensure(h, c, h->qtail[c])) return -1;   /* queue storage first */
  if (h->bump + k > h->n_chunks) return -1;
  uint64_t x = h->bump;
  h->bump += k;
  h->chunk_cls[x] = (int16_t)(CLS_RUN_FREE + c);
  for (uint64_t i = 1; i < k; i++) h->chunk_cls[x + i] = (int16_t)(CLS_RUN_BODY + c);
  h->carves[c] += k;
  h->carved_now[c] += k;
  q_push(h, c, x);
  return 0;
}

static int64_t run_malloc(orc_heap *h, int c) {
  if (h->q[c].n == 0 && run_carve(h, c)) { h->failed[c]++; return -1; }
  uint64_t x = q_pop(h, c);
  h->chunk_cls[x] = (int16_t)c;
  uint64_t off = x * h->chunk_bytes;
  live_set(h, off, 1);
  h->mallocs[c]++;
  return (int64_t)off;
}

/* -------------------------------------------------------------- malloc */
int64_t orc_malloc(orc_heap *h, uint64_t n) {
  if (n == 0) { h->zero_reqs++; return -1; }
  int c = orc_size_class(h->chunk_bytes, n);
  if (c < 0) { h->too_large++; return -1; }
  if (c >= h->n_classes) return run_malloc(h, c);
  uint64_t pb = orc_page_bytes(c);
  uint64_t off;
  if (page_variant(h)) {
    /* Sec. 4.1: a page of the class is taken from the class queue */
    if (h->q[c].n == 0 && carve(h, c)) { h->failed[c]++; return -1; }
    uint64_t id = q_pop(h, c);
    off = id * pb;
  } else {
    /* Sec. 4.2: obtain the front chunk index, then scan it for a free page */
    if (h->q[c].n == 0 && carve(h, c)) { h->failed[c]++; return -1; }
    uint64_t x = fifo_at(&h->q[c], 0);
    uint64_t *w = h->bits + x * h->words_per_chunk;
    uint64_t ppc = pages_per_chunk(h, c), p = 0;
    while (p < ppc && !((w[p >> 6] >> (p & 63)) & 1)) p++;   /* lowest free page */
    w[p >> 6] &= ~(1ull << (p & 63));
    h->free_pages[x]--;
    if (h->free_pages[x] == 0) q_pop(h, c);                   /* full chunks leave */
    off = x * h->chunk_bytes + p * pb;
  }
  live_set(h, off, 1);
  h->mallocs[c]++;
  return (int64_t)off;
}

/* --------------------------------------------------------------- free */
uint32_t orc_free(orc_heap *h, int64_t off_s) {
  if (off_s < 0 || (uint64_t)off_s >= h->bytes) { h->err |= ORC_ERR_BAD_FREE; return ORC_ERR_BAD_FREE; }
  uint64_t off = (uint64_t)off_s;
  uint64_t x = off / h->chunk_bytes;
  int c = h->chunk_cls[x];
  if (c < 0 || c >= CLS_RUN_BODY) { h->err |= ORC_ERR_BAD_FREE; return ORC_ERR_BAD_FREE; }
  if (c >= CLS_RUN_FREE || c >= h->n_classes) {
    /* a run: only its first byte is a block start; a free run is a double free */
    if (off % h->chunk_bytes) { h->err |= ORC_ERR_BAD_FREE; return ORC_ERR_BAD_FREE; }
    if (c >= CLS_RUN_FREE) { h->err |= ORC_ERR_DOUBLE_FREE; return ORC_ERR_DOUBLE_FREE; }
    live_set(h, off, 0);
    h->frees[c]++;
    h->chunk_cls[x] = (int16_t)(CLS_RUN_FREE + c);
    q_push(h, c, x);
    return 0;
  }
  uint64_t pb = orc_page_bytes(c);
  if (off % pb) { h->err |= ORC_ERR_BAD_FREE; return ORC_ERR_BAD_FREE; }
  if (!live_get(h, off)) { h->err |= ORC_ERR_DOUBLE_FREE; return ORC_ERR_DOUBLE_FREE; }
  live_set(h, off, 0);
  h->frees[c]++;
  if (page_variant(h)) {
    q_push(h, c, off / pb);
  } else {
    uint64_t p = (off - x * h->chunk_bytes) / pb;
    h->bits[x * h->words_per_chunk + (p >> 6)] |= 1ull << (p & 63);
    h->free_pages[x]++;
    if (h->free_pages[x] == 1) q_push(h, c, x);   /* a full chunk has a free page again */
  }
  return 0;
}

/* --------------------------------------------------------------- trim */
static int cmp_u64(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return x < y ? -1 : x > y;
}

void orc_trim(orc_heap *h) {
  uint64_t *qcount = (uint64_t *)calloc(h->n_chunks, sizeof(uint64_t));
  uint8_t *reclaim = (uint8_t *)calloc(h->n_chunks, 1);
  if (!qcount || !reclaim) { free(qcount); free(reclaim); return; }
  /* 1. which carved chunks have every page free */
  for (int c = 0; c < h->n_classes; c++) {
    if (page_variant(h)) {
      uint64_t ppc = pages_per_chunk(h, c);
      for (uint64_t i = 0; i < h->q[c].n; i++) qcount[fifo_at(&h->q[c], i) / ppc]++;
    }
  }
  for (uint64_t x = 0; x < h->n_chunks; x++) {
    int c = h->chunk_cls[x];
    if (c < 0 || c >= h->n_classes) continue;   /* runs are handled below */
    uint64_t ppc = pages_per_chunk(h, c);
    uint64_t fr = page_variant(h) ? qcount[x] : h->free_pages[x];
    if (fr == ppc) reclaim[x] = 1;
  }
  /* 2. drop their entries from the queues, keeping the order of the rest */
  for (int c = 0; c < h->n_classes; c++) {
    uint64_t ppc = pages_per_chunk(h, c);
    fifo keep = {0};
    for (uint64_t i = 0; i < h->q[c].n; i++) {
      uint64_t it = fifo_at(&h->q[c], i);
      uint64_t x = page_variant(h) ? it / ppc : it;
      if (!reclaim[x]) fifo_push(&keep, it);
    }
    fifo_free(&h->q[c]);
    h->q[c] = keep;
  }
  /* 3. reclaimed chunks and all queue segments go back to the pool */
  for (uint64_t x = 0; x < h->n_chunks; x++) {
    if (reclaim[x]) {
      h->carved_now[h->chunk_cls[x]]--;
      h->chunk_cls[x] = CLS_NONE;
      if (!page_variant(h)) h->free_pages[x] = 0;
      fifo_push(&h->pool, x);
    } else if (h->chunk_cls[x] == CLS_SEG) {
      h->chunk_cls[x] = CLS_NONE;
      fifo_push(&h->pool, x);
    }
  }
  if (!page_variant(h))
    for (uint64_t x = 0; x < h->n_chunks; x++)
      if (reclaim[x]) memset(h->bits + x * h->words_per_chunk, 0, h->words_per_chunk * 8);
  /* 3b. every chunk of every free run (its class queue) goes back to the pool too */
  for (int c = h->n_classes; c < ORC_MAX_CLASSES; c++) {
    uint64_t k = run_chunks(h, c);
    for (uint64_t i = 0; i < h->q[c].n; i++) {
      uint64_t x = fifo_at(&h->q[c], i);
      for (uint64_t j = 0; j < k; j++) {
        h->chunk_cls[x + j] = CLS_NONE;
        fifo_push(&h->pool, x + j);
      }
      h->carved_now[c] -= k;
    }
    fifo_clear(&h->q[c]);
  }
  /* 4. canonical pool: ascending ids; lower the bump pointer over pooled chunks */
  uint64_t np = h->pool.n;
  uint64_t *pv = (uint64_t *)malloc((np ? np : 1) * sizeof(uint64_t));
  for (uint64_t i = 0; i < np; i++) pv[i] = fifo_at(&h->pool, i);
  qsort(pv, np, sizeof(uint64_t), cmp_u64);
  while (np && pv[np - 1] == h->bump - 1) { np--; h->bump--; }
  fifo_clear(&h->pool);
  for (uint64_t i = 0; i < np; i++) fifo_push(&h->pool, pv[i]);
  free(pv);
  /* 5. virtualized queues are re-laid from position 0, class by class */
  if (virt(h)) {
    for (int c = 0; c < ORC_MAX_CLASSES; c++) {
      fifo items = h->q[c];
      memset(&h->q[c], 0, sizeof(fifo));
      fifo_clear(&h->segs[c]); fifo_clear(&h->spare[c]);
      h->qhead[c] = h->qtail[c] = h->seg_first[c] = 0;
      for (uint64_t i = 0; i < items.n; i++) q_push(h, c, fifo_at(&items, i));
      fifo_free(&items);
    }
  }
  free(qcount);
  free(reclaim);
}

/* --------------------------------------------------------------- stats */
void orc_get_stats(const orc_heap *h, orc_stats *o) {
  memset(o, 0, sizeof(*o));
  o->n_classes = (uint32_t)h->n_classes;
  o->n_large = (uint32_t)(ORC_MAX_CLASSES - h->n_classes);
  for (int c = 0; c < ORC_MAX_CLASSES; c++) {
    o->mallocs[c] = h->mallocs[c];
    o->frees[c] = h->frees[c];
    o->failed[c] = h->failed[c];
    o->carves[c] = h->carves[c];
    o->carved_now[c] = h->carved_now[c];
    o->queued[c] = h->q[c].n;
    o->live[c] = h->mallocs[c] - h->frees[c];
    o->seg_chunks += h->segs[c].n;
    o->spare_chunks += h->spare[c].n;
  }
  o->zero_reqs = h->zero_reqs;
  o->too_large = h->too_large;
  o->bump = h->bump;
  o->pool_size = h->pool.n;
  o->error_bits = h->err;
}

uint64_t orc_queue_items(const orc_heap *h, int c, uint64_t *out, uint64_t max) {
  const fifo *f = &h->q[c];   /* runs above one chunk: first chunks of free runs */
  for (uint64_t i = 0; i < f->n && i < max; i++) out[i] = fifo_at(f, i);
  return f->n;
}
uint64_t orc_pool_items(const orc_heap *h, uint64_t *out, uint64_t max) {
  for (uint64_t i = 0; i < h->pool.n && i < max; i++) out[i] = fifo_at(&h->pool, i);
  return h->pool.n;
}
uint64_t orc_chunk_classes(const orc_heap *h, int16_t *out, uint64_t max) {
  for (uint64_t i = 0; i < h->n_chunks && i < max; i++) out[i] = h->chunk_cls[i];
  return h->n_chunks;
}
uint64_t orc_chunk_free_pages(const orc_heap *h, uint32_t *out, uint64_t max) {
  for (uint64_t i = 0; i < h->n_chunks && i < max; i++)
    out[i] = h->free_pages ? h->free_pages[i] : 0;
  return h->n_chunks;
}
uint64_t orc_seg_chunks(const orc_heap *h, int c, uint64_t *out, uint64_t max) {
  uint64_t n = h->segs[c].n;
  for (uint64_t i = 0; i < n && i < max; i++) out[i] = fifo_at(&h->segs[c], i);
  return n;
}
uint32_t orc_error_bits(const orc_heap *h) { return h->err; }

/* ------------------------------------------------- driver round (Sec. 3) */
uint32_t orc_fmix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x85ebca6bu;
  x ^= x >> 13;
  x *= 0xc2b2ae35u;
  x ^= x >> 16;
  return x;
}

/* The paper writes "some data" and checks it (Sec. 3).  Reading: mode 0
 * stores the thread id in word 0 only; mode 1 fills every word with a
 * sequence keyed by (seed, thread): key + i * 0x9E3779B9, where
 * key = fmix32(seed ^ tid * 0x9E3779B9). */
uint32_t orc_pattern_word(uint32_t seed, uint32_t tid, uint32_t i, int mode) {
  if (mode == 0) return tid;
  uint32_t key = orc_fmix32(seed ^ (tid * 0x9E3779B9u));
  return key + i * 0x9E3779B9u;
}

/* words written for a request of n bytes: mode 0 writes one word; mode 1
 * writes floor(n/4) words plus (n mod 4) tail bytes taken from the low
 * bytes of the next word of the sequence */
static void fold(orc_round_result *r, uint64_t v) { r->xor64 ^= v; r->sum64 += v; r->words++; }

void orc_expected_checksums(const uint32_t *sizes, uint64_t n, uint32_t seed, int mode,
                            orc_round_result *res) {
  memset(res, 0, sizeof(*res));
  for (uint64_t t = 0; t < n; t++) {
    if (mode == 0) { fold(res, orc_pattern_word(seed, (uint32_t)t, 0, 0)); continue; }
    uint64_t nw = sizes[t] / 4, tail = sizes[t] % 4;
    for (uint64_t i = 0; i < nw; i++) fold(res, orc_pattern_word(seed, (uint32_t)t, (uint32_t)i, 1));
    if (tail) {
      uint32_t v = orc_pattern_word(seed, (uint32_t)t, (uint32_t)nw, 1);
      fold(res, v & (uint32_t)((1ull << (8 * tail)) - 1));
    }
  }
}

void orc_round(orc_heap *h, const uint32_t *sizes, uint64_t n, uint32_t seed, int mode,
               uint8_t *mem, int64_t *offs_out, orc_round_result *res) {
  memset(res, 0, sizeof(*res));
  int64_t *offs = offs_out ? offs_out : (int64_t *)malloc((n ? n : 1) * sizeof(int64_t));
  /* allocate */
  for (uint64_t t = 0; t < n; t++) {
    offs[t] = orc_malloc(h, sizes[t]);
    if (offs[t] < 0) res->nulls++;
  }
  /* write */
  if (mem) {
    for (uint64_t t = 0; t < n; t++) {
      if (offs[t] < 0) continue;
      uint8_t *b = mem + offs[t];
      if (mode == 0) {
        uint32_t v = orc_pattern_word(seed, (uint32_t)t, 0, 0);
        memcpy(b, &v, 4);
        continue;
      }
      uint64_t nw = sizes[t] / 4, tail = sizes[t] % 4;
      for (uint64_t i = 0; i < nw; i++) {
        uint32_t v = orc_pattern_word(seed, (uint32_t)t, (uint32_t)i, 1);
        memcpy(b + 4 * i, &v, 4);
      }
      if (tail) {
        uint32_t v = orc_pattern_word(seed, (uint32_t)t, (uint32_t)nw, 1);
        for (uint64_t j = 0; j < tail; j++) b[4 * nw + j] = (uint8_t)(v >> (8 * j));
      }
    }
  }
  /* read back and check */
  for (uint64_t t = 0; t < n; t++) {
    if (offs[t] < 0) continue;
    uint64_t nw = mode == 0 ? 1 : sizes[t] / 4, tail = mode == 0 ? 0 : sizes[t] % 4;
    for (uint64_t i = 0; i < nw; i++) {
      uint32_t want = orc_pattern_word(seed, (uint32_t)t, (uint32_t)i, mode), got = want;
      if (mem) memcpy(&got, mem + offs[t] + 4 * i, 4);
      if (got != want) res->mismatches++;
      fold(res, got);
    }
    if (tail) {
      uint32_t v = orc_pattern_word(seed, (uint32_t)t, (uint32_t)nw, 1), got = 0, want = 0;
      for (uint64_t j = 0; j < tail; j++) {
        uint8_t wb = (uint8_t)(v >> (8 * j));
        uint8_t gb = mem ? mem[offs[t] + 4 * nw + j] : wb;
        if (gb != wb) res->mismatches++;
        got |= (uint32_t)gb << (8 * j);
        want |= (uint32_t)wb << (8 * j);
      }
      (void)want;
      fold(res, got);
    }
  }
  /* free */
  for (uint64_t t = 0; t < n; t++)
    if (offs[t] >= 0) orc_free(h, offs[t]);
  if (!offs_out) free(offs);
}
