/*
 * Sequential CPU oracle of the device-side allocator studied in
 * "Dynamic Memory Management on GPUs with SYCL" (arXiv 2504.18211).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline / reference legs of bench.py may load this library.  The
 * product path (include/ouro.h, the CUDA library) never links, imports or
 * calls it, and this file shares no code, header, table or constant with it.
 *
 * The oracle executes the method one request at a time, in the order the
 * paper states it:
 *   - the host preallocates one heap (Sec. 1, Introduction);
 *   - the heap is cut into chunks whose pages serve requests, one queue per
 *     size (Sec. 1 related work; Sec. 4 Results preamble);
 *   - size classes are powers of two (Sec. 4.2, Chunk allocator);
 *   - the page allocator hands out fixed-size pages from a per-class queue
 *     (Sec. 4.1, Page allocator);
 *   - the chunk allocator keeps a queue of chunks that still hold free pages,
 *     takes the front chunk, then scans it for a free page (Sec. 4.2);
 *   - virtualized queues keep queue storage inside the heap itself (Sec. 4.3);
 *   - the driver round is allocate, write, read back and check, free
 *     (Sec. 3, Methods).
 * Where the paper leaves a point open, the reading taken is stated beside
 * the code that takes it.
 */
#ifndef OURO_ORACLE_H
#define OURO_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_CLASSES 17          /* 16 B .. 1 MiB */

/* queue forms (Sec. 3 lists six: page / chunk queues, each as a plain
 * array, a virtualized array and a virtualized list) */
enum {
  ORC_PAGE_ARRAY = 0, ORC_CHUNK_ARRAY = 1, ORC_PAGE_VLIST = 2, ORC_CHUNK_VLIST = 3,
  ORC_PAGE_VARRAY = 4, ORC_CHUNK_VARRAY = 5
};

/* error bits (sticky) */
enum {
  ORC_ERR_BAD_FREE    = 1u << 0,   /* pointer outside the heap, unaligned, or in an uncarved chunk */
  ORC_ERR_DOUBLE_FREE = 1u << 1,   /* block is not live */
  ORC_ERR_QUEUE_FULL  = 1u << 2    /* a virtualized queue needed a segment and none was left */
};

typedef struct orc_heap orc_heap;

typedef struct {
  uint64_t mallocs[ORC_MAX_CLASSES];   /* successful ouro_malloc per class */
  uint64_t frees[ORC_MAX_CLASSES];     /* successful ouro_free per class */
  uint64_t failed[ORC_MAX_CLASSES];    /* null returns for a valid class */
  uint64_t carves[ORC_MAX_CLASSES];    /* chunks ever carved for the class */
  uint64_t carved_now[ORC_MAX_CLASSES];/* chunks currently owned by the class */
  uint64_t queued[ORC_MAX_CLASSES];    /* entries in the class queue */
  uint64_t live[ORC_MAX_CLASSES];      /* mallocs - frees */
  uint64_t zero_reqs, too_large;       /* size 0 / size > 1 MiB requests */
  uint64_t bump, pool_size, seg_chunks, spare_chunks;
  uint32_t error_bits, n_classes;      /* n_classes: classes that fit in one chunk */
  uint32_t n_large, pad;               /* classes above one chunk (runs of chunks) */
} orc_stats;

/* chunk_bytes: power of two in [256, 1 MiB]; bytes: multiple of chunk_bytes.
 * queue_cap: per-class item limit of page-array queues (0 = default 2^23).
 * Returns NULL on a bad argument or when host memory runs out. */
orc_heap *orc_create(uint64_t bytes, uint64_t chunk_bytes, int variant, uint64_t queue_cap);
void      orc_destroy(orc_heap *h);
void      orc_reset(orc_heap *h);

int       orc_num_classes(uint64_t chunk_bytes);                /* classes within one chunk */
int       orc_num_large(uint64_t chunk_bytes);                  /* classes above one chunk */
int       orc_size_class(uint64_t chunk_bytes, uint64_t n);   /* -1 for 0 or > 1 MiB */
uint64_t  orc_page_bytes(int cls);

/* Returns the byte offset of the block inside the heap, or -1 (null). */
int64_t   orc_malloc(orc_heap *h, uint64_t n);
/* Returns 0, or the error bits raised by this call (never aborts). */
uint32_t  orc_free(orc_heap *h, int64_t off);
/* Quiescent reclaim: every chunk whose pages are all free leaves its queue
 * and returns to the pool, and so does every chunk of a free run; the pool
 * is sorted and the bump pointer lowered over pooled chunks at its top;
 * virtualized queues are re-laid from position 0. */
void      orc_trim(orc_heap *h);

void      orc_get_stats(const orc_heap *h, orc_stats *out);

/* snapshot accessors (copy-out; return the element count) */
uint64_t  orc_queue_items(const orc_heap *h, int cls, uint64_t *out, uint64_t max);
uint64_t  orc_pool_items(const orc_heap *h, uint64_t *out, uint64_t max);
uint64_t  orc_chunk_classes(const orc_heap *h, int16_t *out, uint64_t max);
uint64_t  orc_chunk_free_pages(const orc_heap *h, uint32_t *out, uint64_t max);
uint64_t  orc_seg_chunks(const orc_heap *h, int cls, uint64_t *out, uint64_t max);
uint32_t  orc_error_bits(const orc_heap *h);

/* ---- driver round (Sec. 3, Methods): allocate, write, read back, free ---- */
/* MurmurHash3 32-bit finalizer (Appleby, public domain) */
uint32_t  orc_fmix32(uint32_t h);
/* value of word i of thread tid's block; mode 0: word 0 holds tid, mode 1: keyed Weyl sequence */
uint32_t  orc_pattern_word(uint32_t seed, uint32_t tid, uint32_t i, int mode);

typedef struct {
  uint64_t nulls;        /* requests that returned null */
  uint64_t mismatches;   /* words or tail bytes read back different from what was written */
  uint64_t xor64;        /* XOR of all words read back (tail word zero-extended) */
  uint64_t sum64;        /* wrapping sum of all words read back */
  uint64_t words;        /* words (incl. partial tail words) checked */
} orc_round_result;

/* One round over n requests in thread order: every malloc, then every write,
 * then every read-back check, then every free.  mem: host buffer of the
 * heap's size that receives the payload (NULL: checksums are computed from
 * the pattern without storing it).  offs (optional): receives the offsets. */
void orc_round(orc_heap *h, const uint32_t *sizes, uint64_t n, uint32_t seed, int mode,
               uint8_t *mem, int64_t *offs, orc_round_result *res);
/* Expected checksums of a fully successful round (no allocator involved). */
void orc_expected_checksums(const uint32_t *sizes, uint64_t n, uint32_t seed, int mode,
                            orc_round_result *res);

#ifdef __cplusplus
}
#endif
#endif
