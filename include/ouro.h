/*
 * ouro.h -- C ABI of the GB300 device-side dynamic memory allocator.
 *
 * The method follows "Dynamic Memory Management on GPUs with SYCL"
 * (arXiv 2504.18211), which ports the Ouroboros allocator:
 *   - the host preallocates one block of device memory to act as a heap and
 *     an allocation algorithm runs on the device (Sec. 1, Introduction);
 *   - the heap is divided into chunks; requests are served as pages from
 *     inside chunks, through one lock-free queue per size (Sec. 1; Sec. 4);
 *   - sizes are powers of two (Sec. 4.2);
 *   - page queues hand out fixed-size pages (Sec. 4.1); chunk queues hold
 *     chunks with free pages, which are scanned for a free page (Sec. 4.2);
 *   - virtualized queues keep their storage inside the heap (Sec. 4.3);
 *   - the driver round allocates, writes, reads back and frees (Sec. 3).
 *
 * Conventions for every entry point:
 *   - return an ouro_status (0 = OURO_OK); no entry point aborts or traps;
 *   - "d_" arguments are DEVICE pointers owned by the caller; "h_"/"out"
 *     arguments are HOST pointers owned by the caller;
 *   - calls taking a cudaStream_t are asynchronous on that stream unless the
 *     comment says "syncs"; a NULL stream is the legacy default stream;
 *   - OURO_ECUDA keeps the CUDA error in ouro_last_cuda_error().
 * Device-side use (ouro_malloc / ouro_free inside user kernels) is declared
 * in ouro_device.cuh.
 */
#ifndef OURO_H
#define OURO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int ouro_status;
enum {
  OURO_OK = 0,
  OURO_EINVAL = 1,    /* bad argument */
  OURO_ENOMEM = 2,    /* a host or device allocation failed */
  OURO_ECUDA = 3,     /* a CUDA call failed; see ouro_last_cuda_error() */
  OURO_EDEVICE = 4,   /* the heap's device error word is non-zero (see ouro_stats.error_bits) */
  OURO_ENOTSUP = 5    /* the heap's variant does not offer this operation */
};

/* queue variants (the six of Sec. 3): page or chunk queues (Sec. 4.1, 4.2),
 * each as a plain array, a virtualized list or a virtualized array (Sec. 4.3).
 *   plain array:        a ring of slots outside the heap, per class
 *                       next_pow2(min(bytes/page, array_queue_capacity) + 2^19)
 *                       slots of 8 B;
 *   virtualized list:   slots live in heap chunks (segments) linked in
 *                       position order, found by a walk (with a lookaside);
 *   virtualized array:  slots live in heap chunks found by index through a
 *                       per-class directory of 8-B entries, next_pow2 of
 *                       ceil((bytes/page + 2^20) / segment slots) + 4
 *                       entries (chunk queues: n_chunks in place of
 *                       bytes/page).  A segment returns to its class's spare
 *                       stack once all its positions are produced and
 *                       consumed. */
typedef enum {
  OURO_PAGE_ARRAY = 0,
  OURO_CHUNK_ARRAY = 1,
  OURO_PAGE_VLIST = 2,
  OURO_CHUNK_VLIST = 3,
  OURO_PAGE_VARRAY = 4,
  OURO_CHUNK_VARRAY = 5
} ouro_variant;

/* device error bits (sticky until ouro_heap_reset) */
enum {
  OURO_ERR_BAD_FREE = 1u << 0,       /* pointer outside the heap, unaligned or in an uncarved chunk */
  OURO_ERR_DOUBLE_FREE = 1u << 1,    /* page already free (chunk queues; page queues when checked) */
  OURO_ERR_QUEUE_FULL = 1u << 2,     /* a virtualized queue needed a segment and no chunk was left */
  OURO_ERR_TIMEOUT = 1u << 3,        /* a bounded wait ran out; the request returned null */
  OURO_ERR_QUEUE_OVERFLOW = 1u << 4  /* a queue slot stayed busy for a whole lap */
};

#define OURO_MAX_CLASSES 17            /* 16 B .. 1 MiB */

typedef struct ouro_heap ouro_heap;   /* host handle, opaque */

typedef struct {
  uint32_t spin_limit;            /* iterations of a bounded wait before it gives up (default 1<<20) */
  uint32_t backoff_min_ns;        /* first __nanosleep of a waiting warp (default 32) */
  uint32_t backoff_max_ns;        /* backoff cap (default 2048) */
  uint32_t max_carve;             /* chunks one carve may take at once (default 65536) */
  uint64_t array_queue_capacity;  /* page-array item limit per class (default 1<<23) */
  uint32_t checked;               /* page queues: track live pages to detect double frees */
  uint32_t staging;               /* the library's fused / persistent kernels stage freed pages per
                                     warp in shared memory (ouro_block_ctx), every queue form */
  uint32_t deopt;                 /* the "deoptimised" form of Sec. 2: no warp aggregation (every
                                     request takes its own queue atomics) and a memory fence where
                                     a waiting thread would __nanosleep; for comparison only */
  uint32_t reserved;              /* must be 0 */
} ouro_options;

/* Device view of a heap, passed BY VALUE to kernels that call ouro_malloc /
 * ouro_free.  Filled by ouro_heap_device(); its pointers stay valid until
 * ouro_heap_destroy().  The pointed-to layouts are private to the library. */
typedef struct {
  unsigned char *base;
  unsigned long long bytes, n_chunks;
  unsigned int chunk_bytes, log2_chunk, n_classes, variant;
  unsigned int seg_cap, words_per_chunk;
  unsigned int spin_limit, backoff_min_ns, backoff_max_ns, max_carve;
  unsigned int checked, staging, deopt, pad;
  void *qhdr;                          /* per-class queue headers */
  unsigned long long *cells;           /* array variants: every class ring, back to back */
  unsigned long long ring_off[OURO_MAX_CLASSES];
  unsigned long long ring_mask[OURO_MAX_CLASSES];
  unsigned long long qcap[OURO_MAX_CLASSES];   /* page-array item limit per class */
  unsigned char *chunk_cls;            /* class of each chunk; 0xFF none, 0xFE queue segment */
  int *chunk_free;                     /* chunk queues: free pages per chunk */
  unsigned int *bits;                  /* free-page bitmap (chunk queues; checked page queues) */
  unsigned int *pool;                  /* chunk ids returned by ouro_heap_trim */
  void *glob;                          /* heap-wide counters and error word */
  unsigned long long *stats;           /* sharded per-class counters */
} ouro_heap_dev;

typedef struct {
  uint64_t mallocs[OURO_MAX_CLASSES];     /* successful device mallocs */
  uint64_t frees[OURO_MAX_CLASSES];       /* successful device frees */
  uint64_t failed[OURO_MAX_CLASSES];      /* null returns for a request with a class */
  uint64_t carves[OURO_MAX_CLASSES];      /* chunks ever carved for the class */
  uint64_t carved_now[OURO_MAX_CLASSES];  /* chunks the class owns now (chunk table) */
  uint64_t queued[OURO_MAX_CLASSES];      /* queue entries (quiescent heaps only) */
  uint64_t live[OURO_MAX_CLASSES];        /* mallocs - frees */
  uint64_t repushes[OURO_MAX_CLASSES];    /* items re-queued after a consumer gave up a slot */
  uint64_t dead[OURO_MAX_CLASSES];        /* queue positions answered with null (heap exhausted) */
  uint64_t zero_reqs, too_large;          /* requests of 0 bytes / above 1 MiB */
  uint64_t bump, pool_size, seg_chunks, spare_chunks;
  uint32_t error_bits, n_classes;         /* n_classes: classes that fit in one chunk */
  uint32_t error_site;                    /* where the first error was recorded (device header's OURO_SITE_*) */
  uint32_t n_large;                       /* classes above one chunk: entries n_classes .. n_classes+n_large-1
                                             of the per-class arrays; queued = free runs in the class queue */
} ouro_stats;

/* Host copy of the queue state, for tests (ouro_heap_snapshot).  Arrays are
 * malloc'ed by the library and released by ouro_snapshot_free. */
typedef struct {
  uint32_t n_classes;
  uint64_t n_chunks;
  uint64_t bump;
  uint64_t pool_n;
  uint32_t *pool;                        /* pool_n chunk ids, in pool order */
  uint8_t *chunk_cls;                    /* n_chunks entries */
  int32_t *chunk_free;                   /* n_chunks entries (chunk queues) or NULL */
  uint64_t queue_n[OURO_MAX_CLASSES];
  uint32_t *queue[OURO_MAX_CLASSES];     /* items from head to tail, null answers skipped */
} ouro_snapshot;

/* ---- size classes --------------------------------------------------------
 * A request of n bytes (1 <= n <= 1 MiB) has class c = max(0, ceil(log2 n) - 4),
 * i.e. 16 << c bytes (Sec. 4.2: queues of power-of-two sizes).  Classes that
 * fit in one chunk (c < n_classes = log2(chunk_bytes) - 3) are pages of chunks
 * served by the class queues.  Larger classes (the paper is silent on them)
 * are runs of 2^(c - n_classes + 1) contiguous chunks: a freed run waits in
 * its class queue (same queue form as the other classes) for reuse; a debt
 * is carved by cutting runs at the bump pointer (pooled chunks are not
 * gathered into runs); ouro_heap_trim returns free runs to the pool.
 * 0 bytes and more than 1 MiB: null, counted. */

/* ---- heap life cycle (Sec. 1: the host preallocates the heap) ---------- */

/* Create a heap of `bytes` bytes cut into chunks of `chunk_bytes` with
 * page-array queues and default options.  chunk_bytes: power of two in
 * [256 B, 1 MiB]; bytes: a multiple of chunk_bytes, at most 64 GiB.
 * *out receives the handle.  EINVAL on bad sizes, ENOMEM/ECUDA on
 * allocation failure (nothing is leaked). */
ouro_status ouro_heap_create(size_t bytes, size_t chunk_bytes, ouro_heap **out);

/* As ouro_heap_create with a queue variant, options (NULL = defaults) and
 * optionally a caller-owned device buffer of `bytes` bytes used as the heap
 * (NULL = the library allocates and owns it).  A caller buffer must be
 * 256-byte aligned and outlive the heap. */
ouro_status ouro_heap_create_ex(size_t bytes, size_t chunk_bytes, ouro_variant variant,
                                const ouro_options *opt, void *d_heap_buf, ouro_heap **out);

/* Release every device buffer the heap owns.  NULL is accepted.  Syncs the device. */
ouro_status ouro_heap_destroy(ouro_heap *h);

/* Back to the post-create state: every chunk uncarved, queues empty, counters
 * and error word cleared.  Quiescent: no kernel may use the heap meanwhile. */
ouro_status ouro_heap_reset(ouro_heap *h, void *stream);

/* Quiescent reclaim: every chunk whose pages are all free leaves its class
 * queue and returns to the pool; the pool is sorted; the bump pointer drops
 * over pooled chunks at its top; virtualized queues are re-laid from
 * position 0.  After freeing everything, the state equals the post-create
 * state.  Syncs `stream`. */
ouro_status ouro_heap_trim(ouro_heap *h, void *stream);

/* Fill *out with the device view used by ouro_malloc / ouro_free. */
ouro_status ouro_heap_device(const ouro_heap *h, ouro_heap_dev *out);

/* Read and sum the device counters.  Syncs `stream`.  Returns OURO_EDEVICE
 * (after filling *out) when the device error word is non-zero. */
ouro_status ouro_heap_stats(ouro_heap *h, ouro_stats *out, void *stream);

/* Copy the queue state to host arrays (tests).  Quiescent; syncs `stream`. */
ouro_status ouro_heap_snapshot(ouro_heap *h, ouro_snapshot *out, void *stream);
void ouro_snapshot_free(ouro_snapshot *s);

/* ---- batch API --------------------------------------------------------------- */

/* d_ptrs[i] = ouro_malloc(d_sizes[i]) for i < n; null for failures.  The
 * results, counters and queue states are those of n ouro_malloc calls (the
 * class queues of Sec. 4.1-4.3).  On page queues the kernel takes the head
 * positions of a whole block of requests with one atomic per class, and on
 * plain arrays a batch of at least 4 x 256 x (SM count) requests runs four
 * requests per thread with their slots read together; chunk queues and the
 * deoptimised form take one atomic per warp class group, as ouro_malloc. */
ouro_status ouro_batch_malloc(ouro_heap *h, const uint32_t *d_sizes, void **d_ptrs, size_t n,
                              void *stream);
/* ouro_free(d_ptrs[i]) for i < n; null entries are skipped.  Aggregated like
 * ouro_batch_malloc: tail positions per class and block on page queues,
 * four requests per thread with their slot writes together on plain arrays
 * for large batches. */
ouro_status ouro_batch_free(ouro_heap *h, void *const *d_ptrs, size_t n, void *stream);

/* ---- driver round payload (Sec. 3: write data, read it back, check) ------ */

/* Result of a read-back check, written to device memory by the kernels. */
typedef struct {
  unsigned long long nulls;       /* requests that got null */
  unsigned long long mismatches;  /* words or tail bytes that read back wrong */
  unsigned long long xor64;       /* XOR of every word read back */
  unsigned long long sum64;       /* wrapping sum of every word read back */
  unsigned long long words;       /* words checked (a partial tail counts as one) */
} ouro_check;

/* Pattern of request i: mode 0 writes i into word 0; mode 1 writes
 * floor(size/4) words key_i + w * 0x9E3779B9 (key_i = fmix32(seed ^
 * i * 0x9E3779B9)) and the low size%4 bytes of the next word. */
ouro_status ouro_pattern_write(void *const *d_ptrs, const uint32_t *d_sizes, size_t n,
                               uint32_t seed, int mode, void *stream);
/* Read every block back; *d_out (device) is overwritten with the result. */
ouro_status ouro_pattern_check(void *const *d_ptrs, const uint32_t *d_sizes, size_t n,
                               uint32_t seed, int mode, ouro_check *d_out, void *stream);

/* One whole driver round in ONE kernel: every request allocates, writes its
 * pattern, reads it back and frees.  *d_out (device) receives the check.
 * d_ptrs (device, optional): receives each request's block address. */
ouro_status ouro_round_fused(ouro_heap *h, const uint32_t *d_sizes, size_t n, uint32_t seed,
                             int mode, ouro_check *d_out, void **d_ptrs, void *stream);

/* Same result as ouro_heap_stats, for callers that cannot allocate device
 * memory when they ask: applications whose device memory is all handed out
 * up front by their own pool (a cudaMalloc would fail, or take memory the
 * pool counts on), and latency-bound loops that must not let a cudaMalloc /
 * cudaFree stall the device while other streams are busy.  The paper has no
 * counterpart; this is a service of this library.
 *   - Allocates nothing: no cudaMalloc, no cudaFree, no allocating library
 *     call.  Its scratch (1584 bytes) is a file-scope __device__ array that
 *     every GPU loading the library keeps until the process exits.
 *   - Limit: heaps of at most OURO_MAX_CLASSES size classes (chunks up to
 *     1 MiB); a larger heap is rejected with OURO_EINVAL.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls share the one array, which keeps the last call's contents
 *     (it is cleared at the start of every call): calls that overlap on the
 *     GPU (other streams, other threads) race and may return mixed counts.
 *   - Syncs `stream`; returns OURO_EDEVICE (after filling *out) when the
 *     device error word is non-zero. */
ouro_status ouro_heap_stats_static(ouro_heap *h, ouro_stats *out, void *stream);

/* ---- batching: many request batches per pass ----------------------------- */

/* One kernel for n_batches batches (Sec. 3 driver round per request):
 * request i of batch b (d_sizes[d_offs[b] + i]) allocates, writes its
 * pattern (seed + b, thread id i), reads it back and frees.  Warps pull
 * 256-request tasks from *d_work (device scratch, 1 word, reset here);
 * d_task_offs[b] = sum over batches before b of ceil(count/256), n_tasks
 * its total.  d_out: n_batches checks (overwritten).  blocks_per_sm <= 0:
 * the occupancy limit.  d_offs, d_task_offs: device arrays of n_batches+1. */
ouro_status ouro_batches_persistent(ouro_heap *h, const uint32_t *d_sizes, const unsigned long long *d_offs,
                                    const unsigned long long *d_task_offs, uint32_t n_batches, uint64_t n_tasks,
                                    uint32_t seed, int mode, ouro_check *d_out, unsigned long long *d_work,
                                    int blocks_per_sm, void *stream);

/* Blocks of 256 threads per SM the persistent batching kernel of this
 * heap's variant can keep resident (register limit); 0 on error. */
int ouro_batches_max_blocks_per_sm(const ouro_heap *h);

/* The same pass as one CUDA graph of per-batch launches, captured once.
 * form 0: ouro_round_fused per batch; form 1: ouro_batch_malloc,
 * ouro_pattern_write, ouro_pattern_check, ouro_batch_free per batch (d_ptrs:
 * device scratch for the largest batch).  h_offs: HOST offsets (n_batches+1).
 * Replay with ouro_batch_graph_launch; the captured pointers must stay valid. */
typedef struct ouro_batch_graph ouro_batch_graph;
ouro_status ouro_batch_graph_create(ouro_heap *h, const uint32_t *d_sizes, const unsigned long long *h_offs,
                                    uint32_t n_batches, uint32_t seed, int mode, ouro_check *d_out,
                                    void **d_ptrs, int form, ouro_batch_graph **out);
ouro_status ouro_batch_graph_launch(ouro_batch_graph *g, void *stream);
uint64_t ouro_batch_graph_nodes(const ouro_batch_graph *g);
ouro_status ouro_batch_graph_destroy(ouro_batch_graph *g);

/* ---- serving: a request loop on the device -------------------------------- */

/* Run `steps` serving steps in ONE cooperative kernel.  Sessions (arrival
 * order) arrive at step d_arrive_step[s] and grow by one block of
 * block_bytes per step up to d_blocks[s] blocks (<= max_blocks), then free
 * every block.  Admission, in arrival order: while a slot is free and the
 * committed blocks of admitted sessions plus the newcomer's total stay <=
 * cap_blocks.  Each block gets the driver-round pattern (seed + s, block
 * index) and is read back; the session checksum folds every word.
 * Device buffers (caller-owned; contents overwritten):
 *   d_slot_session n_slots ints, d_slot_k n_slots, d_slot_acc 3*n_slots,
 *   d_tables n_slots*max_blocks pointers, d_sess_out 5*n_sessions words
 *   (xor, sum, mismatches, admit step, done step; all ones if never),
 *   d_step_ns 3*`steps` %globaltimer stamps (after admission, growth and
 *   completion of each step), d_ctl 11 words (barrier state, next
 *   arrival, committed blocks, error flag, mallocs, frees, failed mallocs,
 *   free-slot stack top, sessions finished in the step, one reserved),
 *   d_free_stack 2*n_slots slot ids (the free-slot stack, then the step's
 *   list of finished sessions, whose blocks are freed in tasks of 32 dealt
 *   to the warps in turn).
 * EINVAL unless block_bytes is a non-zero multiple of 16 of at most the
 * heap's chunk_bytes (the block payload moves whole 16-byte units), and for
 * a null buffer or n_slots / max_blocks of 0.
 * ENOTSUP if the device cannot launch cooperative kernels.  A grid barrier
 * whose wait runs out sets d_ctl[4] and ends the kernel. */
ouro_status ouro_serve(ouro_heap *h, const uint32_t *d_arrive_step, const uint32_t *d_blocks, uint32_t n_sessions,
                       uint32_t n_slots, uint32_t max_blocks, int *d_slot_session, uint32_t *d_slot_k,
                       unsigned long long *d_slot_acc, unsigned long long *d_tables, unsigned long long *d_sess_out,
                       unsigned long long *d_step_ns, unsigned long long *d_ctl, uint32_t *d_free_stack,
                       uint32_t steps, uint32_t seed, uint64_t cap_blocks, uint32_t block_bytes, int blocks_per_sm,
                       void *stream);

/* The same loop as plain per-launch kernels: for every step, one launch each
 * for admission, growth, completion and freeing, enqueued on `stream` in
 * order without a host wait (4 * steps + 2 launches).  Kernel boundaries
 * take the place of the grid barriers, so no cooperative launch is needed
 * and no wait can run out.  Arguments, buffers and results are those of
 * ouro_serve and equal its results for the same inputs; d_step_ns stamps
 * are taken at the start of the next phase's launch.  An added comparison
 * form: the paper's driver launches one kernel per phase (Sec. 3). */
ouro_status ouro_serve_per_launch(ouro_heap *h, const uint32_t *d_arrive_step, const uint32_t *d_blocks,
                                  uint32_t n_sessions, uint32_t n_slots, uint32_t max_blocks, int *d_slot_session,
                                  uint32_t *d_slot_k, unsigned long long *d_slot_acc, unsigned long long *d_tables,
                                  unsigned long long *d_sess_out, unsigned long long *d_step_ns,
                                  unsigned long long *d_ctl, uint32_t *d_free_stack, uint32_t steps, uint32_t seed,
                                  uint64_t cap_blocks, uint32_t block_bytes, int blocks_per_sm, void *stream);

/* ---- graph growth: adjacency lists grown in kernels --------------------------- */

/* Bytes of one vertex record (d_vertices holds n_vertices of them, device). */
size_t ouro_graph_vertex_bytes(void);
/* Every vertex gets an empty list of 4 entries (16 B from the heap).
 * d_ctl (device, 4 words, cleared): [0] entries appended, [1] failed
 * mallocs, [2] entries skipped after a lock wait ran out. */
ouro_status ouro_graph_init(ouro_heap *h, void *d_vertices, uint32_t n_vertices, unsigned long long *d_ctl,
                            void *stream);
/* Append edge e's d_dst[e] to vertex d_src[e]'s list for all n_edges: a
 * list that is full doubles (malloc 2x, copy, free old) one step at a time
 * up to one chunk of entries, then grows by chained one-chunk overflow
 * segments.  Per-vertex locks, bounded. */
ouro_status ouro_graph_insert(ouro_heap *h, void *d_vertices, const uint32_t *d_src, const uint32_t *d_dst,
                              uint64_t n_edges, unsigned long long *d_ctl, void *stream);
/* Copy every vertex's entries to d_out[d_offsets[v] ..] (offsets = prefix
 * sum of the degrees) for checking. */
ouro_status ouro_graph_gather(ouro_heap *h, const void *d_vertices, uint32_t n_vertices,
                              const unsigned long long *d_offsets, uint32_t *d_out, void *stream);
/* Free every list and overflow segment. */
ouro_status ouro_graph_free(ouro_heap *h, void *d_vertices, uint32_t n_vertices, void *stream);

/* ---- measurement ------------------------------------------------------------ */

/* L2 atomic throughput probe: `blocks` x 256 threads each do `iters` atomics on
 * d_buf (device, `words` 64-bit words >= 512, contents overwritten).
 * pattern 0: lane 0 of every warp on one shared counter; 1: lane 0 of every
 * warp on one of 32 counters on separate 128-byte lines (one atomic per warp,
 * as a warp group leader issues); 2: every lane, distinct words, consecutive
 * lanes on consecutive words, 64-bit CAS.
 * Time it with events on `stream`. */
ouro_status ouro_probe_atomics(unsigned long long *d_buf, size_t words, int pattern, uint32_t iters,
                               int blocks, void *stream);

/* As ouro_batch_malloc, timing every request with clock64: d_hist (device,
 * 256 words, overwritten) counts requests per latency bin; bin b < 4 holds
 * b cycles, bin b >= 4 holds [2^l + q*2^(l-2), 2^l + (q+1)*2^(l-2)) cycles
 * with l = b >> 2, q = b & 3. */
ouro_status ouro_malloc_latency(ouro_heap *h, const uint32_t *d_sizes, void **d_ptrs, size_t n,
                                unsigned long long *d_hist, void *stream);

/* ---- comparison: CUDA's built-in device malloc (Sec. 1) -------------------- */
/* Size the current context's device-malloc heap (cudaLimitMallocHeapSize;
 * it lasts as long as the context).  Must precede the first launch of any
 * kernel that calls malloc in this context: CUDA fixes the heap then, after
 * which the call returns OURO_ECUDA.  *got_bytes (host, optional): the size
 * CUDA reports back. */
ouro_status ouro_cuda_malloc_heap(size_t bytes, size_t *got_bytes);
/* The driver round of ouro_round_fused with CUDA's device malloc / free in
 * place of this library's heap: every request mallocs its size, writes its
 * pattern, reads it back and frees.  *d_out (device) receives the check. */
ouro_status ouro_cuda_malloc_round(const uint32_t *d_sizes, size_t n, uint32_t seed, int mode,
                                   ouro_check *d_out, void *stream);

/* ---- misc ----------------------------------------------------------------- */
const char *ouro_status_string(ouro_status s);
int ouro_last_cuda_error(void);
/* Number of the library's kernels launched since load (a running count). */
uint64_t ouro_kernel_launches(void);

/* Test aid: advance the producer counter of class `cls` by n without filling
 * the slots, so that the consumers of those slots wait until their bounded
 * wait gives up (OURO_ERR_TIMEOUT) -- used to test liveness without a fault. */
ouro_status ouro_debug_stall_producer(ouro_heap *h, int cls, uint32_t n, void *stream);

#ifdef __cplusplus
}
#endif
#endif
