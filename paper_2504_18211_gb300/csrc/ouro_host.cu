/*
 * Heap life cycle, statistics, snapshot and quiescent reclaim (trim).
 *
 * The host preallocates the heap once (Sec. 1 of arXiv 2504.18211); every
 * table the device allocator needs lives in ONE further device allocation,
 * cut into 256-byte aligned parts.  Maintenance (init, trim, stats,
 * snapshot) runs as kernels on the caller's stream; the host only sums a few
 * kilobytes of counters.
 */
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "ouro_internal.cuh"

using namespace ouro::detail;

namespace ouro {
namespace host {

thread_local int g_last_cuda_error = 0;
static unsigned long long g_launches = 0;

ouro_status cuda_fail(cudaError_t e) {
  g_last_cuda_error = (int)e;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return OURO_ENOMEM;
  }
  return OURO_ECUDA;
}
void count_launch(unsigned n) { __atomic_fetch_add(&g_launches, n, __ATOMIC_RELAXED); }
int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

}  // namespace host
}  // namespace ouro

using namespace ouro::host;

static inline cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }
static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
static inline unsigned long long next_pow2(unsigned long long x) {
  unsigned long long p = 1;
  while (p < x) p <<= 1;
  return p;
}
static inline bool is_page(unsigned v) { return ouro_page_queues((int)v); }
static inline bool is_virtual(unsigned v) { return ouro_qform((int)v) != OURO_QF_RING; }
static inline bool is_varray(unsigned v) { return ouro_qform((int)v) == OURO_QF_VARRAY; }

/* ------------------------------------------------------------- init kernels */
__global__ void k_init_qhdr(ouro_heap_dev h) {
  const int c = blockIdx.x;
  ouro_qhdr *q = qh(h, c);
  unsigned long long *w = reinterpret_cast<unsigned long long *>(q);
  for (unsigned i = threadIdx.x; i < sizeof(ouro_qhdr) / 8; i += blockDim.x) w[i] = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    q->front.v = pack(0, OURO_NIL);
    q->back.v = pack(0, OURO_NIL);
    q->spare.v = pack(0, OURO_NIL);
  }
  for (unsigned i = threadIdx.x; i < OURO_VL_HINTS; i += blockDim.x) q->hint[i] = pack(0, OURO_NIL);
}

/* every ring slot starts empty for its own position (seq = index); every
 * virtualized-array directory entry starts empty for segment index = entry */
__global__ void k_init_cells(ouro_heap_dev h) {
  const unsigned item = ouro_qform((int)h.variant) == OURO_QF_VARRAY ? OURO_NIL : 0u;
  for (int c = 0; c < OURO_MAX_CLASSES; ++c) {
    const unsigned long long R = h.ring_mask[c] + 1;
    unsigned long long *cells = h.cells + h.ring_off[c];
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < R;
         i += (unsigned long long)gridDim.x * blockDim.x)
      cells[i] = slot(i, item);
  }
}

__global__ void k_fill_u8(unsigned char *p, unsigned long long n, unsigned char v) {
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x)
    p[i] = v;
}

static ouro_status init_state(ouro_heap *H, cudaStream_t s) {
  ouro_heap_dev &d = H->d;
  OURO_CUDA(cudaMemsetAsync(H->meta + H->off_glob, 0, sizeof(ouro_glob), s));
  OURO_CUDA(cudaMemsetAsync(H->meta + H->off_stats, 0, H->stats_words * 8, s));
  k_init_qhdr<<<OURO_MAX_CLASSES, 128, 0, s>>>(d);   /* every class, runs above one chunk too */
  OURO_LAUNCHED();
  const int grid = 4 * sm_count();
  k_fill_u8<<<grid, 256, 0, s>>>(d.chunk_cls, d.n_chunks, OURO_CLS_NONE);
  OURO_LAUNCHED();
  if (d.chunk_free) OURO_CUDA(cudaMemsetAsync(d.chunk_free, 0, d.n_chunks * 4, s));
  if (d.bits) OURO_CUDA(cudaMemsetAsync(d.bits, 0, d.n_chunks * (size_t)d.words_per_chunk * 4, s));
  if (H->ring_total) {
    k_init_cells<<<grid, 256, 0, s>>>(d);
    OURO_LAUNCHED();
  }
  return OURO_OK;
}

/* ------------------------------------------------------------------ create */
extern "C" ouro_status ouro_heap_create(size_t bytes, size_t chunk_bytes, ouro_heap **out) {
  return ouro_heap_create_ex(bytes, chunk_bytes, OURO_PAGE_ARRAY, nullptr, nullptr, out);
}

extern "C" ouro_status ouro_heap_create_ex(size_t bytes, size_t chunk_bytes, ouro_variant variant,
                                           const ouro_options *opt, void *d_heap_buf, ouro_heap **out) {
  if (!out) return OURO_EINVAL;
  *out = nullptr;
  if (chunk_bytes < 256 || chunk_bytes > (1u << 20) || (chunk_bytes & (chunk_bytes - 1))) return OURO_EINVAL;
  if (bytes == 0 || bytes % chunk_bytes || bytes > (64ull << 30)) return OURO_EINVAL;
  if (variant < OURO_PAGE_ARRAY || variant > OURO_CHUNK_VARRAY) return OURO_EINVAL;
  if (d_heap_buf && ((uintptr_t)d_heap_buf & 255)) return OURO_EINVAL;
  if (!is_page(variant) && bytes / chunk_bytes > (1ull << 26)) return OURO_EINVAL;   /* chunk id field: 26 bits */

  ouro_options o;
  o.spin_limit = 1u << 20;
  o.backoff_min_ns = 32;
  o.backoff_max_ns = 2048;
  o.max_carve = 1u << 16;
  o.array_queue_capacity = 1ull << 23;
  o.checked = 0;
  o.staging = 0;
  o.deopt = 0;
  o.reserved = 0;
  if (opt) {
    if (opt->spin_limit) o.spin_limit = opt->spin_limit;
    if (opt->backoff_min_ns) o.backoff_min_ns = opt->backoff_min_ns;
    if (opt->backoff_max_ns) o.backoff_max_ns = opt->backoff_max_ns;
    if (opt->max_carve) o.max_carve = opt->max_carve;
    if (opt->array_queue_capacity) o.array_queue_capacity = opt->array_queue_capacity;
    o.checked = opt->checked;
    o.staging = opt->staging;
    o.deopt = opt->deopt;
    if (opt->reserved) return OURO_EINVAL;
  }
  if (o.backoff_max_ns < o.backoff_min_ns) o.backoff_max_ns = o.backoff_min_ns;

  ouro_heap *H = (ouro_heap *)calloc(1, sizeof(ouro_heap));
  if (!H) return OURO_ENOMEM;
  H->opt = o;
  cudaGetDevice(&H->device);
  ouro_heap_dev &d = H->d;
  d.bytes = bytes;
  d.n_chunks = bytes / chunk_bytes;
  d.chunk_bytes = (unsigned)chunk_bytes;
  d.log2_chunk = 0;
  while ((1ull << d.log2_chunk) < chunk_bytes) d.log2_chunk++;
  d.n_classes = d.log2_chunk - 4 + 1;
  d.variant = variant;
  d.seg_cap = (unsigned)((chunk_bytes - OURO_SEG_HDR) / 8);
  d.words_per_chunk = (unsigned)((chunk_bytes / 16 + 31) / 32);
  d.spin_limit = o.spin_limit;
  d.backoff_min_ns = o.backoff_min_ns;
  d.backoff_max_ns = o.backoff_max_ns;
  d.max_carve = o.max_carve;
  d.checked = o.checked ? 1u : 0u;
  d.staging = o.staging ? 1u : 0u;   /* every queue form */
  d.deopt = o.deopt ? 1u : 0u;
  d.pad = 0;

  /* ring sizes (plain arrays); directory sizes (virtualized arrays): a
   * directory spans every position that can be live at once -- all items
   * of the class, plus waiting and in-flight positions -- in whole segments */
  unsigned long long ring_total = 0;
  for (unsigned c = 0; c < OURO_MAX_CLASSES; ++c) {
    unsigned long long cap = 0, R = 0;
    /* items the class can ever hold: pages, chunk ids, or (above one chunk) runs */
    const unsigned long long items = c >= d.n_classes ? d.n_chunks >> (c - d.n_classes + 1)
                                     : is_page(variant) ? bytes >> (4 + c) : d.n_chunks;
    if (variant == OURO_PAGE_ARRAY || variant == OURO_CHUNK_ARRAY) {
      cap = items;
      if (variant == OURO_PAGE_ARRAY && c < d.n_classes && cap > o.array_queue_capacity)
        cap = o.array_queue_capacity;
      R = next_pow2(cap + OURO_RING_SLACK);
    } else if (is_varray(variant)) {
      R = next_pow2((items + OURO_VA_SLACK + d.seg_cap - 1) / d.seg_cap + 4);
    }
    d.qcap[c] = cap;
    d.ring_off[c] = ring_total;
    d.ring_mask[c] = R ? R - 1 : 0;
    ring_total += R;
  }
  H->ring_total = ring_total;

  /* metadata layout */
  const bool need_free = !is_page(variant);
  const bool need_bits = !is_page(variant) || o.checked;
  size_t off = 0;
  H->off_qhdr = off;  off = align256(off + sizeof(ouro_qhdr) * OURO_MAX_CLASSES);
  H->off_glob = off;  off = align256(off + sizeof(ouro_glob));
  H->stats_words = (size_t)(OURO_MAX_CLASSES + 1) * OURO_NSTAT * OURO_SHARDS;   /* + row OURO_ROW_NONE */
  H->off_stats = off; off = align256(off + H->stats_words * 8);
  H->off_cls = off;   off = align256(off + d.n_chunks);
  H->off_pool = off;  off = align256(off + d.n_chunks * 4);
  H->off_free = off;  if (need_free) off = align256(off + d.n_chunks * 4);
  H->off_bits = off;  if (need_bits) off = align256(off + d.n_chunks * (size_t)d.words_per_chunk * 4);
  H->off_cells = off; off = align256(off + ring_total * 8);
  H->off_work = off;  off = align256(off + OURO_WORK_SLOTS * 128);
  H->meta_bytes = off;

  cudaError_t e = cudaMalloc((void **)&H->meta, H->meta_bytes);
  if (e != cudaSuccess) {
    free(H);
    return cuda_fail(e);
  }
  if (d_heap_buf) {
    H->heap_buf = d_heap_buf;
    H->owns_heap = 0;
  } else {
    e = cudaMalloc(&H->heap_buf, bytes);
    if (e != cudaSuccess) {
      cudaFree(H->meta);
      free(H);
      return cuda_fail(e);
    }
    H->owns_heap = 1;
  }
  d.base = (unsigned char *)H->heap_buf;
  d.qhdr = H->meta + H->off_qhdr;
  d.glob = H->meta + H->off_glob;
  d.stats = (unsigned long long *)(H->meta + H->off_stats);
  d.chunk_cls = H->meta + H->off_cls;
  d.pool = (unsigned int *)(H->meta + H->off_pool);
  d.chunk_free = need_free ? (int *)(H->meta + H->off_free) : nullptr;
  d.bits = need_bits ? (unsigned int *)(H->meta + H->off_bits) : nullptr;
  d.cells = ring_total ? (unsigned long long *)(H->meta + H->off_cells) : nullptr;

  ouro_status st = init_state(H, 0);
  if (st == OURO_OK) {
    e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) st = cuda_fail(e);
  }
  if (st != OURO_OK) {
    ouro_heap_destroy(H);
    return st;
  }
  *out = H;
  return OURO_OK;
}

extern "C" ouro_status ouro_heap_destroy(ouro_heap *H) {
  if (!H) return OURO_OK;
  cudaDeviceSynchronize();
  if (H->owns_heap && H->heap_buf) cudaFree(H->heap_buf);
  if (H->meta) cudaFree(H->meta);
  free(H);
  return OURO_OK;
}

extern "C" ouro_status ouro_heap_reset(ouro_heap *H, void *stream) {
  if (!H) return OURO_EINVAL;
  return init_state(H, S(stream));
}

extern "C" ouro_status ouro_heap_device(const ouro_heap *H, ouro_heap_dev *out) {
  if (!H || !out) return OURO_EINVAL;
  *out = H->d;
  return OURO_OK;
}

/* ------------------------------------------------------- queue inspection */
/* Number of positions in [head, tail) of class c holding an item; written
 * to out[c].  Quiescent heaps only.  One block per class. */
__global__ void k_count_queued(ouro_heap_dev h, unsigned long long *out) {
  const int c = blockIdx.x;
  ouro_qhdr *q = qh(h, c);
  const unsigned long long hd = q->head.v, tl = q->tail.v;
  unsigned long long n = 0;
  for (unsigned long long p = hd + threadIdx.x; p < tl; p += blockDim.x) {
    unsigned long long *cell = slot_any(h, c, p);
    if (cell && slot_d(*cell, p) == 1) n++;
  }
  atomicAdd(&out[c], n);
}

/* Items of class c in queue order (quiescent): single thread, compacted. */
__global__ void k_collect_queue(ouro_heap_dev h, int c, unsigned *out, unsigned long long cap,
                                unsigned long long *n_out) {
  ouro_qhdr *q = qh(h, c);
  const unsigned long long hd = q->head.v, tl = q->tail.v;
  unsigned long long n = 0;
  for (unsigned long long p = hd; p < tl; ++p) {
    unsigned long long *cell = slot_any(h, c, p);
    if (!cell) continue;
    unsigned long long v = *cell;
    if (slot_d(v, p) != 1) continue;
    const bool cq = !ouro_page_queues((int)h.variant);
    if (n < cap) out[n] = cq ? OURO_CQ_ID(lo32(v)) : lo32(v);
    n++;
  }
  *n_out = n;
}

/* chunks per class (row n_classes: queue segments) */
__global__ void k_chunk_hist(ouro_heap_dev h, unsigned long long *out) {
  __shared__ unsigned long long sh[OURO_MAX_CLASSES + 1];
  for (unsigned i = threadIdx.x; i <= OURO_MAX_CLASSES; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  for (unsigned long long x = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; x < h.n_chunks;
       x += (unsigned long long)gridDim.x * blockDim.x) {
    unsigned c = h.chunk_cls[x];
    if (c == OURO_CLS_SEG) {
      atomicAdd(&sh[OURO_MAX_CLASSES], 1ull);
      continue;
    }
    if (c != OURO_CLS_NONE && (c & 0xC0u) != 0xC0u) c &= 0x3Fu;   /* runs: start (live or free) and body */
    if (c < OURO_MAX_CLASSES) atomicAdd(&sh[c], 1ull);
  }
  __syncthreads();
  for (unsigned i = threadIdx.x; i <= OURO_MAX_CLASSES; i += blockDim.x)
    if (sh[i]) atomicAdd(&out[i], sh[i]);
}

/* segments on each class spare stack (quiescent) */
__global__ void k_count_spares(ouro_heap_dev h, unsigned long long *out) {
  if (threadIdx.x) return;
  for (unsigned c = 0; c < OURO_MAX_CLASSES; ++c) {
    unsigned x = lo32(qh(h, c)->spare.v);
    unsigned long long n = 0;
    while (x != OURO_NIL && n < h.n_chunks) {
      n++;
      x = seg_of(h, x)->spare_next;
    }
    out[c] = n;
  }
}


struct scratch_buf {
  void *p = nullptr;
  ~scratch_buf() {
    if (p) cudaFree(p);
  }
};

extern "C" ouro_status ouro_heap_stats(ouro_heap *H, ouro_stats *out, void *stream) {
  if (!H || !out) return OURO_EINVAL;
  cudaStream_t s = S(stream);
  const ouro_heap_dev &d = H->d;
  memset(out, 0, sizeof(*out));
  out->n_classes = d.n_classes;
  std::vector<unsigned long long> st(H->stats_words);
  ouro_glob g;
  scratch_buf tmp;
  const size_t nt = 3 * (OURO_MAX_CLASSES + 1);
  OURO_CUDA(cudaMalloc(&tmp.p, nt * 8));
  unsigned long long *dq = (unsigned long long *)tmp.p, *dh = dq + (OURO_MAX_CLASSES + 1),
                     *ds = dh + (OURO_MAX_CLASSES + 1);
  OURO_CUDA(cudaMemsetAsync(tmp.p, 0, nt * 8, s));
  k_count_queued<<<OURO_MAX_CLASSES, 256, 0, s>>>(d, dq);
  OURO_LAUNCHED();
  k_chunk_hist<<<2 * sm_count(), 256, 0, s>>>(d, dh);
  OURO_LAUNCHED();
  if (is_virtual(d.variant)) {
    k_count_spares<<<1, 32, 0, s>>>(d, ds);
    OURO_LAUNCHED();
  }
  std::vector<unsigned long long> hq(nt);
  OURO_CUDA(cudaMemcpyAsync(hq.data(), tmp.p, nt * 8, cudaMemcpyDeviceToHost, s));
  OURO_CUDA(cudaMemcpyAsync(st.data(), d.stats, H->stats_words * 8, cudaMemcpyDeviceToHost, s));
  OURO_CUDA(cudaMemcpyAsync(&g, d.glob, sizeof(g), cudaMemcpyDeviceToHost, s));
  OURO_CUDA(cudaStreamSynchronize(s));
  auto sum = [&](unsigned row, unsigned kind) {
    unsigned long long a = 0;
    for (unsigned i = 0; i < OURO_SHARDS; ++i) a += st[((size_t)row * OURO_NSTAT + kind) * OURO_SHARDS + i];
    return a;
  };
  out->n_large = OURO_MAX_CLASSES - d.n_classes;
  for (unsigned c = 0; c < OURO_MAX_CLASSES; ++c) {
    out->mallocs[c] = sum(c, OURO_ST_MALLOC);
    out->frees[c] = sum(c, OURO_ST_FREE);
    out->failed[c] = sum(c, OURO_ST_FAILED);
    out->carves[c] = sum(c, OURO_ST_CARVE);
    out->repushes[c] = sum(c, OURO_ST_REPUSH);
    out->dead[c] = sum(c, OURO_ST_DEAD);
    out->live[c] = out->mallocs[c] - out->frees[c];
    out->queued[c] = hq[c];
    out->carved_now[c] = hq[(OURO_MAX_CLASSES + 1) + c];
    out->spare_chunks += hq[2 * (OURO_MAX_CLASSES + 1) + c];
  }
  out->seg_chunks = hq[(OURO_MAX_CLASSES + 1) + OURO_MAX_CLASSES];
  if (out->seg_chunks >= out->spare_chunks) out->seg_chunks -= out->spare_chunks;
  out->zero_reqs = sum(OURO_ROW_NONE, OURO_ST_ZERO);
  out->too_large = sum(OURO_ROW_NONE, OURO_ST_TOO_LARGE);
  out->bump = g.bump.v < d.n_chunks ? g.bump.v : d.n_chunks;
  out->pool_size = g.pool_taken.v < g.pool_size ? g.pool_size - g.pool_taken.v : 0;
  out->error_bits = g.error_bits;
  out->error_site = g.error_site;
  return g.error_bits ? OURO_EDEVICE : OURO_OK;
}

/* ---------------------------------------------------------------- snapshot */
extern "C" ouro_status ouro_heap_snapshot(ouro_heap *H, ouro_snapshot *out, void *stream) {
  if (!H || !out) return OURO_EINVAL;
  memset(out, 0, sizeof(*out));
  cudaStream_t s = S(stream);
  const ouro_heap_dev &d = H->d;
  out->n_classes = d.n_classes;
  out->n_chunks = d.n_chunks;
  ouro_glob g;
  OURO_CUDA(cudaMemcpyAsync(&g, d.glob, sizeof(g), cudaMemcpyDeviceToHost, s));
  OURO_CUDA(cudaStreamSynchronize(s));
  out->bump = g.bump.v < d.n_chunks ? g.bump.v : d.n_chunks;
  const unsigned long long pt = g.pool_taken.v < g.pool_size ? g.pool_taken.v : g.pool_size;
  out->pool_n = g.pool_size - pt;
  out->pool = (uint32_t *)malloc((out->pool_n ? out->pool_n : 1) * 4);
  out->chunk_cls = (uint8_t *)malloc(d.n_chunks);
  if (!out->pool || !out->chunk_cls) return OURO_ENOMEM;
  if (out->pool_n)
    OURO_CUDA(cudaMemcpyAsync(out->pool, d.pool + pt, out->pool_n * 4, cudaMemcpyDeviceToHost, s));
  OURO_CUDA(cudaMemcpyAsync(out->chunk_cls, d.chunk_cls, d.n_chunks, cudaMemcpyDeviceToHost, s));
  if (d.chunk_free) {
    out->chunk_free = (int32_t *)malloc(d.n_chunks * 4);
    if (!out->chunk_free) return OURO_ENOMEM;
    OURO_CUDA(cudaMemcpyAsync(out->chunk_free, d.chunk_free, d.n_chunks * 4, cudaMemcpyDeviceToHost, s));
  }
  scratch_buf cnt;
  OURO_CUDA(cudaMalloc(&cnt.p, 8));
  for (unsigned c = 0; c < OURO_MAX_CLASSES; ++c) {   /* runs above one chunk: first chunks of free runs */
    ouro_qhdr hq;
    OURO_CUDA(cudaMemcpyAsync(&hq, qh(d, c), sizeof(hq), cudaMemcpyDeviceToHost, s));
    OURO_CUDA(cudaStreamSynchronize(s));
    unsigned long long span = hq.tail.v > hq.head.v ? hq.tail.v - hq.head.v : 0;
    scratch_buf items;
    OURO_CUDA(cudaMalloc(&items.p, (span ? span : 1) * 4));
    k_collect_queue<<<1, 1, 0, s>>>(d, (int)c, (unsigned *)items.p, span, (unsigned long long *)cnt.p);
    OURO_LAUNCHED();
    unsigned long long n = 0;
    OURO_CUDA(cudaMemcpyAsync(&n, cnt.p, 8, cudaMemcpyDeviceToHost, s));
    OURO_CUDA(cudaStreamSynchronize(s));
    if (n > span) n = span;
    out->queue_n[c] = n;
    out->queue[c] = (uint32_t *)malloc((n ? n : 1) * 4);
    if (!out->queue[c]) return OURO_ENOMEM;
    if (n) OURO_CUDA(cudaMemcpyAsync(out->queue[c], items.p, n * 4, cudaMemcpyDeviceToHost, s));
    OURO_CUDA(cudaStreamSynchronize(s));
  }

  return OURO_OK;
}

extern "C" void ouro_snapshot_free(ouro_snapshot *sn) {
  if (!sn) return;
  free(sn->pool);
  free(sn->chunk_cls);
  free(sn->chunk_free);
  for (int c = 0; c < OURO_MAX_CLASSES; ++c) free(sn->queue[c]);
  memset(sn, 0, sizeof(*sn));
}

/* -------------------------------------------------------------------- trim */
/* 1. count the queued pages of every chunk (page queues) */
__global__ void k_trim_count(ouro_heap_dev h, unsigned *qcount) {
  if (!ouro_page_queues((int)h.variant)) return;   /* counts live in chunk_free */
  const int c = blockIdx.y;
  ouro_qhdr *q = qh(h, c);
  const unsigned long long hd = q->head.v, tl = q->tail.v;
  const unsigned ppc_log = h.log2_chunk - 4 - c;
  for (unsigned long long p = hd + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; p < tl;
       p += (unsigned long long)gridDim.x * blockDim.x) {
    unsigned long long *cell = slot_any(h, c, p);
    if (!cell) continue;
    unsigned long long v = *cell;
    if (slot_d(v, p) == 1) atomicAdd(&qcount[lo32(v) >> ppc_log], 1u);
  }
}

/* 2. chunks whose pages are all free, and queue segments, return to the pool:
 *    keep[x] = 1 for chunks that stay carved; in_pool[x] = 1 for pool chunks */
__global__ void k_trim_mark(ouro_heap_dev h, const unsigned *qcount, unsigned char *in_pool) {
  for (unsigned long long x = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; x < h.n_chunks;
       x += (unsigned long long)gridDim.x * blockDim.x) {
    unsigned c = h.chunk_cls[x];
    unsigned char ip = 0;
    if (c < h.n_classes) {
      unsigned long long ppc = 1ull << (h.log2_chunk - 4 - c);
      const unsigned long long free_pages = h.chunk_free ? (unsigned long long)max(h.chunk_free[x], 0) : qcount[x];
      if (free_pages == ppc) {
        h.chunk_cls[x] = OURO_CLS_NONE;
        ip = 1;
        if (h.chunk_free) h.chunk_free[x] = 0;
        if (h.bits)
          for (unsigned w = 0; w < h.words_per_chunk; ++w) h.bits[x * h.words_per_chunk + w] = 0;
      }
    } else if (c == OURO_CLS_SEG) {
      h.chunk_cls[x] = OURO_CLS_NONE;
      ip = 1;
    }
    in_pool[x] = ip;
  }
}

/* pool entries not yet handed out stay in the pool */
__global__ void k_trim_old_pool(ouro_heap_dev h, unsigned char *in_pool) {
  ouro_glob *g = gl(h);
  const unsigned long long ps = g->pool_size, pt = g->pool_taken.v < ps ? g->pool_taken.v : ps;
  for (unsigned long long i = pt + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < ps;
       i += (unsigned long long)gridDim.x * blockDim.x)
    in_pool[h.pool[i]] = 1;
}

/* free runs: every chunk of every run queued in a class above one chunk
 * joins the pool (the queues are reset afterwards); blockIdx.y = class -
 * n_classes */
__global__ void k_trim_runs(ouro_heap_dev h, unsigned char *in_pool) {
  const unsigned c = h.n_classes + blockIdx.y;
  ouro_qhdr *q = qh(h, c);
  const unsigned long long hd = q->head.v, tl = q->tail.v;
  const unsigned long long k = 1ull << (c - h.n_classes + 1);
  for (unsigned long long p = hd + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; p < tl;
       p += (unsigned long long)gridDim.x * blockDim.x) {
    unsigned long long *cell = slot_any(h, (int)c, p);
    if (!cell) continue;
    const unsigned long long v = *cell;
    if (slot_d(v, p) != 1) continue;
    const unsigned x = lo32(v);
    for (unsigned long long i = 0; i < k; ++i) {
      h.chunk_cls[x + i] = OURO_CLS_NONE;
      in_pool[x + i] = 1;
    }
  }
}

/* 3. surviving queue items of class c, in queue order, into tmp (one block) */
__global__ void k_trim_compact(ouro_heap_dev h, int c, const unsigned char *in_pool, unsigned *tmp,
                               unsigned long long *n_out) {
  ouro_qhdr *q = qh(h, c);
  const unsigned long long hd = q->head.v, tl = q->tail.v;
  const unsigned ppc_log = h.log2_chunk - 4 - c;
  const bool cq = !ouro_page_queues((int)h.variant);
  __shared__ unsigned warp_tot[32];
  __shared__ unsigned long long base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (unsigned long long p0 = hd; p0 < tl; p0 += blockDim.x) {
    unsigned long long p = p0 + threadIdx.x;
    unsigned item = 0;
    bool keep = false;
    if (p < tl) {
      unsigned long long *cell = slot_any(h, c, p);
      if (cell) {
        unsigned long long v = *cell;
        if (slot_d(v, p) == 1) {
          item = lo32(v);
          keep = !in_pool[cq ? OURO_CQ_ID(item) : item >> ppc_log];
          if (cq) item = OURO_CQ_ID(item);
        }
      }
    }
    unsigned b = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) warp_tot[wid] = __popc(b);
    __syncthreads();
    unsigned before = 0, tot = 0;
    for (unsigned w = 0; w < nw; ++w) {
      if (w < wid) before += warp_tot[w];
      tot += warp_tot[w];
    }
    if (keep) tmp[base + before + __popc(b & ((1u << lane) - 1))] = item;
    __syncthreads();
    if (threadIdx.x == 0) base += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_out = base;
}

/* 4. canonical pool: new bump = 1 + highest non-pool chunk below the old bump */
__global__ void k_trim_bump(ouro_heap_dev h, const unsigned char *in_pool, unsigned long long *top) {
  const unsigned long long b = gl(h)->bump.v < h.n_chunks ? gl(h)->bump.v : h.n_chunks;
  for (unsigned long long x = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; x < b;
       x += (unsigned long long)gridDim.x * blockDim.x)
    if (!in_pool[x]) atomicMax(top, x + 1);
}

/* ascending pool list below the new bump (one block, ordered compaction) */
__global__ void k_trim_pool(ouro_heap_dev h, const unsigned char *in_pool, const unsigned long long *top) {
  const unsigned long long nb = *top;
  __shared__ unsigned warp_tot[32];
  __shared__ unsigned long long base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (unsigned long long x0 = 0; x0 < nb; x0 += blockDim.x) {
    unsigned long long x = x0 + threadIdx.x;
    bool inp = x < nb && in_pool[x];
    unsigned b = __ballot_sync(0xffffffffu, inp);
    if (lane == 0) warp_tot[wid] = __popc(b);
    __syncthreads();
    unsigned before = 0, tot = 0;
    for (unsigned w = 0; w < nw; ++w) {
      if (w < wid) before += warp_tot[w];
      tot += warp_tot[w];
    }
    if (inp) h.pool[base + before + __popc(b & ((1u << lane) - 1))] = (unsigned)x;
    __syncthreads();
    if (threadIdx.x == 0) base += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    ouro_glob *g = gl(h);
    g->pool_size = base;
    g->pool_taken.v = 0;
    g->bump.v = nb;
  }
}

/* 5. reset the class queue and re-lay its surviving items from position 0.
 *    Array rings: slots [0, n) hold the items, the rest is empty again.
 *    Lists: segments are taken class by class from the pool front. */
__global__ void k_trim_relay_ring(ouro_heap_dev h, int c, const unsigned *tmp, const unsigned long long *n_in) {
  const unsigned long long n = *n_in, R = h.ring_mask[c] + 1;
  unsigned long long *cells = h.cells + h.ring_off[c];
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < R;
       i += (unsigned long long)gridDim.x * blockDim.x)
    cells[i] = i < n ? slot(i + 1, tmp[i]) : slot(i, 0);
}

__global__ void k_trim_reset_q(ouro_heap_dev h, int c, const unsigned long long *n_in) {
  ouro_qhdr *q = qh(h, c);
  q->head.v = 0;
  q->tail.v = n_in ? *n_in : 0;
  q->lock.v = 0;
  q->front.v = pack(0, OURO_NIL);
  q->back.v = pack(0, OURO_NIL);
  q->spare.v = pack(0, OURO_NIL);
  for (int i = 0; i < OURO_VL_HINTS; ++i) q->hint[i] = pack(0, OURO_NIL);
}

/* chunks each class owns after the trim (from the chunk histogram) */
__global__ void k_trim_carved(ouro_heap_dev h, const unsigned long long *hist) {
  for (unsigned c = threadIdx.x; c < OURO_MAX_CLASSES; c += blockDim.x) qh(h, c)->carved.v = hist[c];
}

/* virtualized-array directory: every entry empty for its own index */
__global__ void k_trim_reset_dir(ouro_heap_dev h, int c) {
  const unsigned long long D = h.ring_mask[c] + 1;
  unsigned long long *dir = h.cells + h.ring_off[c];
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < D;
       i += (unsigned long long)gridDim.x * blockDim.x)
    dir[i] = pack((unsigned)i, OURO_NIL);
}

/* virtualized relay: one block per class call; thread 0 takes segments from
 * the pool and links them (list) or enters them in the directory (array) */
__global__ void k_trim_relay_list(ouro_heap_dev h, int c, const unsigned *tmp, const unsigned long long *n_in) {
  __shared__ unsigned seg_chunk;
  ouro_qhdr *q = qh(h, c);
  const unsigned long long n = *n_in;
  const unsigned cap = h.seg_cap;
  const bool dir = ouro_qform((int)h.variant) == OURO_QF_VARRAY;
  unsigned prev = OURO_NIL;
  for (unsigned long long s = 0; s * cap < n; ++s) {
    if (threadIdx.x == 0) {
      chunk_range r = take_chunks(h, 1);
      unsigned x = r.k1 + r.k2 ? range_chunk(h, r, 0) : OURO_NIL;
      if (x != OURO_NIL) {
        h.chunk_cls[x] = OURO_CLS_SEG;
        seg_of(h, x)->link = pack((unsigned)s, OURO_NIL);
        seg_of(h, x)->done = 0;
        if (dir) {
          *va_entry(h, c, s) = pack((unsigned)s, x);
        } else {
          if (prev == OURO_NIL) q->front.v = pack((unsigned)s, x);
          else seg_of(h, prev)->link = pack((unsigned)(s - 1), x);
          q->back.v = pack((unsigned)s, x);
        }
      } else {
        set_error(h, OURO_ERR_QUEUE_FULL, OURO_SITE_TRIM);
      }
      seg_chunk = x;
    }
    __syncthreads();
    const unsigned x = seg_chunk;
    if (x == OURO_NIL) return;
    unsigned long long *cells = seg_cells(h, x);
    for (unsigned i = threadIdx.x; i < cap; i += blockDim.x) {
      unsigned long long p = s * cap + i;
      cells[i] = p < n ? slot(p + 1, tmp[p]) : slot(p, 0);
    }
    /* positions already produced (and, below n, waiting for consumers) */
    if (threadIdx.x == 0) seg_of(h, x)->done = (unsigned)min((unsigned long long)cap, n - s * cap);
    prev = x;
    __syncthreads();
  }
}

extern "C" ouro_status ouro_heap_trim(ouro_heap *H, void *stream) {
  if (!H) return OURO_EINVAL;
  cudaStream_t s = S(stream);
  const ouro_heap_dev &d = H->d;
  OURO_CUDA(cudaStreamSynchronize(s));
  /* largest queue span decides the temp size */
  unsigned long long span_max = 1;
  std::vector<unsigned long long> spans(d.n_classes);
  for (unsigned c = 0; c < d.n_classes; ++c) {        /* classes within a chunk keep their live pages */
    ouro_qhdr hq;
    OURO_CUDA(cudaMemcpy(&hq, qh(d, c), sizeof(hq), cudaMemcpyDeviceToHost));
    spans[c] = hq.tail.v > hq.head.v ? hq.tail.v - hq.head.v : 0;
    if (spans[c] > span_max) span_max = spans[c];
  }
  scratch_buf qcount, in_pool, tmp, nbuf;
  OURO_CUDA(cudaMalloc(&qcount.p, d.n_chunks * 4));
  OURO_CUDA(cudaMalloc(&in_pool.p, d.n_chunks));
  OURO_CUDA(cudaMalloc(&tmp.p, span_max * 4 * d.n_classes));
  const size_t nwords = OURO_MAX_CLASSES + 1 + OURO_MAX_CLASSES + 1;
  OURO_CUDA(cudaMalloc(&nbuf.p, 8 * nwords));
  /* ncount: items each class keeps (0 for the run classes: all their queued runs are free) */
  unsigned long long *ncount = (unsigned long long *)nbuf.p, *top = ncount + OURO_MAX_CLASSES,
                     *hist = top + 1;
  OURO_CUDA(cudaMemsetAsync(qcount.p, 0, d.n_chunks * 4, s));
  OURO_CUDA(cudaMemsetAsync(nbuf.p, 0, 8 * nwords, s));
  const int grid = 4 * sm_count();
  k_trim_count<<<dim3(grid, d.n_classes), 256, 0, s>>>(d, (unsigned *)qcount.p);
  OURO_LAUNCHED();
  k_trim_mark<<<grid, 256, 0, s>>>(d, (const unsigned *)qcount.p, (unsigned char *)in_pool.p);
  OURO_LAUNCHED();
  k_trim_old_pool<<<grid, 256, 0, s>>>(d, (unsigned char *)in_pool.p);
  OURO_LAUNCHED();
  if (d.n_classes < OURO_MAX_CLASSES) {
    k_trim_runs<<<dim3(grid, OURO_MAX_CLASSES - d.n_classes), 256, 0, s>>>(d, (unsigned char *)in_pool.p);
    OURO_LAUNCHED();
  }
  for (unsigned c = 0; c < d.n_classes; ++c) {
    k_trim_compact<<<1, 1024, 0, s>>>(d, (int)c, (const unsigned char *)in_pool.p,
                                      (unsigned *)tmp.p + (size_t)c * span_max, ncount + c);
    OURO_LAUNCHED();
  }
  k_trim_bump<<<grid, 256, 0, s>>>(d, (const unsigned char *)in_pool.p, top);
  OURO_LAUNCHED();
  k_trim_pool<<<1, 1024, 0, s>>>(d, (const unsigned char *)in_pool.p, top);
  OURO_LAUNCHED();
  for (unsigned c = 0; c < OURO_MAX_CLASSES; ++c) {
    const unsigned *src = (const unsigned *)tmp.p + (size_t)(c < d.n_classes ? c : 0) * span_max;
    if (d.variant == OURO_PAGE_ARRAY || d.variant == OURO_CHUNK_ARRAY) {
      k_trim_relay_ring<<<grid, 256, 0, s>>>(d, (int)c, src, ncount + c);
      OURO_LAUNCHED();
      k_trim_reset_q<<<1, 1, 0, s>>>(d, (int)c, ncount + c);
      OURO_LAUNCHED();
    } else {
      k_trim_reset_q<<<1, 1, 0, s>>>(d, (int)c, ncount + c);
      OURO_LAUNCHED();
      if (is_varray(d.variant)) {
        k_trim_reset_dir<<<grid, 256, 0, s>>>(d, (int)c);
        OURO_LAUNCHED();
      }
      k_trim_relay_list<<<1, 256, 0, s>>>(d, (int)c, src, ncount + c);
      OURO_LAUNCHED();
    }
  }
  k_chunk_hist<<<grid, 256, 0, s>>>(d, hist);
  OURO_LAUNCHED();
  k_trim_carved<<<1, 32, 0, s>>>(d, hist);
  OURO_LAUNCHED();
  OURO_CUDA(cudaStreamSynchronize(s));
  return OURO_OK;
}

/* ------------------------------------------------------------------- misc */
extern "C" const char *ouro_status_string(ouro_status s) {
  switch (s) {
    case OURO_OK: return "ok";
    case OURO_EINVAL: return "invalid argument";
    case OURO_ENOMEM: return "out of memory";
    case OURO_ECUDA: return "CUDA error";
    case OURO_EDEVICE: return "device error bits set";
    case OURO_ENOTSUP: return "not supported by this queue variant";
    default: return "unknown status";
  }
}
extern "C" int ouro_last_cuda_error(void) { return g_last_cuda_error; }
extern "C" uint64_t ouro_kernel_launches(void) {
  return __atomic_load_n(&ouro::host::g_launches, __ATOMIC_RELAXED);
}

__global__ void k_stall_producer(ouro_heap_dev h, int c, unsigned n) {
  atomicAdd(&qh(h, c)->tail.v, (unsigned long long)n);
}
extern "C" ouro_status ouro_debug_stall_producer(ouro_heap *H, int cls, uint32_t n, void *stream) {
  if (!H || cls < 0 || cls >= (int)H->d.n_classes) return OURO_EINVAL;
  k_stall_producer<<<1, 1, 0, S(stream)>>>(H->d, cls, n);
  OURO_LAUNCHED();
  return OURO_OK;
}

/* ------------------------------------------- statistics without allocation */
/* For callers that must not allocate device memory at the time they ask for
 * statistics: applications whose device memory is all handed out up front by
 * their own pool, and latency-bound loops in which a cudaMalloc / cudaFree
 * could stall the device.  The scratch lives in this file-scope device array
 * instead of a cudaMalloc'ed buffer; every device that loads the library
 * holds it (1.5 KiB) until the process exits. */
#define OURO_STATIC_SCRATCH_ROWS (OURO_MAX_CLASSES + 1)
#define OURO_STATIC_SCRATCH_WORDS (OURO_STATIC_SCRATCH_ROWS * (OURO_NSTAT + 3))
static __device__ __align__(256) unsigned long long g_stats_scratch[OURO_STATIC_SCRATCH_WORDS];

/* sum the per-SM shards of every counter row into out[row * OURO_NSTAT + kind] */
__global__ void k_sum_shards(ouro_heap_dev h, unsigned long long *out) {
  const unsigned rows = (OURO_MAX_CLASSES + 1) * OURO_NSTAT;   /* every class row + OURO_ROW_NONE */
  for (unsigned i = threadIdx.x; i < rows; i += blockDim.x) {
    unsigned long long a = 0;
    for (unsigned s = 0; s < OURO_SHARDS; ++s) a += h.stats[(size_t)i * OURO_SHARDS + s];
    out[i] = a;
  }
}

static std::mutex g_scratch_mu;
static unsigned long long *g_scratch_dev[64];   /* device address of the array, per device ordinal */

extern "C" ouro_status ouro_heap_stats_static(ouro_heap *H, ouro_stats *out, void *stream) {
  if (!H || !out) return OURO_EINVAL;
  const ouro_heap_dev &d = H->d;
  if (d.n_classes + 1 > OURO_STATIC_SCRATCH_ROWS) return OURO_EINVAL;   /* larger than the scratch array */
  int dev = 0;
  OURO_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return OURO_EINVAL;
  unsigned long long *scratch;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_dev[dev]) {
      void *p = nullptr;
      OURO_CUDA(cudaGetSymbolAddress(&p, g_stats_scratch));
      g_scratch_dev[dev] = (unsigned long long *)p;
    }
    scratch = g_scratch_dev[dev];
  }
  cudaStream_t s = S(stream);
  const unsigned R = OURO_STATIC_SCRATCH_ROWS;
  unsigned long long *dsum = scratch, *dq = scratch + R * OURO_NSTAT, *dh = dq + R, *ds = dh + R;
  OURO_CUDA(cudaMemsetAsync(scratch, 0, OURO_STATIC_SCRATCH_WORDS * 8, s));
  k_sum_shards<<<1, 256, 0, s>>>(d, dsum);
  OURO_LAUNCHED();
  k_count_queued<<<OURO_MAX_CLASSES, 256, 0, s>>>(d, dq);
  OURO_LAUNCHED();
  k_chunk_hist<<<2 * sm_count(), 256, 0, s>>>(d, dh);
  OURO_LAUNCHED();
  if (is_virtual(d.variant)) {
    k_count_spares<<<1, 32, 0, s>>>(d, ds);
    OURO_LAUNCHED();
  }
  unsigned long long hv[OURO_STATIC_SCRATCH_WORDS];
  ouro_glob g;
  OURO_CUDA(cudaMemcpyAsync(hv, scratch, sizeof(hv), cudaMemcpyDeviceToHost, s));
  OURO_CUDA(cudaMemcpyAsync(&g, d.glob, sizeof(g), cudaMemcpyDeviceToHost, s));
  OURO_CUDA(cudaStreamSynchronize(s));
  const unsigned long long *hs = hv, *hq = hv + R * OURO_NSTAT, *hh = hq + R, *hsp = hh + R;
  memset(out, 0, sizeof(*out));
  out->n_classes = d.n_classes;
  out->n_large = OURO_MAX_CLASSES - d.n_classes;
  for (unsigned c = 0; c < OURO_MAX_CLASSES; ++c) {
    const unsigned long long *row = hs + (size_t)c * OURO_NSTAT;
    out->mallocs[c] = row[OURO_ST_MALLOC];
    out->frees[c] = row[OURO_ST_FREE];
    out->failed[c] = row[OURO_ST_FAILED];
    out->carves[c] = row[OURO_ST_CARVE];
    out->repushes[c] = row[OURO_ST_REPUSH];
    out->dead[c] = row[OURO_ST_DEAD];
    out->live[c] = out->mallocs[c] - out->frees[c];
    out->queued[c] = hq[c];
    out->carved_now[c] = hh[c];
    out->spare_chunks += hsp[c];
  }
  out->seg_chunks = hh[OURO_MAX_CLASSES];
  if (out->seg_chunks >= out->spare_chunks) out->seg_chunks -= out->spare_chunks;
  out->zero_reqs = hs[(size_t)OURO_ROW_NONE * OURO_NSTAT + OURO_ST_ZERO];
  out->too_large = hs[(size_t)OURO_ROW_NONE * OURO_NSTAT + OURO_ST_TOO_LARGE];
  out->bump = g.bump.v < d.n_chunks ? g.bump.v : d.n_chunks;
  out->pool_size = g.pool_taken.v < g.pool_size ? g.pool_size - g.pool_taken.v : 0;
  out->error_bits = g.error_bits;
  out->error_site = g.error_site;
  return g.error_bits ? OURO_EDEVICE : OURO_OK;
}
