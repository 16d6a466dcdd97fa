/*
 * Batch API and driver-round kernels.
 *
 * The paper's driver (Sec. 3 of arXiv 2504.18211) allocates, writes some
 * data, reads it back to check it, and frees, ten times over.  Two forms:
 *   - per launch: ouro_batch_malloc, ouro_pattern_write, ouro_pattern_check,
 *     ouro_batch_free (four kernels per round);
 *   - fused: ouro_round_fused, one kernel per round; the allocator state
 *     stays in L2 while every warp streams its own blocks.
 * Payload traffic is warp-cooperative: the 32 blocks of a warp are cut into
 * 16-byte units that the 32 lanes write and read in turn, so stores and
 * loads are 16-byte vectors that coalesce within each block.
 */
#include "ouro_internal.cuh"
#include "ouro_payload.cuh"
#include "ouro_shard.cuh"

using namespace ouro::detail;

namespace {
/* ------------------------------------------------------------ batch API */
template <int V>
__global__ void k_batch_malloc(ouro_heap_dev h, const uint32_t *sizes, void **ptrs, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    ptrs[i] = malloc_v<V>(h, sizes[i]);
}

template <int V>
__global__ void k_batch_free(ouro_heap_dev h, void *const *ptrs, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    free_v<V, false>(h, ptrs[i]);   /* the blocks were written by earlier kernels */
}

/* Block-aggregated forms (page queues, not the deoptimised form): every
 * request of a block takes its offset in its class's share with one
 * shared-memory atomic, and one thread per class takes the whole block's
 * head (malloc) or tail (free) positions with a single global atomic, so
 * the hot queue counters see one atomic per class per block instead of one
 * per class per warp.  Statistics are counted once per class per block.
 *
 * Each thread carries R requests (r * 256 + thread of the block's span, so
 * loads coalesce).  On plain-array queues a thread first tries all R of its
 * positions at once: R relaxed slot loads (malloc) or R relaxed slot CASes
 * (free) in flight together, behind one acquire / release fence, instead of
 * R chains of dependent round trips.  A position whose slot is not ready
 * (not produced yet, or its previous lap not consumed yet) goes through the
 * warp path with the position already taken, which waits, carves and
 * answers as ouro_malloc / ouro_free do. */
template <int R>
__device__ __forceinline__ void blk_reserve(const int (&cls)[R], unsigned long long (&pos)[R], unsigned *s_cnt) {
#pragma unroll
  for (int r = 0; r < R; ++r)   /* this request's offset in the block's share of its class */
    pos[r] = cls[r] >= 0 ? atomicAdd(&s_cnt[cls[r]], 1u) : 0u;
}

template <int V, int R>
__global__ void __launch_bounds__(256, 4) k_batch_malloc_blk(ouro_heap_dev h, const uint32_t *sizes, void **ptrs,
                                                             size_t n) {
  constexpr bool RING = ouro_qform(V) == OURO_QF_RING;
  __shared__ unsigned s_cnt[OURO_MAX_CLASSES], s_ok[OURO_MAX_CLASSES];
  __shared__ unsigned long long s_pos[OURO_MAX_CLASSES];
  __shared__ unsigned long long *s_ring[OURO_MAX_CLASSES];
  __shared__ unsigned long long s_rmask[OURO_MAX_CLASSES];
  if (threadIdx.x < OURO_MAX_CLASSES) {
    s_ring[threadIdx.x] = h.cells + h.ring_off[threadIdx.x];
    s_rmask[threadIdx.x] = h.ring_mask[threadIdx.x];
  }
  const size_t span = (size_t)blockDim.x * R;
  for (size_t base = (size_t)blockIdx.x * span; base < n; base += (size_t)gridDim.x * span) {
    uint32_t sz[R];
    int cls[R];
    unsigned long long pos[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const size_t i = base + (size_t)r * blockDim.x + threadIdx.x;
      sz[r] = i < n ? sizes[i] : 0;
    }
    if (threadIdx.x < OURO_MAX_CLASSES) s_cnt[threadIdx.x] = s_ok[threadIdx.x] = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const bool act = base + (size_t)r * blockDim.x + threadIdx.x < n;
      cls[r] = act ? size_class(h, sz[r]) : -1;
      if (act && cls[r] < 0) stat_add(h, OURO_ROW_NONE, sz[r] == 0 ? OURO_ST_ZERO : OURO_ST_TOO_LARGE, 1);
    }
    __syncthreads();
    blk_reserve<R>(cls, pos, s_cnt);
    __syncthreads();
    if (threadIdx.x < OURO_MAX_CLASSES && s_cnt[threadIdx.x])
      s_pos[threadIdx.x] = atomicAdd(&qh(h, threadIdx.x)->head.v, (unsigned long long)s_cnt[threadIdx.x]);
    __syncthreads();
    void *res[R];
    bool pend[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (cls[r] >= 0) pos[r] += s_pos[cls[r]];
      res[r] = nullptr;
      pend[r] = cls[r] >= 0;
    }
    if (RING && !h.checked) {   /* fast path: every position's slot at once */
      unsigned long long v[R];
#pragma unroll
      for (int r = 0; r < R; ++r)
        v[r] = pend[r] && cls[r] < (int)h.n_classes ? ld_rlx(s_ring[cls[r]] + (pos[r] & s_rmask[cls[r]])) : 0ull;
      fence_acq_rel();
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!pend[r] || cls[r] >= (int)h.n_classes) continue;
        const int d = slot_d(v[r], pos[r]);
        if (d == 1 || d == 2) {   /* an item, or the heap's null answer: take it, retire the slot */
          st_rlx(s_ring[cls[r]] + (pos[r] & s_rmask[cls[r]]), slot(pos[r] + s_rmask[cls[r]] + 1, 0));
          if (d == 1) res[r] = h.base + ((size_t)lo32(v[r]) << (4 + cls[r]));
          pend[r] = false;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {   /* the rest: the warp path from the taken positions */
      if (!__any_sync(0xffffffffu, pend[r])) continue;
      void *q = page_malloc<V, 1, true>(h, pend[r] ? cls[r] : -1, 0xffffffffu, pos[r]);
      if (pend[r]) res[r] = q;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const size_t i = base + (size_t)r * blockDim.x + threadIdx.x;
      if (i < n) ptrs[i] = res[r];
      if (res[r]) atomicAdd(&s_ok[cls[r]], 1u);
    }
    __syncthreads();
    if (threadIdx.x < OURO_MAX_CLASSES && s_cnt[threadIdx.x]) {
      stat_add(h, threadIdx.x, OURO_ST_MALLOC, s_ok[threadIdx.x]);
      stat_add(h, threadIdx.x, OURO_ST_FAILED, s_cnt[threadIdx.x] - s_ok[threadIdx.x]);
    }
    __syncthreads();
  }
}

template <int V, int R>
__global__ void __launch_bounds__(256) k_batch_free_blk(ouro_heap_dev h, void *const *ptrs, size_t n) {
  constexpr bool RING = ouro_qform(V) == OURO_QF_RING;
  __shared__ unsigned s_cnt[OURO_MAX_CLASSES];
  __shared__ unsigned long long s_pos[OURO_MAX_CLASSES];
  __shared__ unsigned long long *s_ring[OURO_MAX_CLASSES];
  __shared__ unsigned long long s_rmask[OURO_MAX_CLASSES];
  if (threadIdx.x < OURO_MAX_CLASSES) {
    s_ring[threadIdx.x] = h.cells + h.ring_off[threadIdx.x];
    s_rmask[threadIdx.x] = h.ring_mask[threadIdx.x];
  }
  const size_t span = (size_t)blockDim.x * R;
  for (size_t base = (size_t)blockIdx.x * span; base < n; base += (size_t)gridDim.x * span) {
    void *p[R];
    unsigned item[R];
    int cls[R];
    unsigned long long pos[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const size_t i = base + (size_t)r * blockDim.x + threadIdx.x;
      p[r] = i < n ? ptrs[i] : nullptr;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      item[r] = 0;
      cls[r] = free_locate<V>(h, p[r], item[r]);
    }
    if (threadIdx.x < OURO_MAX_CLASSES) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    blk_reserve<R>(cls, pos, s_cnt);
    __syncthreads();
    if (threadIdx.x < OURO_MAX_CLASSES && s_cnt[threadIdx.x]) {
      s_pos[threadIdx.x] = atomicAdd(&qh(h, threadIdx.x)->tail.v, (unsigned long long)s_cnt[threadIdx.x]);
      stat_add(h, threadIdx.x, OURO_ST_FREE, s_cnt[threadIdx.x]);
    }
    __syncthreads();
    bool pend[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (cls[r] >= 0) pos[r] += s_pos[cls[r]];
      pend[r] = cls[r] >= 0;
    }
    if (RING) {   /* fast path: one release fence, then every slot's CAS at once */
      unsigned long long old[R];
      fence_acq_rel();
#pragma unroll
      for (int r = 0; r < R; ++r)
        old[r] = pend[r] ? cas_rlx(s_ring[cls[r]] + (pos[r] & s_rmask[cls[r]]), slot(pos[r], 0), slot(pos[r] + 1, item[r]))
                         : 0ull;
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (pend[r] && old[r] == slot(pos[r], 0)) pend[r] = false;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {   /* the rest: the warp path at the taken positions */
      const unsigned vmask = __ballot_sync(0xffffffffu, pend[r]);
      if (pend[r]) page_free<V, true>(h, cls[r], item[r], vmask, pos[r]);
    }
    __syncthreads();
  }
}

/* Block-aggregated batch free for chunk queues (not the deoptimised form):
 * each request sets its page bit and counts it back on its chunk with its
 * warp, as a single free does (one atomicOr per (chunk, word) group, one
 * count atomic per chunk group); the chunks whose count that lifted take
 * their rank in their class's share of the block with one shared-memory
 * atomic, and one thread per class takes the block's tail positions with a
 * single global atomic.  Per warp, those tail atomics piled up on the class
 * of one page per chunk, where every free lifts a chunk.  Statistics once
 * per class per block; runs above one chunk take the warp path. */
template <int V, int R>
__global__ void __launch_bounds__(256) k_batch_free_cblk(ouro_heap_dev h, void *const *ptrs, size_t n) {
  __shared__ unsigned s_cnt[OURO_MAX_CLASSES], s_free[OURO_MAX_CLASSES];
  __shared__ unsigned long long s_pos[OURO_MAX_CLASSES];
  const size_t span = (size_t)blockDim.x * R;
  for (size_t base = (size_t)blockIdx.x * span; base < n; base += (size_t)gridDim.x * span) {
    void *p[R];
    unsigned item[R], x[R];
    int cls[R];
    bool lift[R];
    unsigned long long pos[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const size_t i = base + (size_t)r * blockDim.x + threadIdx.x;
      p[r] = i < n ? ptrs[i] : nullptr;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      item[r] = 0;
      cls[r] = free_locate<V>(h, p[r], item[r]);   /* a run is marked free here */
    }
    if (threadIdx.x < OURO_MAX_CLASSES) s_cnt[threadIdx.x] = s_free[threadIdx.x] = 0;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      int pc = cls[r] < (int)h.n_classes ? cls[r] : -1;
      lift[r] = chunk_release<false>(h, pc, p[r], 0xffffffffu, x[r]);   /* pc: -1 on a double free */
      if (cls[r] < (int)h.n_classes) cls[r] = pc;
      if (pc >= 0) atomicAdd(&s_free[pc], 1u);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) pos[r] = lift[r] ? atomicAdd(&s_cnt[cls[r]], 1u) : 0u;
    __syncthreads();
    if (threadIdx.x < h.n_classes) {
      if (s_cnt[threadIdx.x])
        s_pos[threadIdx.x] = atomicAdd(&qh(h, threadIdx.x)->tail.v, (unsigned long long)s_cnt[threadIdx.x]);
      if (s_free[threadIdx.x]) stat_add(h, threadIdx.x, OURO_ST_FREE, s_free[threadIdx.x]);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) {   /* the lifted chunks into their class queues, at the taken positions */
      const unsigned vmask = __ballot_sync(0xffffffffu, lift[r]);
      if (lift[r]) page_free<V, true>(h, cls[r], x[r], vmask, s_pos[cls[r]] + pos[r]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {   /* runs above one chunk: the warp path */
      const bool run = cls[r] >= (int)h.n_classes;
      const unsigned rm = __ballot_sync(0xffffffffu, run);
      if (run) page_free<V>(h, cls[r], item[r], rm);
    }
    __syncthreads();
  }
}

/* Block-aggregated batch malloc for chunk queues (not the deoptimised
 * form): every request takes its rank in its class's share of the block
 * with one shared-memory atomic; the shares are cut into tasks of at most
 * 32 whole chunks' pages (what one round of chunk_acquire serves from a
 * queue of whole chunks: 32 queue positions, each lane reserving and
 * claiming its chunk's part), and the block's warps take the tasks in turn,
 * classes with the fewest pages per chunk first, into a shared-memory page
 * list from which every request takes the page of its rank.  A class of
 * one page per chunk thus spreads over several warps instead of costing
 * one warp a round per 32 requests while the others wait at the barrier.
 * Requests above one chunk (runs) take the warp path of page_malloc.
 * Statistics once per class per block. */
template <int V, int R>
__global__ void __launch_bounds__(256) k_batch_malloc_cblk(ouro_heap_dev h, const uint32_t *sizes, void **ptrs,
                                                           size_t n) {
  static_assert(256 * R < 2048, "task offsets and counts are 11-bit fields");
  constexpr unsigned MAX_TASKS = (256 * R) / 32 + OURO_MAX_CLASSES;   /* sum over classes of ceil(share / part) */
  __shared__ unsigned s_cnt[OURO_MAX_CLASSES], s_base[OURO_MAX_CLASSES], s_ok[OURO_MAX_CLASSES];
  __shared__ unsigned s_items[256 * R];
  __shared__ unsigned s_task[MAX_TASKS];   /* class | offset << 5 | count << 16 */
  __shared__ unsigned s_ntask;
  const size_t span = (size_t)blockDim.x * R;
  const unsigned warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (size_t base = (size_t)blockIdx.x * span; base < n; base += (size_t)gridDim.x * span) {
    uint32_t sz[R];
    int cls[R];
    unsigned long long pos[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const size_t i = base + (size_t)r * blockDim.x + threadIdx.x;
      sz[r] = i < n ? sizes[i] : 0;
      cls[r] = i < n ? size_class(h, sz[r]) : -1;
      if (i < n && cls[r] < 0) stat_add(h, OURO_ROW_NONE, sz[r] == 0 ? OURO_ST_ZERO : OURO_ST_TOO_LARGE, 1);
    }
    if (threadIdx.x < OURO_MAX_CLASSES) s_cnt[threadIdx.x] = s_ok[threadIdx.x] = 0;
    __syncthreads();
    int pc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) pc[r] = cls[r] < (int)h.n_classes ? cls[r] : -1;   /* runs: warp path below */
    blk_reserve<R>(pc, pos, s_cnt);
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned acc = 0, nt = 0;
      for (unsigned c = 0; c < h.n_classes; ++c) {
        s_base[c] = acc;
        acc += s_cnt[c];
      }
      for (int c = (int)h.n_classes - 1; c >= 0; --c) {
        const unsigned part = 32u << (h.log2_chunk - 4 - c);
        for (unsigned o = 0; o < s_cnt[c]; o += part)
          s_task[nt++] = (unsigned)c | (o << 5) | (min(part, s_cnt[c] - o) << 16);
      }
      s_ntask = nt;
    }
    __syncthreads();
    for (unsigned t = warp; t < s_ntask; t += nwarps) {
      const unsigned tk = s_task[t], c = tk & 31u, cnt = tk >> 16;
      unsigned *out = s_items + s_base[c] + ((tk >> 5) & 2047u);
      const unsigned got = chunk_acquire<V>(h, (int)c, cnt, out);
      for (unsigned i = got + lane; i < cnt; i += 32) out[i] = OURO_NIL;   /* the heap ran out: null answers */
    }
    __syncthreads();
    void *res[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      res[r] = nullptr;
      if (pc[r] >= 0) {
        const unsigned item = s_items[s_base[pc[r]] + pos[r]];
        if (item != OURO_NIL) {
          res[r] = h.base + ((size_t)item << (4 + pc[r]));
          atomicAdd(&s_ok[pc[r]], 1u);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {   /* runs above one chunk: the warp path */
      const bool run = cls[r] >= (int)h.n_classes;
      if (!__any_sync(0xffffffffu, run)) continue;
      void *q = page_malloc<V>(h, run ? cls[r] : -1, 0xffffffffu);
      if (run) res[r] = q;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const size_t i = base + (size_t)r * blockDim.x + threadIdx.x;
      if (i < n) ptrs[i] = res[r];
    }
    __syncthreads();
    if (threadIdx.x < h.n_classes && s_cnt[threadIdx.x]) {
      stat_add(h, threadIdx.x, OURO_ST_MALLOC, s_ok[threadIdx.x]);
      stat_add(h, threadIdx.x, OURO_ST_FAILED, s_cnt[threadIdx.x] - s_ok[threadIdx.x]);
    }
    __syncthreads();
  }
}

template <int OP>
__global__ void k_pattern(void *const *ptrs, const uint32_t *sizes, size_t n, uint32_t seed, int mode,
                          ouro_check *out) {
  payload_acc a;
  unsigned long long nulls = 0;
  const size_t warps = ((size_t)gridDim.x * blockDim.x) >> 5;
  const size_t wid = (((size_t)blockIdx.x * blockDim.x) + threadIdx.x) >> 5;
  for (size_t base = wid * 32; base < n; base += warps * 32) {
    const size_t i = base + (threadIdx.x & 31);
    unsigned char *p = i < n ? static_cast<unsigned char *>(ptrs[i]) : nullptr;
    const uint32_t sz = i < n ? sizes[i] : 0;
    if (i < n && !p) nulls++;
    warp_payload<OP>(p, sz, (uint32_t)i, seed, mode, a);
  }
  if (OP & PAY_CHECK) flush_acc(a, nulls, out);
}

/* one whole round per thread: malloc, write, read back, free.  Warps pull
 * 32 requests at a time from the launch's work counter, so blocks of
 * uneven sizes balance across warps and the round ends within one task of
 * the last byte.  STAGE: the warp's freed pages serve its next mallocs of
 * the same class from shared memory (page queues, heap option `staging`). */
#ifndef OURO_FUSED_MIN_BLOCKS
#define OURO_FUSED_MIN_BLOCKS 4   /* resident blocks of 256 per SM the fused round is compiled for */
#endif
/* chunk queues: their larger malloc path gets 2 blocks of 256 per SM
 * (128 registers a thread) instead of spilling at 64 */
template <int V, bool STAGE>
__global__ void __launch_bounds__(256, ouro_page_queues(V) ? OURO_FUSED_MIN_BLOCKS : 2) k_round_fused(ouro_heap_dev h, const uint32_t *sizes, size_t n,
                                                     uint32_t seed, int mode, ouro_check *out, void **ptrs,
                                                     unsigned long long *work) {
  __shared__ ouro_block_ctx<8> ctx;
  if (STAGE) ouro_block_begin(ctx);
  payload_acc a;
  unsigned long long nulls = 0;
  const unsigned lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(work, 32ull);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= n) break;
    const size_t i = base + lane;
    const uint32_t sz = i < n ? sizes[i] : 0;
    unsigned char *p = nullptr;
    if (STAGE) {
      p = static_cast<unsigned char *>(stage_malloc_v<V>(ctx, h, sz, i < n));
    } else if (i < n) {
      p = static_cast<unsigned char *>(malloc_v<V>(h, sz));
    }
    if (i < n) {
      if (!p) nulls++;
      if (ptrs) ptrs[i] = p;
    }
    __syncwarp();
    warp_payload<PAY_FUSED>(p, sz, (uint32_t)i, seed, mode, a);
    __syncwarp();
    /* staged: the class of each block is known here, so the free skips the
     * chunk-table lookup (one L2 round trip per task off the warp's chain) */
    if (STAGE) ouro::detail::stage_free<V, 8>(ctx, h, p, __activemask(), p ? size_class(h, sz) : -1);
    else if (i < n) free_v<V>(h, p);
    __syncwarp();
  }
  if (STAGE) ouro_block_end_v<V>(ctx, h);
  flush_acc(a, nulls, out);
}

#if OURO_SHARD_ENTRIES
inline cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }
#endif

template <typename K>
int occupancy_grid(K kernel, int block) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0);
  if (per_sm < 1) per_sm = 1;
  return per_sm * ouro::host::sm_count();
}

inline int grid_for(size_t n, int block, int cap) {
  size_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  return (int)(g < (size_t)cap ? g : (size_t)cap);
}

}  // namespace

/* ------------------------------------------------------- per-form launchers */
namespace ouro {
namespace launch {

/* Requests per thread of the block-aggregated kernels: four on plain arrays
 * (their slots are tried together) once a batch fills every SM with four
 * per thread; one otherwise, and always on virtualized queues, so that a
 * small batch still spreads over many blocks. */
constexpr int BLK_WIDE = 4;
inline bool blk_wide(size_t n) { return n >= (size_t)BLK_WIDE * 256 * ouro::host::sm_count(); }
/* The plain-array batch free takes eight requests per thread in blocks of
 * 128 once a batch fills every SM with four such blocks: a 2^20 batch then
 * runs as one wave (1024 blocks, at most 56 registers a thread). */
constexpr int FREE_WIDE = 8, FREE_BLOCK = 128;
inline bool free_wide(size_t n) { return n >= (size_t)FREE_WIDE * FREE_BLOCK * 4 * ouro::host::sm_count(); }

template <int V>
ouro_status batch_malloc(ouro_heap *H, const uint32_t *d_sizes, void **d_ptrs, size_t n, cudaStream_t s) {
  const int block = 256;
  if constexpr (ouro_page_queues(V)) {
    if (!H->d.deopt) {
      if constexpr (ouro_qform(V) == OURO_QF_RING) {
        if (blk_wide(n)) {
          k_batch_malloc_blk<V, BLK_WIDE><<<grid_for((n + BLK_WIDE - 1) / BLK_WIDE, block, 1 << 20), block, 0, s>>>(
              H->d, d_sizes, d_ptrs, n);
          OURO_LAUNCHED();
          return OURO_OK;
        }
      }
      k_batch_malloc_blk<V, 1><<<grid_for(n, block, 1 << 20), block, 0, s>>>(H->d, d_sizes, d_ptrs, n);
      OURO_LAUNCHED();
      return OURO_OK;
    }
  }
  if constexpr (!ouro_page_queues(V)) {
    if (!H->d.deopt) {
      if (blk_wide(n))
        k_batch_malloc_cblk<V, BLK_WIDE><<<grid_for((n + BLK_WIDE - 1) / BLK_WIDE, block, 1 << 20), block, 0, s>>>(
            H->d, d_sizes, d_ptrs, n);
      else
        k_batch_malloc_cblk<V, 1><<<grid_for(n, block, 1 << 20), block, 0, s>>>(H->d, d_sizes, d_ptrs, n);
      OURO_LAUNCHED();
      return OURO_OK;
    }
  }
  k_batch_malloc<V><<<grid_for(n, block, 1 << 20), block, 0, s>>>(H->d, d_sizes, d_ptrs, n);
  OURO_LAUNCHED();
  return OURO_OK;
}

template <int V>
ouro_status batch_free(ouro_heap *H, void *const *d_ptrs, size_t n, cudaStream_t s) {
  const int block = 256;
  if constexpr (ouro_page_queues(V)) {
    if (!H->d.deopt) {
      if constexpr (ouro_qform(V) == OURO_QF_RING) {
        if (free_wide(n)) {
          k_batch_free_blk<V, FREE_WIDE>
              <<<grid_for((n + FREE_WIDE - 1) / FREE_WIDE, FREE_BLOCK, 1 << 20), FREE_BLOCK, 0, s>>>(H->d, d_ptrs, n);
          OURO_LAUNCHED();
          return OURO_OK;
        }
        if (blk_wide(n)) {
          k_batch_free_blk<V, BLK_WIDE><<<grid_for((n + BLK_WIDE - 1) / BLK_WIDE, block, 1 << 20), block, 0, s>>>(
              H->d, d_ptrs, n);
          OURO_LAUNCHED();
          return OURO_OK;
        }
      }
      k_batch_free_blk<V, 1><<<grid_for(n, block, 1 << 20), block, 0, s>>>(H->d, d_ptrs, n);
      OURO_LAUNCHED();
      return OURO_OK;
    }
  }
  if constexpr (!ouro_page_queues(V)) {
    if (!H->d.deopt) {
      if (blk_wide(n))
        k_batch_free_cblk<V, BLK_WIDE><<<grid_for((n + BLK_WIDE - 1) / BLK_WIDE, block, 1 << 20), block, 0, s>>>(
            H->d, d_ptrs, n);
      else
        k_batch_free_cblk<V, 1><<<grid_for(n, block, 1 << 20), block, 0, s>>>(H->d, d_ptrs, n);
      OURO_LAUNCHED();
      return OURO_OK;
    }
  }
  k_batch_free<V><<<grid_for(n, block, 1 << 20), block, 0, s>>>(H->d, d_ptrs, n);
  OURO_LAUNCHED();
  return OURO_OK;
}

template <int V>
ouro_status round_fused(ouro_heap *H, const uint32_t *d_sizes, size_t n, uint32_t seed, int mode, ouro_check *d_out,
                        void **d_ptrs, unsigned long long *work, cudaStream_t s) {
  const int block = 256;
  if (H->d.staging)
    k_round_fused<V, true><<<grid_for(n, block, occupancy_grid(k_round_fused<V, true>, block)), block, 0, s>>>(
        H->d, d_sizes, n, seed, mode, d_out, d_ptrs, work);
  else
    k_round_fused<V, false><<<grid_for(n, block, occupancy_grid(k_round_fused<V, false>, block)), block, 0, s>>>(
        H->d, d_sizes, n, seed, mode, d_out, d_ptrs, work);
  OURO_LAUNCHED();
  return OURO_OK;
}

#define INST_BATCH_MALLOC(PRE, V) \
  PRE template ouro_status batch_malloc<V>(ouro_heap *, const uint32_t *, void **, size_t, cudaStream_t);
#define INST_BATCH_FREE(PRE, V) \
  PRE template ouro_status batch_free<V>(ouro_heap *, void *const *, size_t, cudaStream_t);
#define INST_ROUND_FUSED(PRE, V)                                                                                 \
  PRE template ouro_status round_fused<V>(ouro_heap *, const uint32_t *, size_t, uint32_t, int, ouro_check *, \
                                          void **, unsigned long long *, cudaStream_t);
OURO_SHARD_INSTANTIATE(INST_BATCH_MALLOC)
OURO_SHARD_INSTANTIATE(INST_BATCH_FREE)
OURO_SHARD_INSTANTIATE(INST_ROUND_FUSED)

}  // namespace launch
}  // namespace ouro

#if OURO_SHARD_ENTRIES
/* ------------------------------------------------------------- C entries */
extern "C" ouro_status ouro_batch_malloc(ouro_heap *H, const uint32_t *d_sizes, void **d_ptrs, size_t n,
                                         void *stream) {
  if (!H || (n && (!d_sizes || !d_ptrs))) return OURO_EINVAL;
  if (!n) return OURO_OK;
  OURO_DISPATCH(H->d.variant, return ouro::launch::batch_malloc<V>(H, d_sizes, d_ptrs, n, S(stream)));
}

extern "C" ouro_status ouro_batch_free(ouro_heap *H, void *const *d_ptrs, size_t n, void *stream) {
  if (!H || (n && !d_ptrs)) return OURO_EINVAL;
  if (!n) return OURO_OK;
  OURO_DISPATCH(H->d.variant, return ouro::launch::batch_free<V>(H, d_ptrs, n, S(stream)));
}

extern "C" ouro_status ouro_pattern_write(void *const *d_ptrs, const uint32_t *d_sizes, size_t n, uint32_t seed,
                                          int mode, void *stream) {
  if (n && (!d_ptrs || !d_sizes)) return OURO_EINVAL;
  if (mode != 0 && mode != 1) return OURO_EINVAL;
  if (!n) return OURO_OK;
  const int block = 256;
  const int g = grid_for((n + 31) / 32 * 32, block, occupancy_grid(k_pattern<PAY_WRITE>, block));
  k_pattern<PAY_WRITE><<<g, block, 0, S(stream)>>>(d_ptrs, d_sizes, n, seed, mode, nullptr);
  OURO_LAUNCHED();
  return OURO_OK;
}

extern "C" ouro_status ouro_pattern_check(void *const *d_ptrs, const uint32_t *d_sizes, size_t n, uint32_t seed,
                                          int mode, ouro_check *d_out, void *stream) {
  if (!d_out || (n && (!d_ptrs || !d_sizes))) return OURO_EINVAL;
  if (mode != 0 && mode != 1) return OURO_EINVAL;
  OURO_CUDA(cudaMemsetAsync(d_out, 0, sizeof(ouro_check), S(stream)));
  if (!n) return OURO_OK;
  const int block = 256;
  const int g = grid_for((n + 31) / 32 * 32, block, occupancy_grid(k_pattern<PAY_CHECK>, block));
  k_pattern<PAY_CHECK><<<g, block, 0, S(stream)>>>(d_ptrs, d_sizes, n, seed, mode, d_out);
  OURO_LAUNCHED();
  return OURO_OK;
}

extern "C" ouro_status ouro_round_fused(ouro_heap *H, const uint32_t *d_sizes, size_t n, uint32_t seed, int mode,
                                        ouro_check *d_out, void **d_ptrs, void *stream) {
  if (!H || !d_out || (n && !d_sizes)) return OURO_EINVAL;
  if (mode != 0 && mode != 1) return OURO_EINVAL;
  OURO_CUDA(cudaMemsetAsync(d_out, 0, sizeof(ouro_check), S(stream)));
  if (!n) return OURO_OK;
  /* this launch's work counter: a slot of the heap's ring, zeroed on the
   * launch's stream (launches in flight at once on one heap: up to 64) */
  const unsigned slot = __atomic_fetch_add(&H->work_seq, 1u, __ATOMIC_RELAXED) % OURO_WORK_SLOTS;
  unsigned long long *work = (unsigned long long *)(H->meta + H->off_work + (size_t)slot * 128);
  OURO_CUDA(cudaMemsetAsync(work, 0, 8, S(stream)));
  OURO_DISPATCH(H->d.variant,
                return ouro::launch::round_fused<V>(H, d_sizes, n, seed, mode, d_out, d_ptrs, work, S(stream)));
}
#endif
