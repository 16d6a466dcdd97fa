/* Device helpers shared by the library's kernels: variant-resolved
 * malloc / free, and the warp-cooperative driver-round payload (Sec. 3 of
 * arXiv 2504.18211: write data into each block, read it back, check it). */
#ifndef OURO_PAYLOAD_CUH
#define OURO_PAYLOAD_CUH

#include "ouro_internal.cuh"

namespace ouro {
namespace detail {


/* Variant-resolved malloc.  want = false: the lane asks for nothing but
 * stays in the call to help its warp carve (see page_malloc).  FILL: slot
 * writes in flight per lane when the warp fills a carve (page queues). */
template <int V, int FILL = 1>
__device__ __forceinline__ void *malloc_v(const ouro_heap_dev &h, unsigned long long n, bool want = true) {
  const unsigned mask = __activemask();
  const int cls = want ? size_class(h, n) : -1;
  if (want && cls < 0) stat_add(h, OURO_ROW_NONE, n == 0 ? OURO_ST_ZERO : OURO_ST_TOO_LARGE, 1);
  if (!__any_sync(mask, cls >= 0)) return nullptr;
  if constexpr (ouro_page_queues(V)) return page_malloc<V, FILL>(h, cls, mask);   /* pages and runs */
  else return chunk_or_run_malloc<V>(h, cls, mask);
}

/* Class and item of a block being freed; -1 for null or an invalid free
 * (recorded).  A run is marked free here; page queues in checked mode clear
 * the page's bit and catch a double free. */
template <int V>
__device__ __forceinline__ int free_locate(const ouro_heap_dev &h, void *p, unsigned &item) {
  int cls = -1;
  if (p) {
    cls = locate(h, p, &item);
    if (cls < 0) set_error(h, OURO_ERR_BAD_FREE, OURO_SITE_BAD_FREE);
    else if (cls >= (int)h.n_classes) {   /* a run */
      if (!run_mark_free(h, cls, item)) cls = -1;
    } else if (h.checked && ouro_page_queues(V)) {
      const unsigned sh = h.log2_chunk - 4 - cls;
      const unsigned pg = item & ((1u << sh) - 1), x = item >> sh, bit = 1u << (pg & 31);
      __threadfence();
      unsigned old = atomicOr(&h.bits[(size_t)x * h.words_per_chunk + (pg >> 5)], bit);
      if (old & bit) {
        set_error(h, OURO_ERR_DOUBLE_FREE, OURO_SITE_PAGE_DOUBLE);
        cls = -1;
      }
    }
  }
  return cls;
}

/* FENCE = false: only for kernels that free blocks written before they began
 * and allocate nothing (the batch free kernel) */
template <int V, bool FENCE = true>
__device__ __forceinline__ void free_v(const ouro_heap_dev &h, void *p) {
  const unsigned mask = __activemask();
  unsigned item = 0;
  const int cls = free_locate<V>(h, p, item);
  if constexpr (!ouro_page_queues(V)) {
    chunk_or_run_free<V, FENCE>(h, cls, item, p, mask);
  } else {
    const unsigned vmask = __ballot_sync(mask, cls >= 0);
    if (cls < 0) return;
    page_free<V>(h, cls, item, vmask);
  }
}

/* Staged malloc / free: the warp's shared-memory stacks first (every queue
 * form), then the heap. */
template <int V, int WARPS>
__device__ __forceinline__ void *stage_malloc_v(ouro_block_ctx<WARPS> &ctx, const ouro_heap_dev &h,
                                                unsigned long long n, bool want) {
  return ouro::detail::stage_malloc<V, WARPS>(ctx, h, n, want);
}

template <int V, int WARPS>
__device__ __forceinline__ void stage_free_v(ouro_block_ctx<WARPS> &ctx, const ouro_heap_dev &h, void *p) {
  ouro::detail::stage_free<V, WARPS>(ctx, h, p);
}

/* ------------------------------------------------------------- payload */
/* MurmurHash3 32-bit finalizer (Appleby, public domain) */
__device__ __forceinline__ uint32_t fmix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x85ebca6bu;
  x ^= x >> 13;
  x *= 0xc2b2ae35u;
  x ^= x >> 16;
  return x;
}
#define OURO_GOLD 0x9E3779B9u

/* per-lane check counters: mismatches and the XOR fold in 32 bits (the
 * words are 32-bit), the sum and the word count in 64 */
struct payload_acc {
  unsigned mism = 0, x = 0;
  unsigned long long s = 0, words = 0;
  __device__ void fold(uint32_t v) {
    x ^= v;
    s += v;
  }
};

/* Warp-cooperative payload over the 32 blocks of a warp, one block at a
 * time: all 32 lanes stride over the block's 16-byte units, several units in
 * flight per lane.  Every lane of the warp must call (a lane without a block
 * passes p = null).
 *   WRITE:  store the pattern.
 *   CHECK:  read back, compare, fold the checksums into a.
 *   FUSED:  write the block, then (after __syncwarp) read it back through L2
 *           with every lane checking the units its neighbour wrote.
 * mode 0: word 0 = tid.  mode 1: floor(size/4) words key + w*GOLD, then the
 * low size%4 bytes of word floor(size/4). */
enum { PAY_WRITE = 1, PAY_CHECK = 2, PAY_FUSED = 3 };

__device__ __forceinline__ uint4 pat4(uint32_t key, uint32_t w0) {
  return make_uint4(key + w0 * OURO_GOLD, key + (w0 + 1) * OURO_GOLD, key + (w0 + 2) * OURO_GOLD,
                    key + (w0 + 3) * OURO_GOLD);
}

__device__ __forceinline__ void check4(const uint4 &got, const uint4 &want, payload_acc &a) {
  a.mism += (got.x != want.x) + (got.y != want.y) + (got.z != want.z) + (got.w != want.w);
  a.x ^= got.x ^ got.y ^ got.z ^ got.w;
  a.s += (unsigned long long)got.x + got.y + got.z + got.w;
}

/* words [4*units, nw) and the tail bytes of one block: one lane */
template <bool WRITE>
__device__ void block_rest(unsigned char *bp, uint32_t key, uint32_t nw, uint32_t tail, payload_acc &a) {
  uint32_t *wp = reinterpret_cast<uint32_t *>(bp);
  for (uint32_t w = nw & ~3u; w < nw; ++w) {
    const uint32_t want = key + w * OURO_GOLD;
    if (WRITE) wp[w] = want;
    else {
      uint32_t got = __ldcg(wp + w);
      a.mism += got != want;
      a.fold(got);
    }
  }
  if (tail) {
    const uint32_t v = key + nw * OURO_GOLD;
    unsigned char *tb = bp + 4ull * nw;
    if (WRITE) {
      for (uint32_t b = 0; b < tail; ++b) tb[b] = (unsigned char)(v >> (8 * b));
    } else {
      uint32_t got = 0;
      for (uint32_t b = 0; b < tail; ++b) {
        unsigned char gb = __ldcg(tb + b);
        a.mism += gb != (unsigned char)(v >> (8 * b));
        got |= (uint32_t)gb << (8 * b);
      }
      a.fold(got);
    }
  }
}

template <int OP>
__device__ void warp_payload(unsigned char *p, uint32_t size, uint32_t tid, uint32_t seed, int mode, payload_acc &a) {
  const unsigned lane = laneid();
  if (mode == 0) {
    if (p) {
      if (OP & PAY_WRITE) *reinterpret_cast<uint32_t *>(p) = tid;
      if (OP == PAY_FUSED) __syncwarp(__activemask());
      if (OP & PAY_CHECK) {
        uint32_t v = __ldcg(reinterpret_cast<const uint32_t *>(p));
        a.mism += v != tid;
        a.fold(v);
        a.words++;
      }
    }
    return;
  }
  const uint32_t key = fmix32(seed ^ (tid * OURO_GOLD));
  const unsigned rd = OP == PAY_FUSED ? (lane + 1) & 31 : lane;   /* unit lane that this lane checks */
  for (int j = 0; j < 32; ++j) {
    const unsigned long long bpi = __shfl_sync(0xffffffffu, (unsigned long long)p, j);
    const uint32_t bsize = __shfl_sync(0xffffffffu, size, j);
    const uint32_t bkey = __shfl_sync(0xffffffffu, key, j);
    if (!bpi) continue;
    unsigned char *bp = reinterpret_cast<unsigned char *>(bpi);
    uint4 *u4 = reinterpret_cast<uint4 *>(bp);
    const uint32_t nw = bsize >> 2, tail = bsize & 3, units = nw >> 2;
    const unsigned rest_lane = units & 31;
    if (OP & PAY_WRITE) {
#pragma unroll 4
      for (uint32_t u = lane; u < units; u += 32) u4[u] = pat4(bkey, 4 * u);
      if (lane == rest_lane) block_rest<true>(bp, bkey, nw, tail, a);
    }
    if (OP == PAY_FUSED) __syncwarp();
    if (OP & PAY_CHECK) {
      uint32_t u = rd;
      for (; u + 96 < units; u += 128) {          /* four independent 16-byte loads in flight */
        const uint4 g0 = __ldcg(u4 + u), g1 = __ldcg(u4 + u + 32), g2 = __ldcg(u4 + u + 64),
                    g3 = __ldcg(u4 + u + 96);
        check4(g0, pat4(bkey, 4 * u), a);
        check4(g1, pat4(bkey, 4 * (u + 32)), a);
        check4(g2, pat4(bkey, 4 * (u + 64)), a);
        check4(g3, pat4(bkey, 4 * (u + 96)), a);
      }
      for (; u < units; u += 32) check4(__ldcg(u4 + u), pat4(bkey, 4 * u), a);
      if (lane == (OP == PAY_FUSED ? (rest_lane + 31) & 31 : rest_lane)) {
        block_rest<false>(bp, bkey, nw, tail, a);
        a.words += nw + (tail != 0);
      }
    }
  }
}

/* block reduction of the check counters into *out */
__device__ inline void flush_acc(payload_acc &a, unsigned long long nulls, ouro_check *out) {
  __shared__ unsigned long long sm[5];
  if (threadIdx.x < 5) sm[threadIdx.x] = 0;
  __syncthreads();
  unsigned long long mism = a.mism;   /* per lane 32 bits; summed over the warp in 64 */
  for (int o = 16; o; o >>= 1) {
    mism += __shfl_xor_sync(0xffffffffu, mism, o);
    a.x ^= __shfl_xor_sync(0xffffffffu, a.x, o);
    a.s += __shfl_xor_sync(0xffffffffu, a.s, o);
    a.words += __shfl_xor_sync(0xffffffffu, a.words, o);
    nulls += __shfl_xor_sync(0xffffffffu, nulls, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&sm[0], nulls);
    atomicAdd(&sm[1], mism);
    atomicXor(&sm[2], (unsigned long long)a.x);
    atomicAdd(&sm[3], a.s);
    atomicAdd(&sm[4], a.words);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (sm[0]) atomicAdd(&out->nulls, sm[0]);
    if (sm[1]) atomicAdd(&out->mismatches, sm[1]);
    atomicXor(&out->xor64, sm[2]);
    atomicAdd(&out->sum64, sm[3]);
    atomicAdd(&out->words, sm[4]);
  }
}


/* warp reduction of the check counters; lane 0 adds them to *out */
__device__ inline void warp_flush(payload_acc &a, unsigned long long nulls, ouro_check *out) {
  unsigned long long mism = a.mism;   /* per lane 32 bits; summed over the warp in 64 */
  for (int o = 16; o; o >>= 1) {
    mism += __shfl_xor_sync(0xffffffffu, mism, o);
    a.x ^= __shfl_xor_sync(0xffffffffu, a.x, o);
    a.s += __shfl_xor_sync(0xffffffffu, a.s, o);
    a.words += __shfl_xor_sync(0xffffffffu, a.words, o);
    nulls += __shfl_xor_sync(0xffffffffu, nulls, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (nulls) atomicAdd(&out->nulls, nulls);
    if (mism) atomicAdd(&out->mismatches, mism);
    atomicXor(&out->xor64, (unsigned long long)a.x);
    atomicAdd(&out->sum64, a.s);
    atomicAdd(&out->words, a.words);
  }
}

}  // namespace detail
}  // namespace ouro

#define OURO_DISPATCH(VAR, CALL)                                                 \
  switch (VAR) {                                                                 \
    case OURO_PAGE_ARRAY: { constexpr int V = OURO_PAGE_ARRAY; CALL; break; }   \
    case OURO_PAGE_VLIST: { constexpr int V = OURO_PAGE_VLIST; CALL; break; }   \
    case OURO_CHUNK_ARRAY: { constexpr int V = OURO_CHUNK_ARRAY; CALL; break; } \
    case OURO_CHUNK_VLIST: { constexpr int V = OURO_CHUNK_VLIST; CALL; break; } \
    case OURO_PAGE_VARRAY: { constexpr int V = OURO_PAGE_VARRAY; CALL; break; } \
    case OURO_CHUNK_VARRAY: { constexpr int V = OURO_CHUNK_VARRAY; CALL; break; } \
    default: return OURO_ENOTSUP;                                                \
  }

#endif
