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

using namespace ouro::detail;

namespace {

template <int V>
__device__ __forceinline__ void *malloc_v(const ouro_heap_dev &h, unsigned long long n) {
  const unsigned mask = __activemask();
  const int cls = size_class(h, n);
  const unsigned vmask = __ballot_sync(mask, cls >= 0);
  if (cls < 0) {
    stat_add(h, h.n_classes, n == 0 ? OURO_ST_ZERO : OURO_ST_TOO_LARGE, 1);
    return nullptr;
  }
  if constexpr (V == OURO_PAGE_ARRAY || V == OURO_PAGE_VLIST) return page_malloc<V>(h, cls, vmask);
  else return chunk_malloc<V>(h, cls, vmask);
}

template <int V>
__device__ __forceinline__ void free_v(const ouro_heap_dev &h, void *p) {
  const unsigned mask = __activemask();
  unsigned item = 0;
  int cls = -1;
  if (p) {
    cls = locate(h, p, &item);
    if (cls < 0) set_error(h, OURO_ERR_BAD_FREE, OURO_SITE_BAD_FREE);
    else if (h.checked && (V == OURO_PAGE_ARRAY || V == OURO_PAGE_VLIST)) {
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
  if constexpr (V == OURO_CHUNK_ARRAY || V == OURO_CHUNK_VLIST) {
    chunk_free_impl<V>(h, cls, p, mask);
  } else {
    const unsigned vmask = __ballot_sync(mask, cls >= 0);
    if (cls < 0) return;
    page_free<V>(h, cls, item, vmask);
  }
}

/* ------------------------------------------------------------ batch API */
template <int V>
__global__ void k_batch_malloc(ouro_heap_dev h, const uint32_t *sizes, void **ptrs, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    ptrs[i] = malloc_v<V>(h, sizes[i]);
}

template <int V>
__global__ void k_batch_free(ouro_heap_dev h, void *const *ptrs, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    free_v<V>(h, ptrs[i]);
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

struct acc {
  unsigned long long mism = 0, x = 0, s = 0, words = 0;
  __device__ void fold(uint32_t v) {
    x ^= v;
    s += v;
    words++;
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

__device__ __forceinline__ void check4(const uint4 &got, const uint4 &want, acc &a) {
  a.mism += (got.x != want.x) + (got.y != want.y) + (got.z != want.z) + (got.w != want.w);
  a.x ^= (unsigned long long)(got.x ^ got.y ^ got.z ^ got.w);
  a.s += (unsigned long long)got.x + got.y + got.z + got.w;
  a.words += 4;
}

/* words [4*units, nw) and the tail bytes of one block: one lane */
template <bool WRITE>
__device__ void block_rest(unsigned char *bp, uint32_t key, uint32_t nw, uint32_t tail, acc &a) {
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
__device__ void warp_payload(unsigned char *p, uint32_t size, uint32_t tid, uint32_t seed, int mode, acc &a) {
  const unsigned lane = laneid();
  if (mode == 0) {
    if (p) {
      if (OP & PAY_WRITE) *reinterpret_cast<uint32_t *>(p) = tid;
      if (OP == PAY_FUSED) __syncwarp(__activemask());
      if (OP & PAY_CHECK) {
        uint32_t v = __ldcg(reinterpret_cast<const uint32_t *>(p));
        a.mism += v != tid;
        a.fold(v);
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
      if (lane == (OP == PAY_FUSED ? (rest_lane + 31) & 31 : rest_lane)) block_rest<false>(bp, bkey, nw, tail, a);
    }
  }
}

/* block reduction of the check counters into *out */
__device__ void flush_acc(acc &a, unsigned long long nulls, ouro_check *out) {
  __shared__ unsigned long long sm[5];
  if (threadIdx.x < 5) sm[threadIdx.x] = 0;
  __syncthreads();
  for (int o = 16; o; o >>= 1) {
    a.mism += __shfl_xor_sync(0xffffffffu, a.mism, o);
    a.x ^= __shfl_xor_sync(0xffffffffu, a.x, o);
    a.s += __shfl_xor_sync(0xffffffffu, a.s, o);
    a.words += __shfl_xor_sync(0xffffffffu, a.words, o);
    nulls += __shfl_xor_sync(0xffffffffu, nulls, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&sm[0], nulls);
    atomicAdd(&sm[1], a.mism);
    atomicXor(&sm[2], a.x);
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

template <int OP>
__global__ void k_pattern(void *const *ptrs, const uint32_t *sizes, size_t n, uint32_t seed, int mode,
                          ouro_check *out) {
  acc a;
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

/* one whole round per thread: malloc, write, read back, free */
template <int V>
__global__ void __launch_bounds__(256, 4) k_round_fused(ouro_heap_dev h, const uint32_t *sizes, size_t n,
                                                     uint32_t seed, int mode, ouro_check *out, void **ptrs) {
  acc a;
  unsigned long long nulls = 0;
  const size_t warps = ((size_t)gridDim.x * blockDim.x) >> 5;
  const size_t wid = (((size_t)blockIdx.x * blockDim.x) + threadIdx.x) >> 5;
  for (size_t base = wid * 32; base < n; base += warps * 32) {
    const size_t i = base + (threadIdx.x & 31);
    const uint32_t sz = i < n ? sizes[i] : 0;
    unsigned char *p = nullptr;
    if (i < n) {
      p = static_cast<unsigned char *>(malloc_v<V>(h, sz));
      if (!p) nulls++;
      if (ptrs) ptrs[i] = p;
    }
    __syncwarp();
    warp_payload<PAY_FUSED>(p, sz, (uint32_t)i, seed, mode, a);
    __syncwarp();
    if (i < n) free_v<V>(h, p);
    __syncwarp();
  }
  flush_acc(a, nulls, out);
}

inline cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }

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

/* ------------------------------------------------------------- C entries */
#define OURO_DISPATCH(VAR, CALL)                                   \
  switch (VAR) {                                                   \
    case OURO_PAGE_ARRAY: { constexpr int V = OURO_PAGE_ARRAY; CALL; break; }   \
    case OURO_PAGE_VLIST: { constexpr int V = OURO_PAGE_VLIST; CALL; break; }   \
    case OURO_CHUNK_ARRAY: { constexpr int V = OURO_CHUNK_ARRAY; CALL; break; } \
    case OURO_CHUNK_VLIST: { constexpr int V = OURO_CHUNK_VLIST; CALL; break; } \
    default: return OURO_ENOTSUP;                                  \
  }

extern "C" ouro_status ouro_batch_malloc(ouro_heap *H, const uint32_t *d_sizes, void **d_ptrs, size_t n,
                                         void *stream) {
  if (!H || (n && (!d_sizes || !d_ptrs))) return OURO_EINVAL;
  if (!n) return OURO_OK;
  const int block = 256;
  const int g = grid_for(n, block, 1 << 20);
  OURO_DISPATCH(H->d.variant, (k_batch_malloc<V><<<g, block, 0, S(stream)>>>(H->d, d_sizes, d_ptrs, n)));
  OURO_LAUNCHED();
  return OURO_OK;
}

extern "C" ouro_status ouro_batch_free(ouro_heap *H, void *const *d_ptrs, size_t n, void *stream) {
  if (!H || (n && !d_ptrs)) return OURO_EINVAL;
  if (!n) return OURO_OK;
  const int block = 256;
  const int g = grid_for(n, block, 1 << 20);
  OURO_DISPATCH(H->d.variant, (k_batch_free<V><<<g, block, 0, S(stream)>>>(H->d, d_ptrs, n)));
  OURO_LAUNCHED();
  return OURO_OK;
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
  const int block = 256;
  OURO_DISPATCH(H->d.variant, (k_round_fused<V><<<grid_for(n, block, occupancy_grid(k_round_fused<V>, block)),
                                                 block, 0, S(stream)>>>(H->d, d_sizes, n, seed, mode, d_out, d_ptrs)));
  OURO_LAUNCHED();
  return OURO_OK;
}
