/*
 * A user's kernels on the public device API (include/ouro_device.cuh), for
 * the GPU tests: the allocator called from inside a kernel on a heap the host
 * preallocated (arXiv 2504.18211, Sec. 1), as an application would call it.
 * The kernels include the public header only: ouro_malloc / ouro_free on an
 * ouro_heap_dev and their warp-collective forms ouro_malloc_warp /
 * ouro_free_warp (ouro_user_plain.cu), and the staged forms after
 * ouro_block_begin(ctx, h) (ouro_user_staged.cu); all pick the heap's queue
 * form at run time.  Built into a test-only
 * library (tests/cuda/build_user.py -> libouro_user.so), not libouro.so.
 *
 * Round of one thread t (t < n), in divergent code:
 *   phase A  lanes with lane % 3 != 2: p = ouro_malloc(size_a[t]); write the
 *            pattern of (seed, t), read it back; odd t free p at once (a
 *            free in the middle of the kernel), even t keep it in keep[t];
 *   phase B  lanes below 20: q = ouro_malloc(size_b[t]); pattern of
 *            (seed + 1, t); free q.
 * A second kernel frees keep[t]; lanes t % 5 == 4 call only for a non-null
 * pointer, the others call with null entries too (a no-op).  The
 * warp-collective kernels run the same round with every lane calling at each
 * step (want = false / p = null for the lanes that sit a phase out).
 * Pattern: floor(size/4) words key + i * 0x9E3779B9 with key =
 * fmix32(seed ^ t * 0x9E3779B9), then size mod 4 bytes of the next word,
 * low bytes first; the read-back is folded into XOR / sum / word counts.
 */
#ifndef OURO_USER_COMMON_CUH
#define OURO_USER_COMMON_CUH

#include <cuda_runtime.h>
#include <stdint.h>

#include "ouro_device.cuh"

/* Each kernel file compiles twice: UT_COLLECTIVE=0 for the lane-private
 * calls, 1 for the warp-collective ones (entry points suffixed _warp). */
#ifndef UT_COLLECTIVE
#define UT_COLLECTIVE 0
#endif
#if UT_COLLECTIVE
#define UT_ENTRY(name) name##_warp
#else
#define UT_ENTRY(name) name
#endif

namespace ut {

constexpr uint32_t kGold = 0x9E3779B9u;

/* MurmurHash3 32-bit finalizer (Appleby, public domain) */
__device__ __forceinline__ uint32_t fmix(uint32_t x) {
  x ^= x >> 16;
  x *= 0x85ebca6bu;
  x ^= x >> 13;
  x *= 0xc2b2ae35u;
  x ^= x >> 16;
  return x;
}

struct acc_t {
  unsigned long long x = 0, s = 0, w = 0, mism = 0, nulls = 0;
};

/* write the pattern of (seed, t) into the n bytes at p, read it back, fold it */
__device__ __forceinline__ void pattern_round(unsigned char *p, uint32_t n, uint32_t seed, uint32_t t, acc_t &a) {
  const uint32_t key = fmix(seed ^ (t * kGold));
  const uint32_t nw = n / 4, tail = n % 4;
  uint32_t *w = reinterpret_cast<uint32_t *>(p);
  for (uint32_t i = 0; i < nw; ++i) w[i] = key + i * kGold;
  const uint32_t last = key + nw * kGold;
  for (uint32_t j = 0; j < tail; ++j) p[4 * nw + j] = (unsigned char)(last >> (8 * j));
  __threadfence_block();
  for (uint32_t i = 0; i < nw; ++i) {
    const uint32_t v = *reinterpret_cast<volatile uint32_t *>(w + i);
    a.mism += v != key + i * kGold;
    a.x ^= v;
    a.s += v;
    a.w++;
  }
  if (tail) {
    uint32_t v = 0;
    for (uint32_t j = 0; j < tail; ++j)
      v |= (uint32_t)(*reinterpret_cast<volatile unsigned char *>(p + 4 * nw + j)) << (8 * j);
    a.mism += v != (last & ((1u << (8 * tail)) - 1));
    a.x ^= v;
    a.s += v;
    a.w++;
  }
}

__device__ __forceinline__ void flush(const acc_t &a, unsigned long long *out) {
  atomicXor(&out[0], a.x);
  atomicAdd(&out[1], a.s);
  atomicAdd(&out[2], a.w);
  atomicAdd(&out[3], a.mism);
  atomicAdd(&out[4], a.nulls);
}

__device__ __forceinline__ bool in_a(unsigned lane) { return lane % 3 != 2; }
__device__ __forceinline__ bool in_b(unsigned lane) { return lane < 20; }

/* pattern round on a block (or count the null), logged per request */
__device__ __forceinline__ void use(void *p, uint32_t n, uint32_t seed, uint64_t t, acc_t &a, unsigned long long *log,
                                    int phase) {
  const unsigned long long m0 = a.mism;
  if (p) pattern_round(static_cast<unsigned char *>(p), n, seed, (uint32_t)t, a);
  else a.nulls++;
  if (log) {
    log[4 * t + phase] = reinterpret_cast<unsigned long long>(p);
    log[4 * t + 2 + phase] = a.mism - m0;
  }
}

inline unsigned grid_of(uint64_t n) { return (unsigned)(n ? (n + 255) / 256 : 1); }

}  // namespace ut

#endif
