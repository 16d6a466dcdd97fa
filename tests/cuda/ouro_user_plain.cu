/* User kernels on ouro_malloc / ouro_free (any lane, divergent code) and on
 * ouro_malloc_warp / ouro_free_warp (warp-collective) with an ouro_heap_dev
 * (see ouro_user_common.cuh). */
#include "ouro_user_common.cuh"

namespace {

#if !UT_COLLECTIVE
__global__ void k_user_round(ouro_heap_dev h, const uint32_t *size_a, const uint32_t *size_b, uint64_t n,
                             uint32_t seed, void **keep, unsigned long long *out, unsigned long long *log) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned lane = threadIdx.x & 31;
  ut::acc_t a;
  if (t < n) {
    void *p = nullptr;
    if (ut::in_a(lane)) {
      p = ouro_malloc(h, size_a[t]);
      ut::use(p, size_a[t], seed, t, a, log, 0);
      if (t & 1) {
        ouro_free(h, p);
        p = nullptr;
      }
    }
    keep[t] = p;
    if (ut::in_b(lane)) {
      void *q = ouro_malloc(h, size_b[t]);
      ut::use(q, size_b[t], seed + 1, t, a, log, 1);
      ouro_free(h, q);
    }
  }
  ut::flush(a, out);
}

#else
/* the same round, warp-collective: every lane calls, want / null say who asks */
__global__ void k_user_round_warp(ouro_heap_dev h, const uint32_t *size_a, const uint32_t *size_b, uint64_t n,
                                  uint32_t seed, void **keep, unsigned long long *out, unsigned long long *log) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned lane = threadIdx.x & 31;
  const bool live = t < n;
  ut::acc_t a;
  const bool wa = live && ut::in_a(lane), wb = live && ut::in_b(lane);
  void *p = ouro_malloc_warp(h, wa ? size_a[t] : 0, wa);
  if (wa) ut::use(p, size_a[t], seed, t, a, log, 0);
  ouro_free_warp(h, (wa && (t & 1)) ? p : nullptr);
  if (wa && (t & 1)) p = nullptr;
  if (live) keep[t] = p;
  void *q = ouro_malloc_warp(h, wb ? size_b[t] : 0, wb);
  if (wb) ut::use(q, size_b[t], seed + 1, t, a, log, 1);
  ouro_free_warp(h, q);
  ut::flush(a, out);
}

#endif

#if !UT_COLLECTIVE
__global__ void k_user_free(ouro_heap_dev h, void **keep, uint64_t n) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n && (t % 5 != 4 || keep[t])) ouro_free(h, keep[t]);
}

#else
__global__ void k_user_free_warp(ouro_heap_dev h, void **keep, uint64_t n) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  ouro_free_warp(h, t < n ? keep[t] : nullptr);
}

#endif

}  // namespace

/* out[5] (device, zeroed here): XOR, sum, words, mismatches, null returns of
 * the round.  keep: device array of n pointers.  log (device, nullable): 4
 * words per request (block of phase A and of phase B, mismatching words of
 * each).  h: host copy of the heap's ouro_heap_dev.  collective: the
 * warp-collective calls.  Returns the cudaError_t of the launch. */
extern "C" int UT_ENTRY(ut_round_plain)(const ouro_heap_dev *h, const uint32_t *size_a, const uint32_t *size_b,
                              uint64_t n, uint32_t seed, void **keep, unsigned long long *out,
                              unsigned long long *log, void *stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(out, 0, 5 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return (int)e;
#if UT_COLLECTIVE
  k_user_round_warp<<<ut::grid_of(n), 256, 0, s>>>(*h, size_a, size_b, n, seed, keep, out, log);
#else
  k_user_round<<<ut::grid_of(n), 256, 0, s>>>(*h, size_a, size_b, n, seed, keep, out, log);
#endif
  return (int)cudaGetLastError();
}

extern "C" int UT_ENTRY(ut_free_plain)(const ouro_heap_dev *h, void **keep, uint64_t n, void *stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
#if UT_COLLECTIVE
  k_user_free_warp<<<ut::grid_of(n), 256, 0, s>>>(*h, keep, n);
#else
  k_user_free<<<ut::grid_of(n), 256, 0, s>>>(*h, keep, n);
#endif
  return (int)cudaGetLastError();
}
