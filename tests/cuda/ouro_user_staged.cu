/* User kernels on the staged public form: ouro_block_begin(ctx, h),
 * ouro_malloc(ctx, n) / ouro_free(ctx, p) (any lane, divergent code) or
 * ouro_malloc_warp(ctx, n, want) / ouro_free_warp(ctx, p) (warp-collective),
 * ouro_block_end(ctx) (see ouro_user_common.cuh).  Blocks of 256 threads,
 * one ouro_block_ctx<8>. */
#include "ouro_user_common.cuh"

namespace {

#if !UT_COLLECTIVE
__global__ void __launch_bounds__(256) k_user_round_staged(ouro_heap_dev h, const uint32_t *size_a,
                                                           const uint32_t *size_b, uint64_t n, uint32_t seed,
                                                           void **keep, unsigned long long *out,
                                                           unsigned long long *log) {
  __shared__ ouro_block_ctx<8> ctx;
  ouro_block_begin(ctx, h);
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned lane = threadIdx.x & 31;
  ut::acc_t a;
  if (t < n) {
    void *p = nullptr;
    if (ut::in_a(lane)) {
      p = ouro_malloc(ctx, size_a[t]);
      ut::use(p, size_a[t], seed, t, a, log, 0);
      if (t & 1) {
        ouro_free(ctx, p);
        p = nullptr;
      }
    }
    keep[t] = p;
    if (ut::in_b(lane)) {
      void *q = ouro_malloc(ctx, size_b[t]);
      ut::use(q, size_b[t], seed + 1, t, a, log, 1);
      ouro_free(ctx, q);
    }
  }
  ouro_block_end(ctx);
  ut::flush(a, out);
}

#else
__global__ void __launch_bounds__(256) k_user_round_staged_warp(ouro_heap_dev h, const uint32_t *size_a,
                                                                const uint32_t *size_b, uint64_t n, uint32_t seed,
                                                                void **keep, unsigned long long *out,
                                                                unsigned long long *log) {
  __shared__ ouro_block_ctx<8> ctx;
  ouro_block_begin(ctx, h);
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned lane = threadIdx.x & 31;
  const bool live = t < n;
  ut::acc_t a;
  const bool wa = live && ut::in_a(lane), wb = live && ut::in_b(lane);
  void *p = ouro_malloc_warp(ctx, wa ? size_a[t] : 0, wa);
  if (wa) ut::use(p, size_a[t], seed, t, a, log, 0);
  ouro_free_warp(ctx, (wa && (t & 1)) ? p : nullptr);
  if (wa && (t & 1)) p = nullptr;
  if (live) keep[t] = p;
  void *q = ouro_malloc_warp(ctx, wb ? size_b[t] : 0, wb);
  if (wb) ut::use(q, size_b[t], seed + 1, t, a, log, 1);
  ouro_free_warp(ctx, q);
  ouro_block_end(ctx);
  ut::flush(a, out);
}

#endif

#if !UT_COLLECTIVE
__global__ void __launch_bounds__(256) k_user_free_staged(ouro_heap_dev h, void **keep, uint64_t n) {
  __shared__ ouro_block_ctx<8> ctx;
  ouro_block_begin(ctx, h);
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n && (t % 5 != 4 || keep[t])) ouro_free(ctx, keep[t]);
  ouro_block_end(ctx);
}

#else
__global__ void __launch_bounds__(256) k_user_free_staged_warp(ouro_heap_dev h, void **keep, uint64_t n) {
  __shared__ ouro_block_ctx<8> ctx;
  ouro_block_begin(ctx, h);
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  ouro_free_warp(ctx, t < n ? keep[t] : nullptr);
  ouro_block_end(ctx);
}

#endif

}  // namespace

/* as ut_round_plain, through the staged form */
extern "C" int UT_ENTRY(ut_round_staged)(const ouro_heap_dev *h, const uint32_t *size_a, const uint32_t *size_b,
                               uint64_t n, uint32_t seed, void **keep, unsigned long long *out,
                               unsigned long long *log, void *stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(out, 0, 5 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return (int)e;
#if UT_COLLECTIVE
  k_user_round_staged_warp<<<ut::grid_of(n), 256, 0, s>>>(*h, size_a, size_b, n, seed, keep, out, log);
#else
  k_user_round_staged<<<ut::grid_of(n), 256, 0, s>>>(*h, size_a, size_b, n, seed, keep, out, log);
#endif
  return (int)cudaGetLastError();
}

extern "C" int UT_ENTRY(ut_free_staged)(const ouro_heap_dev *h, void **keep, uint64_t n, void *stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
#if UT_COLLECTIVE
  k_user_free_staged_warp<<<ut::grid_of(n), 256, 0, s>>>(*h, keep, n);
#else
  k_user_free_staged<<<ut::grid_of(n), 256, 0, s>>>(*h, keep, n);
#endif
  return (int)cudaGetLastError();
}
