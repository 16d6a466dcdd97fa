/*
 * Measurement kernels: the L2 atomic rates that bound the allocator, and a
 * per-request malloc latency histogram.
 *
 * The allocator's queue traffic is atomics: one same-address atomic per
 * warp group on a class head or tail counter, one distinct-address
 * compare-and-swap per lane on a queue slot.  ouro_probe_atomics measures
 * those two rates on the running GPU so the bench can state achieved
 * allocator throughput as a fraction of them.
 */
#include "ouro_internal.cuh"
#include "ouro_payload.cuh"

using namespace ouro::detail;

namespace {

/* pattern 0: lane 0 of every warp, one 64-bit counter (returning atomicAdd),
 *            as a warp group leader on a class head or tail
 * pattern 1: lane 0 of every warp, one of 32 counters on separate lines
 * pattern 2: distinct addresses, consecutive lanes on consecutive words
 *            (like queue slots), 64-bit CAS that always succeeds
 * (an atomic issued by all 32 lanes on one address is merged by the
 * hardware, so patterns 0 and 1 issue one atomic per warp) */
__global__ void k_probe(unsigned long long *buf, unsigned long long words, int pattern, unsigned iters,
                        unsigned long long *sink) {
  const unsigned long long tid = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned long long nthreads = (unsigned long long)gridDim.x * blockDim.x;
  unsigned long long acc = 0;
  if (pattern == 0) {
    if ((threadIdx.x & 31) == 0)
      for (unsigned i = 0; i < iters; ++i) acc += atomicAdd(&buf[0], 1ull);
  } else if (pattern == 1) {
    unsigned long long *p = &buf[((tid >> 5) & 31) * 16];
    if ((threadIdx.x & 31) == 0)
      for (unsigned i = 0; i < iters; ++i) acc += atomicAdd(p, 1ull);
  } else {
    for (unsigned i = 0; i < iters; ++i) {
      unsigned long long w = (tid + (unsigned long long)i * nthreads) % words;
      unsigned long long v = buf[w];
      acc += atomicCAS(&buf[w], v, v + 1);
    }
  }
  if (acc == 0x5A5A5A5A5A5A5A5Aull) *sink = acc;   /* keeps the loop alive */
}

/* clock64 around every malloc: 4 sub-buckets per octave of cycles */
__device__ __forceinline__ unsigned lat_bin(unsigned long long d) {
  if (d < 4) return (unsigned)d;
  const unsigned l = 63 - __clzll(d);
  return (l << 2) | (unsigned)((d >> (l - 2)) & 3);
}

template <int V>
__global__ void k_malloc_timed(ouro_heap_dev h, const uint32_t *sizes, void **ptrs, size_t n,
                               unsigned long long *hist) {
  __shared__ unsigned long long sh[256];
  for (unsigned i = threadIdx.x; i < 256; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const unsigned long long t0 = clock64();
    void *p;
    p = malloc_v<V>(h, sizes[i]);
    const unsigned long long t1 = clock64();
    ptrs[i] = p;
    atomicAdd(&sh[min(lat_bin(t1 - t0), 255u)], 1ull);
  }
  __syncthreads();
  for (unsigned i = threadIdx.x; i < 256; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

/* The fused driver round on CUDA's built-in device allocator: the same
 * warp payload, with malloc / free of the CUDA runtime. */
__global__ void __launch_bounds__(256) k_cuda_malloc_round(const uint32_t *sizes, size_t n, uint32_t seed,
                                                           int mode, ouro_check *out) {
  payload_acc a;
  unsigned long long nulls = 0;
  const size_t warps = ((size_t)gridDim.x * blockDim.x) >> 5;
  const size_t wid = (((size_t)blockIdx.x * blockDim.x) + threadIdx.x) >> 5;
  for (size_t base = wid * 32; base < n; base += warps * 32) {
    const size_t i = base + (threadIdx.x & 31);
    const uint32_t sz = i < n ? sizes[i] : 0;
    unsigned char *p = i < n ? static_cast<unsigned char *>(malloc(sz)) : nullptr;
    if (i < n && !p) nulls++;
    __syncwarp();
    warp_payload<PAY_FUSED>(p, sz, (uint32_t)i, seed, mode, a);
    __syncwarp();
    if (p) free(p);
  }
  flush_acc(a, nulls, out);
}

inline cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

extern "C" ouro_status ouro_probe_atomics(unsigned long long *d_buf, size_t words, int pattern, uint32_t iters,
                                          int blocks, void *stream) {
  if (!d_buf || words < 32 * 16 || pattern < 0 || pattern > 2 || blocks <= 0) return OURO_EINVAL;
  k_probe<<<blocks, 256, 0, S(stream)>>>(d_buf, words, pattern, iters, d_buf + words - 1);
  OURO_LAUNCHED();
  return OURO_OK;
}

extern "C" ouro_status ouro_cuda_malloc_heap(size_t bytes, size_t *got_bytes) {
  if (!bytes) return OURO_EINVAL;
  OURO_CUDA(cudaDeviceSetLimit(cudaLimitMallocHeapSize, bytes));
  size_t got = 0;
  OURO_CUDA(cudaDeviceGetLimit(&got, cudaLimitMallocHeapSize));
  if (got_bytes) *got_bytes = got;
  return OURO_OK;
}

extern "C" ouro_status ouro_cuda_malloc_round(const uint32_t *d_sizes, size_t n, uint32_t seed, int mode,
                                              ouro_check *d_out, void *stream) {
  if (!d_out || (n && !d_sizes)) return OURO_EINVAL;
  if (mode != 0 && mode != 1) return OURO_EINVAL;
  OURO_CUDA(cudaMemsetAsync(d_out, 0, sizeof(ouro_check), S(stream)));
  if (!n) return OURO_OK;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cuda_malloc_round, 256, 0);
  if (per_sm < 1) per_sm = 1;
  size_t g = (n + 255) / 256;
  const size_t cap = (size_t)per_sm * ouro::host::sm_count();
  if (g > cap) g = cap;
  k_cuda_malloc_round<<<(int)g, 256, 0, S(stream)>>>(d_sizes, n, seed, mode, d_out);
  OURO_LAUNCHED();
  return OURO_OK;
}

extern "C" ouro_status ouro_malloc_latency(ouro_heap *H, const uint32_t *d_sizes, void **d_ptrs, size_t n,
                                           unsigned long long *d_hist, void *stream) {
  if (!H || !d_hist || (n && (!d_sizes || !d_ptrs))) return OURO_EINVAL;
  OURO_CUDA(cudaMemsetAsync(d_hist, 0, 256 * 8, S(stream)));
  if (!n) return OURO_OK;
  const int block = 256;
  size_t g = (n + block - 1) / block;
  if (g > (1u << 20)) g = 1u << 20;
  switch (H->d.variant) {
    case OURO_PAGE_ARRAY: k_malloc_timed<OURO_PAGE_ARRAY><<<(int)g, block, 0, S(stream)>>>(H->d, d_sizes, d_ptrs, n, d_hist); break;
    case OURO_PAGE_VLIST: k_malloc_timed<OURO_PAGE_VLIST><<<(int)g, block, 0, S(stream)>>>(H->d, d_sizes, d_ptrs, n, d_hist); break;
    case OURO_CHUNK_ARRAY: k_malloc_timed<OURO_CHUNK_ARRAY><<<(int)g, block, 0, S(stream)>>>(H->d, d_sizes, d_ptrs, n, d_hist); break;
    case OURO_CHUNK_VLIST: k_malloc_timed<OURO_CHUNK_VLIST><<<(int)g, block, 0, S(stream)>>>(H->d, d_sizes, d_ptrs, n, d_hist); break;
    case OURO_PAGE_VARRAY: k_malloc_timed<OURO_PAGE_VARRAY><<<(int)g, block, 0, S(stream)>>>(H->d, d_sizes, d_ptrs, n, d_hist); break;
    case OURO_CHUNK_VARRAY: k_malloc_timed<OURO_CHUNK_VARRAY><<<(int)g, block, 0, S(stream)>>>(H->d, d_sizes, d_ptrs, n, d_hist); break;
    default: return OURO_ENOTSUP;
  }
  OURO_LAUNCHED();
  return OURO_OK;
}
