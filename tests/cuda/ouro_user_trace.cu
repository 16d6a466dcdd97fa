/* A user's kernels compiled with -DOURO_TRACE: the allocator's slow events
 * (carves, null answers, new queue segments, errors) land in this
 * translation unit's device event ring, read back with ouro_trace_copy. */
#include "ouro_user_common.cuh"

namespace {

/* every lane of every warp calls: lanes t < n ask for `size` bytes */
__global__ void k_trace_fill(ouro_heap_dev h, uint32_t size, uint64_t n, void **ptrs) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool want = t < n;
  void *p = ouro_malloc_warp(h, want ? size : 0, want);
  if (want) ptrs[t] = p;
}

__global__ void k_trace_free(ouro_heap_dev h, void *p) { ouro_free(h, p); }

}  // namespace

/* n requests of `size` bytes, warp-collective; ptrs: device array of n */
extern "C" int ut_trace_fill(const ouro_heap_dev *h, uint32_t size, uint64_t n, void **ptrs, void *stream) {
  k_trace_fill<<<ut::grid_of(n), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(*h, size, n, ptrs);
  return (int)cudaGetLastError();
}

/* one free of p (any pointer, valid or not) by one thread */
extern "C" int ut_trace_free(const ouro_heap_dev *h, void *p, void *stream) {
  k_trace_free<<<1, 1, 0, reinterpret_cast<cudaStream_t>(stream)>>>(*h, p);
  return (int)cudaGetLastError();
}

/* the newest events of this translation unit's ring (see ouro_trace_copy) */
extern "C" int ut_trace_read(ouro_trace_event *out, unsigned cap, unsigned long long *total, int clear) {
  return (int)ouro_trace_copy(out, cap, total, clear);
}
