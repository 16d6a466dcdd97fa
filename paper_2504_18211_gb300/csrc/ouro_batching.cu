/*
 * Batching: many request batches of uneven size, each request allocating,
 * writing its pattern, reading it back and freeing (the driver round of
 * Sec. 3 of arXiv 2504.18211, applied to a stream of batches).
 *
 * Forms:
 *   - per launch:  one fused-round launch per batch (ouro_round_fused), or
 *                  four launches per batch (malloc / write / check / free);
 *   - CUDA graph:  the per-batch launches captured once and replayed;
 *   - persistent:  ONE kernel for all batches; warps pull 256-request tasks
 *                  from a device work counter, so uneven batches overlap
 *                  and the allocator state never leaves L2 between them.
 * Request i of batch b uses pattern seed (seed + b) and thread id i (its
 * index inside the batch), in every form, so the per-batch checks agree.
 */
#include <algorithm>
#include <vector>

#include "ouro_internal.cuh"
#include "ouro_payload.cuh"
#include "ouro_shard.cuh"

using namespace ouro::detail;

namespace {

constexpr unsigned TASK_REQ = 256;   /* requests per persistent task: 8 warp iterations */

template <int V, bool STAGE>
__global__ void __launch_bounds__(256, ouro_page_queues(V) ? 4 : 2)   /* chunk queues: no spills at 2 per SM */
k_batches_persistent(ouro_heap_dev h, const uint32_t *sizes, const unsigned long long *offs,
                     const unsigned long long *task_offs, unsigned n_batches, uint32_t seed, int mode,
                     ouro_check *out, unsigned long long *work, unsigned long long n_tasks) {
  __shared__ ouro_block_ctx<8> ctx;
  if (STAGE) ouro_block_begin(ctx);
  const unsigned lane = laneid();
  for (;;) {
    unsigned long long task = 0;
    if (lane == 0) task = atomicAdd(work, 1ull);
    task = __shfl_sync(0xffffffffu, task, 0);
    if (task >= n_tasks) break;
    unsigned lo = 0, hi = n_batches;       /* task_offs[lo] <= task < task_offs[hi] */
    while (hi - lo > 1) {
      const unsigned mid = (lo + hi) >> 1;
      if (task_offs[mid] <= task) lo = mid;
      else hi = mid;
    }
    const unsigned b = lo;
    const unsigned long long base = offs[b], count = offs[b + 1] - offs[b];
    const unsigned long long local0 = (task - task_offs[b]) * TASK_REQ;
    payload_acc a;
    unsigned long long nulls = 0;
    for (unsigned r = 0; r < TASK_REQ / 32; ++r) {
      const unsigned long long i = local0 + r * 32 + lane;
      const bool active = i < count;
      if (!__any_sync(0xffffffffu, active)) break;
      const uint32_t sz = active ? sizes[base + i] : 0;
      unsigned char *p = nullptr;
      if (STAGE) p = static_cast<unsigned char *>(stage_malloc_v<V>(ctx, h, sz, active));
      else if (active) p = static_cast<unsigned char *>(malloc_v<V>(h, sz));
      if (active && !p) nulls++;
      __syncwarp();
      warp_payload<PAY_FUSED>(p, sz, (uint32_t)i, seed + b, mode, a);
      __syncwarp();
      if (STAGE) stage_free_v<V>(ctx, h, p);
      else if (active) free_v<V>(h, p);
      __syncwarp();
    }
    warp_flush(a, nulls, &out[b]);
  }
  if (STAGE) ouro_block_end_v<V>(ctx, h);
}

#if OURO_SHARD_ENTRIES
inline cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }
#endif

}  // namespace

/* ------------------------------------------------------- per-form launchers */
namespace ouro {
namespace launch {

template <int V, bool STAGE>
int persistent_blocks_per_sm(int blocks_per_sm) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batches_persistent<V, STAGE>, 256, 0);
  if (blocks_per_sm > 0 && blocks_per_sm < per_sm) per_sm = blocks_per_sm;
  return per_sm;
}

template <int V>
ouro_status batches_persistent(ouro_heap *H, const uint32_t *d_sizes, const unsigned long long *d_offs,
                               const unsigned long long *d_task_offs, uint32_t n_batches, uint64_t n_tasks,
                               uint32_t seed, int mode, ouro_check *d_out, unsigned long long *d_work,
                               int blocks_per_sm, cudaStream_t s) {
  if (H->d.staging) {
    const int per_sm = std::max(1, persistent_blocks_per_sm<V, true>(blocks_per_sm));
    k_batches_persistent<V, true><<<per_sm * ouro::host::sm_count(), 256, 0, s>>>(
        H->d, d_sizes, d_offs, d_task_offs, n_batches, seed, mode, d_out, d_work, n_tasks);
  } else {
    const int per_sm = std::max(1, persistent_blocks_per_sm<V, false>(blocks_per_sm));
    k_batches_persistent<V, false><<<per_sm * ouro::host::sm_count(), 256, 0, s>>>(
        H->d, d_sizes, d_offs, d_task_offs, n_batches, seed, mode, d_out, d_work, n_tasks);
  }
  OURO_LAUNCHED();
  return OURO_OK;
}

/* blocks of 256 per SM the unstaged persistent kernel keeps resident */
template <int V>
int batches_max_blocks_per_sm() { return persistent_blocks_per_sm<V, false>(0); }

#define INST_BATCHES_PERSISTENT(PRE, V)                                                                         \
  PRE template ouro_status batches_persistent<V>(ouro_heap *, const uint32_t *, const unsigned long long *,   \
                                                 const unsigned long long *, uint32_t, uint64_t, uint32_t, int, \
                                                 ouro_check *, unsigned long long *, int, cudaStream_t);
#define INST_BATCHES_MAX_BLOCKS(PRE, V) PRE template int batches_max_blocks_per_sm<V>();
OURO_SHARD_INSTANTIATE(INST_BATCHES_PERSISTENT)
OURO_SHARD_INSTANTIATE(INST_BATCHES_MAX_BLOCKS)

}  // namespace launch
}  // namespace ouro

#if OURO_SHARD_ENTRIES
struct ouro_batch_graph {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  size_t nodes;
  size_t kernels;   /* kernel nodes: the library's launches per replay */
};

extern "C" ouro_status ouro_batches_persistent(ouro_heap *H, const uint32_t *d_sizes, const unsigned long long *d_offs,
                                               const unsigned long long *d_task_offs, uint32_t n_batches,
                                               uint64_t n_tasks, uint32_t seed, int mode, ouro_check *d_out,
                                               unsigned long long *d_work, int blocks_per_sm, void *stream) {
  if (!H || !d_sizes || !d_offs || !d_task_offs || !d_out || !d_work || n_batches == 0) return OURO_EINVAL;
  if (mode != 0 && mode != 1) return OURO_EINVAL;
  OURO_CUDA(cudaMemsetAsync(d_out, 0, sizeof(ouro_check) * n_batches, S(stream)));
  OURO_CUDA(cudaMemsetAsync(d_work, 0, 8, S(stream)));
  if (!n_tasks) return OURO_OK;
  OURO_DISPATCH(H->d.variant,
                return ouro::launch::batches_persistent<V>(H, d_sizes, d_offs, d_task_offs, n_batches, n_tasks, seed,
                                                           mode, d_out, d_work, blocks_per_sm, S(stream)));
}

extern "C" int ouro_batches_max_blocks_per_sm(const ouro_heap *H) {
  if (!H) return 0;
  switch (H->d.variant) {
#define CASE_MAX_BLOCKS(PRE, V) \
  case V: return ouro::launch::batches_max_blocks_per_sm<V>();
    OURO_SHARD_EACH(CASE_MAX_BLOCKS, )
#undef CASE_MAX_BLOCKS
    default: return 0;
  }
}

/* Capture the per-batch launches of one pass over all batches.
 * form 0: one fused-round launch per batch; form 1: malloc / write / check
 * / free per batch (d_ptrs: device scratch of max batch size pointers).
 * h_offs: HOST array of n_batches+1 request offsets into d_sizes. */
extern "C" ouro_status ouro_batch_graph_create(ouro_heap *H, const uint32_t *d_sizes, const unsigned long long *h_offs,
                                               uint32_t n_batches, uint32_t seed, int mode, ouro_check *d_out,
                                               void **d_ptrs, int form, ouro_batch_graph **out) {
  if (!H || !d_sizes || !h_offs || !d_out || !out || n_batches == 0 || (form == 1 && !d_ptrs) || form < 0 || form > 1)
    return OURO_EINVAL;
  *out = nullptr;
  cudaStream_t cs;
  OURO_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  ouro_status st = OURO_OK;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return ouro::host::cuda_fail(e);
  }
  for (uint32_t b = 0; b < n_batches && st == OURO_OK; ++b) {
    const size_t n = (size_t)(h_offs[b + 1] - h_offs[b]);
    const uint32_t *sz = d_sizes + h_offs[b];
    if (form == 0) {
      st = ouro_round_fused(H, sz, n, seed + b, mode, d_out + b, nullptr, cs);
    } else {
      st = ouro_batch_malloc(H, sz, d_ptrs, n, cs);
      if (st == OURO_OK) st = ouro_pattern_write(d_ptrs, sz, n, seed + b, mode, cs);
      if (st == OURO_OK) st = ouro_pattern_check(d_ptrs, sz, n, seed + b, mode, d_out + b, cs);
      if (st == OURO_OK) st = ouro_batch_free(H, d_ptrs, n, cs);
    }
  }
  e = cudaStreamEndCapture(cs, &g);
  if (st == OURO_OK && e != cudaSuccess) st = ouro::host::cuda_fail(e);
  ouro_batch_graph *G = nullptr;
  if (st == OURO_OK) {
    G = new ouro_batch_graph{g, nullptr, 0, 0};
    e = cudaGraphInstantiate(&G->exec, g, 0);
    if (e != cudaSuccess) st = ouro::host::cuda_fail(e);
    cudaGraphGetNodes(g, nullptr, &G->nodes);
    std::vector<cudaGraphNode_t> nodes(G->nodes);
    if (G->nodes) cudaGraphGetNodes(g, nodes.data(), &G->nodes);
    for (auto nd : nodes) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) G->kernels++;
    }
  }
  cudaStreamDestroy(cs);
  if (st != OURO_OK) {
    if (G) {
      if (G->exec) cudaGraphExecDestroy(G->exec);
      delete G;
    }
    if (g) cudaGraphDestroy(g);
    return st;
  }
  *out = G;
  return OURO_OK;
}

extern "C" ouro_status ouro_batch_graph_launch(ouro_batch_graph *G, void *stream) {
  if (!G) return OURO_EINVAL;
  OURO_CUDA(cudaGraphLaunch(G->exec, S(stream)));
  ouro::host::count_launch((unsigned)G->kernels);
  return OURO_OK;
}

extern "C" uint64_t ouro_batch_graph_nodes(const ouro_batch_graph *G) { return G ? G->nodes : 0; }

extern "C" ouro_status ouro_batch_graph_destroy(ouro_batch_graph *G) {
  if (!G) return OURO_OK;
  cudaGraphExecDestroy(G->exec);
  cudaGraphDestroy(G->graph);
  delete G;
  return OURO_OK;
}
#endif
