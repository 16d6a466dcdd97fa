/*
 * Graph growth: adjacency lists that grow inside kernels through the device
 * allocator (a dynamically partitioned workload of the kind Sec. 1 of
 * arXiv 2504.18211 names: graph algorithms need memory repartitioned
 * while the kernel runs).
 *
 * Vertex v owns a list of uint32 neighbours.  It starts with 4 entries
 * (16 B).  When an append does not fit, the list doubles (malloc 2x, copy,
 * free the old list), one doubling at a time, until it reaches one chunk.
 * Past one chunk, entries go to overflow segments of one chunk each, chained
 * newest first: [next pointer (8 B)][entries].
 *
 * Each thread owns 16 edges.  A block sorts its 4096 (src, dst) pairs in
 * shared memory, so that a warp appends a whole run of one source under
 * that vertex's lock, taken once.  The per-vertex locks are bounded spins;
 * a lock that cannot be taken sets the heap's TIMEOUT bit and skips the run
 * (counted in ctl[2]).
 */
#include "ouro_internal.cuh"
#include "ouro_payload.cuh"
#include "ouro_shard.cuh"

using namespace ouro::detail;

namespace {

struct vertex {
  unsigned long long ptr;   /* plain list */
  unsigned long long ovf;   /* newest overflow segment (0: none) */
  unsigned cnt;             /* entries in the plain list */
  unsigned cap;             /* capacity of the plain list (entries) */
  unsigned ovf_cnt;         /* entries in the newest overflow segment */
  unsigned lock;
  unsigned deg;             /* all entries */
  unsigned pad;
};

constexpr int EDGES_PER_THREAD = 16;
constexpr int GB_THREADS = 256;
constexpr int GB_EDGES = EDGES_PER_THREAD * GB_THREADS;   /* 4096 pairs per block */

template <int V>
__global__ void k_graph_init(ouro_heap_dev h, vertex *vt, unsigned nv, unsigned long long *ctl) {
  for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
    void *p = malloc_v<V>(h, 16);
    vt[v].ptr = reinterpret_cast<unsigned long long>(p);
    vt[v].ovf = 0;
    vt[v].cnt = vt[v].ovf_cnt = vt[v].lock = vt[v].deg = 0;
    vt[v].cap = p ? 4 : 0;
    if (!p) atomicAdd(&ctl[1], 1ull);
  }
}

__device__ bool vlock(vertex *vx, unsigned spin_limit) {
  unsigned ns = 32;
  for (unsigned it = 0; it < spin_limit; ++it) {
    if (atomicCAS(&vx->lock, 0u, 1u) == 0u) {
      __threadfence();
      return true;
    }
    __nanosleep(ns);
    ns = min(ns * 2, 1024u);
  }
  return false;
}

__device__ void vunlock(vertex *vx) {
  __threadfence();
  atomicExch(&vx->lock, 0u);
}

/* Append the n neighbours in the low words of keys[0..n) (shared memory)
 * to vertex vx; the whole warp calls, lane 0 holds the lock and talks to the
 * allocator.  Vertex fields and list entries written by other SMs are read
 * past L1 (volatile / ld.cg); every lane fences its stores before unlock. */
template <int V>
__device__ void warp_append(const ouro_heap_dev &h, vertex *vx, const unsigned long long *keys, unsigned n,
                            unsigned long long *ctl) {
  const unsigned lane = laneid();
  const unsigned max_plain = h.chunk_bytes >> 2;          /* entries in one chunk */
  const unsigned seg_cap = (h.chunk_bytes - 8) >> 2;     /* entries per overflow segment */
  int ok = 1;
  if (lane == 0) ok = vlock(vx, h.spin_limit) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (!ok) {
    if (lane == 0) {
      set_error(h, OURO_ERR_TIMEOUT, OURO_SITE_GRAPH_LOCK);
      atomicAdd(&ctl[2], (unsigned long long)n);
    }
    return;
  }
  __syncwarp();
  volatile vertex *vv = vx;
  unsigned done = 0;
  for (int guard = 0; done < n && guard < 64; ++guard) {
    unsigned cnt = vv->cnt, cap = vv->cap;
    unsigned long long ptr = vv->ptr;
    if (cnt == cap && cap < max_plain && cap) {
      /* one doubling: malloc 2x, copy, free the old list */
      /* lane 0 asks, the other lanes help the warp's carves */
      unsigned long long np = reinterpret_cast<unsigned long long>(malloc_v<V>(h, (size_t)cap * 8, lane == 0));
      np = __shfl_sync(0xffffffffu, np, 0);
      if (!np) {
        if (lane == 0) atomicAdd(&ctl[1], (unsigned long long)(n - done));
        break;
      }
      const unsigned *src = reinterpret_cast<const unsigned *>(ptr);
      unsigned *dst = reinterpret_cast<unsigned *>(np);
      for (unsigned i = lane; i < cnt; i += 32) dst[i] = __ldcg(src + i);
      __syncwarp();
      if (lane == 0) {
        free_v<V>(h, reinterpret_cast<void *>(ptr));
        vv->ptr = np;
        vv->cap = cap * 2;
      }
      __syncwarp();
      continue;
    }
    if (cnt < cap) {
      const unsigned m = min(cap - cnt, n - done);
      unsigned *dst = reinterpret_cast<unsigned *>(ptr) + cnt;
      for (unsigned i = lane; i < m; i += 32) dst[i] = (unsigned)keys[done + i];
      __syncwarp();
      if (lane == 0) vv->cnt = cnt + m;
      done += m;
      __syncwarp();
      continue;
    }
    /* plain list full at one chunk: overflow segments */
    unsigned long long seg = vv->ovf;
    unsigned oc = vv->ovf_cnt;
    if (!seg || oc == seg_cap) {
      unsigned long long ns = reinterpret_cast<unsigned long long>(malloc_v<V>(h, h.chunk_bytes, lane == 0));
      if (lane == 0) {
        if (ns) {
          *reinterpret_cast<unsigned long long *>(ns) = seg;
          vv->ovf = ns;
          vv->ovf_cnt = 0;
        }
      }
      ns = __shfl_sync(0xffffffffu, ns, 0);
      if (!ns) {
        if (lane == 0) atomicAdd(&ctl[1], (unsigned long long)(n - done));
        break;
      }
      seg = ns;
      oc = 0;
    }
    const unsigned m = min(seg_cap - oc, n - done);
    unsigned *dst = reinterpret_cast<unsigned *>(seg + 8) + oc;
    for (unsigned i = lane; i < m; i += 32) dst[i] = (unsigned)keys[done + i];
    __syncwarp();
    if (lane == 0) vv->ovf_cnt = oc + m;
    done += m;
    __syncwarp();
  }
  __threadfence();
  __syncwarp();
  if (lane == 0) {
    vv->deg = vv->deg + done;
    atomicAdd(&ctl[0], (unsigned long long)done);
    vunlock(vx);
  }
  __syncwarp();
}

/* Each thread owns 16 edges; the block sorts its 4096 pairs by (src, dst)
 * with a bitonic network in shared memory, then warps append source runs. */
template <int V>
__global__ void __launch_bounds__(GB_THREADS) k_graph_insert(ouro_heap_dev h, vertex *vt, const unsigned *src,
                                                             const unsigned *dst, unsigned long long n_edges,
                                                             unsigned long long *ctl) {
  __shared__ unsigned long long key[GB_EDGES];
  __shared__ unsigned short run_start[GB_EDGES + 1];
  __shared__ unsigned n_runs;
  const unsigned long long base = (unsigned long long)blockIdx.x * GB_EDGES;
  for (unsigned i = threadIdx.x; i < GB_EDGES; i += GB_THREADS) {
    const unsigned long long e = base + i;
    key[i] = e < n_edges ? ((unsigned long long)src[e] << 32) | dst[e] : ~0ull;
  }
  __syncthreads();
  for (unsigned k = 2; k <= GB_EDGES; k <<= 1) {
    for (unsigned j = k >> 1; j > 0; j >>= 1) {
      for (unsigned i = threadIdx.x; i < GB_EDGES; i += GB_THREADS) {
        const unsigned ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long a = key[i], b = key[ixj];
          const bool up = (i & k) == 0;
          if ((a > b) == up) {
            key[i] = b;
            key[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) n_runs = 0;
  __syncthreads();
  /* run starts, in order (ordered compaction by one warp) */
  if (threadIdx.x < 32) {
    unsigned count = 0;
    for (unsigned i0 = 0; i0 < GB_EDGES; i0 += 32) {
      const unsigned i = i0 + threadIdx.x;
      const bool valid = key[i] != ~0ull;
      const bool start = valid && (i == 0 || (key[i] >> 32) != (key[i - 1] >> 32));
      const unsigned b = __ballot_sync(0xffffffffu, start);
      if (start) run_start[count + __popc(b & ((1u << threadIdx.x) - 1))] = (unsigned short)i;
      count += __popc(b);
    }
    if (threadIdx.x == 0) {
      n_runs = count;
      unsigned end = GB_EDGES;
      while (end > 0 && key[end - 1] == ~0ull) --end;
      run_start[count] = (unsigned short)(end == GB_EDGES ? 0 : end);   /* GB_EDGES does not fit: 0 marks it */
    }
  }
  __syncthreads();
  const unsigned warp = threadIdx.x >> 5;
  for (unsigned r = warp; r < n_runs; r += GB_THREADS / 32) {
    const unsigned a = run_start[r];
    const unsigned b = (r + 1 == n_runs && run_start[r + 1] == 0) ? GB_EDGES : run_start[r + 1];
    const unsigned v = (unsigned)(key[a] >> 32);
    warp_append<V>(h, &vt[v], key + a, b - a, ctl);
  }
}

/* Every vertex's entries, plain list then overflow segments (newest first),
 * into out[off[v] .. off[v] + deg[v]). */
__global__ void k_graph_gather(const vertex *vt, unsigned nv, const unsigned long long *off, unsigned *out,
                               unsigned chunk_bytes) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned seg_cap = (chunk_bytes - 8) >> 2;
  for (unsigned v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < nv; v += (gridDim.x * blockDim.x) >> 5) {
    unsigned long long o = off[v];
    const vertex x = vt[v];
    const unsigned *pl = reinterpret_cast<const unsigned *>(x.ptr);
    for (unsigned i = lane; i < x.cnt; i += 32) out[o + i] = pl[i];
    o += x.cnt;
    unsigned long long seg = x.ovf;
    unsigned take = x.ovf_cnt;
    for (unsigned guard = 0; seg && guard < (1u << 26); ++guard) {
      const unsigned *e = reinterpret_cast<const unsigned *>(seg + 8);
      for (unsigned i = lane; i < take; i += 32) out[o + i] = e[i];
      o += take;
      seg = *reinterpret_cast<const unsigned long long *>(seg);
      take = seg_cap;
    }
  }
}

template <int V>
__global__ void k_graph_free(ouro_heap_dev h, vertex *vt, unsigned nv) {
  for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
    free_v<V>(h, reinterpret_cast<void *>(vt[v].ptr));
    unsigned long long seg = vt[v].ovf;
    for (unsigned guard = 0; seg && guard < (1u << 26); ++guard) {
      const unsigned long long nx = *reinterpret_cast<const unsigned long long *>(seg);
      free_v<V>(h, reinterpret_cast<void *>(seg));
      seg = nx;
    }
    vt[v].ptr = vt[v].ovf = 0;
  }
}

#if OURO_SHARD_ENTRIES
inline cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }
#endif

}  // namespace

/* ------------------------------------------------------- per-form launchers */
namespace ouro {
namespace launch {

template <int V>
ouro_status graph_init(ouro_heap *H, void *d_vertices, uint32_t n_vertices, unsigned long long *d_ctl,
                       cudaStream_t s) {
  k_graph_init<V><<<4 * ouro::host::sm_count(), 256, 0, s>>>(H->d, (vertex *)d_vertices, n_vertices, d_ctl);
  OURO_LAUNCHED();
  return OURO_OK;
}

template <int V>
ouro_status graph_insert(ouro_heap *H, void *d_vertices, const uint32_t *d_src, const uint32_t *d_dst,
                         uint64_t n_edges, unsigned long long *d_ctl, cudaStream_t s) {
  const unsigned blocks = (unsigned)((n_edges + GB_EDGES - 1) / GB_EDGES);
  k_graph_insert<V><<<blocks, GB_THREADS, 0, s>>>(H->d, (vertex *)d_vertices, d_src, d_dst, n_edges, d_ctl);
  OURO_LAUNCHED();
  return OURO_OK;
}

template <int V>
ouro_status graph_free(ouro_heap *H, void *d_vertices, uint32_t n_vertices, cudaStream_t s) {
  k_graph_free<V><<<4 * ouro::host::sm_count(), 256, 0, s>>>(H->d, (vertex *)d_vertices, n_vertices);
  OURO_LAUNCHED();
  return OURO_OK;
}

#define INST_GRAPH_INIT(PRE, V) \
  PRE template ouro_status graph_init<V>(ouro_heap *, void *, uint32_t, unsigned long long *, cudaStream_t);
#define INST_GRAPH_INSERT(PRE, V)                                                                          \
  PRE template ouro_status graph_insert<V>(ouro_heap *, void *, const uint32_t *, const uint32_t *, uint64_t, \
                                           unsigned long long *, cudaStream_t);
#define INST_GRAPH_FREE(PRE, V) PRE template ouro_status graph_free<V>(ouro_heap *, void *, uint32_t, cudaStream_t);
OURO_SHARD_INSTANTIATE(INST_GRAPH_INIT)
OURO_SHARD_INSTANTIATE(INST_GRAPH_INSERT)
OURO_SHARD_INSTANTIATE(INST_GRAPH_FREE)

}  // namespace launch
}  // namespace ouro

#if OURO_SHARD_ENTRIES
extern "C" size_t ouro_graph_vertex_bytes(void) { return sizeof(vertex); }

extern "C" ouro_status ouro_graph_init(ouro_heap *H, void *d_vertices, uint32_t n_vertices, unsigned long long *d_ctl,
                                       void *stream) {
  if (!H || !d_vertices || !d_ctl || !n_vertices) return OURO_EINVAL;
  OURO_CUDA(cudaMemsetAsync(d_ctl, 0, 4 * 8, S(stream)));
  OURO_DISPATCH(H->d.variant, return ouro::launch::graph_init<V>(H, d_vertices, n_vertices, d_ctl, S(stream)));
}

extern "C" ouro_status ouro_graph_insert(ouro_heap *H, void *d_vertices, const uint32_t *d_src, const uint32_t *d_dst,
                                         uint64_t n_edges, unsigned long long *d_ctl, void *stream) {
  if (!H || !d_vertices || !d_ctl || (n_edges && (!d_src || !d_dst))) return OURO_EINVAL;
  if (!n_edges) return OURO_OK;
  OURO_DISPATCH(H->d.variant,
                return ouro::launch::graph_insert<V>(H, d_vertices, d_src, d_dst, n_edges, d_ctl, S(stream)));
}

extern "C" ouro_status ouro_graph_gather(ouro_heap *H, const void *d_vertices, uint32_t n_vertices,
                                         const unsigned long long *d_offsets, uint32_t *d_out, void *stream) {
  if (!H || !d_vertices || !d_offsets || !d_out) return OURO_EINVAL;
  const int g = 8 * ouro::host::sm_count();
  k_graph_gather<<<g, 256, 0, S(stream)>>>((const vertex *)d_vertices, n_vertices, d_offsets, d_out, H->d.chunk_bytes);
  OURO_LAUNCHED();
  return OURO_OK;
}

extern "C" ouro_status ouro_graph_free(ouro_heap *H, void *d_vertices, uint32_t n_vertices, void *stream) {
  if (!H || !d_vertices) return OURO_EINVAL;
  OURO_DISPATCH(H->d.variant, return ouro::launch::graph_free<V>(H, d_vertices, n_vertices, S(stream)));
}
#endif
