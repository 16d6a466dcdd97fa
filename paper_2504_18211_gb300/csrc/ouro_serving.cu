/*
 * Serving: a request loop that stays on the device (one cooperative,
 * persistent kernel for all steps) over sessions whose memory grows.
 *
 * Each step:
 *   1. admission (block 0, warp 0): sessions that have arrived are admitted
 *      in arrival order while a session slot is free and the blocks committed
 *      to admitted sessions, plus the newcomer's total, stay within the
 *      admission cap (95 % of the heap's blocks); the warp weighs 32
 *      arrivals at a time and admits the longest run of them, from the
 *      first, that passes;
 *   2. growth (all warps): every active session allocates one block with
 *      ouro_malloc, records it in its block table, writes its pattern
 *      (seed + session id, block index) and reads it back through L2,
 *      folding the words into the session checksum;
 *   3. completion: a session that reached its size reports its checksum and
 *      its slot is free for the next step (one thread per slot); after a
 *      barrier, the finished sessions' blocks are cut into tasks of 32 (one
 *      round of a warp) dealt to the warps in turn, so that the step's
 *      frees spread over the grid and one long session does not hold the
 *      step for a single warp.
 * The allocator state, the session table and the block tables stay resident
 * for the whole run; requests that arrive while others are running are
 * admitted as slots and memory free up, and their work overlaps on the GPU.
 * Step boundaries are a grid barrier of this file (every wait bounded); one
 * thread stamps %globaltimer after each step for the latency histogram.
 *
 * The same phases also run as the plain per-launch form (ouro_serve_per_launch):
 * one kernel per phase and step in stream order, kernel boundaries in place
 * of the grid barriers, for comparison with the one-launch loop.
 */
#include <algorithm>

#include "ouro_internal.cuh"
#include "ouro_payload.cuh"
#include "ouro_shard.cuh"

using namespace ouro::detail;

namespace {

struct serve_args {
  ouro_heap_dev h;
  /* sessions, in arrival order */
  const uint32_t *arrive_step;   /* step at which the session has arrived */
  const uint32_t *blocks;        /* total blocks the session grows to */
  uint32_t n_sessions;
  /* slots */
  uint32_t n_slots, max_blocks;
  int *slot_session;             /* session id or -1 */
  uint32_t *slot_k;              /* blocks allocated so far */
  unsigned long long *slot_acc;  /* per slot: xor, sum, mismatches */
  unsigned long long *tables;    /* n_slots x max_blocks block pointers */
  /* results */
  unsigned long long *sess_out;  /* per session: xor, sum, mismatches, admit step, done step (u64 each) */
  unsigned long long *step_ns;   /* per step: %globaltimer after admission, growth and completion (3 words) */
  unsigned long long *ctl;       /* [0] barrier count, [1] barrier generation, [2] next arrival,
                                    [3] committed blocks, [4] error, [5] mallocs, [6] frees, [7] failed,
                                    [8] free-slot stack top, [9] sessions finished this step,
                                    [10] reserved */
  uint32_t *free_stack;          /* free slot ids (stack of n_slots) */
  uint32_t *done_list;           /* slots whose sessions finished this step (n_slots) */
  uint32_t steps;
  uint32_t seed;
  unsigned long long cap_blocks; /* admission cap */
  uint32_t block_bytes;
  uint32_t spin_limit;
};

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

/* grid barrier for a cooperative launch; a wait that runs out sets ctl[4] */
__device__ bool grid_barrier(unsigned long long *ctl, unsigned nblocks, unsigned limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned long long gen = ld_acq(&ctl[1]);
    __threadfence();
    if (atomicAdd(&ctl[0], 1ull) == nblocks - 1) {
      st_rlx(&ctl[0], 0ull);
      __threadfence();
      atomicAdd(&ctl[1], 1ull);
    } else {
      unsigned it = 0;
      while (ld_acq(&ctl[1]) == gen) {
        if (++it > limit) {
          atomicExch(&ctl[4], 1ull);
          ok = 0;
          break;
        }
        __nanosleep(128);
      }
    }
    if (ld_acq(&ctl[4])) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

/* Pattern of one block, written and read back by the whole warp; the
 * block's folded checksum lands in (x, s, mism) of every lane. */
__device__ void serve_block_payload(unsigned char *bp, uint32_t bytes, uint32_t key, unsigned long long &x,
                                    unsigned long long &s, unsigned long long &mism) {
  const unsigned lane = laneid();
  uint4 *u4 = reinterpret_cast<uint4 *>(bp);
  const uint32_t units = bytes >> 4;
#pragma unroll 4
  for (uint32_t u = lane; u < units; u += 32) u4[u] = pat4(key, 4 * u);
  __syncwarp();
  payload_acc a;
  for (uint32_t u = (lane + 1) & 31; u < units; u += 32) check4(__ldcg(u4 + u), pat4(key, 4 * u), a);
  unsigned long long m = a.mism;
  for (int o = 16; o; o >>= 1) {
    a.x ^= __shfl_xor_sync(0xffffffffu, a.x, o);
    a.s += __shfl_xor_sync(0xffffffffu, a.s, o);
    m += __shfl_xor_sync(0xffffffffu, m, o);
  }
  x = a.x;
  s = a.s;
  mism = m;
}

/* ---------------------------------------------------------------- phases
 * Each phase is a device function over the whole grid; the cooperative
 * kernel separates them with grid barriers, the per-launch form with kernel
 * boundaries on one stream. */

/* the free-slot stack holds every slot */
__device__ void serve_init(const serve_args &A) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n_slots; i += gridDim.x * blockDim.x)
    A.free_stack[i] = A.n_slots - 1 - i;
  if (blockIdx.x == 0 && threadIdx.x == 0) A.ctl[8] = A.n_slots;
}

/* 1. admission (warp 0 of block 0): arrival order, a free slot (stack),
 *    committed + newcomer <= cap */
__device__ void serve_admit(const serve_args &A, uint32_t step) {
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  const unsigned lane = laneid();
  if (lane == 0) A.ctl[9] = 0;       /* the previous step's frees are all done */
  unsigned long long next = A.ctl[2], committed = A.ctl[3], top = A.ctl[8];
  for (;;) {
    const unsigned long long i = next + lane;
    const bool arrived = i < A.n_sessions && A.arrive_step[i] <= step;
    unsigned long long cum = arrived ? A.blocks[i] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, cum, o);
      if ((int)lane >= o) cum += y;
    }
    const bool ok = arrived && committed + cum <= A.cap_blocks && lane < top;
    const unsigned okm = __ballot_sync(0xffffffffu, ok);
    const unsigned n_adm = okm == 0xffffffffu ? 32u : (unsigned)(__ffs(~okm) - 1);   /* leading run */
    if (lane < n_adm) {
      const uint32_t slot = A.free_stack[top - 1 - lane];
      A.slot_session[slot] = (int)i;
      A.slot_k[slot] = 0;
      A.slot_acc[3 * slot] = A.slot_acc[3 * slot + 1] = A.slot_acc[3 * slot + 2] = 0;
      A.sess_out[5 * i + 3] = step;
    }
    if (n_adm) committed += __shfl_sync(0xffffffffu, cum, n_adm - 1);
    next += n_adm;
    top -= n_adm;
    if (n_adm < 32) break;
  }
  if (lane == 0) {
    A.ctl[2] = next;
    A.ctl[3] = committed;
    A.ctl[8] = top;
  }
  __threadfence();
}

/* 2. growth: one session per warp: lane 0 allocates, the warp writes and
 *    reads back the block */
template <int V>
__device__ void serve_grow(const serve_args &A) {
  const unsigned lane = laneid();
  const unsigned warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
  const ouro_heap_dev &h = A.h;
  for (uint32_t slot = warp; slot < A.n_slots; slot += nwarps) {
    const int sess = A.slot_session[slot];
    if (sess < 0) continue;
    const uint32_t k = A.slot_k[slot];
    if (k >= A.blocks[sess]) continue;
    /* lane 0 asks; the other 31 lanes help the warp's carves */
    /* (a step's growth can carve thousands of chunks: eight slot writes per
     *  lane in flight while the warp fills them) */
    unsigned long long bp = reinterpret_cast<unsigned long long>(malloc_v<V, 8>(h, A.block_bytes, lane == 0));
    if (lane == 0) {
      if (bp) {
        A.tables[(size_t)slot * A.max_blocks + k] = bp;
        A.slot_k[slot] = k + 1;
        atomicAdd(&A.ctl[5], 1ull);
      } else {
        atomicAdd(&A.ctl[7], 1ull);
      }
    }
    bp = __shfl_sync(0xffffffffu, bp, 0);
    if (!bp) continue;
    const uint32_t key = fmix32((A.seed + (uint32_t)sess) ^ (k * OURO_GOLD));
    unsigned long long x, sum, mism;
    serve_block_payload(reinterpret_cast<unsigned char *>(bp), A.block_bytes, key, x, sum, mism);
    if (lane == 0) {
      A.slot_acc[3 * slot] ^= x;
      A.slot_acc[3 * slot + 1] += sum;
      A.slot_acc[3 * slot + 2] += mism;
    }
  }
}

/* 3a. completion: a session that reached its size reports, releases its
 *     slot (reused from the next step on) and is listed for freeing */
__device__ void serve_complete(const serve_args &A, uint32_t step) {
  for (uint32_t slot = blockIdx.x * blockDim.x + threadIdx.x; slot < A.n_slots; slot += gridDim.x * blockDim.x) {
    const int sess = A.slot_session[slot];
    if (sess < 0 || A.slot_k[slot] < A.blocks[sess]) continue;
    A.sess_out[5 * sess + 0] = A.slot_acc[3 * slot];
    A.sess_out[5 * sess + 1] = A.slot_acc[3 * slot + 1];
    A.sess_out[5 * sess + 2] = A.slot_acc[3 * slot + 2];
    A.sess_out[5 * sess + 4] = step;
    atomicAdd(&A.ctl[6], (unsigned long long)A.slot_k[slot]);
    atomicAdd(&A.ctl[3], 0ull - (unsigned long long)A.blocks[sess]);
    A.slot_session[slot] = -1;
    A.free_stack[atomicAdd(&A.ctl[8], 1ull)] = slot;
    A.done_list[atomicAdd(&A.ctl[9], 1ull)] = slot;
  }
}

/* blocks of a finished session freed per task: one warp round, so that the
 * step's frees spread over as many warps as there are rounds of work */
constexpr uint32_t SERVE_FREE_TASK = 32;

/* 3b. the listed sessions' blocks, in tasks of SERVE_FREE_TASK blocks; warp
 *     w takes tasks w, w + nwarps, ... (tasks are of equal size, so a static
 *     share balances without a shared counter): task c is piece
 *     c - (pieces of the earlier list entries) of the first entry whose
 *     running piece count passes c */
template <int V>
__device__ void serve_free(const serve_args &A) {
  const unsigned lane = laneid();
  const unsigned long long nwarps = (gridDim.x * blockDim.x) >> 5;
  const ouro_heap_dev &h = A.h;
  const unsigned long long nl = *(volatile unsigned long long *)&A.ctl[9];
  for (unsigned long long c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;; c += nwarps) {
    unsigned long long before = 0;
    uint32_t slot = 0, nb = 0;
    bool found = false;
    for (unsigned long long i0 = 0; i0 < nl && !found; i0 += 32) {
      const unsigned long long i = i0 + lane;
      const uint32_t s_i = i < nl ? A.done_list[i] : 0;
      const uint32_t nb_i = i < nl ? A.slot_k[s_i] : 0;
      unsigned long long pc = (nb_i + SERVE_FREE_TASK - 1) / SERVE_FREE_TASK, incl = pc;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += y;
      }
      const unsigned hit = __ballot_sync(0xffffffffu, i < nl && before + incl > c);
      if (hit) {
        const int l = __ffs(hit) - 1;
        slot = __shfl_sync(0xffffffffu, s_i, l);
        nb = __shfl_sync(0xffffffffu, nb_i, l);
        before += __shfl_sync(0xffffffffu, incl - pc, l);
        found = true;
      } else {
        before += __shfl_sync(0xffffffffu, incl, 31);
      }
    }
    if (!found) break;
    const uint32_t b_lo = (uint32_t)(c - before) * SERVE_FREE_TASK, b_hi = min(nb, b_lo + SERVE_FREE_TASK);
    for (uint32_t b0 = b_lo; b0 < b_hi; b0 += 32) {
      const uint32_t b = b0 + lane;
      void *p = b < b_hi ? reinterpret_cast<void *>(A.tables[(size_t)slot * A.max_blocks + b]) : nullptr;
      if (b < b_hi) free_v<V>(h, p);
      __syncwarp();
    }
  }
}

/* The cooperative form: every step in one launch, phases separated by grid
 * barriers; block 0 stamps %globaltimer after admission, growth and freeing. */
template <int V>
__global__ void __launch_bounds__(256) k_serve(serve_args A) {
  serve_init(A);
  if (!grid_barrier(A.ctl, gridDim.x, A.spin_limit)) return;
  for (uint32_t step = 0; step < A.steps; ++step) {
    serve_admit(A, step);
    if (!grid_barrier(A.ctl, gridDim.x, A.spin_limit)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) A.step_ns[3 * step] = globaltimer();
    serve_grow<V>(A);
    if (!grid_barrier(A.ctl, gridDim.x, A.spin_limit)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) A.step_ns[3 * step + 1] = globaltimer();
    serve_complete(A, step);
    if (!grid_barrier(A.ctl, gridDim.x, A.spin_limit)) return;
    serve_free<V>(A);
    if (!grid_barrier(A.ctl, gridDim.x, A.spin_limit)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) A.step_ns[3 * step + 2] = globaltimer();
  }
}

/* The per-launch form: one kernel per phase and step, in stream order.  A
 * phase kernel first stamps %globaltimer into step_ns[stamp] (stamp >= 0):
 * the moment the previous phase had finished on the whole grid. */
enum { PH_INIT, PH_ADMIT, PH_GROW, PH_COMPLETE, PH_FREE, PH_STAMP };

template <int V, int PH>
__global__ void __launch_bounds__(256) k_serve_phase(serve_args A, uint32_t step, int stamp) {
  if (stamp >= 0 && blockIdx.x == 0 && threadIdx.x == 0) A.step_ns[stamp] = globaltimer();
  if (PH == PH_INIT) serve_init(A);
  if (PH == PH_ADMIT) serve_admit(A, step);
  if (PH == PH_GROW) serve_grow<V>(A);
  if (PH == PH_COMPLETE) serve_complete(A, step);
  if (PH == PH_FREE) serve_free<V>(A);
}

#if OURO_SHARD_ENTRIES
inline cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }
#endif

}  // namespace

/* ------------------------------------------------------- per-form launcher */
namespace ouro {
namespace launch {

/* args: the kernel's serve_args, set up by ouro_serve */
template <int V>
ouro_status serve(const void *args, int blocks_per_sm, cudaStream_t s) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_serve<V>, 256, 0);
  if (blocks_per_sm > 0 && blocks_per_sm < per_sm) per_sm = blocks_per_sm;
  if (per_sm < 1) per_sm = 1;
  void *argv[] = {const_cast<void *>(args)};
  OURO_CUDA(cudaLaunchCooperativeKernel((const void *)k_serve<V>, dim3(per_sm * ouro::host::sm_count()), dim3(256),
                                        argv, 0, s));
  OURO_LAUNCHED();
  return OURO_OK;
}

/* the per-launch form: four launches per step (admission, growth,
 * completion, freeing) plus the set-up and a final stamp, in stream order */
template <int V>
ouro_status serve_steps(const void *args, int blocks_per_sm, cudaStream_t s) {
  const serve_args &A = *static_cast<const serve_args *>(args);
  const int sms = ouro::host::sm_count();
  int grow_sm = 0, free_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&grow_sm, k_serve_phase<V, PH_GROW>, 256, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&free_sm, k_serve_phase<V, PH_FREE>, 256, 0);
  if (blocks_per_sm > 0) {
    grow_sm = std::min(grow_sm, blocks_per_sm);
    free_sm = std::min(free_sm, blocks_per_sm);
  }
  /* growth: a warp per slot at most; slots: a thread per slot */
  const unsigned grow_g = (unsigned)std::max(1, std::min(grow_sm * sms, (int)((A.n_slots + 7) / 8)));
  const unsigned free_g = (unsigned)std::max(1, free_sm * sms);
  const unsigned slot_g = (unsigned)std::max(1u, std::min((A.n_slots + 255) / 256, 8u * sms));
  k_serve_phase<V, PH_INIT><<<slot_g, 256, 0, s>>>(A, 0, -1);
  OURO_LAUNCHED();
  for (uint32_t step = 0; step < A.steps; ++step) {
    k_serve_phase<V, PH_ADMIT><<<1, 32, 0, s>>>(A, step, step ? (int)(3 * step - 1) : -1);
    OURO_LAUNCHED();
    k_serve_phase<V, PH_GROW><<<grow_g, 256, 0, s>>>(A, step, (int)(3 * step));
    OURO_LAUNCHED();
    k_serve_phase<V, PH_COMPLETE><<<slot_g, 256, 0, s>>>(A, step, (int)(3 * step + 1));
    OURO_LAUNCHED();
    k_serve_phase<V, PH_FREE><<<free_g, 256, 0, s>>>(A, step, -1);
    OURO_LAUNCHED();
  }
  if (A.steps) {
    k_serve_phase<V, PH_STAMP><<<1, 32, 0, s>>>(A, 0, (int)(3 * A.steps - 1));
    OURO_LAUNCHED();
  }
  return OURO_OK;
}

#define INST_SERVE(PRE, V) PRE template ouro_status serve<V>(const void *, int, cudaStream_t);
#define INST_SERVE_STEPS(PRE, V) PRE template ouro_status serve_steps<V>(const void *, int, cudaStream_t);
OURO_SHARD_INSTANTIATE(INST_SERVE)
OURO_SHARD_INSTANTIATE(INST_SERVE_STEPS)

}  // namespace launch
}  // namespace ouro

#if OURO_SHARD_ENTRIES
namespace {
/* checks the arguments, resets the loop's state on the stream and fills A */
ouro_status serve_prepare(ouro_heap *H, const uint32_t *d_arrive_step, const uint32_t *d_blocks, uint32_t n_sessions,
                          uint32_t n_slots, uint32_t max_blocks, int *d_slot_session, uint32_t *d_slot_k,
                          unsigned long long *d_slot_acc, unsigned long long *d_tables,
                          unsigned long long *d_sess_out, unsigned long long *d_step_ns, unsigned long long *d_ctl,
                          uint32_t *d_free_stack, uint32_t steps, uint32_t seed, uint64_t cap_blocks,
                          uint32_t block_bytes, cudaStream_t s, serve_args &A) {
  if (!H || !d_arrive_step || !d_blocks || !d_slot_session || !d_slot_k || !d_slot_acc || !d_tables ||
      !d_sess_out || !d_step_ns || !d_ctl || !d_free_stack || n_slots == 0 || max_blocks == 0 || (block_bytes & 15) ||
      block_bytes == 0 || block_bytes > H->d.chunk_bytes)
    return OURO_EINVAL;
  OURO_CUDA(cudaMemsetAsync(d_slot_session, 0xFF, n_slots * sizeof(int), s));
  OURO_CUDA(cudaMemsetAsync(d_ctl, 0, 11 * 8, s));
  OURO_CUDA(cudaMemsetAsync(d_sess_out, 0xFF, (size_t)n_sessions * 5 * 8, s));
  A.h = H->d;
  A.arrive_step = d_arrive_step;
  A.blocks = d_blocks;
  A.n_sessions = n_sessions;
  A.n_slots = n_slots;
  A.max_blocks = max_blocks;
  A.slot_session = d_slot_session;
  A.slot_k = d_slot_k;
  A.slot_acc = d_slot_acc;
  A.tables = d_tables;
  A.sess_out = d_sess_out;
  A.step_ns = d_step_ns;
  A.ctl = d_ctl;
  A.free_stack = d_free_stack;
  A.done_list = d_free_stack + n_slots;
  A.steps = steps;
  A.seed = seed;
  A.cap_blocks = cap_blocks;
  A.block_bytes = block_bytes;
  A.spin_limit = 1u << 24;   /* barrier wait: ~2 s of 128 ns naps, far above any step */
  return OURO_OK;
}
}  // namespace

extern "C" ouro_status ouro_serve(ouro_heap *H, const uint32_t *d_arrive_step, const uint32_t *d_blocks,
                                  uint32_t n_sessions, uint32_t n_slots, uint32_t max_blocks, int *d_slot_session,
                                  uint32_t *d_slot_k, unsigned long long *d_slot_acc, unsigned long long *d_tables,
                                  unsigned long long *d_sess_out, unsigned long long *d_step_ns,
                                  unsigned long long *d_ctl, uint32_t *d_free_stack, uint32_t steps, uint32_t seed,
                                  uint64_t cap_blocks, uint32_t block_bytes, int blocks_per_sm, void *stream) {
  cudaStream_t s = S(stream);
  serve_args A;
  const ouro_status st = serve_prepare(H, d_arrive_step, d_blocks, n_sessions, n_slots, max_blocks, d_slot_session,
                                       d_slot_k, d_slot_acc, d_tables, d_sess_out, d_step_ns, d_ctl, d_free_stack,
                                       steps, seed, cap_blocks, block_bytes, s, A);
  if (st != OURO_OK) return st;
  int dev = 0, coop = 0;
  OURO_CUDA(cudaGetDevice(&dev));
  OURO_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return OURO_ENOTSUP;
  OURO_DISPATCH(H->d.variant, return ouro::launch::serve<V>(&A, blocks_per_sm, s));
}

extern "C" ouro_status ouro_serve_per_launch(ouro_heap *H, const uint32_t *d_arrive_step, const uint32_t *d_blocks,
                                             uint32_t n_sessions, uint32_t n_slots, uint32_t max_blocks,
                                             int *d_slot_session, uint32_t *d_slot_k, unsigned long long *d_slot_acc,
                                             unsigned long long *d_tables, unsigned long long *d_sess_out,
                                             unsigned long long *d_step_ns, unsigned long long *d_ctl,
                                             uint32_t *d_free_stack, uint32_t steps, uint32_t seed,
                                             uint64_t cap_blocks, uint32_t block_bytes, int blocks_per_sm,
                                             void *stream) {
  cudaStream_t s = S(stream);
  serve_args A;
  const ouro_status st = serve_prepare(H, d_arrive_step, d_blocks, n_sessions, n_slots, max_blocks, d_slot_session,
                                       d_slot_k, d_slot_acc, d_tables, d_sess_out, d_step_ns, d_ctl, d_free_stack,
                                       steps, seed, cap_blocks, block_bytes, s, A);
  if (st != OURO_OK) return st;
  OURO_DISPATCH(H->d.variant, return ouro::launch::serve_steps<V>(&A, blocks_per_sm, s));
}
#endif
