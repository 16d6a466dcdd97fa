/* Internal declarations shared by the library's translation units. */
#ifndef OURO_INTERNAL_CUH
#define OURO_INTERNAL_CUH

#include <cuda_runtime.h>

#include "ouro.h"
#include "ouro_device.cuh"

/* Ring slack: at most this many threads can be resident on the GPU at once
 * (152 SMs x 2048), so a ring of (capacity + slack) slots never makes a
 * producer wait for a consumer that is still in flight one lap behind. */
#define OURO_RING_SLACK (1ull << 19)
/* virtualized-array directories also span positions that are waiting for a
 * producer or in flight (more than twice the resident threads of 152 SMs) */
#define OURO_VA_SLACK (1ull << 20)
/* work counters of fused rounds: one per launch in flight on a heap, each on
 * its own 128-byte line, handed out round robin */
#define OURO_WORK_SLOTS 64

struct ouro_heap {
  ouro_heap_dev d;
  int device;
  void *heap_buf;
  int owns_heap;
  unsigned char *meta;          /* one device allocation for every metadata table */
  size_t meta_bytes;
  size_t off_qhdr, off_glob, off_stats, off_cls, off_pool, off_free, off_bits, off_cells, off_work;
  unsigned work_seq;            /* next work-counter slot (atomic) */
  size_t stats_words;
  unsigned long long ring_total;
  ouro_options opt;
};

namespace ouro {
namespace host {
extern thread_local int g_last_cuda_error;
ouro_status cuda_fail(cudaError_t e);
void count_launch(unsigned n = 1);
int sm_count();
}  // namespace host
}  // namespace ouro

#define OURO_CUDA(call)                                            \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return ouro::host::cuda_fail(e_);       \
  } while (0)

#define OURO_LAUNCHED()                                            \
  do {                                                             \
    cudaError_t e_ = cudaGetLastError();                           \
    if (e_ != cudaSuccess) return ouro::host::cuda_fail(e_);       \
    ouro::host::count_launch();                                    \
  } while (0)

#endif
