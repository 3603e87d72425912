// dqmc_op_flush_f64_noalloc: the rank-m flush of dqmc_op_flush_f64 with its
// N x K scratch (the factor A = G[:, S] alpha^T) in a fixed device array
// instead of a stream-ordered allocation, so that the call allocates no
// device memory at all.
//
// Callers that cannot allocate: a process that has handed all device memory
// to its own pool or caching allocator up front (a serving process with a
// fixed footprint), where a cudaMallocAsync here could fail or grow a pool
// that must stay fixed; and host code that must not block on the device
// while it runs, since cudaFree synchronises.
#include <mutex>
#include <vector>

#include "kernels.cuh"

namespace dq {

// Largest scratch: N = 3888 (L = 36) at the largest delay rank K = 64,
// 248,832 doubles (1.9 MiB), part of the module's static device memory.
constexpr int kNoAllocMaxN = 3888;
constexpr int kNoAllocMaxK = 64;
constexpr size_t kNoAllocScratchDoubles = (size_t)kNoAllocMaxN * kNoAllocMaxK;

static __device__ __align__(256) double g_flush_scratch[kNoAllocScratchDoubles];

// Device address of the scratch, resolved once per device with that device
// current (the first call on a device does it) and kept for the process: a
// cudaDeviceReset on that device would leave it pointing into the destroyed
// context, so the entry point is not for use across a reset.
static std::mutex g_scratch_mu;
static std::vector<void *> g_scratch_addr;

static dqmc_status flush_scratch(void **out) {
  int dev = 0;
  DQ_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if ((int)g_scratch_addr.size() <= dev) g_scratch_addr.resize(dev + 1, nullptr);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_flush_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(flush scratch)");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return DQMC_OK;
}

}  // namespace dq

using namespace dq;

extern "C" dqmc_status dqmc_op_flush_f64_noalloc(int N, int site0, int kb, double *G,
                                                 const double *Gcol, const double *Grow,
                                                 const double *alpha, const double *beta,
                                                 const int *accept_count, void *stream) try {
  if (N < 1 || kb < 1 || kb > 64 || site0 < 0 || site0 + kb > N)
    return fail(DQMC_EINVAL, "need 1 <= kb <= 64 and 0 <= site0, site0 + kb <= N");
  if (!G || !Gcol || !Grow || !alpha || !beta || !accept_count) return fail(DQMC_EINVAL, "null pointer");
  int K = 4;
  while (K < kb) K <<= 1;
  if ((size_t)N * K > kNoAllocScratchDoubles)
    return fail(DQMC_EINVAL, "N * K exceeds the fixed flush scratch of 248832 doubles (N <= 3888 at "
                             "K = 64, K = kb rounded up to a power of two >= 4)");
  void *A = nullptr;
  const dqmc_status s = flush_scratch(&A);
  if (s != DQMC_OK) return s;
  // The A kernel writes all N x K entries of the scratch (zeros beyond the
  // accepted count) before the flush reads them: nothing has to start at zero.
  FlushArgs a{N, site0, kb, 0, 0, 0, kb, kb, kb};
  const cudaError_t e = launch_flush<double>(K, a, G, Gcol, Grow, alpha, beta, accept_count, A,
                                             nullptr, nullptr, false, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "flush");
  return DQMC_OK;
} DQ_API_CATCH
