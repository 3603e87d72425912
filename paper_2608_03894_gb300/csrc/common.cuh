// Shared device/host helpers of the GB300 kagome DQMC library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <exception>
#include <new>
#include <string>

#include "../../include/dqmc.h"

namespace dq {

// ------------------------------------------------------------------ errors
// Thread-local last-error message behind dqmc_last_error().
void set_error(const std::string &msg);
dqmc_status fail(dqmc_status st, const std::string &msg);
dqmc_status cuda_fail(cudaError_t e, const char *what);

// Records msg without throwing (used where a C++ exception was caught).
dqmc_status fail_host(dqmc_status st, const char *msg) noexcept;

// Tail of the function-try-block of every C ABI entry point: no C++
// exception (a failed host allocation or thread creation) crosses the C
// boundary; it becomes DQMC_ENOMEM with its message.
#define DQ_API_CATCH                                                              \
  catch (const std::bad_alloc &) {                                                \
    return ::dq::fail_host(DQMC_ENOMEM, "host memory exhausted");                 \
  }                                                                               \
  catch (const std::exception &_x) {                                              \
    return ::dq::fail_host(DQMC_ENOMEM, _x.what());                               \
  }                                                                               \
  catch (...) {                                                                   \
    return ::dq::fail_host(DQMC_ENOMEM, "host exception");                        \
  }

#define DQ_CUDA(call)                                     \
  do {                                                    \
    cudaError_t _e = (call);                              \
    if (_e != cudaSuccess) return ::dq::cuda_fail(_e, #call); \
  } while (0)

#define DQ_CHECK(st)                   \
  do {                                 \
    dqmc_status _s = (st);             \
    if (_s != DQMC_OK) return _s;      \
  } while (0)

// ------------------------------------------------------------------ small types
template <typename T> struct cpx { T x, y; };

template <typename T> __host__ __device__ __forceinline__ cpx<T> mkc(T a, T b) { return cpx<T>{a, b}; }

// Supported torus sizes (one register-resident FFT instantiation each).
constexpr int kSupportedL[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 36};
inline bool supported_L(int L) {
  for (int v : kSupportedL)
    if (v == L) return true;
  return false;
}

// ------------------------------------------------------------------ Philox4x32-10
// Written from its published definition (Salmon, Moraes, Dror, Shaw, SC'11):
// two 32x32->64 multiplies per round on words 0 and 2, the high halves mixed
// with words 1 and 3 and the round key, key bumped by the Weyl constants.
__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = mulhi32(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = mulhi32(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// u in [0,1) from 53 bits: ((r0 >> 5) 2^26 + (r1 >> 6)) 2^-53.
__host__ __device__ __forceinline__ double uniform53(uint32_t r0, uint32_t r1) {
  return ((double)(r0 >> 5) * 67108864.0 + (double)(r1 >> 6)) * (1.0 / 9007199254740992.0);
}

constexpr uint32_t kDomainMetropolis = 0u;
constexpr uint32_t kDomainInit = 1u;

// ------------------------------------------------------------------ launch helpers
inline int ceil_div(long a, long b) { return (int)((a + b - 1) / b); }

// Kernel families for per-family device timing (dqmc_stats.ms_kernel).
// kernel families for timing and work accounting (order = dqmc_stats arrays)
enum KFam {
  KF_PROP = 0,    // FFT propagation
  KF_METRO,       // Metropolis block
  KF_FLUSH,       // rank-m flush
  KF_GEMM,        // stabilisation GEMMs
  KF_QRPANEL,     // Householder panels
  KF_MEASURE,     // measurements
  KF_OTHER,       // remaining small kernels (exp(V), field init, drift)
  KF_SLICE,       // operand splitting of the digit-slice / double-float GEMMs
  KF_BLOCKAUX,    // delayed-update helpers: gathers, A/B factors, look-ahead block
  KF_STABAUX,     // stabilisation helpers: T factors, triangular inverses, pivoting, scaling
  KF_COUNT
};

// Optional per-launch event recorder, installed by the engine for the calling
// thread while a context runs with per-kernel timing; every launch site wraps
// its launch in a KScope, which also counts launches.
struct KTimerSink {
  virtual void begin(int fam, cudaStream_t st) = 0;
  virtual void end(int fam, cudaStream_t st) = 0;
  virtual ~KTimerSink() {}
};
KTimerSink *&ktimer_sink();
void count_launch();
unsigned long long launch_count();
// Algorithmic work of the launches issued by the calling thread, per family
// (flops of the mathematical operation, bytes of one read of every input and
// one write of every output); read by the engine for the roofline figures.
void add_work(int fam, double flops, double bytes);
const double *work_flops();
const double *work_bytes();

struct KScope {
  int fam;
  cudaStream_t st;
  KScope(int f, cudaStream_t s) : fam(f), st(s) {
    if (ktimer_sink()) ktimer_sink()->begin(f, s);
  }
  ~KScope() {
    count_launch();
    if (ktimer_sink()) ktimer_sink()->end(fam, st);
  }
};
#define DQ_KSCOPE_CAT2(a, b) a##b
#define DQ_KSCOPE_CAT(a, b) DQ_KSCOPE_CAT2(a, b)
#define DQ_KSCOPE(fam, st) ::dq::KScope DQ_KSCOPE_CAT(dq_kscope_, __LINE__)(fam, st)

}  // namespace dq
