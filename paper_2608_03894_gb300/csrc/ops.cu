// Stateless operator entry points of include/dqmc.h: one hot-path step on
// caller-owned device memory.
#include <algorithm>
#include <cmath>
#include <complex>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "kernels.cuh"
#include "lattice_host.h"
#include "linalg.cuh"

namespace dq {

// block tables for the operator API (cached per device, L, scale, precision)
static std::mutex g_op_mu;
static std::map<std::tuple<int, int, int, double>, void *> g_op_tables;

static dqmc_status op_table(int L, double scale, int prec, const void **out) {
  int dev = 0;
  DQ_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_op_mu);
  auto key = std::make_tuple(dev, L, prec, scale);
  auto it = g_op_tables.find(key);
  if (it != g_op_tables.end()) {
    *out = it->second;
    return DQMC_OK;
  }
  std::vector<cd> tab = block_exp_table(L, scale);
  void *d = nullptr;
  if (prec == 0) {
    std::vector<cpx<double>> h(tab.size());
    for (size_t q = 0; q < tab.size(); ++q) h[q] = cpx<double>{tab[q].real(), tab[q].imag()};
    DQ_CUDA(cudaMalloc(&d, h.size() * sizeof(h[0])));
    DQ_CUDA(cudaMemcpy(d, h.data(), h.size() * sizeof(h[0]), cudaMemcpyHostToDevice));
  } else if (prec == 1) {
    std::vector<cpx<float>> h(tab.size());
    for (size_t q = 0; q < tab.size(); ++q) h[q] = cpx<float>{(float)tab[q].real(), (float)tab[q].imag()};
    DQ_CUDA(cudaMalloc(&d, h.size() * sizeof(h[0])));
    DQ_CUDA(cudaMemcpy(d, h.data(), h.size() * sizeof(h[0]), cudaMemcpyHostToDevice));
  } else {
    std::vector<cpx<df64>> h(tab.size());
    for (size_t q = 0; q < tab.size(); ++q) h[q] = cpx<df64>{df64(tab[q].real()), df64(tab[q].imag())};
    DQ_CUDA(cudaMalloc(&d, h.size() * sizeof(h[0])));
    DQ_CUDA(cudaMemcpy(d, h.data(), h.size() * sizeof(h[0]), cudaMemcpyHostToDevice));
  }
  g_op_tables[key] = d;
  *out = d;
  return DQMC_OK;
}

static dqmc_status check_prop(int L, int side, const void *X, void *Y, int nvec, int ld) {
  if (!supported_L(L)) return fail(DQMC_EINVAL, "unsupported L");
  if (side != 0 && side != 1) return fail(DQMC_EINVAL, "side must be 0 (left) or 1 (right)");
  if (!X || !Y) return fail(DQMC_EINVAL, "X and Y must be device pointers");
  const int N = 3 * L * L;
  if (nvec < 0) return fail(DQMC_EINVAL, "nvec must be >= 0");
  if (ld < (side == 0 ? nvec : N)) return fail(DQMC_EINVAL, "ld too small");
  return DQMC_OK;
}

}  // namespace dq

using namespace dq;

extern "C" {

dqmc_status dqmc_op_propagate_f64(int L, double scale, int side, const double *X, double *Y,
                                  int nvec, int ld, const double *pre, const double *post,
                                  const double *vscale, void *stream) try {
  DQ_CHECK(check_prop(L, side, X, Y, nvec, ld));
  const void *E = nullptr;
  DQ_CHECK(op_table(L, scale, 0, &E));
  DQ_CUDA(launch_prop_f64(L, side, X, Y, nvec, ld, static_cast<const cpx<double> *>(E), pre, post,
                          vscale, static_cast<cudaStream_t>(stream)));
  return DQMC_OK;
} DQ_API_CATCH

dqmc_status dqmc_op_propagate_df(int L, double scale, int side, const double *X, double *Y,
                                 int nvec, int ld, const double *pre, const double *post,
                                 const double *vscale, void *stream) try {
  DQ_CHECK(check_prop(L, side, X, Y, nvec, ld));
  const void *E = nullptr;
  DQ_CHECK(op_table(L, scale, 2, &E));
  DQ_CUDA(launch_prop_df(L, side, X, Y, nvec, ld, static_cast<const cpx<df64> *>(E), pre, post,
                         vscale, static_cast<cudaStream_t>(stream)));
  return DQMC_OK;
} DQ_API_CATCH

dqmc_status dqmc_op_propagate_f32(int L, double scale, int side, const float *X, float *Y,
                                  int nvec, int ld, const float *pre, const float *post,
                                  const float *vscale, void *stream) try {
  DQ_CHECK(check_prop(L, side, X, Y, nvec, ld));
  const void *E = nullptr;
  DQ_CHECK(op_table(L, scale, 1, &E));
  DQ_CUDA(launch_prop_f32(L, side, X, Y, nvec, ld, static_cast<const cpx<float> *>(E), pre, post,
                          vscale, static_cast<cudaStream_t>(stream)));
  return DQMC_OK;
} DQ_API_CATCH

static dqmc_status op_metropolis(int N, int site0, int kb, const double *g, int ld_g, int8_t *s,
                                 double lambda, uint64_t seed, uint32_t chain, uint32_t sweep_pass,
                                 int slice1, const uint8_t *forced, double *alpha, double *beta,
                                 int *accept_count, int *status, void *stream, bool df) {
  if (N < 1 || kb < 1 || kb > 64 || site0 < 0 || site0 + kb > N)
    return fail(DQMC_EINVAL, "need 1 <= kb <= 64 and 0 <= site0, site0 + kb <= N");
  if (!g || !s || !alpha || !beta || !accept_count || !status) return fail(DQMC_EINVAL, "null pointer");
  if (ld_g < kb) return fail(DQMC_EINVAL, "ld_g < kb");
  if (!(lambda >= 0.0)) return fail(DQMC_EINVAL, "lambda must be >= 0");
  if (slice1 < 1) return fail(DQMC_EINVAL, "slice1 is 1-based");
  MetroArgs a;
  a.N = N;
  a.s0 = site0;
  a.kb = kb;
  a.K = kb;
  a.ld_g = ld_g;
  a.e2l = std::exp(2.0 * lambda);
  a.em2l = std::exp(-2.0 * lambda);
  a.k0 = (uint32_t)(seed & 0xffffffffu);
  a.k1 = (uint32_t)(seed >> 32);
  a.c2 = sweep_pass;
  a.c3 = (chain & 0xffffffu) | (kDomainMetropolis << 24);
  a.slice0 = slice1 - 1;
  DQ_CUDA(launch_metropolis(a, g, false, s, forced, alpha, beta, accept_count, status, nullptr,
                            static_cast<cudaStream_t>(stream), df));
  return DQMC_OK;
}

dqmc_status dqmc_op_metropolis_block(int N, int site0, int kb, const double *g, int ld_g,
                                     int8_t *s, double lambda, uint64_t seed, uint32_t chain,
                                     uint32_t sweep_pass, int slice1, const uint8_t *forced,
                                     double *alpha, double *beta, int *accept_count, int *status,
                                     void *stream) try {
  return op_metropolis(N, site0, kb, g, ld_g, s, lambda, seed, chain, sweep_pass, slice1, forced, alpha,
                       beta, accept_count, status, stream, false);
} DQ_API_CATCH

dqmc_status dqmc_op_metropolis_block_df(int N, int site0, int kb, const double *g, int ld_g,
                                        int8_t *s, double lambda, uint64_t seed, uint32_t chain,
                                        uint32_t sweep_pass, int slice1, const uint8_t *forced,
                                        double *alpha, double *beta, int *accept_count, int *status,
                                        void *stream) try {
  return op_metropolis(N, site0, kb, g, ld_g, s, lambda, seed, chain, sweep_pass, slice1, forced, alpha,
                       beta, accept_count, status, stream, true);
} DQ_API_CATCH

}  // extern "C"

template <typename T>
static dqmc_status op_flush(int N, int site0, int kb, T *G, const T *Gcol, const T *Grow,
                            const double *alpha, const double *beta, const int *accept_count,
                            bool df, void *stream) {
  if (N < 1 || kb < 1 || kb > 64 || site0 < 0 || site0 + kb > N)
    return fail(DQMC_EINVAL, "need 1 <= kb <= 64 and 0 <= site0, site0 + kb <= N");
  if (!G || !Gcol || !Grow || !alpha || !beta || !accept_count) return fail(DQMC_EINVAL, "null pointer");
  int K = 4;
  while (K < kb) K <<= 1;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // scratch for the N x K factor A (and, double-float, the K x N factor B), stream-ordered
  void *Abuf = nullptr;
  DQ_CUDA(cudaMallocAsync(&Abuf, (size_t)N * K * 8 * (df ? 2 : 1), st));
  FlushArgs a{N, site0, kb, 0, 0, 0, kb, kb, kb};
  cudaError_t e = launch_flush<T>(K, a, G, Gcol, Grow, alpha, beta, accept_count, Abuf, nullptr,
                                  nullptr, df, st);
  cudaError_t e2 = cudaFreeAsync(Abuf, st);
  if (e != cudaSuccess) return cuda_fail(e, "flush");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
  return DQMC_OK;
}

extern "C" {

dqmc_status dqmc_op_flush_f64(int N, int site0, int kb, double *G, const double *Gcol,
                              const double *Grow, const double *alpha, const double *beta,
                              const int *accept_count, void *stream) try {
  return op_flush<double>(N, site0, kb, G, Gcol, Grow, alpha, beta, accept_count, false, stream);
} DQ_API_CATCH

dqmc_status dqmc_op_flush_df(int N, int site0, int kb, double *G, const double *Gcol,
                             const double *Grow, const double *alpha, const double *beta,
                             const int *accept_count, void *stream) try {
  return op_flush<double>(N, site0, kb, G, Gcol, Grow, alpha, beta, accept_count, true, stream);
} DQ_API_CATCH

dqmc_status dqmc_op_flush_f32(int N, int site0, int kb, float *G, const float *Gcol,
                              const float *Grow, const double *alpha, const double *beta,
                              const int *accept_count, void *stream) try {
  return op_flush<float>(N, site0, kb, G, Gcol, Grow, alpha, beta, accept_count, false, stream);
} DQ_API_CATCH

dqmc_status dqmc_op_flush_tc(int N, int site0, int kb, double *G, const double *Gcol,
                             const double *Grow, const double *alpha, const double *beta,
                             const int *accept_count, void *stream) try {
  if (N < 1 || kb < 1 || kb > 32 || site0 < 0 || site0 + kb > N)
    return fail(DQMC_EINVAL, "need 1 <= kb <= 32 and 0 <= site0, site0 + kb <= N");
  if (!G || !Gcol || !Grow || !alpha || !beta || !accept_count) return fail(DQMC_EINVAL, "null pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t wb = flush_tc_workspace_bytes(N);
  void *ws = nullptr;
  DQ_CUDA(cudaMallocAsync(&ws, wb, st));
  FlushArgs a{N, site0, kb, 0, 0, 0, kb, kb, kb};
  cudaError_t e = cudaMemsetAsync(ws, 0, wb, st);
  if (e == cudaSuccess) e = launch_flush_tc(a, G, Gcol, Grow, alpha, beta, accept_count, ws, nullptr, nullptr, st);
  const cudaError_t e2 = cudaFreeAsync(ws, st);
  if (e != cudaSuccess) return cuda_fail(e, "flush_tc");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
  if (flush_tc_timed_out(st)) return fail(DQMC_ETIMEOUT, "a bounded wait of the tcgen05 flush gave up");
  return DQMC_OK;
} DQ_API_CATCH

dqmc_status dqmc_op_gemm_f64(int mode, int ta, int tb, int M, int N, int K, double alpha,
                             const double *A, int lda, const double *B, int ldb, double beta,
                             double *C, int ldc, void *stream) try {
  if (mode < 0 || mode > 3)
    return fail(DQMC_EINVAL, "mode must be 0 (FP64), 1 (double-float), 2 (digit slices, mma.sync) or 3 "
                             "(digit slices, tcgen05)");
  if (M < 0 || N < 0 || K < 0) return fail(DQMC_EINVAL, "negative size");
  if ((M && N && K) && (!A || !B)) return fail(DQMC_EINVAL, "null operand");
  if (M && N && !C) return fail(DQMC_EINVAL, "null C");
  if (lda < (ta ? M : K) || ldb < (tb ? K : N) || ldc < N) return fail(DQMC_EINVAL, "leading dimension too small");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void *ws = nullptr;
  int *ex = nullptr;
  double *sk = nullptr;
  cudaError_t e = cudaSuccess;
  DQ_CUDA(cudaMallocAsync((void **)&sk, splitk_ws_doubles() * sizeof(double), st));
  set_splitk_workspace(sk, splitk_ws_doubles());
  if (mode == 1) {
    DQ_CUDA(cudaMallocAsync(&ws, ((size_t)M * K + (size_t)K * N + 1) * sizeof(float2), st));
    set_df_workspace(static_cast<float2 *>(ws), (size_t)M * K + (size_t)K * N + 1);
    e = dfgemm(ta != 0, tb != 0, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, nullptr, nullptr, st, 0, 304);
    set_df_workspace(nullptr, 0);
  } else if (mode == 2 || mode == 3) {
    const size_t bytes = oz_workspace_bytes(M, N, K) + 16;
    DQ_CUDA(cudaMallocAsync(&ws, bytes, st));
    DQ_CUDA(cudaMallocAsync((void **)&ex, ((size_t)M + N + 1) * sizeof(int), st));
    set_oz_workspace(ws, bytes, ex, (size_t)M + N + 1);
    set_gemm_oz_tc(mode == 3, true);
    e = ozgemm(ta != 0, tb != 0, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, nullptr, nullptr, st);
    set_gemm_oz_tc(false);
    set_oz_workspace(nullptr, 0, nullptr, 0);
  } else {
    e = dgemm(ta != 0, tb != 0, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, nullptr, nullptr, st);
  }
  set_splitk_workspace(nullptr, 0);
  cudaFreeAsync(sk, st);
  if (ws) cudaFreeAsync(ws, st);
  if (ex) cudaFreeAsync(ex, st);
  if (e != cudaSuccess) return cuda_fail(e, "gemm");
  return DQMC_OK;
} DQ_API_CATCH

dqmc_status dqmc_op_trial_state(int L, int n_occ, double eps, double *P_out) try {
  if (!supported_L(L)) return fail(DQMC_EINVAL, "unsupported L");
  const int N = 3 * L * L;
  if (n_occ < 1 || n_occ >= N) return fail(DQMC_EINVAL, "need 1 <= n_occ < N");
  if (!P_out) return fail(DQMC_EINVAL, "P_out is NULL");
  if (!std::isfinite(eps)) return fail(DQMC_EINVAL, "eps must be finite");
  std::vector<double> P;
  const int rc = trial_orbitals(L, n_occ, eps, 1.0, 1e-9, P);
  if (rc == 2) return fail(DQMC_EINVAL, "open shell: the lowest n_occ states are not separated by a gap");
  if (rc != 0) return fail(DQMC_EINVAL, "bad trial-state arguments");
  std::copy(P.begin(), P.end(), P_out);
  return DQMC_OK;
} DQ_API_CATCH

dqmc_status dqmc_op_measure(int L, const double *G, int site_offsets, double *out, void *stream) try {
  if (!supported_L(L)) return fail(DQMC_EINVAL, "unsupported L");
  if (!G || !out) return fail(DQMC_EINVAL, "null pointer");
  const int N = 3 * L * L;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // phase tables (same conventions as the context measurement)
  std::vector<double> h(6 * (size_t)N);
  std::vector<int> nb(4 * (size_t)N), fill(N, 0);
  const double two_pi = 6.283185307179586476925286766559;
  const double fA[3][2] = {{0.0, 0.0}, {0.0, -0.5}, {-0.5, 0.0}};
  const bool haveK = (L % 3 == 0);
  const int km1 = L / 3, km2 = 2 * L / 3;
  for (int x1 = 0; x1 < L; ++x1)
    for (int x2 = 0; x2 < L; ++x2)
      for (int a = 0; a < 3; ++a) {
        const int i = (x1 * L + x2) * 3 + a;
        const double f1 = x1 + (site_offsets ? fA[a][0] : 0.0);
        const double th = two_pi * ((double)(1 % L) * f1 / L);
        const double pa = two_pi * a / 3.0;
        const double pk = two_pi * ((double)((km1 * x1 + km2 * x2) % L) / L) + pa;
        h[i] = std::cos(th);
        h[N + i] = std::sin(th);
        h[2 * N + i] = std::cos(pa);
        h[3 * N + i] = std::sin(pa);
        h[4 * N + i] = std::cos(pk);
        h[5 * N + i] = std::sin(pk);
      }
  for (const Bond &bd : kKagomeBonds)
    for (int x1 = 0; x1 < L; ++x1)
      for (int x2 = 0; x2 < L; ++x2) {
        const int i = (x1 * L + x2) * 3 + bd.a;
        const int y1 = ((x1 + bd.d1) % L + L) % L, y2 = ((x2 + bd.d2) % L + L) % L;
        const int j = (y1 * L + y2) * 3 + bd.b;
        nb[4 * (size_t)i + fill[i]++] = j;
        nb[4 * (size_t)j + fill[j]++] = i;
      }
  double *d = nullptr;
  int *dn = nullptr;
  DQ_CUDA(cudaMalloc(&d, (6 * (size_t)N + 16 + 8) * sizeof(double)));
  DQ_CUDA(cudaMalloc(&dn, 4 * (size_t)N * sizeof(int)));
  DQ_CUDA(cudaMemcpyAsync(d, h.data(), 6 * (size_t)N * sizeof(double), cudaMemcpyHostToDevice, st));
  DQ_CUDA(cudaMemcpyAsync(dn, nb.data(), 4 * (size_t)N * sizeof(int), cudaMemcpyHostToDevice, st));
  MeasTables t{d, d + N, d + 2 * N, d + 3 * N, haveK ? d + 4 * N : nullptr,
               haveK ? d + 5 * N : nullptr, dn};
  double *raw = d + 6 * (size_t)N, *obs = raw + 16;
  cudaError_t e = launch_measure(G, N, t, raw, 1.0, obs, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, obs, 6 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  cudaFree(dn);
  if (e != cudaSuccess) return cuda_fail(e, "dqmc_op_measure");
  return DQMC_OK;
} DQ_API_CATCH

}  // extern "C"
