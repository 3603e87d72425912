// DQMC chain engine and the C ABI of include/dqmc.h.
//
// The sweep is a fixed sequence of kernel launches on one stream; the host
// never waits inside a sweep. Per slice visit (up pass):
//   wrap   G <- e^{V} e^{-dtau K} G e^{+dtau K} e^{-V}     2 FFT propagator passes
//   update gather block 0; per block of k sites: Metropolis (1 CTA) + rank-k flush
//   stab   every n_stab slices: UDV stack update (FFT propagation of the
//          orthogonal factor in FP64, pre-pivoted Householder QR) and the
//          scale-separated recomputation of G; drift = max |G - G_fresh|
// The down pass runs the same steps in reverse order (update, then unwrap).
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <array>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <system_error>
#include <thread>
#include <vector>

#include "kernels.cuh"
#include "lattice_host.h"
#include "linalg.cuh"

namespace dq {

// ---------------------------------------------------------------- errors
static thread_local std::string g_last_error;
void set_error(const std::string &msg) { g_last_error = msg; }
dqmc_status fail(dqmc_status st, const std::string &msg) {
  set_error(msg);
  return st;
}
dqmc_status fail_host(dqmc_status st, const char *msg) noexcept {
  try {
    g_last_error = std::string("host: ") + msg;
  } catch (...) {
  }
  return st;
}
dqmc_status cuda_fail(cudaError_t e, const char *what) {
  return fail(DQMC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// ---------------------------------------------------------------- launch accounting
// per host thread: a context is driven by one thread at a time, so the
// difference of this counter around a call is that context's launches
static thread_local unsigned long long t_launches = 0;
static thread_local KTimerSink *t_sink = nullptr;
KTimerSink *&ktimer_sink() { return t_sink; }
void count_launch() { ++t_launches; }
unsigned long long launch_count() { return t_launches; }
static thread_local double t_flops[KF_COUNT] = {};
static thread_local double t_bytes[KF_COUNT] = {};
void add_work(int fam, double flops, double bytes) {
  t_flops[fam] += flops;
  t_bytes[fam] += bytes;
}
const double *work_flops() { return t_flops; }
const double *work_bytes() { return t_bytes; }

// ---------------------------------------------------------------- shared-memory opt-in
// cudaFuncSetAttribute is per device; remember (function, device) pairs.
static std::mutex g_attr_mu;
static std::map<std::pair<const void *, int>, int> g_attr;
cudaError_t ensure_smem_attr(const void *func, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_attr_mu);
  auto key = std::make_pair(func, dev);
  auto it = g_attr.find(key);
  if (it != g_attr.end() && it->second >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) g_attr[key] = bytes;
  return e;
}

// ---------------------------------------------------------------- small kernels
// e^{V_i} = e^{lambda s_i + dtau mu}: two values, computed on the host
__global__ void expv_kernel(const int8_t *s, int N, double vp, double vm, double *ev64,
                            double *evi64, float *ev32, float *evi32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double v = s[i] > 0 ? vp : vm;
  const double vi = s[i] > 0 ? 1.0 / vp : 1.0 / vm;
  ev64[i] = v;
  evi64[i] = vi;
  ev32[i] = (float)v;
  evi32[i] = (float)vi;
}

// initial field from Philox, domain 1: s = +1 iff the low bit of word 0 is set
__global__ void init_field_kernel(int8_t *s, int M, int N, uint32_t k0, uint32_t k1, uint32_t c3) {
  const long total = (long)M * N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int l = (int)(e / N), i = (int)(e % N);
    const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)l, 0u, c3), k0, k1);
    s[e] = (r.x & 1u) ? (int8_t)1 : (int8_t)-1;
  }
}

// ---------------------------------------------------------------- block table cache
struct TableKey {
  int dev, L, prec;
  uint64_t scale_bits;
  bool operator<(const TableKey &o) const {
    if (dev != o.dev) return dev < o.dev;
    if (L != o.L) return L < o.L;
    if (prec != o.prec) return prec < o.prec;
    return scale_bits < o.scale_bits;
  }
};
static std::mutex g_tab_mu;
static std::map<TableKey, void *> g_tables;

// Device table of e^{scale H(k)} / L^2 (half spectrum), FP64 (prec 0) or FP32 (prec 1).
static dqmc_status get_table(int L, double scale, int prec, const void **out) {
  int dev = 0;
  DQ_CUDA(cudaGetDevice(&dev));
  uint64_t bits;
  std::memcpy(&bits, &scale, sizeof(bits));
  TableKey key{dev, L, prec, bits};
  std::lock_guard<std::mutex> lk(g_tab_mu);
  auto it = g_tables.find(key);
  if (it != g_tables.end()) {
    *out = it->second;
    return DQMC_OK;
  }
  std::vector<cd> tab = block_exp_table(L, scale);
  void *d = nullptr;
  if (prec == 0) {
    std::vector<cpx<double>> h(tab.size());
    for (size_t q = 0; q < tab.size(); ++q) h[q] = cpx<double>{tab[q].real(), tab[q].imag()};
    DQ_CUDA(cudaMalloc(&d, h.size() * sizeof(cpx<double>)));
    DQ_CUDA(cudaMemcpy(d, h.data(), h.size() * sizeof(cpx<double>), cudaMemcpyHostToDevice));
  } else if (prec == 1) {
    std::vector<cpx<float>> h(tab.size());
    for (size_t q = 0; q < tab.size(); ++q)
      h[q] = cpx<float>{(float)tab[q].real(), (float)tab[q].imag()};
    DQ_CUDA(cudaMalloc(&d, h.size() * sizeof(cpx<float>)));
    DQ_CUDA(cudaMemcpy(d, h.data(), h.size() * sizeof(cpx<float>), cudaMemcpyHostToDevice));
  } else {
    std::vector<cpx<df64>> h(tab.size());
    for (size_t q = 0; q < tab.size(); ++q) h[q] = cpx<df64>{df64(tab[q].real()), df64(tab[q].imag())};
    DQ_CUDA(cudaMalloc(&d, h.size() * sizeof(cpx<df64>)));
    DQ_CUDA(cudaMemcpy(d, h.data(), h.size() * sizeof(cpx<df64>), cudaMemcpyHostToDevice));
  }
  g_tables[key] = d;
  *out = d;
  return DQMC_OK;
}

}  // namespace dq

using namespace dq;

// ---------------------------------------------------------------- context
static_assert(KF_COUNT == DQMC_KERNEL_FAMILIES, "dqmc_stats arrays follow the kernel families");

struct UDVd {
  double *U = nullptr, *D = nullptr, *T = nullptr;
};

struct dqmc_ctx {
  // parameters
  int L = 0, N = 0, M = 0;
  double beta = 0, dtau = 0, U = 0, mu = 0, thop = 1.0, lam = 0;
  uint64_t seed = 0;
  // options
  int k = 32, n_stab = 10, precision = 0, chain = 0, timing = 0, site_offsets = 1, bin = 10;
  double drift_limit = 1e-3;
  // runtime
  cudaStream_t stream = nullptr;
  bool own_stream = false;  // created by dqmc_batch_create, destroyed with the context
  void *(*ualloc)(size_t, void *) = nullptr;
  void (*ufree)(void *, void *) = nullptr;
  void *uuser = nullptr;
  std::vector<void *> allocs;
  int device = 0;
  bool allocated = false, ready = false, poisoned = false, started = false;
  int C = 0;
  std::vector<int> tau;
  int cur_slice = 0;
  // device buffers
  int8_t *field = nullptr;
  double *G64 = nullptr;  // working G (fp64 mode) / scratch fp64 copy (mixed)
  float *G32 = nullptr;   // working G (mixed)
  double *Gf = nullptr;   // fresh G
  const cpx<double> *E64m = nullptr, *E64p = nullptr;
  const cpx<float> *E32m = nullptr, *E32p = nullptr;
  const cpx<df64> *EDFm = nullptr, *EDFp = nullptr;
  std::vector<UDVd> right, left;
  UDVd tmpA, tmpB;                       // scratch UDVs for dqmc_green
  double *X = nullptr, *Xp = nullptr, *Tp = nullptr, *Dp = nullptr, *norms = nullptr;
  int *perm = nullptr;
  double *Mm = nullptr, *Bm = nullptr, *Z = nullptr;
  double *drmax_inv = nullptr, *drmin = nullptr, *dlmax_inv = nullptr, *dlmin = nullptr;
  QRWork qr;
  double *ev64 = nullptr, *evi64 = nullptr;
  float *ev32 = nullptr, *evi32 = nullptr;
  void *Gcol[2] = {nullptr, nullptr}, *Grow[2] = {nullptr, nullptr};
  double *coef_a = nullptr, *coef_b = nullptr;  // 2 x K x K alpha / beta vectors (block parity)
  double *gnext = nullptr;                      // K x K look-ahead G[S', S'] of the next block
  cudaStream_t side = nullptr;                  // Metropolis of the next block runs here
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  void *Abuf = nullptr;                       // N x K rank-m factor A (or its FP32 pairs)
  int df_flush = 1;   // mixed: rank-m flush as double-float product (else FP64)
  int df_prop = 0;    // mixed: FFT propagation in double-float arithmetic (default: FP64)
  int pipeline = 1;   // next block's Metropolis on the side stream beside the flush (0: one stream)
  int df_metro = 1;   // mixed: Metropolis decisions and Woodbury coefficients in double-float
  int metro_reserve = 200 * 1024;  // shared memory the look-ahead Metropolis claims (own SM)
  int stab_gemm = 2;  // mixed: stabilisation GEMMs 0 FP64, 1 double-float, 2 tensor-core digit slices
  int stab_qr = 0;    // 0 Householder QR, 1 CholeskyQR2, -1 = CholeskyQR2 in mixed precision only
  int tc_gemm = 1;    // mixed, digit slices: tcgen05 GEMM (else the mma.sync one)
  int flush_tc = 1;   // mixed, k = 32: rank-m flush as digit slices on tcgen05 (else double-float)
  int df_panel = 0;   // mixed: Householder panel column loop in double-float arithmetic
  int refl_gram = 1;  // mixed: Gram matrix of each block reflector (0 digit slices, 1 parallel FP64, 2 double-float)
  int refl_tw = 1;    // mixed: op(T) W of each block reflector (0 digit slices, 1 parallel FP64, 2 double-float)
  void *tcws = nullptr;  // its digit tiles and row exponents
  int *tcperm = nullptr;  // 2 x k: the accepted sites of a block (block parity), for the digit tiles
  bool cholqr = false;  // the sweep's stabilisation uses CholeskyQR2 (resolved at allocation)
  unsigned gemm_sites = 0xffffffffu;  // mixed: GEMM call sites (GemmSite bits) that use stab_gemm
  unsigned gemm_df_sites = 0u;        // mixed: of those, the sites that use double-float products
  void *ozws = nullptr;  // digit-slice workspace
  size_t ozws_bytes = 0;
  int *ozexp = nullptr;
  int *acc = nullptr, *status = nullptr;
  uint8_t *flip_flags = nullptr;  // dqmc_replay: M x N forced-flip flags, then the M x N target
  unsigned long long *total_acc = nullptr;
  double *drift = nullptr, *drift_max = nullptr;
  double *meas_raw = nullptr, *meas_obs = nullptr;  // obs: capacity meas_cap x 6
  int meas_cap = 0, meas_n = 0;
  double *ph_pc = nullptr, *ph_ps = nullptr, *ph_wgc = nullptr, *ph_wgs = nullptr,
         *ph_wkc = nullptr, *ph_wks = nullptr;
  int *nbr = nullptr;
  double *skws = nullptr;  // split-K partial products of the stabilisation GEMMs
  float2 *dfws = nullptr;  // double-float GEMM workspace (mixed precision)
  size_t dfws_elems = 0;
  bool haveK = false;
  bool reference_chain = false;  // dqmc_green: Householder QR after every slice, whatever the mode
  // host statistics
  long sweeps = 0, proposed = 0, accepted = 0;
  double max_drift = 0.0, last_drift = 0.0;
  std::vector<std::array<double, 6>> samples;
  double ms_wrap = 0, ms_update = 0, ms_stab = 0, ms_measure = 0;
  double ms_kernel[KF_COUNT] = {};
  long n_kernel[KF_COUNT] = {};
  double flops_kernel[KF_COUNT] = {};
  double bytes_kernel[KF_COUNT] = {};
  unsigned long long launches = 0;
};

namespace {

dqmc_status ctx_alloc(dqmc_ctx *c, void **p, size_t bytes) {
  void *q = nullptr;
  if (bytes == 0) bytes = 16;
  if (c->ualloc) {
    q = c->ualloc(bytes, c->uuser);
    if (!q) return fail(DQMC_ENOMEM, "allocator callback returned NULL");
  } else {
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) return fail(DQMC_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  c->allocs.push_back(q);
  *p = q;
  return DQMC_OK;
}
template <typename T> dqmc_status ctx_alloc_n(dqmc_ctx *c, T **p, size_t n) {
  void *q = nullptr;
  DQ_CHECK(ctx_alloc(c, &q, n * sizeof(T)));
  *p = static_cast<T *>(q);
  return DQMC_OK;
}

dqmc_status poison(dqmc_ctx *c, dqmc_status st) {
  if (st == DQMC_ECUDA || st == DQMC_ETIMEOUT) c->poisoned = true;
  return st;
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return poison(c, cuda_fail(_e, #call)); \
  } while (0)

bool valid_k(int k) { return k == 4 || k == 8 || k == 16 || k == 32 || k == 64; }

// ---------------------------------------------------------------- allocation
dqmc_status ensure_alloc(dqmc_ctx *c) {
  if (c->allocated) return DQMC_OK;
  CK(cudaGetDevice(&c->device));
  const int N = c->N, M = c->M;
  const size_t NN = (size_t)N * N;
  c->C = (M + c->n_stab - 1) / c->n_stab;
  c->tau.resize(c->C + 1);
  for (int q = 0; q <= c->C; ++q) c->tau[q] = std::min(q * c->n_stab, M);

  DQ_CHECK(ctx_alloc_n(c, &c->field, (size_t)M * N));
  DQ_CHECK(ctx_alloc_n(c, &c->G64, NN));
  DQ_CHECK(ctx_alloc_n(c, &c->Gf, NN));
  if (c->precision == 2) DQ_CHECK(ctx_alloc_n(c, &c->G32, NN));
  c->right.resize(c->C + 1);
  c->left.resize(c->C + 1);
  for (int q = 0; q <= c->C; ++q) {
    for (UDVd *u : {&c->right[q], &c->left[q]}) {
      DQ_CHECK(ctx_alloc_n(c, &u->U, NN));
      DQ_CHECK(ctx_alloc_n(c, &u->T, NN));
      DQ_CHECK(ctx_alloc_n(c, &u->D, (size_t)N));
    }
  }
  for (UDVd *u : {&c->tmpA, &c->tmpB}) {
    DQ_CHECK(ctx_alloc_n(c, &u->U, NN));
    DQ_CHECK(ctx_alloc_n(c, &u->T, NN));
    DQ_CHECK(ctx_alloc_n(c, &u->D, (size_t)N));
  }
  DQ_CHECK(ctx_alloc_n(c, &c->X, NN));
  DQ_CHECK(ctx_alloc_n(c, &c->Xp, NN));
  DQ_CHECK(ctx_alloc_n(c, &c->Tp, NN));
  DQ_CHECK(ctx_alloc_n(c, &c->Dp, (size_t)N));
  DQ_CHECK(ctx_alloc_n(c, &c->norms, (size_t)N));
  DQ_CHECK(ctx_alloc_n(c, &c->perm, (size_t)N));
  DQ_CHECK(ctx_alloc_n(c, &c->Mm, NN));
  DQ_CHECK(ctx_alloc_n(c, &c->Bm, NN));
  DQ_CHECK(ctx_alloc_n(c, &c->Z, NN));
  DQ_CHECK(ctx_alloc_n(c, &c->drmax_inv, (size_t)N));
  DQ_CHECK(ctx_alloc_n(c, &c->drmin, (size_t)N));
  DQ_CHECK(ctx_alloc_n(c, &c->dlmax_inv, (size_t)N));
  DQ_CHECK(ctx_alloc_n(c, &c->dlmin, (size_t)N));
  double *qrmem = nullptr;
  DQ_CHECK(ctx_alloc_n(c, &qrmem, qr_work_doubles(N)));
  qr_work_bind(c->qr, N, qrmem);
  CK(cudaMemsetAsync(qrmem, 0, qr_work_doubles(N) * sizeof(double), c->stream));
  DQ_CHECK(ctx_alloc_n(c, &c->ev64, (size_t)N));
  DQ_CHECK(ctx_alloc_n(c, &c->evi64, (size_t)N));
  DQ_CHECK(ctx_alloc_n(c, &c->ev32, (size_t)N));
  DQ_CHECK(ctx_alloc_n(c, &c->evi32, (size_t)N));
  DQ_CHECK(ctx_alloc_n(c, &c->skws, splitk_ws_doubles()));
  c->cholqr = c->stab_qr == 1 || (c->stab_qr < 0 && c->precision == 1);
  if (c->precision == 1 && (c->stab_gemm == 1 || c->gemm_df_sites != 0)) {
    // split operands of the double-float GEMMs: at most M*K + K*N = 2 N^2 pairs
    c->dfws_elems = 2 * NN;
    DQ_CHECK(ctx_alloc_n(c, &c->dfws, c->dfws_elems));
  }
  if (c->precision == 1 && c->stab_gemm == 2) {
    c->ozws_bytes = oz_workspace_bytes(N, N, N);
    DQ_CHECK(ctx_alloc(c, &c->ozws, c->ozws_bytes));
    DQ_CHECK(ctx_alloc_n(c, &c->ozexp, 2 * (size_t)N));
  }
  const size_t es = c->precision == 2 ? sizeof(float) : sizeof(double);
  for (int b = 0; b < 2; ++b) {
    DQ_CHECK(ctx_alloc(c, &c->Gcol[b], (size_t)N * c->k * es));
    DQ_CHECK(ctx_alloc(c, &c->Grow[b], (size_t)N * c->k * es));
    CK(cudaMemsetAsync(c->Gcol[b], 0, (size_t)N * c->k * es, c->stream));
    CK(cudaMemsetAsync(c->Grow[b], 0, (size_t)N * c->k * es, c->stream));
  }
  DQ_CHECK(ctx_alloc_n(c, &c->coef_a, 2 * (size_t)c->k * c->k));
  DQ_CHECK(ctx_alloc_n(c, &c->coef_b, 2 * (size_t)c->k * c->k));
  DQ_CHECK(ctx_alloc_n(c, &c->gnext, (size_t)c->k * c->k));
  if (!c->side) {
    // highest priority: the serial Metropolis block is the critical path, its
    // CTA should take the first SM that the concurrent flush frees
    int prio_lo = 0, prio_hi = 0;
    CK(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
    CK(cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_hi));
    CK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  }
  DQ_CHECK(ctx_alloc(c, &c->Abuf, 2 * (size_t)N * c->k * sizeof(double)));
  if (c->precision == 1 && c->df_flush && c->flush_tc && c->k == 32) {
    // digit tiles: rows beyond N are never written and must stay zero
    const size_t b = flush_tc_workspace_bytes(N);
    DQ_CHECK(ctx_alloc(c, &c->tcws, b));
    CK(cudaMemsetAsync(c->tcws, 0, b, c->stream));
    DQ_CHECK(ctx_alloc_n(c, &c->tcperm, 2 * (size_t)c->k));
  }
  DQ_CHECK(ctx_alloc_n(c, &c->acc, 4));
  DQ_CHECK(ctx_alloc_n(c, &c->status, 4));
  DQ_CHECK(ctx_alloc_n(c, &c->total_acc, 1));
  DQ_CHECK(ctx_alloc_n(c, &c->drift, 1));
  DQ_CHECK(ctx_alloc_n(c, &c->drift_max, 1));
  DQ_CHECK(ctx_alloc_n(c, &c->meas_raw, 16));
  CK(cudaMemsetAsync(c->status, 0, 4 * sizeof(int), c->stream));
  CK(cudaMemsetAsync(c->total_acc, 0, sizeof(unsigned long long), c->stream));
  CK(cudaMemsetAsync(c->drift_max, 0, sizeof(double), c->stream));

  // tables
  const void *t = nullptr;
  DQ_CHECK(get_table(c->L, -c->dtau, 0, &t));
  c->E64m = static_cast<const cpx<double> *>(t);
  DQ_CHECK(get_table(c->L, c->dtau, 0, &t));
  c->E64p = static_cast<const cpx<double> *>(t);
  DQ_CHECK(get_table(c->L, -c->dtau, 1, &t));
  c->E32m = static_cast<const cpx<float> *>(t);
  DQ_CHECK(get_table(c->L, c->dtau, 1, &t));
  c->E32p = static_cast<const cpx<float> *>(t);
  DQ_CHECK(get_table(c->L, -c->dtau, 2, &t));
  c->EDFm = static_cast<const cpx<df64> *>(t);
  DQ_CHECK(get_table(c->L, c->dtau, 2, &t));
  c->EDFp = static_cast<const cpx<df64> *>(t);

  // measurement phases
  const int L = c->L;
  std::vector<double> pc(N), ps(N), wgc(N), wgs(N), wkc(N), wks(N);
  std::vector<int> nb(4 * (size_t)N);
  const double two_pi = 6.283185307179586476925286766559;
  const double fA[3][2] = {{0.0, 0.0}, {0.0, -0.5}, {-0.5, 0.0}};  // tau_a in units of a1, a2
  c->haveK = (L % 3 == 0);
  const int km1 = L / 3, km2 = 2 * L / 3;  // Dirac point K where the dispersive bands touch
  std::vector<int> fill(N, 0);
  for (int x1 = 0; x1 < L; ++x1)
    for (int x2 = 0; x2 < L; ++x2)
      for (int a = 0; a < 3; ++a) {
        const int i = (x1 * L + x2) * 3 + a;
        double f1 = x1, f2 = x2;
        if (c->site_offsets) {
          f1 += fA[a][0];
          f2 += fA[a][1];
        }
        const double th = two_pi * ((double)(1 % L) * f1 / L);  // Gamma + dk = (1, 0)
        pc[i] = std::cos(th);
        ps[i] = std::sin(th);
        const double pa = two_pi * a / 3.0;
        wgc[i] = std::cos(pa);
        wgs[i] = std::sin(pa);
        const double pk = two_pi * ((double)((km1 * x1 + km2 * x2) % std::max(L, 1)) / L) + pa;
        wkc[i] = std::cos(pk);
        wks[i] = std::sin(pk);
      }
  for (const Bond &bd : kKagomeBonds) {
    for (int x1 = 0; x1 < L; ++x1)
      for (int x2 = 0; x2 < L; ++x2) {
        const int i = (x1 * L + x2) * 3 + bd.a;
        const int y1 = ((x1 + bd.d1) % L + L) % L, y2 = ((x2 + bd.d2) % L + L) % L;
        const int j = (y1 * L + y2) * 3 + bd.b;
        nb[4 * (size_t)i + fill[i]++] = j;
        nb[4 * (size_t)j + fill[j]++] = i;
      }
  }
  DQ_CHECK(ctx_alloc_n(c, &c->ph_pc, (size_t)N));
  DQ_CHECK(ctx_alloc_n(c, &c->ph_ps, (size_t)N));
  DQ_CHECK(ctx_alloc_n(c, &c->ph_wgc, (size_t)N));
  DQ_CHECK(ctx_alloc_n(c, &c->ph_wgs, (size_t)N));
  DQ_CHECK(ctx_alloc_n(c, &c->ph_wkc, (size_t)N));
  DQ_CHECK(ctx_alloc_n(c, &c->ph_wks, (size_t)N));
  DQ_CHECK(ctx_alloc_n(c, &c->nbr, 4 * (size_t)N));
  CK(cudaMemcpyAsync(c->ph_pc, pc.data(), N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->ph_ps, ps.data(), N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->ph_wgc, wgc.data(), N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->ph_wgs, wgs.data(), N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->ph_wkc, wkc.data(), N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->ph_wks, wks.data(), N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->nbr, nb.data(), 4 * (size_t)N * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));

  // initial field
  const uint32_t k0 = (uint32_t)(c->seed & 0xffffffffu), k1 = (uint32_t)(c->seed >> 32);
  const uint32_t c3 = ((uint32_t)c->chain & 0xffffffu) | (kDomainInit << 24);
  DQ_KSCOPE(KF_OTHER, c->stream);
  init_field_kernel<<<256, 256, 0, c->stream>>>(c->field, M, N, k0, k1, c3);
  CK(cudaGetLastError());
  c->allocated = true;
  return DQMC_OK;
}

// ---------------------------------------------------------------- propagation helpers
dqmc_status compute_expv(dqmc_ctx *c, int l) {
  const double vp = std::exp(c->lam + c->dtau * c->mu), vm = std::exp(-c->lam + c->dtau * c->mu);
  DQ_KSCOPE(KF_OTHER, c->stream);
  expv_kernel<<<(c->N + 255) / 256, 256, 0, c->stream>>>(c->field + (size_t)(l - 1) * c->N, c->N,
                                                         vp, vm, c->ev64, c->evi64, c->ev32,
                                                         c->evi32);
  CK(cudaGetLastError());
  return DQMC_OK;
}

// e^{sign dtau K} on an FP64 N x N operand in place (side 0: X <- E X,
// side 1: X <- X E), in FP64 or, in mixed precision, double-float arithmetic
cudaError_t prop64(dqmc_ctx *c, int side, int sign, double *X, const double *pre,
                   const double *post, const double *vscale) {
  const int N = c->N;
  if (c->precision == 1 && c->df_prop)
    return launch_prop_df(c->L, side, X, X, N, N, sign < 0 ? c->EDFm : c->EDFp, pre, post, vscale,
                          c->stream);
  return launch_prop_f64(c->L, side, X, X, N, N, sign < 0 ? c->E64m : c->E64p, pre, post, vscale,
                         c->stream);
}

// G <- e^{V} e^{-dtau K} G e^{+dtau K} e^{-V}
dqmc_status wrap(dqmc_ctx *c, int l) {
  DQ_CHECK(compute_expv(c, l));
  const int N = c->N;
  if (c->precision != 2) {
    CK(prop64(c, 0, -1, c->G64, nullptr, nullptr, nullptr));
    CK(prop64(c, 1, +1, c->G64, nullptr, c->evi64, c->ev64));
  } else {
    CK(launch_prop_f32(c->L, 0, c->G32, c->G32, N, N, c->E32m, nullptr, nullptr, nullptr, c->stream));
    CK(launch_prop_f32(c->L, 1, c->G32, c->G32, N, N, c->E32p, nullptr, c->evi32, c->ev32, c->stream));
  }
  return DQMC_OK;
}

// G <- e^{+dtau K} e^{-V} G e^{V} e^{-dtau K}
dqmc_status unwrap(dqmc_ctx *c, int l) {
  DQ_CHECK(compute_expv(c, l));
  const int N = c->N;
  if (c->precision != 2) {
    CK(prop64(c, 0, +1, c->G64, c->evi64, nullptr, c->ev64));
    CK(prop64(c, 1, -1, c->G64, nullptr, nullptr, nullptr));
  } else {
    CK(launch_prop_f32(c->L, 0, c->G32, c->G32, N, N, c->E32p, c->evi32, nullptr, c->ev32, c->stream));
    CK(launch_prop_f32(c->L, 1, c->G32, c->G32, N, N, c->E32m, nullptr, nullptr, nullptr, c->stream));
  }
  return DQMC_OK;
}

// ---------------------------------------------------------------- delayed update of one slice
// The blocks of one slice, pipelined over two streams. On the context's
// stream: A = G[:, S_b] alpha_b^T, the look-ahead G'[S_{b+1}, S_{b+1}], then
// the rank-m flush of block b (which also gathers the rows / columns of
// block b+1). On the side stream, between the look-ahead and the next A
// kernel: the Metropolis block b+1, so that its serial decisions overlap the
// flush of block b. Coefficients alternate between two buffers by block parity.
template <typename T>
dqmc_status update_slice_t(dqmc_ctx *c, T *G, int l, int pas, const uint8_t *forced) {
  const int N = c->N, K = c->k;
  const int nblk = (N + K - 1) / K;
  const size_t KK = (size_t)K * K;
  T *Gc[2] = {static_cast<T *>(c->Gcol[0]), static_cast<T *>(c->Gcol[1])};
  T *Gr[2] = {static_cast<T *>(c->Grow[0]), static_cast<T *>(c->Grow[1])};
  const bool df = (c->precision == 1 && c->df_flush);
  CK(launch_gather<T>(N, 0, std::min(K, N), K, G, Gc[0], Gr[0], c->stream));
  const bool dfm = (c->precision == 1 && c->df_metro);
  MetroArgs ma;
  ma.N = N;
  ma.K = K;
  ma.e2l = std::exp(2.0 * c->lam);
  ma.em2l = std::exp(-2.0 * c->lam);
  ma.k0 = (uint32_t)(c->seed & 0xffffffffu);
  ma.k1 = (uint32_t)(c->seed >> 32);
  ma.c2 = (uint32_t)(2 * c->sweeps + pas);
  ma.c3 = ((uint32_t)c->chain & 0xffffffu) | (kDomainMetropolis << 24);
  ma.slice0 = l - 1;
  int8_t *s = c->field + (size_t)(l - 1) * N;
  if constexpr (std::is_same<T, double>::value) {
    if (df && c->tcws && K == 32) {
      // tensor-core flush. Per block on the context's stream: the digit
      // tiles (whose warps for the next block's rows of A also form the
      // look-ahead G'[S', S'] from the pre-flush G), then the flush, which
      // gathers the next block's rows and columns; the next block's
      // Metropolis runs on the side stream between the digit tiles and the
      // next block's, beside the flush.
      ma.s0 = 0;
      ma.kb = std::min(K, N);
      ma.ld_g = N;
      ma.perm = c->tcperm;
      CK(launch_metropolis(ma, Gr[0], false, s, forced, c->coef_a, c->coef_b, c->acc, c->status, c->total_acc,
                           c->stream, dfm));
      for (int b = 0; b < nblk; ++b) {
        const int s0 = b * K, kb = std::min(K, N - s0);
        const int par = b & 1;
        double *al = c->coef_a + par * KK, *be = c->coef_b + par * KK;
        int *acc = c->acc + par;
        FlushArgs fa;
        fa.N = N;
        fa.s0 = s0;
        fa.kb = kb;
        fa.ns0 = (b + 1 < nblk) ? s0 + K : 0;
        fa.nkb = (b + 1 < nblk) ? std::min(K, N - s0 - K) : 0;
        fa.rows_per_cta = 0;
        fa.ldc = K;
        fa.ldb = K;
        fa.lda = K;
        // the digit tiles, and the next block's G'[S', S'] from the pre-flush G
        CK(launch_flush_tc_prep(fa, Gc[par], Gr[par], al, be, acc, c->tcws, nullptr, c->stream, c->tcperm + par * K, G,
                                fa.nkb > 0 ? c->gnext : nullptr));
        if (fa.nkb > 0) {
          cudaStream_t ms = c->stream;
          if (c->pipeline) {
            CK(cudaEventRecord(c->ev_fork, c->stream));
            CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
            ms = c->side;
          }
          MetroArgs mn = ma;
          mn.s0 = fa.ns0;
          mn.kb = fa.nkb;
          mn.ld_g = fa.nkb;
          mn.perm = c->tcperm + (par ^ 1) * K;
          CK(launch_metropolis(mn, c->gnext, false, s, forced ? forced + fa.ns0 : nullptr,
                               c->coef_a + (par ^ 1) * KK, c->coef_b + (par ^ 1) * KK, c->acc + (par ^ 1),
                               c->status, c->total_acc, ms, dfm));
          if (c->pipeline) CK(cudaEventRecord(c->ev_join, c->side));
        }
        CK(launch_flush_tc_update(fa, G, acc, c->tcws, Gc[par ^ 1], Gr[par ^ 1], c->stream));
        if (fa.nkb > 0 && c->pipeline) CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
      }
      c->proposed += N;
      return DQMC_OK;
    }
  }
  // block 0: decisions on the context's stream from the gathered rows
  ma.s0 = 0;
  ma.kb = std::min(K, N);
  ma.ld_g = N;
  CK(launch_metropolis(ma, Gr[0], sizeof(T) == 4, s, forced, c->coef_a, c->coef_b, c->acc,
                       c->status, c->total_acc, c->stream, dfm));
  for (int b = 0; b < nblk; ++b) {
    const int s0 = b * K, kb = std::min(K, N - s0);
    const int par = b & 1;
    double *al = c->coef_a + par * KK, *be = c->coef_b + par * KK;
    int *acc = c->acc + par;
    FlushArgs fa;
    fa.N = N;
    fa.s0 = s0;
    fa.kb = kb;
    fa.ns0 = (b + 1 < nblk) ? s0 + K : 0;
    fa.nkb = (b + 1 < nblk) ? std::min(K, N - s0 - K) : 0;
    fa.rows_per_cta = 0;
    fa.ldc = K;
    fa.ldb = K;
    fa.lda = K;
    CK(launch_amat<T>(K, fa, Gc[par], Gr[par], al, be, acc, c->Abuf, df, c->stream));
    if (fa.nkb > 0) {
      CK(launch_lookahead_g<T>(K, fa, G, c->Abuf, df, Gr[par], be, acc, c->gnext, c->stream));
      // pipelined: the next block's Metropolis on the side stream, beside the
      // flush; single-stream (pipeline = 0): before the flush on this stream
      cudaStream_t ms = c->stream;
      if (c->pipeline) {
        CK(cudaEventRecord(c->ev_fork, c->stream));
        CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
        ms = c->side;
      }
      MetroArgs mn = ma;
      mn.s0 = fa.ns0;
      mn.kb = fa.nkb;
      mn.ld_g = fa.nkb;
      CK(launch_metropolis(mn, c->gnext, false, s, forced ? forced + fa.ns0 : nullptr,
                           c->coef_a + (par ^ 1) * KK, c->coef_b + (par ^ 1) * KK, c->acc + (par ^ 1),
                           c->status, c->total_acc, ms, dfm, c->pipeline ? c->metro_reserve : 0));
      if (c->pipeline) CK(cudaEventRecord(c->ev_join, c->side));
    }
    CK(launch_flush_update<T>(K, fa, G, c->Abuf, Gr[par], be, acc, Gc[par ^ 1], Gr[par ^ 1], df,
                              c->stream));
    if (fa.nkb > 0 && c->pipeline) CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
  }
  c->proposed += N;
  return DQMC_OK;
}

// forced != NULL (N flags of slice l): site i flips iff forced[i] != 0
dqmc_status update_slice(dqmc_ctx *c, int l, int pas, const uint8_t *forced = nullptr) {
  return c->precision != 2 ? update_slice_t<double>(c, c->G64, l, pas, forced)
                           : update_slice_t<float>(c, c->G32, l, pas, forced);
}

// ---------------------------------------------------------------- UDV stacks (FP64)
// dst = (chunk) src, chunk = B_{l1} ... B_{l0} (right, l0 < l1) applied as
// X <- e^{V} e^{-dtau K} X, or B_{l0}^T ... B_{l1}^T (transposed left form)
// applied as X <- e^{-dtau K} e^{V} X, slices visited in the given order.
dqmc_status udv_advance(dqmc_ctx *c, const UDVd &src, UDVd &dst, const std::vector<int> &slices,
                        bool transposed) {
  const int N = c->N;
  const size_t NN = (size_t)N * N;
  CK(cudaMemcpyAsync(c->X, src.U, NN * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  for (int l : slices) {
    DQ_CHECK(compute_expv(c, l));
    if (!transposed)
      CK(prop64(c, 0, -1, c->X, nullptr, c->ev64, nullptr));
    else
      CK(prop64(c, 0, -1, c->X, c->ev64, nullptr, nullptr));
  }
  // pre-pivoting: columns ordered by ||X_j|| D_j, descending
  CK(column_norms_scaled(c->X, N, src.D, c->norms, c->stream));
  CK(argsort_desc(c->norms, N, c->perm, c->stream));
  CK(permute_udv(c->X, src.D, src.T, c->perm, N, c->Xp, c->Dp, c->Tp, c->stream));
  if (c->cholqr && !c->reference_chain) {
    // Xp = U R by CholeskyQR2: U to dst.U, R to Mm (scratch X, Z, Bm and the
    // QR workspace's V), then R'' = diag(D_new)^{-1} R diag(Dp), T_new = R'' P^T T_old
    set_gemm_site(GS_CHOLQR);
    CK(cholqr2(c->Xp, N, dst.U, c->Mm, c->X, c->Z, c->Bm, c->qr.V, c->status + 1, c->stream));
    CK(udv_diag_and_scale(c->Mm, N, c->Dp, dst.D, c->stream));
    set_gemm_site(GS_T_UPDATE);
    CK(dgemm(false, false, N, N, N, 1.0, c->Mm, N, c->Tp, N, 0.0, dst.T, N, nullptr, nullptr, c->stream));
    return DQMC_OK;
  }
  set_gemm_site(GS_QR_UPDATE);
  CK(qr_factor(c->Xp, N, c->qr, c->stream));
  set_gemm_site(GS_FORM_Q);
  CK(qr_form_q(dst.U, N, c->qr, c->stream));
  CK(udv_diag_and_scale(c->Xp, N, c->Dp, dst.D, c->stream));
  // T_new = R'' (P^T T_old)
  set_gemm_site(GS_T_UPDATE);
  CK(dgemm(false, false, N, N, N, 1.0, c->Xp, N, c->Tp, N, 0.0, dst.T, N, nullptr, nullptr, c->stream));
  return DQMC_OK;
}

dqmc_status udv_identity(dqmc_ctx *c, UDVd &u) {
  CK(set_identity(u.U, c->N, c->N, c->stream));
  CK(set_identity(u.T, c->N, c->N, c->stream));
  CK(set_value(u.D, c->N, 1.0, c->stream));
  return DQMC_OK;
}

// G_fresh = (I + B(tau,0) B(beta,tau))^{-1} from right = B(tau,0) = U_r D_r T_r and
// left = B(beta,tau)^T = U' D_l T' by the scale-separated inversion:
//   G = U' Dlmax^{-1} [Drmax^{-1} U_r^T U' Dlmax^{-1} + Drmin T_r T'^T Dlmin]^{-1} Drmax^{-1} U_r^T
dqmc_status combine(dqmc_ctx *c, const UDVd &r, const UDVd &lf, double *Gout) {
  const int N = c->N;
  CK(split_scales(r.D, N, c->drmax_inv, c->drmin, c->stream));
  CK(split_scales(lf.D, N, c->dlmax_inv, c->dlmin, c->stream));
  set_gemm_site(GS_UU);
  CK(dgemm(true, false, N, N, N, 1.0, r.U, N, lf.U, N, 0.0, c->Mm, N, c->drmax_inv, c->dlmax_inv, c->stream));
  set_gemm_site(GS_TT);
  CK(dgemm(false, true, N, N, N, 1.0, r.T, N, lf.T, N, 1.0, c->Mm, N, c->drmin, c->dlmin, c->stream));
  CK(transpose_scale(r.U, N, c->Bm, N, c->drmax_inv, c->stream));
  if (c->cholqr && !c->reference_chain) {
    // M^{-1} B by shifted CholeskyQR3 of M (Fukaya, Kannan, Nakatsukasa,
    // Yamamoto, Yanagisawa 2020): a first pass on M^T M + s I, s = 11 (n^2 +
    // n (n + 1)) u tr(M^T M), keeps the Cholesky factorisation defined up to
    // cond(M) ~ 1/u (the scale-separated matrix of a random field reaches
    // 1e7 - 1e8 here), then CholeskyQR2 of the result: M = Q R, R = R2 R1 R0,
    // Z = R0^{-1} R1^{-1} R2^{-1} Q^T B.
    const double shift = 11.0 * (2.0 * (double)N * N + N) * 0x1p-53;
    set_gemm_site(GS_CHOLQR);
    CK(dgemm(true, false, N, N, N, 1.0, c->Mm, N, c->Mm, N, 0.0, c->Z, N, nullptr, nullptr, c->stream));
    CK(shift_diag(c->Z, N, N, shift, c->stream));
    CK(chol_inv(c->Z, N, c->X, N, c->Xp, N, N, c->status + 1, c->stream));               // R0^{-1} -> X
    CK(dgemm(false, false, N, N, N, 1.0, c->Mm, N, c->X, N, 0.0, c->Tp, N, nullptr, nullptr, c->stream));   // Q0
    CK(dgemm(true, false, N, N, N, 1.0, c->Tp, N, c->Tp, N, 0.0, c->Z, N, nullptr, nullptr, c->stream));
    CK(chol_inv(c->Z, N, c->Xp, N, c->Mm, N, N, c->status + 1, c->stream));              // R1^{-1} -> Xp
    CK(dgemm(false, false, N, N, N, 1.0, c->Tp, N, c->Xp, N, 0.0, c->Mm, N, nullptr, nullptr, c->stream));  // Q1
    CK(dgemm(false, false, N, N, N, 1.0, c->X, N, c->Xp, N, 0.0, c->Tp, N, nullptr, nullptr, c->stream));   // R0^{-1} R1^{-1}
    CK(dgemm(true, false, N, N, N, 1.0, c->Mm, N, c->Mm, N, 0.0, c->Z, N, nullptr, nullptr, c->stream));
    CK(chol_inv(c->Z, N, c->Xp, N, c->X, N, N, c->status + 1, c->stream));               // R2^{-1} -> Xp
    CK(dgemm(false, false, N, N, N, 1.0, c->Mm, N, c->Xp, N, 0.0, c->X, N, nullptr, nullptr, c->stream));   // Q
    CK(dgemm(false, false, N, N, N, 1.0, c->Tp, N, c->Xp, N, 0.0, c->Mm, N, nullptr, nullptr, c->stream));  // R^{-1}
    CK(dgemm(true, false, N, N, N, 1.0, c->X, N, c->Bm, N, 0.0, c->Tp, N, nullptr, nullptr, c->stream));    // Q^T B
    CK(dgemm(false, false, N, N, N, 1.0, c->Mm, N, c->Tp, N, 0.0, c->Z, N, nullptr, nullptr, c->stream));
  } else {
    set_gemm_site(GS_QRM);
    CK(qr_factor(c->Mm, N, c->qr, c->stream));
    set_gemm_site(GS_APPLY_QT);
    CK(qr_apply_qt(c->Bm, N, N, N, c->qr, c->stream));
    set_gemm_site(GS_TRSM);
    CK(qr_solve_r(c->Mm, N, c->Bm, c->Z, N, c->qr, c->stream));
  }
  CK(scale_rows_cols(c->Z, N, N, c->dlmax_inv, nullptr, c->stream));
  set_gemm_site(GS_FINAL);
  CK(dgemm(false, false, N, N, N, 1.0, lf.U, N, c->Z, N, 0.0, Gout, N, nullptr, nullptr, c->stream));
  return DQMC_OK;
}

// replace the running G by G_fresh(stack c), recording the drift
dqmc_status refresh(dqmc_ctx *c, int q, bool record_drift) {
  const int N = c->N;
  DQ_CHECK(combine(c, c->right[q], c->left[q], c->Gf));
  if (c->precision != 2) {
    if (record_drift) CK(max_abs_diff_f64(c->Gf, c->G64, N, c->drift, c->stream));
    CK(cudaMemcpyAsync(c->G64, c->Gf, (size_t)N * N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  } else {
    if (record_drift) CK(max_abs_diff_f32(c->Gf, c->G32, N, c->drift, c->stream));
    CK(convert_f64_to_f32(c->Gf, c->G32, (long)N * N, c->stream));
  }
  return DQMC_OK;
}

// flags[q] = 1 where the current spin differs from the target spin
__global__ void flip_flags_kernel(const int8_t *field, const int8_t *target, long n, uint8_t *flags) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x)
    flags[q] = field[q] != target[q] ? 1 : 0;
}

// *flag = 1 if the two fields differ anywhere (flag cleared by the caller)
__global__ void field_differs_kernel(const int8_t *a, const int8_t *b, long n, int *flag) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x)
    if (a[q] != b[q]) {
      *flag = 1;
      break;
    }
}

__global__ void drift_max_kernel(const double *d, double *mx) {
  const double v = *d;
  if (v != v || v > *mx) *mx = v;
}

// In mixed precision the stabilisation GEMMs of the sweep run FP64-accurate
// on faster units: digit slices on the bf16 tensor cores (default) or
// double-float products on the FP32 units.
struct GemmModeScope {
  explicit GemmModeScope(dqmc_ctx *c) {
    set_splitk_workspace(c->skws, splitk_ws_doubles());
    if (c->precision != 1) return;
    set_qr_panel_df(c->df_panel != 0);
    set_reflector_modes(c->refl_gram, c->refl_tw);
    if (c->stab_gemm == 1 && c->dfws) {
      set_df_workspace(c->dfws, c->dfws_elems);
      set_gemm_df(true);
    } else if (c->stab_gemm == 2 && c->ozws) {
      set_oz_workspace(c->ozws, c->ozws_bytes, c->ozexp, 2 * (size_t)c->N);
      set_gemm_oz(true);
      set_gemm_oz_tc(c->tc_gemm != 0);
      if (c->gemm_df_sites && c->dfws) {
        set_df_workspace(c->dfws, c->dfws_elems);
        set_gemm_df(true);
      }
    }
    set_gemm_site_mask(c->gemm_sites);
    set_gemm_df_site_mask(c->stab_gemm == 2 ? c->gemm_df_sites : 0u);
  }
  ~GemmModeScope() {
    set_splitk_workspace(nullptr, 0);
    set_qr_panel_df(false);
    set_reflector_modes(0, 0);
    set_gemm_df(false);
    set_gemm_oz(false);
    set_gemm_oz_tc(false);
    set_gemm_df_site_mask(0u);
  }
};

dqmc_status ensure_ready(dqmc_ctx *c) {
  DQ_CHECK(ensure_alloc(c));
  if (c->ready) return DQMC_OK;
  GemmModeScope gm(c);
  DQ_CHECK(udv_identity(c, c->left[c->C]));
  for (int q = c->C - 1; q >= 0; --q) {
    std::vector<int> sl;
    for (int l = c->tau[q + 1]; l > c->tau[q]; --l) sl.push_back(l);
    DQ_CHECK(udv_advance(c, c->left[q + 1], c->left[q], sl, true));
  }
  DQ_CHECK(udv_identity(c, c->right[0]));
  DQ_CHECK(refresh(c, 0, false));
  c->cur_slice = 0;
  c->ready = true;
  CK(cudaStreamSynchronize(c->stream));
  return DQMC_OK;
}

dqmc_status measure_now(dqmc_ctx *c) {
  if (c->meas_n >= c->meas_cap) {
    // grow: keep old contents
    const int cap = std::max(64, 2 * c->meas_cap);
    double *nb = nullptr;
    DQ_CHECK(ctx_alloc_n(c, &nb, (size_t)cap * 6));
    if (c->meas_obs && c->meas_n)
      CK(cudaMemcpyAsync(nb, c->meas_obs, (size_t)c->meas_n * 6 * sizeof(double),
                         cudaMemcpyDeviceToDevice, c->stream));
    c->meas_obs = nb;
    c->meas_cap = cap;
  }
  MeasTables t{c->ph_pc, c->ph_ps, c->ph_wgc, c->ph_wgs, c->haveK ? c->ph_wkc : nullptr,
               c->haveK ? c->ph_wks : nullptr, c->nbr};
  CK(launch_measure(c->Gf, c->N, t, c->meas_raw, c->thop, c->meas_obs + (size_t)c->meas_n * 6, c->stream));
  c->meas_n++;
  return DQMC_OK;
}

// Per-phase events (timing >= 1) and, as the thread's kernel sink, per-launch
// events grouped by kernel family (timing == 2). Also attributes the launches
// issued while it lives to the context.
struct PhaseTimer : KTimerSink {
  dqmc_ctx *c;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[4];
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> kev[KF_COUNT];
  std::vector<cudaEvent_t> open[KF_COUNT];
  unsigned long long launches0;
  double f0[KF_COUNT], b0[KF_COUNT];
  KTimerSink *prev;
  explicit PhaseTimer(dqmc_ctx *cc) : c(cc), launches0(launch_count()), prev(ktimer_sink()) {
    if (c->timing >= 2) ktimer_sink() = this;
    for (int f = 0; f < KF_COUNT; ++f) {
      f0[f] = work_flops()[f];
      b0[f] = work_bytes()[f];
    }
  }
  ~PhaseTimer() override {
    ktimer_sink() = prev;
    c->launches += launch_count() - launches0;
    for (int f = 0; f < KF_COUNT; ++f) {
      c->flops_kernel[f] += work_flops()[f] - f0[f];
      c->bytes_kernel[f] += work_bytes()[f] - b0[f];
    }
    if (c->timing) {
      cudaStreamSynchronize(c->stream);
      collect();
    }
  }
  void begin(int fam, cudaStream_t st) override {
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, st);
    open[fam].push_back(e);
  }
  void end(int fam, cudaStream_t st) override {
    if (open[fam].empty()) return;
    cudaEvent_t s = open[fam].back(), e;
    open[fam].pop_back();
    cudaEventCreate(&e);
    cudaEventRecord(e, st);
    kev[fam].push_back({s, e});
  }
  void start(int ph, cudaEvent_t *e) {
    if (!c->timing) return;
    cudaEventCreate(e);
    cudaEventRecord(*e, c->stream);
    (void)ph;
  }
  void stop(int ph, cudaEvent_t s) {
    if (!c->timing) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, c->stream);
    ev[ph].push_back({s, e});
  }
  void collect() {
    double *acc[4] = {&c->ms_wrap, &c->ms_update, &c->ms_stab, &c->ms_measure};
    for (int ph = 0; ph < 4; ++ph) {
      for (auto &p : ev[ph]) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p.first, p.second);
        *acc[ph] += ms;
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
      }
      ev[ph].clear();
    }
    for (int f = 0; f < KF_COUNT; ++f) {
      for (auto &p : kev[f]) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p.first, p.second);
        c->ms_kernel[f] += ms;
        c->n_kernel[f] += 1;
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
      }
      kev[f].clear();
    }
  }
};

dqmc_status one_sweep(dqmc_ctx *c, bool measure, PhaseTimer &tm) {
  GemmModeScope gm(c);
  int q = 1;
  cudaEvent_t e0 = nullptr;
  for (int l = 1; l <= c->M; ++l) {
    tm.start(0, &e0);
    DQ_CHECK(wrap(c, l));
    tm.stop(0, e0);
    tm.start(1, &e0);
    DQ_CHECK(update_slice(c, l, 0));
    tm.stop(1, e0);
    c->cur_slice = l;
    if (l == c->tau[q]) {
      tm.start(2, &e0);
      std::vector<int> sl;
      for (int m = c->tau[q - 1] + 1; m <= c->tau[q]; ++m) sl.push_back(m);
      DQ_CHECK(udv_advance(c, c->right[q - 1], c->right[q], sl, false));
      DQ_CHECK(refresh(c, q, true));
      DQ_KSCOPE(KF_OTHER, c->stream);
      drift_max_kernel<<<1, 1, 0, c->stream>>>(c->drift, c->drift_max);
      tm.stop(2, e0);
      if (measure) {
        tm.start(3, &e0);
        DQ_CHECK(measure_now(c));
        tm.stop(3, e0);
      }
      ++q;
    }
  }
  q = c->C - 1;
  for (int l = c->M; l >= 1; --l) {
    tm.start(1, &e0);
    DQ_CHECK(update_slice(c, l, 1));
    tm.stop(1, e0);
    tm.start(0, &e0);
    DQ_CHECK(unwrap(c, l));
    tm.stop(0, e0);
    c->cur_slice = l - 1;
    if (q >= 0 && l - 1 == c->tau[q]) {
      tm.start(2, &e0);
      std::vector<int> sl;
      for (int m = c->tau[q + 1]; m > c->tau[q]; --m) sl.push_back(m);
      DQ_CHECK(udv_advance(c, c->left[q + 1], c->left[q], sl, true));
      DQ_CHECK(refresh(c, q, true));
      DQ_KSCOPE(KF_OTHER, c->stream);
      drift_max_kernel<<<1, 1, 0, c->stream>>>(c->drift, c->drift_max);
      tm.stop(2, e0);
      --q;
    }
  }
  c->sweeps++;
  return DQMC_OK;
}

dqmc_status check_ctx(dqmc_ctx *c) {
  if (!c) return fail(DQMC_EINVAL, "null context");
  if (c->poisoned) return fail(DQMC_ESTATE, "context is unusable after an earlier CUDA failure");
  return DQMC_OK;
}

dqmc_status read_status(dqmc_ctx *c) {
  int st[4] = {0, 0, 0, 0};
  CK(cudaMemcpyAsync(st, c->status, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
  unsigned long long tot = 0;
  CK(cudaMemcpyAsync(&tot, c->total_acc, sizeof(tot), cudaMemcpyDeviceToHost, c->stream));
  double dm = 0.0;
  CK(cudaMemcpyAsync(&dm, c->drift_max, sizeof(dm), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->accepted = (long)tot;
  c->last_drift = dm;
  c->max_drift = std::max(c->max_drift, dm);
  if (c->precision == 1 && c->stab_gemm == 2 && c->tc_gemm && oz_tc_timed_out(c->stream))
    return poison(c, fail(DQMC_ETIMEOUT, "a bounded wait of the tcgen05 GEMM gave up"));
  if (c->tcws && flush_tc_timed_out(c->stream))
    return poison(c, fail(DQMC_ETIMEOUT, "a bounded wait of the tcgen05 flush gave up"));
  if (st[0] != 0) return fail(DQMC_ENUMERIC, "non-positive or non-finite acceptance ratio");
  if (st[1] != 0)
    return fail(DQMC_ENUMERIC, "non-positive pivot in the Cholesky factorisation of the CholeskyQR2 "
                               "stabilisation (set stab_qr = 0 for Householder QR)");
  if (!(dm <= c->drift_limit)) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "stabilisation drift %.3e above the limit %.3e", dm, c->drift_limit);
    return fail(DQMC_ENUMERIC, buf);
  }
  return DQMC_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

const char *dqmc_version(void) { return "dqmc-gb300 0.1 (sm_103a)"; }

const char *dqmc_last_error(void) { return g_last_error.c_str(); }

dqmc_status dqmc_create(int L, double beta, double dtau, double U, double mu, uint64_t seed,
                        dqmc_ctx **out) try {
  if (!out) return fail(DQMC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!supported_L(L)) return fail(DQMC_EINVAL, "unsupported L (supported: 1,2,3,4,6,8,12,16,24,36)");
  if (!(dtau > 0.0) || !(beta > 0.0)) return fail(DQMC_EINVAL, "beta and dtau must be positive");
  const double Mr = beta / dtau;
  if (std::fabs(Mr - std::round(Mr)) > 1e-9 || std::round(Mr) < 1)
    return fail(DQMC_EINVAL, "beta / dtau must be a positive integer");
  if (!(U <= 0.0)) return fail(DQMC_EINVAL, "U must be <= 0 (attractive, paper's sign)");
  if (!std::isfinite(mu)) return fail(DQMC_EINVAL, "mu must be finite");
  dqmc_ctx *c = new (std::nothrow) dqmc_ctx();
  if (!c) return fail(DQMC_ENOMEM, "host allocation failed");
  c->L = L;
  c->N = 3 * L * L;
  c->M = (int)std::lround(Mr);
  c->beta = beta;
  c->dtau = dtau;
  c->U = U;
  c->mu = mu;
  c->seed = seed;
  c->lam = std::acosh(std::exp(dtau * std::fabs(U) / 2.0));
  if (c->N < c->k) c->k = 4;
  *out = c;
  return DQMC_OK;
} DQ_API_CATCH

dqmc_status dqmc_set_option(dqmc_ctx *c, const char *key, double v) try {
  DQ_CHECK(check_ctx(c));
  if (!key) return fail(DQMC_EINVAL, "key is NULL");
  const std::string k(key);
  const bool fixed = (k == "k" || k == "n_stab" || k == "precision" || k == "chain");
  if (fixed && c->allocated) return fail(DQMC_ESTATE, "option '" + k + "' is fixed after the first sweep");
  if (k == "k") {
    if (!valid_k((int)v) || (double)(int)v != v) return fail(DQMC_EINVAL, "k must be one of 4, 8, 16, 32, 64");
    c->k = (int)v;
  } else if (k == "n_stab") {
    if (v < 1 || (double)(int)v != v) return fail(DQMC_EINVAL, "n_stab must be a positive integer");
    c->n_stab = (int)v;
  } else if (k == "precision") {
    if (v != 0.0 && v != 1.0 && v != 2.0)
      return fail(DQMC_EINVAL, "precision must be 0 (fp64), 1 (mixed) or 2 (fp32)");
    c->precision = (int)v;
  } else if (k == "chain") {
    if (v < 0 || v > 0xffffff || (double)(int)v != v) return fail(DQMC_EINVAL, "chain must be in [0, 2^24)");
    c->chain = (int)v;
  } else if (k == "timing") {
    if (v != 0.0 && v != 1.0 && v != 2.0) return fail(DQMC_EINVAL, "timing must be 0, 1 or 2");
    c->timing = (int)v;
  } else if (k == "site_offsets") {
    c->site_offsets = v != 0.0;
  } else if (k == "bin") {
    if (v < 1) return fail(DQMC_EINVAL, "bin must be >= 1");
    c->bin = (int)v;
  } else if (k == "df_flush") {
    if (c->allocated) return fail(DQMC_ESTATE, "option '" + k + "' is fixed after the first sweep");
    c->df_flush = v != 0.0;
  } else if (k == "metro_reserve") {
    if (v < 0 || v > 224 * 1024) return fail(DQMC_EINVAL, "metro_reserve must be in [0, 229376] bytes");
    c->metro_reserve = (int)v;
  } else if (k == "df_metro") {
    if (c->allocated) return fail(DQMC_ESTATE, "option '" + k + "' is fixed after the first sweep");
    c->df_metro = v != 0.0;
  } else if (k == "df_prop") {
    if (c->allocated) return fail(DQMC_ESTATE, "option '" + k + "' is fixed after the first sweep");
    c->df_prop = v != 0.0;
  } else if (k == "gemm_sites") {
    if (v < 0 || v > 4294967295.0) return fail(DQMC_EINVAL, "gemm_sites is a 32-bit mask");
    c->gemm_sites = (unsigned)v;
  } else if (k == "gemm_df_sites") {
    if (c->allocated) return fail(DQMC_ESTATE, "option '" + k + "' is fixed after the first sweep");
    if (v < 0 || v > 4294967295.0) return fail(DQMC_EINVAL, "gemm_df_sites is a 32-bit mask");
    c->gemm_df_sites = (unsigned)v;
  } else if (k == "stab_gemm") {
    if (c->allocated) return fail(DQMC_ESTATE, "option '" + k + "' is fixed after the first sweep");
    if (v != 0.0 && v != 1.0 && v != 2.0) return fail(DQMC_EINVAL, "stab_gemm must be 0, 1 or 2");
    c->stab_gemm = (int)v;
  } else if (k == "tc_gemm") {
    c->tc_gemm = v != 0.0;
  } else if (k == "df_panel") {
    c->df_panel = v != 0.0;
  } else if (k == "refl_gram") {
    if (v != 0.0 && v != 1.0 && v != 2.0) return fail(DQMC_EINVAL, "refl_gram must be 0, 1 or 2");
    c->refl_gram = (int)v;
  } else if (k == "refl_tw") {
    if (v != 0.0 && v != 1.0 && v != 2.0) return fail(DQMC_EINVAL, "refl_tw must be 0, 1 or 2");
    c->refl_tw = (int)v;
  } else if (k == "flush_tc") {
    if (c->allocated) return fail(DQMC_ESTATE, "option '" + k + "' is fixed after the first sweep");
    c->flush_tc = v != 0.0;
  } else if (k == "stab_qr") {
    if (c->allocated) return fail(DQMC_ESTATE, "option '" + k + "' is fixed after the first sweep");
    if (v != 0.0 && v != 1.0 && v != -1.0) return fail(DQMC_EINVAL, "stab_qr must be -1 (auto), 0 or 1");
    c->stab_qr = (int)v;
  } else if (k == "pipeline") {
    c->pipeline = v != 0.0;
  } else if (k == "drift_limit") {
    if (!(v > 0.0)) return fail(DQMC_EINVAL, "drift_limit must be positive");
    c->drift_limit = v;
  } else {
    return fail(DQMC_EINVAL, "unknown option '" + k + "'");
  }
  return DQMC_OK;
} DQ_API_CATCH

dqmc_status dqmc_set_stream(dqmc_ctx *c, void *stream) try {
  DQ_CHECK(check_ctx(c));
  c->stream = static_cast<cudaStream_t>(stream);
  return DQMC_OK;
} DQ_API_CATCH

dqmc_status dqmc_set_allocator(dqmc_ctx *c, void *(*alloc)(size_t, void *),
                               void (*release)(void *, void *), void *user) try {
  DQ_CHECK(check_ctx(c));
  if (c->allocated) return fail(DQMC_ESTATE, "allocator must be set before the first allocation");
  if ((alloc == nullptr) != (release == nullptr)) return fail(DQMC_EINVAL, "alloc and release go together");
  c->ualloc = alloc;
  c->ufree = release;
  c->uuser = user;
  return DQMC_OK;
} DQ_API_CATCH

dqmc_status dqmc_sweep(dqmc_ctx *c, int n_sweeps, int measure) try {
  DQ_CHECK(check_ctx(c));
  if (n_sweeps < 0) return fail(DQMC_EINVAL, "n_sweeps must be >= 0");
  DQ_CHECK(ensure_ready(c));
  PhaseTimer tm(c);
  for (int s = 0; s < n_sweeps; ++s) {
    CK(cudaMemsetAsync(c->drift_max, 0, sizeof(double), c->stream));
    dqmc_status st = one_sweep(c, measure != 0, tm);
    if (st != DQMC_OK) return st;
    st = read_status(c);
    if (st != DQMC_OK) return st;
    tm.collect();
  }
  if (measure && c->meas_n > 0) {
    std::vector<double> h((size_t)c->meas_n * 6);
    CK(cudaMemcpyAsync(h.data(), c->meas_obs, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int q = 0; q < c->meas_n; ++q) {
      std::array<double, 6> a;
      for (int j = 0; j < 6; ++j) a[j] = h[(size_t)q * 6 + j];
      c->samples.push_back(a);
    }
    c->meas_n = 0;
  }
  return DQMC_OK;
} DQ_API_CATCH

dqmc_status dqmc_green(dqmc_ctx *c, int slice, double *G_out) try {
  DQ_CHECK(check_ctx(c));
  if (!G_out) return fail(DQMC_EINVAL, "G_out is NULL");
  if (slice < 0 || slice > c->M) return fail(DQMC_EINVAL, "slice out of range");
  PhaseTimer tm(c);
  DQ_CHECK(ensure_ready(c));
  struct SplitKScope {
    explicit SplitKScope(dqmc_ctx *cc) { set_splitk_workspace(cc->skws, splitk_ws_doubles()); }
    ~SplitKScope() { set_splitk_workspace(nullptr, 0); }
  } sk(c);
  struct RefScope {
    dqmc_ctx *cc;
    explicit RefScope(dqmc_ctx *x) : cc(x) { cc->reference_chain = true; }
    ~RefScope() { cc->reference_chain = false; }
  } ref(c);
  // right chain B(slice, 0) in tmpA, left chain B(beta, slice)^T in tmpB, QR every n_stab slices
  DQ_CHECK(udv_identity(c, c->tmpA));
  // reference-quality chains: a pivoted QR after every slice
  for (int l0 = 0; l0 < slice; ++l0) {
    std::vector<int> sl{l0 + 1};
    DQ_CHECK(udv_advance(c, c->tmpA, c->tmpA, sl, false));
  }
  DQ_CHECK(udv_identity(c, c->tmpB));
  for (int l1 = c->M; l1 > slice; --l1) {
    std::vector<int> sl{l1};
    DQ_CHECK(udv_advance(c, c->tmpB, c->tmpB, sl, true));
  }
  DQ_CHECK(combine(c, c->tmpA, c->tmpB, c->Xp));
  CK(cudaMemcpyAsync(G_out, c->Xp, (size_t)c->N * c->N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return DQMC_OK;
} DQ_API_CATCH

dqmc_status dqmc_get_running_green(dqmc_ctx *c, double *G_out, int *slice) try {
  DQ_CHECK(check_ctx(c));
  if (!G_out) return fail(DQMC_EINVAL, "G_out is NULL");
  PhaseTimer tm(c);
  DQ_CHECK(ensure_ready(c));
  const size_t NN = (size_t)c->N * c->N;
  if (c->precision != 2) {
    CK(cudaMemcpyAsync(G_out, c->G64, NN * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  } else {
    CK(convert_f32_to_f64(c->G32, c->X, (long)NN, c->stream));
    CK(cudaMemcpyAsync(G_out, c->X, NN * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  if (slice) *slice = c->cur_slice;
  return DQMC_OK;
} DQ_API_CATCH

dqmc_status dqmc_measure(dqmc_ctx *c, dqmc_obs *o) try {
  DQ_CHECK(check_ctx(c));
  if (!o) return fail(DQMC_EINVAL, "out is NULL");
  std::memset(o, 0, sizeof(*o));
  const long n = (long)c->samples.size();
  o->n_samples = n;
  const int bs = std::max(1, c->bin);
  const long nb = n / bs;
  o->n_bins = nb;
  double mean[6] = {0, 0, 0, 0, 0, 0};
  for (const auto &a : c->samples)
    for (int j = 0; j < 6; ++j) mean[j] += a[j];
  for (int j = 0; j < 6; ++j) mean[j] = n ? mean[j] / n : std::nan("");
  o->S_pair_G = mean[0];
  o->S_pair_dk = mean[1];
  o->phi2_G = mean[2];
  o->phi2_K = mean[3];
  o->density = mean[4];
  o->ekin = mean[5];
  std::vector<std::array<double, 6>> bins(nb);
  for (long b = 0; b < nb; ++b) {
    for (int j = 0; j < 6; ++j) {
      double s = 0;
      for (int q = 0; q < bs; ++q) s += c->samples[b * bs + q][j];
      bins[b][j] = s / bs;
    }
  }
  for (int j = 0; j < 6; ++j) {
    if (nb < 2) {
      o->err[j] = std::nan("");
      continue;
    }
    double m = 0, v = 0;
    for (long b = 0; b < nb; ++b) m += bins[b][j];
    m /= nb;
    for (long b = 0; b < nb; ++b) v += (bins[b][j] - m) * (bins[b][j] - m);
    o->err[j] = std::sqrt(v / (nb - 1) / nb);
  }
  // jackknife over bins for R_pair and P
  const double N = c->N;
  auto Rf = [&](double sG, double sdk) { return 1.0 - sdk / sG; };
  auto Pf = [&](double sG) { return std::sqrt(sG / N); };
  o->R_pair = Rf(mean[0], mean[1]);
  o->P = Pf(mean[0]);
  o->D_G = std::sqrt(mean[2]);
  o->D_K = std::sqrt(mean[3]);
  if (nb >= 2) {
    double tot0 = 0, tot1 = 0;
    for (long b = 0; b < nb; ++b) {
      tot0 += bins[b][0];
      tot1 += bins[b][1];
    }
    std::vector<double> jr(nb), jp(nb);
    double mr = 0, mp = 0;
    for (long b = 0; b < nb; ++b) {
      const double s0 = (tot0 - bins[b][0]) / (nb - 1), s1 = (tot1 - bins[b][1]) / (nb - 1);
      jr[b] = Rf(s0, s1);
      jp[b] = Pf(s0);
      mr += jr[b];
      mp += jp[b];
    }
    mr /= nb;
    mp /= nb;
    double vr = 0, vp = 0;
    for (long b = 0; b < nb; ++b) {
      vr += (jr[b] - mr) * (jr[b] - mr);
      vp += (jp[b] - mp) * (jp[b] - mp);
    }
    o->R_pair_err = std::sqrt((nb - 1.0) / nb * vr);
    o->P_err = std::sqrt((nb - 1.0) / nb * vp);
  } else {
    o->R_pair_err = std::nan("");
    o->P_err = std::nan("");
  }
  return DQMC_OK;
} DQ_API_CATCH

dqmc_status dqmc_get_stats(dqmc_ctx *c, dqmc_stats *o) try {
  if (!c) return fail(DQMC_EINVAL, "null context");
  if (!o) return fail(DQMC_EINVAL, "out is NULL");
  o->sweeps = c->sweeps;
  o->proposed = c->proposed;
  o->accepted = c->accepted;
  o->max_drift = c->max_drift;
  o->last_drift = c->last_drift;
  o->ms_wrap = c->ms_wrap;
  o->ms_update = c->ms_update;
  o->ms_stab = c->ms_stab;
  o->ms_measure = c->ms_measure;
  for (int f = 0; f < KF_COUNT; ++f) {
    o->ms_kernel[f] = c->ms_kernel[f];
    o->n_kernel[f] = c->n_kernel[f];
    o->flops_kernel[f] = c->flops_kernel[f];
    o->bytes_kernel[f] = c->bytes_kernel[f];
  }
  o->launches = c->launches;
  return DQMC_OK;
} DQ_API_CATCH

dqmc_status dqmc_get_field(dqmc_ctx *c, int8_t *s_out) try {
  DQ_CHECK(check_ctx(c));
  if (!s_out) return fail(DQMC_EINVAL, "s_out is NULL");
  DQ_CHECK(ensure_alloc(c));
  CK(cudaMemcpyAsync(s_out, c->field, (size_t)c->M * c->N, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return DQMC_OK;
} DQ_API_CATCH

dqmc_status dqmc_set_field(dqmc_ctx *c, const int8_t *s) try {
  DQ_CHECK(check_ctx(c));
  if (!s) return fail(DQMC_EINVAL, "s is NULL");
  const size_t n = (size_t)c->M * c->N;
  for (size_t q = 0; q < n; ++q)
    if (s[q] != 1 && s[q] != -1) return fail(DQMC_EINVAL, "field values must be +1 or -1");
  PhaseTimer tm(c);
  DQ_CHECK(ensure_alloc(c));
  if (c->ready && c->cur_slice == 0) {
    // Setting the state the chain is already in changes nothing: G and the
    // UDV stacks stay valid. The new field is staged on the device and
    // compared there; only a different field is installed and rebuilt from.
    if (!c->flip_flags) DQ_CHECK(ctx_alloc_n(c, &c->flip_flags, 2 * n));
    int8_t *stage = reinterpret_cast<int8_t *>(c->flip_flags + n);
    CK(cudaMemcpyAsync(stage, s, n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(c->status + 3, 0, sizeof(int), c->stream));
    {
      DQ_KSCOPE(KF_OTHER, c->stream);
      const int grid = (int)std::min<long>(4096, ((long)n + 255) / 256);
      field_differs_kernel<<<grid, 256, 0, c->stream>>>(c->field, stage, (long)n, c->status + 3);
      CK(cudaGetLastError());
    }
    int differs = 1;
    CK(cudaMemcpyAsync(&differs, c->status + 3, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (!differs) return DQMC_OK;
    CK(cudaMemcpyAsync(c->field, stage, n, cudaMemcpyDeviceToDevice, c->stream));
  } else {
    CK(cudaMemcpyAsync(c->field, s, n, cudaMemcpyHostToDevice, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  c->ready = false;
  return ensure_ready(c);
} DQ_API_CATCH

dqmc_status dqmc_replay(dqmc_ctx *c, const int8_t *target, int slice, double *G_out) try {
  DQ_CHECK(check_ctx(c));
  if (!target || !G_out) return fail(DQMC_EINVAL, "target and G_out must not be NULL");
  if (slice < 1 || slice > c->M) return fail(DQMC_EINVAL, "slice must be in [1, M]");
  const int N = c->N;
  const size_t n = (size_t)c->M * N;
  for (size_t q = 0; q < n; ++q)
    if (target[q] != 1 && target[q] != -1) return fail(DQMC_EINVAL, "field values must be +1 or -1");
  PhaseTimer tm(c);
  DQ_CHECK(ensure_ready(c));
  if (c->cur_slice != 0) return fail(DQMC_ESTATE, "replay starts at slice 0");
  if (!c->flip_flags) DQ_CHECK(ctx_alloc_n(c, &c->flip_flags, 2 * n));
  int8_t *tgt = reinterpret_cast<int8_t *>(c->flip_flags + n);
  CK(cudaMemcpyAsync(tgt, target, n, cudaMemcpyHostToDevice, c->stream));
  {
    DQ_KSCOPE(KF_OTHER, c->stream);
    const int grid = (int)std::min<long>(4096, ((long)n + 255) / 256);
    flip_flags_kernel<<<grid, 256, 0, c->stream>>>(c->field, tgt, (long)n, c->flip_flags);
    CK(cudaGetLastError());
  }
  GemmModeScope gm(c);
  int q = 1;
  for (int l = 1; l <= slice; ++l) {
    DQ_CHECK(wrap(c, l));
    DQ_CHECK(update_slice(c, l, 0, c->flip_flags + (size_t)(l - 1) * N));
    c->cur_slice = l;
    if (l == slice) break;
    if (l == c->tau[q]) {
      std::vector<int> sl;
      for (int m = c->tau[q - 1] + 1; m <= c->tau[q]; ++m) sl.push_back(m);
      DQ_CHECK(udv_advance(c, c->right[q - 1], c->right[q], sl, false));
      DQ_CHECK(refresh(c, q, true));
      DQ_KSCOPE(KF_OTHER, c->stream);
      drift_max_kernel<<<1, 1, 0, c->stream>>>(c->drift, c->drift_max);
      ++q;
    }
  }
  const size_t NN = (size_t)N * N;
  if (c->precision != 2) {
    CK(cudaMemcpyAsync(G_out, c->G64, NN * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  } else {
    CK(convert_f32_to_f64(c->G32, c->X, (long)NN, c->stream));
    CK(cudaMemcpyAsync(G_out, c->X, NN * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  // the stacks no longer describe the field: the next call rebuilds them
  c->ready = false;
  c->cur_slice = 0;
  return read_status(c);
} DQ_API_CATCH

dqmc_status dqmc_save(dqmc_ctx *c, const char *path) try {
  DQ_CHECK(check_ctx(c));
  if (!path) return fail(DQMC_EINVAL, "path is NULL");
  DQ_CHECK(ensure_alloc(c));
  std::vector<int8_t> f((size_t)c->M * c->N);
  CK(cudaMemcpyAsync(f.data(), c->field, f.size(), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  FILE *fp = std::fopen(path, "wb");
  if (!fp) return fail(DQMC_EINVAL, std::string("cannot open ") + path);
  const char magic[8] = {'D', 'Q', 'M', 'C', 'G', 'B', '3', '1'};
  double par[5] = {(double)c->L, c->beta, c->dtau, c->U, c->mu};
  int opt[7] = {c->k, c->n_stab, c->precision, c->chain, c->site_offsets, c->bin, 0};
  long st[3] = {c->sweeps, c->proposed, c->accepted};
  long ns = (long)c->samples.size();
  bool ok = std::fwrite(magic, 1, 8, fp) == 8 && std::fwrite(par, sizeof(double), 5, fp) == 5 &&
            std::fwrite(&c->seed, sizeof(uint64_t), 1, fp) == 1 &&
            std::fwrite(opt, sizeof(int), 7, fp) == 7 && std::fwrite(st, sizeof(long), 3, fp) == 3 &&
            std::fwrite(&c->max_drift, sizeof(double), 1, fp) == 1 &&
            std::fwrite(f.data(), 1, f.size(), fp) == f.size() &&
            std::fwrite(&ns, sizeof(long), 1, fp) == 1;
  for (long q = 0; ok && q < ns; ++q) ok = std::fwrite(c->samples[q].data(), sizeof(double), 6, fp) == 6;
  std::fclose(fp);
  if (!ok) return fail(DQMC_EINVAL, "short write");
  return DQMC_OK;
} DQ_API_CATCH

dqmc_status dqmc_load(dqmc_ctx *c, const char *path) try {
  DQ_CHECK(check_ctx(c));
  if (!path) return fail(DQMC_EINVAL, "path is NULL");
  FILE *fp = std::fopen(path, "rb");
  if (!fp) return fail(DQMC_EINVAL, std::string("cannot open ") + path);
  char magic[8];
  double par[5];
  uint64_t seed;
  int opt[7];
  long st[3], ns = 0;
  double md;
  bool ok = std::fread(magic, 1, 8, fp) == 8 && std::memcmp(magic, "DQMCGB31", 8) == 0 &&
            std::fread(par, sizeof(double), 5, fp) == 5 && std::fread(&seed, sizeof(uint64_t), 1, fp) == 1 &&
            std::fread(opt, sizeof(int), 7, fp) == 7 && std::fread(st, sizeof(long), 3, fp) == 3 &&
            std::fread(&md, sizeof(double), 1, fp) == 1;
  if (!ok) {
    std::fclose(fp);
    return fail(DQMC_EINVAL, "not a checkpoint file");
  }
  if ((int)par[0] != c->L || par[1] != c->beta || par[2] != c->dtau || par[3] != c->U || par[4] != c->mu) {
    std::fclose(fp);
    return fail(DQMC_EINVAL, "checkpoint parameters do not match this context");
  }
  // a damaged file must not reach the allocator or the kernels
  if (!valid_k(opt[0]) || opt[1] < 1 || opt[2] < 0 || opt[2] > 2 || opt[3] < 0 || opt[3] > 0xffffff ||
      opt[5] < 1 || st[0] < 0 || st[1] < 0 || st[2] < 0 || st[2] > st[1] || !(md >= 0.0)) {
    std::fclose(fp);
    return fail(DQMC_EINVAL, "corrupt checkpoint header");
  }
  if (c->allocated && (opt[0] != c->k || opt[1] != c->n_stab || opt[2] != c->precision || opt[3] != c->chain)) {
    std::fclose(fp);
    return fail(DQMC_ESTATE, "checkpoint options differ from an already started context");
  }
  std::vector<int8_t> f((size_t)c->M * c->N);
  ok = std::fread(f.data(), 1, f.size(), fp) == f.size() && std::fread(&ns, sizeof(long), 1, fp) == 1;
  // the samples must be exactly what is left of the file
  if (ok) {
    const long pos = std::ftell(fp);
    ok = pos >= 0 && std::fseek(fp, 0, SEEK_END) == 0;
    const long end = ok ? std::ftell(fp) : -1;
    ok = ok && end >= pos && ns >= 0 && ns <= (end - pos) / (long)(6 * sizeof(double)) &&
         (end - pos) == ns * (long)(6 * sizeof(double)) && std::fseek(fp, pos, SEEK_SET) == 0;
  }
  std::vector<std::array<double, 6>> smp(ok ? (size_t)ns : 0);
  for (long q = 0; ok && q < ns; ++q) ok = std::fread(smp[q].data(), sizeof(double), 6, fp) == 6;
  std::fclose(fp);
  if (!ok) return fail(DQMC_EINVAL, "truncated or damaged checkpoint");
  for (const int8_t v : f)
    if (v != 1 && v != -1) return fail(DQMC_EINVAL, "checkpoint field values must be +1 or -1");
  if (!c->allocated) {
    c->k = opt[0];
    c->n_stab = opt[1];
    c->precision = opt[2];
    c->chain = opt[3];
  }
  c->seed = seed;
  c->site_offsets = opt[4];
  c->bin = opt[5];
  DQ_CHECK(ensure_alloc(c));
  CK(cudaMemcpyAsync(c->field, f.data(), f.size(), cudaMemcpyHostToDevice, c->stream));
  unsigned long long acc = (unsigned long long)st[2];
  CK(cudaMemcpyAsync(c->total_acc, &acc, sizeof(acc), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->sweeps = st[0];
  c->proposed = st[1];
  c->accepted = st[2];
  c->max_drift = md;
  c->samples = smp;
  c->ready = false;
  return ensure_ready(c);
} DQ_API_CATCH

dqmc_status dqmc_batch_create(int n, const double *params, dqmc_ctx **out) try {
  if (n < 1 || !params || !out) return fail(DQMC_EINVAL, "need n >= 1, params and out");
  for (int i = 0; i < n; ++i) out[i] = nullptr;
  for (int i = 0; i < n; ++i) {
    const double *p = params + 6 * (size_t)i;
    if (p[0] != std::floor(p[0]) || !(p[5] >= 0.0) || p[5] != std::floor(p[5]) || p[5] > 9007199254740992.0)
      return fail(DQMC_EINVAL, "chain " + std::to_string(i) + ": L and seed must be non-negative integers");
  }
  int dev = 0;
  for (int i = 0; i < n; ++i) {
    const double *p = params + 6 * (size_t)i;
    dqmc_status st = dqmc_create((int)p[0], p[1], p[2], p[3], p[4], (uint64_t)p[5], &out[i]);
    if (st == DQMC_OK) {
      dqmc_ctx *c = out[i];
      c->chain = i;
      cudaError_t e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) {
        c->stream = nullptr;
        st = cuda_fail(e, "chain stream");
      } else {
        c->own_stream = true;
        c->device = dev;
      }
    } else {
      set_error("chain " + std::to_string(i) + ": " + g_last_error);
    }
    if (st != DQMC_OK) {
      const std::string msg = g_last_error;
      for (int j = 0; j <= i; ++j) {
        dqmc_destroy(out[j]);
        out[j] = nullptr;
      }
      set_error(msg);
      return st;
    }
  }
  return DQMC_OK;
} DQ_API_CATCH

dqmc_status dqmc_batch_sweep(dqmc_ctx **ctxs, int n, int n_sweeps, int measure) try {
  if (n < 1 || !ctxs) return fail(DQMC_EINVAL, "need n >= 1 and the contexts");
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return fail(DQMC_EINVAL, "context " + std::to_string(i) + " is NULL");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return fail(DQMC_EINVAL, "a context appears twice");
  }
  std::vector<dqmc_status> rs(n, DQMC_OK);
  std::vector<std::string> errs(n);
  std::vector<std::thread> th;
  th.reserve(n);
  auto run = [&](int i) {
    cudaSetDevice(ctxs[i]->device);
    rs[i] = dqmc_sweep(ctxs[i], n_sweeps, measure);
    if (rs[i] != DQMC_OK) errs[i] = g_last_error;
  };
  // chains [0, spawned) on their own threads; if the host refuses a thread,
  // the rest run one after another on the calling thread (its current
  // device restored afterwards), concurrently with the spawned ones
  int spawned = 0;
  for (; spawned < n; ++spawned) {
    try {
      th.emplace_back(run, spawned);
    } catch (const std::system_error &) {
      break;
    }
  }
  if (spawned < n) {
    int dev = 0;
    const bool have_dev = cudaGetDevice(&dev) == cudaSuccess;
    for (int i = spawned; i < n; ++i) run(i);
    if (have_dev) cudaSetDevice(dev);
  }
  for (auto &t : th) t.join();
  for (int i = 0; i < n; ++i)
    if (rs[i] != DQMC_OK) return fail(rs[i], "chain " + std::to_string(i) + ": " + errs[i]);
  return DQMC_OK;
} DQ_API_CATCH

void dqmc_destroy(dqmc_ctx *c) {
  if (!c) return;
  if (c->allocated || !c->allocs.empty()) cudaStreamSynchronize(c->stream);
  if (c->side) {
    cudaStreamSynchronize(c->side);
    cudaStreamDestroy(c->side);
    cudaEventDestroy(c->ev_fork);
    cudaEventDestroy(c->ev_join);
  }

  if (c->own_stream && c->stream) {
    cudaStreamSynchronize(c->stream);
    cudaStreamDestroy(c->stream);
    c->stream = nullptr;
  }
  for (void *p : c->allocs) {
    if (c->ufree)
      c->ufree(p, c->uuser);
    else
      cudaFree(p);
  }
  delete c;
}

}  // extern "C"
