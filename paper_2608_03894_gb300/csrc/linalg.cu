// FP64 dense linear algebra for the UDV stabilisation.
//
// The stabilisation (not in the paper; standard DQMC practice) needs QR
// factorisations of N x N matrices, explicit Q factors, Q^T applied to a
// matrix and triangular solves, all in FP64. Blocked Householder QR: a panel
// of nb columns is factorised by one thread-block cluster (16 CTAs where the
// part allows it, else 8) whose CTAs
// each hold a slice of the panel rows in shared memory and combine their
// partial column dot products through distributed shared memory; the
// trailing update is two GEMMs with the compact-WY factors V and
// Y = V T^T (Q_panel = I - V T V^T).
#include <cooperative_groups.h>
#include <algorithm>
#include <mutex>

#include "linalg.cuh"
#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace dq {

// ====================================================================== GEMM
// 64 x 64 tile, BK = 16, 256 threads, 4 x 4 outputs per thread (rows ty+16i,
// columns tx+16j). DFMA throughput bound on GB300; the tile keeps operand
// reuse at 16 FMAs per 8 shared loads.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256)
    dgemm_kernel(int M, int N, int K, double alpha, const double *__restrict__ A, int lda,
                 const double *__restrict__ B, int ldb, double beta, double *__restrict__ C,
                 int ldc, const double *__restrict__ rs, const double *__restrict__ cs, int klen,
                 double *__restrict__ part) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kbeg = blockIdx.z * klen;
  const int kend = min(K, kbeg + klen);
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int e = tid; e < BM * BK; e += 256) {
      int mm, kk;
      if (!TA) {
        kk = e % BK;
        mm = e / BK;
      } else {
        mm = e % BM;
        kk = e / BM;
      }
      const int gm = m0 + mm, gk = k0 + kk;
      double v = 0.0;
      if (gm < M && gk < kend) v = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
      As[kk][mm] = v;
    }
#pragma unroll
    for (int e = tid; e < BN * BK; e += 256) {
      int nn, kk;
      if (!TB) {
        nn = e % BN;
        kk = e / BN;
      } else {
        kk = e % BK;
        nn = e / BK;
      }
      const int gn = n0 + nn, gk = k0 + kk;
      double v = 0.0;
      if (gn < N && gk < kend) v = TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
    const double r = rs ? rs[gm] : 1.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      const double v = alpha * r * acc[i][j] * (cs ? cs[gn] : 1.0);
      double *cp = C + (size_t)gm * ldc + gn;
      if (part)
        part[((size_t)blockIdx.z * M + gm) * N + gn] = v;
      else
        *cp = (beta != 0.0) ? v + beta * (*cp) : v;
    }
  }
}

__global__ void scale_matrix_kernel(double *C, int M, int N, int ldc, double beta) {
  const long total = (long)M * N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e / N), j = (int)(e % N);
    double *p = C + (size_t)i * ldc + j;
    *p = (beta == 0.0) ? 0.0 : beta * (*p);
  }
}

static int grid_for(long work, int per) {
  long g = (work + per - 1) / per;
  if (g > 8192) g = 8192;
  if (g < 1) g = 1;
  return (int)g;
}

// ---------------------------------------------------------------------- split K
static thread_local double *t_skws = nullptr;
static thread_local size_t t_skws_n = 0;

void set_splitk_workspace(double *ws, size_t n) {
  t_skws = ws;
  t_skws_n = ws ? n : 0;
}

// The GEMMs split K only while their 64 x 64 tiles number fewer than 304, and
// then into at most ceil(304 / tiles) splits: splits * M * N < 608 * 64 * 64.
size_t splitk_ws_doubles() { return (size_t)608 * 64 * 64; }

double *splitk_partials(int splits, int M, int N) {
  if (splits <= 1) return nullptr;
  const size_t need = (size_t)splits * M * N;
  return (t_skws && need <= t_skws_n) ? t_skws : nullptr;
}

__global__ void splitk_reduce_kernel(const double *__restrict__ part, int splits, int M, int N,
                                     double beta, double *__restrict__ C, int ldc) {
  const long total = (long)M * N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += part[(size_t)z * total + e];
    const int i = (int)(e / N), j = (int)(e % N);
    double *cp = C + (size_t)i * ldc + j;
    *cp = (beta != 0.0) ? s + beta * (*cp) : s;
  }
}

static int grid_for(long work, int per = 256);

cudaError_t splitk_reduce(const double *part, int splits, int M, int N, double beta, double *C,
                          int ldc, cudaStream_t st) {
  DQ_KSCOPE(KF_STABAUX, st);
  splitk_reduce_kernel<<<grid_for((long)M * N), 256, 0, st>>>(part, splits, M, N, beta, C, ldc);
  return cudaGetLastError();
}

static thread_local int t_site = 0;
static thread_local unsigned t_site_mask = 0xffffffffu;
static thread_local unsigned t_df_site_mask = 0u;
void set_gemm_site(int site) { t_site = site; }
void set_gemm_site_mask(unsigned mask) { t_site_mask = mask; }
void set_gemm_df_site_mask(unsigned mask) { t_df_site_mask = mask; }

cudaError_t scale_matrix(double *C, int M, int N, int ldc, double beta, cudaStream_t st) {
  DQ_KSCOPE(KF_STABAUX, st);
  scale_matrix_kernel<<<grid_for((long)M * N), 256, 0, st>>>(C, M, N, ldc, beta);
  return cudaGetLastError();
}

cudaError_t dgemm(bool ta, bool tb, int M, int N, int K, double alpha, const double *A, int lda,
                  const double *B, int ldb, double beta, double *C, int ldc, const double *rs,
                  const double *cs, cudaStream_t st, int splitk) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const bool fast_site = (t_site_mask >> t_site) & 1u;
  if (K > 0 && fast_site && ((t_df_site_mask >> t_site) & 1u) && gemm_df())
    return dfgemm(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, rs, cs, st, splitk, 304);
  if (K > 0 && fast_site && gemm_oz())
    return ozgemm(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, rs, cs, st);
  if (K > 0 && fast_site && gemm_df())
    return dfgemm(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, rs, cs, st, splitk, 304);
  return dgemm_fp64(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, rs, cs, st, splitk);
}

cudaError_t dgemm_fp64(bool ta, bool tb, int M, int N, int K, double alpha, const double *A,
                       int lda, const double *B, int ldb, double beta, double *C, int ldc,
                       const double *rs, const double *cs, cudaStream_t st, int splitk) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (K <= 0) {
    DQ_KSCOPE(KF_STABAUX, st);
    scale_matrix_kernel<<<grid_for((long)M * N), 256, 0, st>>>(C, M, N, ldc, beta);
    return cudaGetLastError();
  }
  const int tiles = ((M + 63) / 64) * ((N + 63) / 64);
  if (splitk <= 0) {
    // aim for ~2 waves over 152 SMs, each split at least 128 deep
    splitk = 1;
    if (tiles < 304) {
      splitk = (304 + tiles - 1) / tiles;
      const int maxs = (K + 127) / 128;
      if (splitk > maxs) splitk = maxs;
      if (splitk < 1) splitk = 1;
    }
  }
  int klen = (K + splitk - 1) / splitk;
  klen = ((klen + 15) / 16) * 16;
  splitk = (K + klen - 1) / klen;
  double *part = splitk_partials(splitk, M, N);
  if (splitk > 1 && !part) {
    splitk = 1;
    klen = ((K + 15) / 16) * 16;
  }
  dim3 grid((N + 63) / 64, (M + 63) / 64, splitk);
  DQ_KSCOPE(KF_GEMM, st);
  add_work(KF_GEMM, 2.0 * M * (double)N * K,
           8.0 * ((double)M * K + (double)K * N + (beta != 0.0 ? 2.0 : 1.0) * (double)M * N));
  if (!ta && !tb)
    dgemm_kernel<false, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, rs, cs, klen, part);
  else if (ta && !tb)
    dgemm_kernel<true, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, rs, cs, klen, part);
  else if (!ta && tb)
    dgemm_kernel<false, true><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, rs, cs, klen, part);
  else
    dgemm_kernel<true, true><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, rs, cs, klen, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !part) return e;
  return splitk_reduce(part, splitk, M, N, beta, C, ldc, st);
}

// ====================================================================== QR panel
// The panel runs on one thread-block cluster: 16 CTAs (non-portable size)
// when the device co-schedules such a cluster with the panel's shared
// memory, else 8. FP64 issue rate per SM is low on this part, so the cluster
// is made as wide as possible and the panel kernel does only the column
// loop; the Gram matrix V^T V, the T factor and every product with V run as
// GEMMs over the whole GPU.
static int g_qr_ctas = 0;

static size_t qr_panel_smem_rows(int rows_per, int nb) {
  return ((size_t)rows_per * (nb + 2) + 16 * (size_t)nb + 64) * sizeof(double);
}

template <int NB> __global__ void qr_panel_kernel(double *, int, int, int, double *, double *);
template <int NB> __global__ void qr_panel_df_kernel(double *, int, int, int, double *, double *);

static std::mutex g_qr_mu;

static int qr_cluster_ctas() {
  std::lock_guard<std::mutex> lk(g_qr_mu);
  if (g_qr_ctas) return g_qr_ctas;
  int ctas = 8;
  const int want = 16;
  if (cudaFuncSetAttribute(qr_panel_kernel<64>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
          cudaSuccess &&
      cudaFuncSetAttribute(qr_panel_kernel<32>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
          cudaSuccess &&
      cudaFuncSetAttribute(qr_panel_df_kernel<64>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
          cudaSuccess &&
      cudaFuncSetAttribute(qr_panel_df_kernel<32>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
          cudaSuccess) {
    // the largest panel used here (L = 36, N = 3888) with nb = 64
    const size_t smem = qr_panel_smem_rows((3888 + want - 1) / want, 64);
    if (cudaFuncSetAttribute(qr_panel_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(want);
      cfg.blockDim = dim3(256);
      cfg.dynamicSmemBytes = smem;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = want;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, qr_panel_kernel<64>, &cfg) == cudaSuccess &&
          nclusters >= 1)
        ctas = want;
    }
  }
  cudaGetLastError();  // a refused query leaves no sticky error; clear the last one
  g_qr_ctas = ctas;
  return ctas;
}

int qr_panel_width(int n) {
  // nb = 64 when one CTA's share of the panel rows fits in shared memory, else 32
  const int ctas = qr_cluster_ctas();
  const int rows_per = (n + ctas - 1) / ctas;
  return qr_panel_smem_rows(rows_per, 64) <= 220 * 1024 ? 64 : 32;
}

size_t qr_work_doubles(int n) {
  const int nb = qr_panel_width(n);
  const int nblk = (n + nb - 1) / nb;
  // V, tau, W, W2, Gram, T blocks, Rinv blocks
  return (size_t)n * n + (size_t)n + 2 * (size_t)nb * n + (size_t)nb * nb +
         2 * (size_t)nblk * nb * nb;
}

void qr_work_bind(QRWork &w, int n, double *mem) {
  w.n = n;
  w.nb = qr_panel_width(n);
  w.ctas = qr_cluster_ctas();
  const int nblk = (n + w.nb - 1) / w.nb;
  w.V = mem;
  w.tau = w.V + (size_t)n * n;
  w.W = w.tau + n;
  w.W2 = w.W + (size_t)w.nb * n;
  w.Gram = w.W2 + (size_t)w.nb * n;
  w.T = w.Gram + (size_t)w.nb * w.nb;
  w.Rinv = w.T + (size_t)nblk * w.nb * w.nb;
}

// Factorises the panel A[p:n, p:p+nc] (nc <= NB) in place. Rows are split
// over the CTAs of the cluster; CTA r owns panel rows [r R, (r+1) R).
// Per column jj: every CTA forms partial dot products of the column with the
// remaining panel columns over its rows, the cluster combines them through
// DSMEM, every CTA computes the same reflector (LAPACK convention:
// H = I - tau v v^T, v_0 = 1, H x = beta e_1) and updates its own rows.
// Output: R and the reflectors in A, V explicit (unit lower trapezoidal,
// zeros above) and tau.
template <int NB>
__global__ void __launch_bounds__(256)
    qr_panel_kernel(double *A, int n, int p, int nc, double *V, double *tau_out) {
  cg::cluster_group cluster = cg::this_cluster();
  const int ncta = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int m = n - p;
  const int rows_per = (m + ncta - 1) / ncta;
  const int lr0 = rank * rows_per;
  const int myrows = max(0, min(m, lr0 + rows_per) - lr0);
  constexpr int LDP = NB + 1;
  extern __shared__ __align__(16) double sm[];
  double *P = sm;                            // rows_per x LDP
  double *red = P + (size_t)rows_per * LDP;  // 8 x NB
  double *part = red + 8 * NB;               // 2 x NB
  double *piv = part + 2 * NB;               // 2 x NB
  double *sD = piv + 2 * NB;                 // NB
  double *sy0 = sD + NB;                     // NB
  double *sw = sy0 + NB;                     // NB
  double *stau = sw + NB;                    // NB
  double *tvs = stau + NB;                   // rows_per: tau v_r of this CTA's rows
  __shared__ double ssc[3];                  // tau, beta, scal of the current reflector
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int e = tid; e < myrows * NB; e += 256) {
    const int r = e / NB, c = e % NB;
    P[r * LDP + c] = (c < nc) ? A[(size_t)(p + lr0 + r) * n + p + c] : 0.0;
  }
  __syncthreads();

  for (int jj = 0; jj < nc; ++jj) {
    const int buf = jj & 1;
    const int owner = jj / rows_per;
    // column dot products over this CTA's rows below the diagonal: thread
    // (column c, row group g) with two independent accumulators
    {
      const int c = tid % NB, g = tid / NB;
      constexpr int NG = 256 / NB;
      double acc0 = 0.0, acc1 = 0.0;
      if (c >= jj && c < nc) {
        const int rs = max(0, jj + 1 - lr0);  // first local row below the diagonal
        int r = rs + ((g - rs) % NG + NG) % NG;
        for (; r + NG < myrows; r += 2 * NG) {
          acc0 = fma(P[r * LDP + jj], P[r * LDP + c], acc0);
          acc1 = fma(P[(r + NG) * LDP + jj], P[(r + NG) * LDP + c], acc1);
        }
        if (r < myrows) acc0 = fma(P[r * LDP + jj], P[r * LDP + c], acc0);
      }
      red[g * NB + c] = acc0 + acc1;
    }
    if (rank == owner)
      for (int c = tid; c < NB; c += 256) piv[buf * NB + c] = P[(jj - lr0) * LDP + c];
    __syncthreads();
    if (tid < NB) {
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < 256 / NB; ++w) s += red[w * NB + tid];
      part[buf * NB + tid] = s;
    }
    // the partial sums and the owner's pivot row become visible cluster-wide;
    // a CTA can only reuse this buffer parity after the next cluster barrier,
    // which every CTA reaches after its reads below
    cluster.sync();
    {
      // 256 / NB threads per column, each summing every (256 / NB)-th rank's
      // partial: the remote loads are independent and overlap. The summation
      // order is fixed, so every CTA gets bit-identical sums.
      constexpr int NG = 256 / NB;
      const int c = tid % NB, g = tid / NB;
      double D = 0.0;
      for (int r2 = g; r2 < ncta; r2 += NG) D += cluster.map_shared_rank(part, r2)[buf * NB + c];
      red[g * NB + c] = D;
      if (g == 0) sy0[c] = cluster.map_shared_rank(piv, owner)[buf * NB + c];
    }
    __syncthreads();
    if (tid < NB) {
      double D = 0.0;
#pragma unroll
      for (int g = 0; g < 256 / NB; ++g) D += red[g * NB + tid];
      sD[tid] = D;
      if (tid == jj) {
        // the reflector's scalars, once (FP64 sqrt and divisions are slow on this part)
        const double alpha = sy0[jj], sigma = D;
        double tau = 0.0, beta = alpha, scal = 0.0;
        if (sigma > 0.0) {
          const double nrm = sqrt(alpha * alpha + sigma);
          beta = (alpha >= 0.0) ? -nrm : nrm;
          tau = (beta - alpha) / beta;
          scal = 1.0 / (alpha - beta);
        }
        ssc[0] = tau;
        ssc[1] = beta;
        ssc[2] = scal;
        stau[jj] = tau;
      }
    }
    __syncthreads();
    const double tau = ssc[0], beta = ssc[1], scal = ssc[2];
    // the reflector of each row (v = x scal below the diagonal), tau v, and w
    for (int r = tid; r < myrows; r += 256) {
      const int lr = lr0 + r;
      double *row = P + r * LDP;
      if (lr > jj) {
        const double v = row[jj] * scal;
        tvs[r] = tau * v;
        row[jj] = v;
      } else if (lr == jj) {
        tvs[r] = tau;
        row[jj] = beta;
      } else {
        tvs[r] = 0.0;
      }
    }
    if (tid < NB) sw[tid] = (tid > jj && tid < nc) ? sy0[tid] + scal * sD[tid] : 0.0;
    __syncthreads();
    // rank-one update of the columns after jj: thread (column offset lane,
    // row offset warp), the column's w in registers
    {
      const int c0 = jj + 1 + lane, c1 = c0 + 32;
      const double w0 = c0 < nc ? sw[c0] : 0.0, w1 = c1 < nc ? sw[c1] : 0.0;
      const int rs = max(0, jj - lr0);  // rows at or below the diagonal
      if (c0 < nc) {
        for (int r = rs + ((warp - rs) % 8 + 8) % 8; r < myrows; r += 8) {
          const double t = tvs[r];
          P[r * LDP + c0] = fma(-t, w0, P[r * LDP + c0]);
          if (c1 < nc) P[r * LDP + c1] = fma(-t, w1, P[r * LDP + c1]);
        }
      }
    }
    __syncthreads();
  }

  // write back R / V into A and the explicit V
  for (int e = tid; e < myrows * nc; e += 256) {
    const int r = e / nc, c = e % nc;
    const int lr = lr0 + r;
    const double pv = P[r * LDP + c];
    A[(size_t)(p + lr) * n + p + c] = pv;
    V[(size_t)(p + lr) * n + p + c] = (lr > c) ? pv : (lr == c ? 1.0 : 0.0);
  }
  if (rank == 0)
    for (int j = tid; j < nc; j += 256) tau_out[p + j] = stau[j];
  // no CTA leaves while another may still read its shared memory
  cluster.sync();
}

// The same panel in double-float arithmetic (mixed precision): the column
// dot products and row updates run as FP32 pairs (~2^-47) on the FP32 units
// instead of the FP64 pipe (1/64 of the FP32 rate on this part); the
// reflector's scalars stay FP64. Each column is first scaled by a power of two
// 2^-e_c (e_c from the cluster-wide largest exponent of the column) so that
// its entries, their squares and sums stay inside the FP32 range; the
// reflectors v and tau do not change under a column scaling, and the entries
// of R are scaled back on the way out. Entries below 2^-126 of their column's
// largest are dropped.
__device__ __forceinline__ df64 df_from_scaled(double x, int es) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  const int e2 = e - es;
  if (e == 0 || e2 <= 0) return df64(0.f, 0.f);
  return df_from(__longlong_as_double((long long)((b & ~(0x7ffull << 52)) | ((unsigned long long)e2 << 52))));
}
__device__ __forceinline__ double scale_pow2(double y, int es) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(y);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0) return y;  // zero (or subnormal, which the panel does not produce)
  const int e2 = e + es;
  if (e2 <= 0) return 0.0;
  return __longlong_as_double((long long)((b & ~(0x7ffull << 52)) | ((unsigned long long)e2 << 52)));
}

template <int NB>
__global__ void __launch_bounds__(256)
    qr_panel_df_kernel(double *A, int n, int p, int nc, double *V, double *tau_out) {
  cg::cluster_group cluster = cg::this_cluster();
  const int ncta = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int m = n - p;
  const int rows_per = (m + ncta - 1) / ncta;
  const int lr0 = rank * rows_per;
  const int myrows = max(0, min(m, lr0 + rows_per) - lr0);
  constexpr int LDP = NB + 1;
  extern __shared__ __align__(16) double sm[];
  df64 *P = reinterpret_cast<df64 *>(sm);   // rows_per x LDP
  df64 *red = P + (size_t)rows_per * LDP;   // 8 x NB
  df64 *part = red + 8 * NB;                // 2 x NB
  df64 *piv = part + 2 * NB;                // 2 x NB
  df64 *sD = piv + 2 * NB;                  // NB
  df64 *sy0 = sD + NB;                      // NB
  df64 *sw = sy0 + NB;                      // NB
  double *stau = reinterpret_cast<double *>(sw + NB);  // NB
  df64 *tvs = reinterpret_cast<df64 *>(stau + NB);     // rows_per: tau v_r of this CTA's rows
  __shared__ int ecol[NB], emine[NB];
  __shared__ df64 ssc[3];                   // tau, beta, scal of the current reflector
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // column scales: the cluster-wide largest exponent of each panel column
  if (tid < NB) emine[tid] = 0;
  __syncthreads();
  for (int e = tid; e < myrows * NB; e += 256) {
    const int r = e / NB, c = e % NB;
    if (c < nc) {
      const double x = A[(size_t)(p + lr0 + r) * n + p + c];
      atomicMax(&emine[c], (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ff));
    }
  }
  cluster.sync();
  if (tid < NB) {
    int mx = 0;
    for (int r2 = 0; r2 < ncta; ++r2) mx = max(mx, cluster.map_shared_rank(emine, r2)[tid]);
    ecol[tid] = mx > 0 ? mx - 1023 : 0;  // the column's largest entry scales into [1, 2)
  }
  __syncthreads();
  for (int e = tid; e < myrows * NB; e += 256) {
    const int r = e / NB, c = e % NB;
    P[r * LDP + c] = (c < nc) ? df_from_scaled(A[(size_t)(p + lr0 + r) * n + p + c], ecol[c]) : df64(0.f, 0.f);
  }
  __syncthreads();

  for (int jj = 0; jj < nc; ++jj) {
    const int buf = jj & 1;
    const int owner = jj / rows_per;
    {
      const int c = tid % NB, g = tid / NB;
      constexpr int NG = 256 / NB;
      df64 acc0(0.f, 0.f), acc1(0.f, 0.f);
      if (c >= jj && c < nc) {
        const int rs = max(0, jj + 1 - lr0);
        int r = rs + ((g - rs) % NG + NG) % NG;
        for (; r + NG < myrows; r += 2 * NG) {
          acc0 = P[r * LDP + jj] * P[r * LDP + c] + acc0;
          acc1 = P[(r + NG) * LDP + jj] * P[(r + NG) * LDP + c] + acc1;
        }
        if (r < myrows) acc0 = P[r * LDP + jj] * P[r * LDP + c] + acc0;
      }
      red[g * NB + c] = acc0 + acc1;
    }
    if (rank == owner)
      for (int c = tid; c < NB; c += 256) piv[buf * NB + c] = P[(jj - lr0) * LDP + c];
    __syncthreads();
    if (tid < NB) {
      df64 sacc(0.f, 0.f);
#pragma unroll
      for (int w = 0; w < 256 / NB; ++w) sacc = sacc + red[w * NB + tid];
      part[buf * NB + tid] = sacc;
    }
    // the partial sums and the owner's pivot row become visible cluster-wide;
    // a CTA can only reuse this buffer parity after the next cluster barrier,
    // which every CTA reaches after its reads below
    cluster.sync();
    {
      constexpr int NG = 256 / NB;
      const int c = tid % NB, g = tid / NB;
      df64 D(0.f, 0.f);
      for (int r2 = g; r2 < ncta; r2 += NG) D = D + cluster.map_shared_rank(part, r2)[buf * NB + c];
      red[g * NB + c] = D;
      if (g == 0) sy0[c] = cluster.map_shared_rank(piv, owner)[buf * NB + c];
    }
    __syncthreads();
    if (tid < NB) {
      df64 D(0.f, 0.f);
#pragma unroll
      for (int g = 0; g < 256 / NB; ++g) D = D + red[g * NB + tid];
      sD[tid] = D;
      if (tid == jj) {
        // the reflector's scalars in FP64, once
        const double alpha = df_to(sy0[jj]), sigma = df_to(D);
        double tau = 0.0, beta = alpha, scal = 0.0;
        if (sigma > 0.0) {
          const double nrm = sqrt(alpha * alpha + sigma);
          beta = (alpha >= 0.0) ? -nrm : nrm;
          tau = (beta - alpha) / beta;
          scal = 1.0 / (alpha - beta);
        }
        ssc[0] = df_from(tau);
        ssc[1] = df_from(beta);
        ssc[2] = df_from(scal);
        stau[jj] = tau;
      }
    }
    __syncthreads();
    const df64 tau = ssc[0], beta = ssc[1], scal = ssc[2];
    for (int r = tid; r < myrows; r += 256) {
      const int lr = lr0 + r;
      df64 *row = P + r * LDP;
      if (lr > jj) {
        const df64 v = row[jj] * scal;
        tvs[r] = -(tau * v);
        row[jj] = v;
      } else if (lr == jj) {
        tvs[r] = -tau;
        row[jj] = beta;
      } else {
        tvs[r] = df64(0.f, 0.f);
      }
    }
    if (tid < NB) sw[tid] = (tid > jj && tid < nc) ? scal * sD[tid] + sy0[tid] : df64(0.f, 0.f);
    __syncthreads();
    {
      const int c0 = jj + 1 + lane, c1 = c0 + 32;
      const df64 w0 = c0 < nc ? sw[c0] : df64(0.f, 0.f), w1 = c1 < nc ? sw[c1] : df64(0.f, 0.f);
      const int rs = max(0, jj - lr0);
      if (c0 < nc) {
        for (int r = rs + ((warp - rs) % 8 + 8) % 8; r < myrows; r += 8) {
          const df64 t = tvs[r];
          P[r * LDP + c0] = t * w0 + P[r * LDP + c0];
          if (c1 < nc) P[r * LDP + c1] = t * w1 + P[r * LDP + c1];
        }
      }
    }
    __syncthreads();
  }

  // write back R (scaled back by 2^e_c) / V into A and the explicit V
  for (int e = tid; e < myrows * nc; e += 256) {
    const int r = e / nc, c = e % nc;
    const int lr = lr0 + r;
    const double pv = df_to(P[r * LDP + c]);
    A[(size_t)(p + lr) * n + p + c] = (lr > c) ? pv : scale_pow2(pv, ecol[c]);
    V[(size_t)(p + lr) * n + p + c] = (lr > c) ? pv : (lr == c ? 1.0 : 0.0);
  }
  if (rank == 0)
    for (int j = tid; j < nc; j += 256) tau_out[p + j] = stau[j];
  // no CTA leaves while another may still read its shared memory
  cluster.sync();
}

// T (nc x nc, upper triangular, leading dimension NB) of the compact WY form
// H_0 H_1 ... H_{nc-1} = I - V T V^T. With every tau_j != 0,
//     T^{-1} = diag(1/tau) + strictly-upper(V^T V)
// (the product of two reflectors gives T = [[t0, -t0 t1 g], [0, t1]], whose
// inverse is [[1/t0, g], [0, 1/t1]], g = v0^T v1; the same block argument
// extends it to nc reflectors), so each column c of T is an independent back
// substitution X[c][c] = tau_c, X[i][c] = -tau_i sum_{k>i} G[i][k] X[k][c]:
// 16 warps, warp w takes columns w, 16 + w, nc - 1 - w and nc - 17 - w
// (balanced lengths; a column two warps share is computed identically by
// both), the dot products over k split over the lanes. If some tau_j = 0
// (H_j = I) the serial recurrence T[0:j, j] = -tau_j T[0:j, 0:j] G[0:j, j],
// T_jj = tau_j is used instead. nc <= 64.
__global__ void __launch_bounds__(512)
    qr_t_kernel(const double *Gram, int ldg, const double *tau, int nc, int NB, double *T) {
  __shared__ double g[64][64];
  __shared__ double x[16][64];
  __shared__ double st[64];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < 64 * 64; e += blockDim.x) {
    const int i = e / 64, k = e % 64;
    g[i][k] = (i < nc && k < nc) ? Gram[(size_t)i * ldg + k] : 0.0;
  }
  if (tid < 64) st[tid] = tid < nc ? tau[tid] : 0.0;
  const int zero_tau = __syncthreads_or(tid < nc && tau[tid] == 0.0);
  if (!zero_tau) {
    const int cand[4] = {warp, 16 + warp, nc - 1 - warp, nc - 17 - warp};
    for (int h = 0; h < 4; ++h) {
      const int c = cand[h];
      bool dup = c < 0 || c >= nc;
      for (int h2 = 0; h2 < h; ++h2) dup = dup || cand[h2] == c;
      if (dup) continue;
      double *xs = x[warp];
      for (int i = c; i >= 0; --i) {
        double part = 0.0;
        for (int k = i + 1 + lane; k <= c; k += 32) part = fma(g[i][k], xs[k], part);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        const double xi = (i == c) ? st[c] : -st[i] * part;
        __syncwarp();
        if (lane == 0) xs[i] = xi;
        __syncwarp();
      }
      for (int i = lane; i < NB; i += 32) T[(size_t)i * NB + c] = i <= c ? xs[i] : 0.0;
    }
    for (int e = tid; e < NB * NB; e += blockDim.x)
      if (e % NB >= nc) T[e] = 0.0;  // columns beyond the panel
  } else if (warp == 0) {
    // serial recurrence by one warp, T built in global memory (only this warp touches it)
    for (int e = lane; e < NB * NB; e += 32) T[e] = 0.0;
    __syncwarp();
    for (int j = 0; j < nc; ++j) {
      for (int i = lane; i < j; i += 32) {
        double acc = 0.0;
        for (int k = i; k < j; ++k) acc = fma(T[(size_t)i * NB + k], g[k][j], acc);
        T[(size_t)i * NB + j] = -st[j] * acc;
      }
      if (lane == 0) T[(size_t)j * NB + j] = st[j];
      __syncwarp();
      __threadfence_block();
    }
  }
}

static thread_local bool t_qr_df = false;
void set_qr_panel_df(bool on) { t_qr_df = on; }
static thread_local int t_refl_gram = 0, t_refl_tw = 0;
void set_reflector_modes(int gram, int tw) {
  t_refl_gram = gram;
  t_refl_tw = tw;
}

// Gram matrix V^T V (nc x nc, nc <= 64) of a panel's reflectors, for the
// compact-WY factor T, in FP64 or in double-float arithmetic (the reflector
// entries are bounded by 1 in magnitude, inside the FP32 range). CTA z sums
// rows [z R, (z + 1) R) into its own 64 x 64 partial (16 x 16 threads, a
// 4 x 4 block each, rows staged 16 at a time); the partials are then summed
// in split order (splitk_reduce), so the result is deterministic. Replaces a
// digit-slice GEMM whose single output tile leaves most of the GPU idle and
// which costs two operand-slicing launches. The double-float form loses
// orthogonality of the block reflectors at the 2^-47 level, which shows in
// the drift at L = 36.
template <bool DF>
__global__ void __launch_bounds__(256)
    gram_kernel(const double *__restrict__ V, int ldv, int m, int nc, int rows_per, double *__restrict__ part) {
  if constexpr (!DF) {
    // FP64: thread (ty, tx) owns the 4 x 4 block; rows staged 16 at a time
    __shared__ double sd[16][64];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int r0 = blockIdx.x * rows_per, r1 = min(m, r0 + rows_per);
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    for (int rb = r0; rb < r1; rb += 16) {
      __syncthreads();
      for (int e = tid; e < 16 * 64; e += 256) {
        const int rr = e / 64, c = e % 64;
        const int r = rb + rr;
        sd[rr][c] = (r < r1 && c < nc) ? V[(size_t)r * ldv + c] : 0.0;
      }
      __syncthreads();
      const int nr = min(16, r1 - rb);
      for (int rr = 0; rr < nr; ++rr) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fma(sd[rr][4 * ty + a], sd[rr][4 * tx + b], acc[a][b]);
      }
    }
    double *out = part + (size_t)blockIdx.x * nc * nc;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int i = 4 * ty + a, j = 4 * tx + b;
        if (i < nc && j < nc) out[(size_t)i * nc + j] = acc[a][b];
      }
    return;
  }
  __shared__ float2 sv[16][64];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int r0 = blockIdx.x * rows_per, r1 = min(m, r0 + rows_per);
  float sh[4][4], sl[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) sh[a][b] = sl[a][b] = 0.f;
  for (int rb = r0; rb < r1; rb += 16) {
    __syncthreads();
    for (int e = tid; e < 16 * 64; e += 256) {
      const int rr = e / 64, c = e % 64;
      const int r = rb + rr;
      sv[rr][c] = (r < r1 && c < nc) ? split_df_bits(V[(size_t)r * ldv + c]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int nr = min(16, r1 - rb);
    for (int rr = 0; rr < nr; ++rr) {
      float2 x[4], y[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        x[a] = sv[rr][4 * ty + a];
        y[a] = sv[rr][4 * tx + a];
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          // double-float multiply-add (FMA residual product, TwoSum accumulation)
          const float pp = x[a].x * y[b].x;
          float e = fmaf(x[a].x, y[b].x, -pp);
          e = fmaf(x[a].x, y[b].y, e);
          e = fmaf(x[a].y, y[b].x, e);
          const float t = sh[a][b] + pp;
          const float z = t - sh[a][b];
          const float err = (sh[a][b] - (t - z)) + (pp - z);
          sh[a][b] = t;
          sl[a][b] += err + e;
        }
    }
  }
  double *out = part + (size_t)blockIdx.x * nc * nc;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = 4 * ty + a, j = 4 * tx + b;
      if (i < nc && j < nc) out[(size_t)i * nc + j] = f2d_bits(sh[a][b]) + f2d_bits(sl[a][b]);
    }
}

// df = false: FP64 products on 256 CTAs (the partials summed in order), df =
// true: double-float on 64
static cudaError_t gram_par(bool df, const double *V, int ldv, int m, int nc, double *G, int ldg, cudaStream_t st) {
  const int splits = std::max(1, std::min(df ? 64 : 256, (m + (df ? 15 : 3)) / (df ? 16 : 4)));
  const int rows_per = (m + splits - 1) / splits;
  double *part = splitk_partials(splits, nc, nc);
  if (!part)  // a panel of at most 16 rows (or no partials workspace): FP64
    return dgemm_fp64(true, false, nc, nc, m, 1.0, V, ldv, V, ldv, 0.0, G, ldg, nullptr, nullptr, st);
  {
    DQ_KSCOPE(KF_GEMM, st);
    add_work(KF_GEMM, 2.0 * m * (double)nc * nc, 8.0 * m * (double)nc);
    if (df)
      gram_kernel<true><<<splits, 256, 0, st>>>(V, ldv, m, nc, rows_per, part);
    else
      gram_kernel<false><<<splits, 256, 0, st>>>(V, ldv, m, nc, rows_per, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return splitk_reduce(part, splits, nc, nc, 0.0, G, ldg, st);
}

// Panel p (Householder column loop on one cluster), its Gram matrix V^T V and T.
template <int NB>
static cudaError_t launch_qr_panel(double *A, int n, int p, int nc, QRWork &w, cudaStream_t st) {
  const int ctas = w.ctas;
  const int rows_per = (n - p + ctas - 1) / ctas;
  const size_t smem = qr_panel_smem_rows(rows_per, NB);
  const void *fn = t_qr_df ? (const void *)qr_panel_df_kernel<NB> : (const void *)qr_panel_kernel<NB>;
  cudaError_t e = ensure_smem_attr(fn, (int)qr_panel_smem_rows((n + ctas - 1) / ctas, NB));
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = ctas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  {
    DQ_KSCOPE(KF_QRPANEL, st);
    // Householder column loop: ~2 m nc^2 flops; the m x nc panel read and written once
    add_work(KF_QRPANEL, 2.0 * (n - p) * (double)nc * nc, 16.0 * (n - p) * (double)nc);
    e = t_qr_df ? cudaLaunchKernelEx(&cfg, qr_panel_df_kernel<NB>, A, n, p, nc, w.V, w.tau)
                : cudaLaunchKernelEx(&cfg, qr_panel_kernel<NB>, A, n, p, nc, w.V, w.tau);
    if (e != cudaSuccess) return e;
  }
  // Gram = V_p^T V_p, then T_p
  const int m = n - p;
  const double *Vp = w.V + (size_t)p * n + p;
  e = (gemm_oz() && t_refl_gram) ? gram_par(t_refl_gram == 2, Vp, n, m, nc, w.Gram, w.nb, st)
                : dgemm(true, false, nc, nc, m, 1.0, Vp, n, Vp, n, 0.0, w.Gram, w.nb, nullptr, nullptr, st);
  if (e != cudaSuccess) return e;
  DQ_KSCOPE(KF_STABAUX, st);
  qr_t_kernel<<<1, 512, 0, st>>>(w.Gram, w.nb, w.tau + p, nc, w.nb,
                                                                   w.T + (size_t)(p / w.nb) * w.nb * w.nb);
  return cudaGetLastError();
}

// W2 = op(T) W (nc x ncols, nc <= 64, T nc x nc with leading dimension ldt)
// in double-float arithmetic (mixed precision): the middle product of a
// block reflector, 64 x ncols x 64, too small to fill the GPU as a digit-slice
// GEMM. The columns of W carry the graded scales of the matrix the reflector
// is applied to, so each column is scaled by a power of two (its largest
// exponent) into the FP32 range before the product and scaled back after;
// T's entries are bounded. CTA per 16 columns, thread (column, 4 rows).
template <bool TT>
__global__ void __launch_bounds__(256)
    tw_df_kernel(const double *__restrict__ T, int ldt, const double *__restrict__ W, int ldw, int nc, int ncols,
                 double *__restrict__ W2, int ldw2) {
  __shared__ df64 st[64][65];   // op(T)[i][k]
  __shared__ df64 sw[64][16];   // scaled W[k][j0 + c]
  __shared__ int emax[16];
  const int tid = threadIdx.x, c = tid & 15, ig = tid >> 4;  // ig: rows 4 ig .. 4 ig + 3
  const int j0 = blockIdx.x * 16, j = j0 + c;
  if (tid < 16) emax[tid] = 0;
  for (int e = tid; e < 64 * 64; e += 256) {
    const int i = e / 64, k = e % 64;
    const double t = (i < nc && k < nc) ? (TT ? T[(size_t)k * ldt + i] : T[(size_t)i * ldt + k]) : 0.0;
    st[i][k] = df_from(t);
  }
  __syncthreads();
  for (int e = tid; e < 64 * 16; e += 256) {
    const int k = e / 16, cc = e % 16;
    if (k < nc && j0 + cc < ncols) {
      const double w = W[(size_t)k * ldw + j0 + cc];
      atomicMax(&emax[cc], (int)(((unsigned long long)__double_as_longlong(w) >> 52) & 0x7ff));
    }
  }
  __syncthreads();
  for (int e = tid; e < 64 * 16; e += 256) {
    const int k = e / 16, cc = e % 16;
    const int es = emax[cc] > 0 ? emax[cc] - 1023 : 0;
    sw[k][cc] = (k < nc && j0 + cc < ncols) ? df_from_scaled(W[(size_t)k * ldw + j0 + cc], es) : df64(0.f, 0.f);
  }
  __syncthreads();
  if (j >= ncols) return;
  const int es = emax[c] > 0 ? emax[c] - 1023 : 0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = 4 * ig + a;
    if (i >= nc) continue;
    df64 acc(0.f, 0.f);
    for (int k = 0; k < nc; ++k) acc = st[i][k] * sw[k][c] + acc;
    W2[(size_t)i * ldw2 + j] = scale_pow2(df_to(acc), es);
  }
}

// The same product in FP64, on a CTA per 8 columns (216 CTAs for 1728
// columns, so the whole GPU's FP64 pipes share the 2 nc^2 ncols flops): op(T)
// staged in shared memory (read along T's rows, stored transposed when
// op = T^T), thread (column c, rows 2 ig and 2 ig + 1), the sum over k in
// order with fused multiply-adds.
template <bool TT>
__global__ void __launch_bounds__(256)
    tw_fp64_kernel(const double *__restrict__ T, int ldt, const double *__restrict__ W, int ldw, int nc, int ncols,
                   double *__restrict__ W2, int ldw2) {
  __shared__ double st[64][65];  // op(T)[i][k]
  __shared__ double sw[64][8];   // W[k][j0 + c]
  const int tid = threadIdx.x, c = tid & 7, ig = tid >> 3;
  const int j0 = blockIdx.x * 8, j = j0 + c;
  for (int e = tid; e < 64 * 64; e += 256) {
    const int r = e / 64, q = e % 64;  // T[r][q]
    const double t = (r < nc && q < nc) ? T[(size_t)r * ldt + q] : 0.0;
    if (TT)
      st[q][r] = t;
    else
      st[r][q] = t;
  }
  for (int e = tid; e < 64 * 8; e += 256) {
    const int k = e / 8, cc = e % 8;
    sw[k][cc] = (k < nc && j0 + cc < ncols) ? W[(size_t)k * ldw + j0 + cc] : 0.0;
  }
  __syncthreads();
  if (j >= ncols) return;
  const int i0 = 2 * ig, i1 = i0 + 1;
  double acc0 = 0.0, acc1 = 0.0;
  for (int k = 0; k < nc; ++k) {
    const double w = sw[k][c];
    acc0 = fma(st[i0][k], w, acc0);
    acc1 = fma(st[i1][k], w, acc1);
  }
  if (i0 < nc) W2[(size_t)i0 * ldw2 + j] = acc0;
  if (i1 < nc) W2[(size_t)i1 * ldw2 + j] = acc1;
}

// W2 = op(T) W by the double-float (df) or the FP64 kernel
static cudaError_t tw_par(bool df, bool trans_t, const double *T, int ldt, const double *W, int ldw, int nc,
                          int ncols, double *W2, int ldw2, cudaStream_t st) {
  DQ_KSCOPE(KF_GEMM, st);
  add_work(KF_GEMM, 2.0 * nc * (double)nc * ncols, 8.0 * (2.0 * nc * (double)ncols + (double)nc * nc));
  if (df) {
    const int grid = (ncols + 15) / 16;
    if (trans_t)
      tw_df_kernel<true><<<grid, 256, 0, st>>>(T, ldt, W, ldw, nc, ncols, W2, ldw2);
    else
      tw_df_kernel<false><<<grid, 256, 0, st>>>(T, ldt, W, ldw, nc, ncols, W2, ldw2);
  } else {
    const int grid = (ncols + 7) / 8;
    if (trans_t)
      tw_fp64_kernel<true><<<grid, 256, 0, st>>>(T, ldt, W, ldw, nc, ncols, W2, ldw2);
    else
      tw_fp64_kernel<false><<<grid, 256, 0, st>>>(T, ldt, W, ldw, nc, ncols, W2, ldw2);
  }
  return cudaGetLastError();
}

// B[p:, 0:ncols] <- (I - V_p op(T_p) V_p^T) B[p:, 0:ncols], op = T^T (Q^T side) or T (Q side)
static cudaError_t apply_block_reflector(const QRWork &w, int p, int nc, bool trans_t, double *B,
                                         int ldb, int ncols, cudaStream_t st) {
  const int n = w.n, m = n - p;
  const double *Vp = w.V + (size_t)p * n + p;
  const double *Tp = w.T + (size_t)(p / w.nb) * w.nb * w.nb;
  cudaError_t e = dgemm(true, false, nc, ncols, m, 1.0, Vp, n, B, ldb, 0.0, w.W, ncols, nullptr,
                        nullptr, st);
  if (e != cudaSuccess) return e;
  e = (gemm_oz() && t_refl_tw) ? tw_par(t_refl_tw == 2, trans_t, Tp, w.nb, w.W, ncols, nc, ncols, w.W2, ncols, st)
                : dgemm(trans_t, false, nc, ncols, nc, 1.0, Tp, w.nb, w.W, ncols, 0.0, w.W2, ncols, nullptr,
                        nullptr, st);
  if (e != cudaSuccess) return e;
  return dgemm(false, false, m, ncols, nc, -1.0, Vp, n, w.W2, ncols, 1.0, B, ldb, nullptr, nullptr,
               st, 1);
}

cudaError_t qr_factor(double *A, int n, QRWork &w, cudaStream_t st) {
  const int nb = w.nb;
  for (int p = 0; p < n; p += nb) {
    const int nc = min(nb, n - p);
    cudaError_t e = (nb == 64) ? launch_qr_panel<64>(A, n, p, nc, w, st)
                               : launch_qr_panel<32>(A, n, p, nc, w, st);
    if (e != cudaSuccess) return e;
    const int ntr = n - p - nc;
    if (ntr > 0) {
      // A[p:, p+nc:] <- H^T A[p:, p+nc:] = (I - V T^T V^T) A[p:, p+nc:]
      e = apply_block_reflector(w, p, nc, true, A + (size_t)p * n + p + nc, n, ntr, st);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

cudaError_t qr_form_q(double *Q, int n, QRWork &w, cudaStream_t st) {
  cudaError_t e = set_identity(Q, n, n, st);
  if (e != cudaSuccess) return e;
  const int nb = w.nb;
  const int last = ((n - 1) / nb) * nb;
  for (int p = last; p >= 0; p -= nb) {
    const int nc = min(nb, n - p);
    // Q[p:, p:] <- (I - V T V^T) Q[p:, p:]  (Q = H_0 H_1 ... applied right to left)
    e = apply_block_reflector(w, p, nc, false, Q + (size_t)p * n + p, n, n - p, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t qr_apply_qt(double *B, int n, int ncols, int ldb, QRWork &w, cudaStream_t st) {
  const int nb = w.nb;
  for (int p = 0; p < n; p += nb) {
    const int nc = min(nb, n - p);
    cudaError_t e = apply_block_reflector(w, p, nc, true, B + (size_t)p * ldb, ldb, ncols, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Inverse of each nb x nb upper-triangular diagonal block of R (in A).
// One CTA per block; thread j solves column j of U X = I by back substitution.
__global__ void tri_inv_upper_blocks_kernel(const double *A, int n, int nb, double *Rinv) {
  const int b = blockIdx.x;
  const int p = b * nb;
  const int bs = min(nb, n - p);
  extern __shared__ double su[];  // bs x bs
  for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
    const int i = e / bs, j = e % bs;
    su[e] = A[(size_t)(p + i) * n + p + j];
  }
  __syncthreads();
  double *X = Rinv + (size_t)b * nb * nb;
  const int j = threadIdx.x;
  if (j < nb) {
    for (int i = 0; i < nb; ++i) X[i * nb + j] = 0.0;
  }
  if (j < bs) {
    X[j * nb + j] = 1.0 / su[j * bs + j];
    for (int i = j - 1; i >= 0; --i) {
      double s = 0.0;
      for (int k = i + 1; k <= j; ++k) s = fma(su[i * bs + k], X[k * nb + j], s);
      X[i * nb + j] = -s / su[i * bs + i];
    }
  }
}

cudaError_t qr_solve_r(const double *A, int n, double *B, double *Z, int ncols, QRWork &w,
                       cudaStream_t st) {
  const int nb = w.nb;
  const int nblk = (n + nb - 1) / nb;
  DQ_KSCOPE(KF_STABAUX, st);
  tri_inv_upper_blocks_kernel<<<nblk, 64, (size_t)nb * nb * sizeof(double), st>>>(A, n, nb, w.Rinv);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int b = nblk - 1; b >= 0; --b) {
    const int p = b * nb;
    const int bs = min(nb, n - p);
    // Z[p:p+bs] = Rinv_b B[p:p+bs]
    e = dgemm(false, false, bs, ncols, bs, 1.0, w.Rinv + (size_t)b * nb * nb, nb,
              B + (size_t)p * ncols, ncols, 0.0, Z + (size_t)p * ncols, ncols, nullptr, nullptr,
              st, 1);
    if (e != cudaSuccess) return e;
    if (p > 0) {
      // B[0:p] -= R[0:p, p:p+bs] Z[p:p+bs]
      e = dgemm(false, false, p, ncols, bs, -1.0, A + p, n, Z + (size_t)p * ncols, ncols, 1.0, B,
                ncols, nullptr, nullptr, st, 1);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// ====================================================================== helpers
__global__ void set_identity_kernel(double *A, int n, int ld) {
  const long total = (long)n * n;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    A[(size_t)i * ld + j] = (i == j) ? 1.0 : 0.0;
  }
}
cudaError_t set_identity(double *A, int n, int ld, cudaStream_t st) {
  DQ_KSCOPE(KF_STABAUX, st);
  set_identity_kernel<<<grid_for((long)n * n), 256, 0, st>>>(A, n, ld);
  return cudaGetLastError();
}

__global__ void set_value_kernel(double *x, long n, double v) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    x[e] = v;
}
cudaError_t set_value(double *x, long n, double v, cudaStream_t st) {
  DQ_KSCOPE(KF_STABAUX, st);
  set_value_kernel<<<grid_for(n), 256, 0, st>>>(x, n, v);
  return cudaGetLastError();
}

// 32 x 32 tiled transpose with row scaling of the output
__global__ void transpose_scale_kernel(const double *in, int ld, double *out, int n,
                                       const double *rs) {
  __shared__ double t[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = by + r, j = bx + threadIdx.x;
    t[r][threadIdx.x] = (i < n && j < n) ? in[(size_t)i * ld + j] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = bx + r, j = by + threadIdx.x;  // out[i][j] = in[j][i]
    if (i < n && j < n) out[(size_t)i * n + j] = t[threadIdx.x][r] * (rs ? rs[i] : 1.0);
  }
}
cudaError_t transpose_scale(const double *in, int ld, double *out, int n, const double *rs,
                            cudaStream_t st) {
  dim3 grid((n + 31) / 32, (n + 31) / 32), block(32, 8);
  DQ_KSCOPE(KF_STABAUX, st);
  transpose_scale_kernel<<<grid, block, 0, st>>>(in, ld, out, n, rs);
  return cudaGetLastError();
}

__global__ void scale_rows_cols_kernel(double *X, int n, int ld, const double *rs, const double *cs) {
  const long total = (long)n * n;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    double v = X[(size_t)i * ld + j];
    if (rs) v *= rs[i];
    if (cs) v *= cs[j];
    X[(size_t)i * ld + j] = v;
  }
}
cudaError_t scale_rows_cols(double *X, int n, int ld, const double *rs, const double *cs,
                            cudaStream_t st) {
  DQ_KSCOPE(KF_STABAUX, st);
  scale_rows_cols_kernel<<<grid_for((long)n * n), 256, 0, st>>>(X, n, ld, rs, cs);
  return cudaGetLastError();
}

__global__ void column_norms_kernel(const double *X, int n, const double *D, double *norms) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0.0;
  for (int i = 0; i < n; ++i) {
    const double v = X[(size_t)i * n + j];
    s = fma(v, v, s);
  }
  norms[j] = sqrt(s) * (D ? D[j] : 1.0);
}
cudaError_t column_norms_scaled(const double *X, int n, const double *D, double *norms,
                                cudaStream_t st) {
  DQ_KSCOPE(KF_STABAUX, st);
  column_norms_kernel<<<(n + 127) / 128, 128, 0, st>>>(X, n, D, norms);
  return cudaGetLastError();
}

// Bitonic sort of (key desc, index asc) in one CTA.
__global__ void argsort_desc_kernel(const double *key, int n, int npow2, int *perm) {
  extern __shared__ unsigned char raw[];
  double *k = reinterpret_cast<double *>(raw);
  int *ix = reinterpret_cast<int *>(k + npow2);
  // real keys are norms >= 0 (NaN mapped to -0.5); padding is -inf, so the
  // first n sorted entries are always real indices < n
  for (int i = threadIdx.x; i < npow2; i += blockDim.x) {
    const double kv = (i < n) ? key[i] : 0.0;
    k[i] = (i < n) ? (kv != kv ? -0.5 : kv) : -1.0 / 0.0;
    ix[i] = i;
  }
  __syncthreads();
  for (int size = 2; size <= npow2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < npow2; i += blockDim.x) {
        const int jx = i ^ stride;
        if (jx > i) {
          // "before(a, b)": a sorts before b if key larger, ties by smaller index
          const bool up = ((i & size) == 0);
          const bool i_before_j = (k[i] > k[jx]) || (k[i] == k[jx] && ix[i] < ix[jx]);
          if (up != i_before_j) {
            const double tk = k[i];
            k[i] = k[jx];
            k[jx] = tk;
            const int ti = ix[i];
            ix[i] = ix[jx];
            ix[jx] = ti;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) perm[i] = ix[i];
}
cudaError_t argsort_desc(const double *key, int n, int *perm, cudaStream_t st) {
  int np = 1;
  while (np < n) np <<= 1;
  if (np > 8192) return cudaErrorInvalidValue;
  const size_t smem = (size_t)np * (sizeof(double) + sizeof(int));
  cudaError_t e = cudaFuncSetAttribute(argsort_desc_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  DQ_KSCOPE(KF_STABAUX, st);
  argsort_desc_kernel<<<1, 1024, smem, st>>>(key, n, np, perm);
  return cudaGetLastError();
}

__global__ void permute_udv_kernel(const double *X, const double *D, const double *T,
                                   const int *perm, int n, double *Xp, double *Dp, double *Tp) {
  const long total = (long)n * n;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), c = (int)(e % n);
    Xp[e] = X[(size_t)i * n + perm[c]];
    Tp[e] = T[(size_t)perm[i] * n + c];
    if (i == 0) Dp[c] = D[perm[c]];
  }
}
cudaError_t permute_udv(const double *X, const double *D, const double *T, const int *perm, int n,
                        double *Xp, double *Dp, double *Tp, cudaStream_t st) {
  DQ_KSCOPE(KF_STABAUX, st);
  permute_udv_kernel<<<grid_for((long)n * n), 256, 0, st>>>(X, D, T, perm, n, Xp, Dp, Tp);
  return cudaGetLastError();
}

__global__ void udv_diag_kernel(const double *R, int n, const double *Dp, double *Dnew) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) Dnew[i] = fabs(R[(size_t)i * n + i]) * Dp[i];
}
__global__ void udv_scale_kernel(double *R, int n, const double *Dp, const double *Dnew) {
  const long total = (long)n * n;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    R[e] = (j >= i) ? R[e] * (Dp[j] / Dnew[i]) : 0.0;
  }
}
cudaError_t udv_diag_and_scale(double *R, int n, const double *Dp, double *Dnew, cudaStream_t st) {
  {
    DQ_KSCOPE(KF_STABAUX, st);
    udv_diag_kernel<<<(n + 255) / 256, 256, 0, st>>>(R, n, Dp, Dnew);
  }
  DQ_KSCOPE(KF_STABAUX, st);
  udv_scale_kernel<<<grid_for((long)n * n), 256, 0, st>>>(R, n, Dp, Dnew);
  return cudaGetLastError();
}

template <typename TB>
__global__ void max_abs_diff_kernel(const double *A, const TB *B, long total, double *out) {
  double mx = 0.0;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const double d = fabs(A[e] - (double)B[e]);
    mx = (d > mx || d != d) ? d : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double v = __shfl_down_sync(0xffffffffu, mx, o);
    mx = (v > mx || v != v) ? v : mx;
  }
  if ((threadIdx.x & 31) == 0) {
    // non-negative doubles order like their bit patterns; NaN maps above +inf
    const unsigned long long bits = (mx != mx) ? 0x7ff8000000000000ull
                                               : (unsigned long long)__double_as_longlong(mx);
    atomicMax(reinterpret_cast<unsigned long long *>(out), bits);
  }
}
cudaError_t max_abs_diff_f64(const double *A, const double *B, int n, double *out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  DQ_KSCOPE(KF_STABAUX, st);
  max_abs_diff_kernel<double><<<grid_for((long)n * n, 1024), 256, 0, st>>>(A, B, (long)n * n, out);
  return cudaGetLastError();
}
cudaError_t max_abs_diff_f32(const double *A, const float *B, int n, double *out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  DQ_KSCOPE(KF_STABAUX, st);
  max_abs_diff_kernel<float><<<grid_for((long)n * n, 1024), 256, 0, st>>>(A, B, (long)n * n, out);
  return cudaGetLastError();
}

__global__ void f64_to_f32_kernel(const double *A, float *B, long n) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    B[e] = (float)A[e];
}
__global__ void f32_to_f64_kernel(const float *A, double *B, long n) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    B[e] = (double)A[e];
}
cudaError_t convert_f64_to_f32(const double *A, float *B, long n, cudaStream_t st) {
  DQ_KSCOPE(KF_STABAUX, st);
  f64_to_f32_kernel<<<grid_for(n), 256, 0, st>>>(A, B, n);
  return cudaGetLastError();
}
cudaError_t convert_f32_to_f64(const float *A, double *B, long n, cudaStream_t st) {
  DQ_KSCOPE(KF_STABAUX, st);
  f32_to_f64_kernel<<<grid_for(n), 256, 0, st>>>(A, B, n);
  return cudaGetLastError();
}

__global__ void split_scales_kernel(const double *D, int n, double *dmax_inv, double *dmin) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double d = D[i];
    dmax_inv[i] = 1.0 / fmax(d, 1.0);
    dmin[i] = fmin(d, 1.0);
  }
}
cudaError_t split_scales(const double *D, int n, double *dmax_inv, double *dmin, cudaStream_t st) {
  DQ_KSCOPE(KF_STABAUX, st);
  split_scales_kernel<<<(n + 255) / 256, 256, 0, st>>>(D, n, dmax_inv, dmin);
  return cudaGetLastError();
}

}  // namespace dq
