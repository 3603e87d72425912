// Delayed-update Metropolis over one time slice.
//
// Sites are proposed in index order in blocks S of k consecutive sites. For a
// block, everything the sequential Sherman-Morrison updates need lies in the
// k x k sub-block g = G[S,S] (submatrix form of the delayed update): the
// decisions follow the current block g~ under the accepted flips, and the m
// accepted flips P then compose into one Woodbury update of the whole G,
//     G' = G - G[:,P] Gamma (E_P - G[P,:]),  Gamma = (Delta^{-1} + I - G[P,P])^{-1},
// which equals the sequential rank-one updates exactly. The flush is that
// rank-m update, written as G' = G - A B^T with A = G[:,S] alpha^T and
// B^T = beta (E_S - G[S,:]), where alpha^T beta = Gamma on (P, P).
//
// Kernels: the Metropolis block (one CTA: 16 warps with the block in
// registers for k <= 32, else a shared-memory form; FP64 or double-float),
// the A factor (and, for the double-float flush, the B factor), the
// look-ahead G'[S',S'] of the next block from the pre-flush G (so that the
// next block's decisions can run while this block's flush streams G), and
// the flush itself -- FP64 / FP32 by column stripes, or double-float by
// 64 x 64 tiles -- whose epilogue gathers G[:,S'] and G[S',:] of the next
// block. The tensor-core flush of the mixed precision sweep is in
// flush_tc.cu.
#include <algorithm>
#include <type_traits>

#include "df64.cuh"
#include "kernels.cuh"

namespace dq {

// ----------------------------------------------------------------- gather
// Gcol[i*K + t] = G[i, s0 + t] (t < kb, zero for kb <= t < K),
// Grow[t*N + j] = G[s0 + t, j].
template <typename T>
__global__ void gather_block_kernel(int N, int s0, int kb, int K, const T *__restrict__ G,
                                    T *__restrict__ Gcol, T *__restrict__ Grow) {
  const long total = (long)N * K;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e / K), t = (int)(e % K);
    Gcol[e] = (t < kb) ? G[(size_t)i * N + s0 + t] : T(0);
  }
  const long total2 = (long)kb * N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total2;
       e += (long)gridDim.x * blockDim.x) {
    const int t = (int)(e / N), j = (int)(e % N);
    Grow[e] = G[(size_t)(s0 + t) * N + j];
  }
}

template <typename T>
cudaError_t launch_gather(int N, int s0, int kb, int K, const T *G, T *Gcol, T *Grow,
                          cudaStream_t st) {
  const long work = (long)N * K;
  int grid = (int)((work + 255) / 256);
  if (grid > 4096) grid = 4096;
  if (grid < 1) grid = 1;
  DQ_KSCOPE(KF_BLOCKAUX, st);
  gather_block_kernel<T><<<grid, 256, 0, st>>>(N, s0, kb, K, G, Gcol, Grow);
  return cudaGetLastError();
}
template cudaError_t launch_gather<double>(int, int, int, int, const double *, double *, double *,
                                           cudaStream_t);
template cudaError_t launch_gather<float>(int, int, int, int, const float *, float *, float *,
                                          cudaStream_t);

// ----------------------------------------------------------------- Metropolis block
// Decisions and the Woodbury coefficients of one block S of kb <= 64 sites.
//
// The decisions need only the current k x k block g~ = G~[S,S]: the ratio of
// site j is r = 1 + delta_j (1 - g~_jj) with delta_j = e^{-2 lambda s_j} - 1,
// R = e^{2 lambda s_j} r^2, and an accepted flip changes the block by the
// Sherman-Morrison step g~ <- g~ - (delta/r) g~[:,j] (e_j - g~[j,:]). Only the
// trailing part (rows and columns after j) matters for later decisions, so
// each accepted flip updates that part in shared memory (right-looking).
//
// The m accepted flips P = (p_1 .. p_m), in order, then compose into one
// Woodbury update of the whole G:
//     G' = G - G[:,P] Gamma (E_P - G[P,:]),   Gamma = (Delta^{-1} + I - G[P,P])^{-1},
// Delta = diag(delta_p), G the block's input. Gauss-Jordan elimination of
// Delta^{-1} + I - G[P,P] in acceptance order without pivoting has exactly the
// sequential quantities r_p / delta_p as pivots (the Schur complements), so
// it is as stable as the one-at-a-time updates. Gamma is computed in FP64.
// Output in the form of the flush kernels: row r of alpha is column r of
// Gamma scattered to the block positions of P, row r of beta selects p_r:
//     alpha^T beta = Gamma on (P, P), zero elsewhere.
//
// Arithmetic of the block: FP64, or double-float (df64, ~2^-47, on the FP32
// units) in mixed precision, where the FP64 pipe (1/64 of FP32 on this part)
// would make the serial decision chain the critical path.
template <typename T> struct MetroMath;
template <> struct MetroMath<double> {
  static __device__ __forceinline__ double from(double x) { return x; }
  static __device__ __forceinline__ double to(double x) { return x; }
  static __device__ __forceinline__ double mad(double a, double b, double c) { return fma(a, b, c); }
  static __device__ __forceinline__ double div(double a, double b) { return a / b; }
  static __device__ __forceinline__ bool positive(double a) { return a > 0.0; }
  static __device__ __forceinline__ bool finite(double a) { return isfinite(a); }
  static __device__ __forceinline__ float hi(double a) { return (float)a; }
};
template <> struct MetroMath<df64> {
  static __device__ __forceinline__ df64 from(double x) { return df_from(x); }
  static __device__ __forceinline__ double to(df64 x) { return df_to(x); }
  static __device__ __forceinline__ df64 mad(df64 a, df64 b, df64 c) { return a * b + c; }
  // one FP32 quotient refined by one double-float residual step
  static __device__ __forceinline__ df64 div(df64 a, df64 b) {
    const float q1 = a.hi / b.hi;
    const df64 r = a - b * df64(q1, 0.f);
    const float q2 = r.hi / b.hi;
    return fast_two_sum(q1, q2);
  }
  static __device__ __forceinline__ bool positive(df64 a) { return a.hi > 0.f || (a.hi == 0.f && a.lo > 0.f); }
  static __device__ __forceinline__ bool finite(df64 a) { return isfinite(a.hi); }
  static __device__ __forceinline__ float hi(df64 a) { return a.hi; }
};

// One CTA of 4 x NC threads (NC = 32 or 64 block columns): thread (w, v) owns
// column v and the rows i = w (mod 4) of the block, so that the work of a
// trailing update is spread over the four SM sub-partitions. The decision of
// site j is taken by the thread that also wrote g~_jj last (column j, row
// group j mod 4), and the one barrier per site publishes it.
template <int NC, typename T>
__global__ void __launch_bounds__(4 * NC)
    metropolis_block_kernel(MetroArgs a, const void *__restrict__ g_, int g_is_f32, int8_t *s,
                            const uint8_t *__restrict__ forced, double *__restrict__ alpha_out,
                            double *__restrict__ beta_out, int *accept_count, int *status,
                            unsigned long long *total) {
  using MM = MetroMath<T>;
  constexpr int LD = NC + 1;
  extern __shared__ __align__(16) unsigned char msm_raw[];
  T *g = reinterpret_cast<T *>(msm_raw);  // NC x LD: current block, then Delta^{-1} + I - G[P,P] -> Gamma
  T *g0 = g + NC * LD;                    // NC x LD: the input block
  __shared__ T s_c[2], s_pinv;
  __shared__ int s_dec[2];
  __shared__ int s_P[NC];
  __shared__ T s_delta[NC];
  __shared__ double s_u[NC];
  __shared__ int s_spin[NC];
  const int kb = a.kb;
  const int tid = threadIdx.x, v = tid % NC, w = tid / NC;

  for (int e = tid; e < kb * kb; e += 4 * NC) {
    const int r = e / kb, c = e % kb;
    const size_t off = (size_t)r * a.ld_g + c;
    const double x = g_is_f32 ? (double)static_cast<const float *>(g_)[off]
                              : static_cast<const double *>(g_)[off];
    g[r * LD + c] = MM::from(x);
    g0[r * LD + c] = MM::from(x);
  }
  if (w == 0 && v < kb) {
    const uint4 r = philox4x32_10(make_uint4((uint32_t)(a.s0 + v), (uint32_t)a.slice0, a.c2, a.c3),
                                  a.k0, a.k1);
    s_u[v] = uniform53(r.x, r.y);
    s_spin[v] = (int)s[a.s0 + v];
  }
  __syncthreads();

  const T one = MM::from(1.0);
  const T dpos = MM::from(a.em2l - 1.0), dneg = MM::from(a.e2l - 1.0);  // delta for s = +1 / -1
  const T epos = MM::from(a.e2l), eneg = MM::from(a.em2l);
  int m = 0;
  bool failed = false;
  for (int j = 0; j < kb; ++j) {
    if (v == j && w == (j & 3)) {
      // delta = e^{-2 lambda s} - 1, r = 1 + delta (1 - g~_jj), R = e^{2 lambda s} r^2
      const int sj = s_spin[j];
      const T delta = sj > 0 ? dpos : dneg;
      const T r = MM::mad(delta, one - g[j * LD + j], one);
      const T R = (sj > 0 ? epos : eneg) * r * r;
      int dec;
      if (!MM::positive(R) || !MM::finite(R))
        dec = -1;
      else if (forced)
        dec = forced[j] ? 1 : 0;
      else
        dec = MM::positive(R - MM::from(s_u[j])) ? 1 : 0;  // accept iff u < R
      s_dec[j & 1] = dec;
      if (dec > 0) s_c[j & 1] = MM::div(delta, r);
    }
    __syncthreads();
    const int dec = s_dec[j & 1];
    if (dec < 0) {
      failed = true;
      break;
    }
    if (!dec) continue;
    if (tid == 0) {
      s_P[m] = j;
      s_delta[m] = s_spin[j] > 0 ? dpos : dneg;
      s_spin[j] = -s_spin[j];
      s[a.s0 + j] = (int8_t)s_spin[j];
    }
    ++m;
    // trailing update g~[i][v] += c g~[j][v] g~[i][j] for i, v > j
    // (the e_j term of the step only touches column j, which is done with)
    if (v > j && v < kb) {
      const T cg = s_c[j & 1] * g[j * LD + v];
      int i = j + 1;
      i += (w - i) & 3;  // first row > j in this thread's row group
      for (; i < kb; i += 4) g[i * LD + v] = MM::mad(cg, g[i * LD + j], g[i * LD + v]);
    }
  }
  __syncthreads();

  // Gamma = (Delta^{-1} + I - G[P,P])^{-1} by in-place Gauss-Jordan, P in order
  for (int e = tid; e < m * m; e += 4 * NC) {
    const int r = e / m, c = e % m;
    const T dinv = MM::div(one, s_delta[r]);
    g[r * LD + c] = (r == c ? one + dinv : MM::from(0.0)) - g0[s_P[r] * LD + s_P[c]];
  }
  __syncthreads();
  for (int p = 0; p < m; ++p) {
    if (tid == 0) s_pinv = MM::div(one, g[p * LD + p]);
    __syncthreads();
    const T pinv = s_pinv;
    if (w == (p & 3) && v < m) g[p * LD + v] = (v == p) ? pinv : g[p * LD + v] * pinv;
    T f[NC / 4];
#pragma unroll
    for (int q = 0; q < NC / 4; ++q) {
      const int i = w + 4 * q;
      f[q] = (i < m && i != p) ? g[i * LD + p] : MM::from(0.0);
    }
    __syncthreads();
    if (v < m) {
      const T rp = g[p * LD + v];
#pragma unroll
      for (int q = 0; q < NC / 4; ++q) {
        const int i = w + 4 * q;
        if (i < m && i != p)
          g[i * LD + v] = (v == p) ? -(f[q] * pinv) : MM::mad(-f[q], rp, g[i * LD + v]);
      }
    }
    __syncthreads();
  }

  // alpha[r][P_q] = Gamma[q][r], beta[r][P_r] = 1 (row stride K); the rest zero
  for (int e = tid; e < a.K * a.K; e += 4 * NC) {
    alpha_out[e] = 0.0;
    beta_out[e] = 0.0;
  }
  __syncthreads();
  for (int e = tid; e < m * m; e += 4 * NC) {
    const int q = e / m, r = e % m;
    alpha_out[r * a.K + s_P[q]] = MM::to(g[q * LD + r]);
  }
  for (int r = tid; r < m; r += 4 * NC) beta_out[r * a.K + s_P[r]] = 1.0;
  if (tid == 0) {
    *accept_count = m;
    if (failed) *status = 1;
    if (total) atomicAdd(total, (unsigned long long)m);
  }
}

// The same block for kb <= 32 on 16 warps, the block in registers. Warp w
// holds rows w and w + 16 of g~ (lane v = column v), so that the trailing
// update of an accepted flip costs every warp two multiply-adds. Site j: the
// warp holding row j takes the decision (an FP32 screen decides unless the
// uniform lies within 1e-5 of the ratio, the full arithmetic otherwise, so
// the decisions are those of metropolis_block_kernel), publishes the decision,
// its coefficient delta / r and row j in shared memory, and one CTA barrier
// hands them to the other warps, which update their rows i > j with one
// broadcast of column j within the warp. Gauss-Jordan on Delta^{-1} + I -
// G[P,P] then runs on the same layout with one barrier per pivot; the pivot of
// step p is the Schur complement r_p / delta_p of the decision chain, so its
// reciprocal is the flip's coefficient delta_p / r_p. All global loads are
// issued before the conversions that use them.
template <typename T>
__device__ __forceinline__ T shfl_t(T x, int src);
template <>
__device__ __forceinline__ double shfl_t<double>(double x, int src) {
  return __shfl_sync(0xffffffffu, x, src);
}
template <>
__device__ __forceinline__ df64 shfl_t<df64>(df64 x, int src) {
  return df64(__shfl_sync(0xffffffffu, x.hi, src), __shfl_sync(0xffffffffu, x.lo, src));
}

constexpr int kMetroCta = 512;

template <typename T>
__global__ void __launch_bounds__(kMetroCta)
    metropolis_cta_kernel(MetroArgs a, const void *__restrict__ g_, int g_is_f32, int8_t *s,
                          const uint8_t *__restrict__ forced, double *__restrict__ alpha_out,
                          double *__restrict__ beta_out, int *accept_count, int *status,
                          unsigned long long *total) {
  using MM = MetroMath<T>;
  __shared__ T s_row[2][32];
  __shared__ T s_c[2];
  __shared__ int s_dec[2];
  __shared__ int s_P[32];
  __shared__ T s_dinv[32], s_cinv[32];
  __shared__ double s_u[32];
  __shared__ int s_spin[32], s_forced[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int kb = a.kb;
  auto gin = [&](int r, int c) -> double {
    const size_t off = (size_t)r * a.ld_g + c;
    return g_is_f32 ? (double)static_cast<const float *>(g_)[off] : static_cast<const double *>(g_)[off];
  };
  const T one = MM::from(1.0), zero = MM::from(0.0);
  const T dpos = MM::from(a.em2l - 1.0), dneg = MM::from(a.e2l - 1.0);  // delta for s = +1 / -1
  const T epos = MM::from(a.e2l), eneg = MM::from(a.em2l);
  const float dposf = (float)(a.em2l - 1.0), dnegf = (float)(a.e2l - 1.0);
  const float eposf = (float)a.e2l, enegf = (float)a.em2l;

  T x[2];
  {
    double gr[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = warp + 16 * q;
      gr[q] = (i < kb && lane < kb) ? gin(i, lane) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) x[q] = MM::from(gr[q]);
  }
  if (tid < kb) {
    const uint4 r = philox4x32_10(make_uint4((uint32_t)(a.s0 + tid), (uint32_t)a.slice0, a.c2, a.c3), a.k0, a.k1);
    s_u[tid] = uniform53(r.x, r.y);
    s_spin[tid] = (int)s[a.s0 + tid];
    s_forced[tid] = forced ? (int)forced[tid] : 0;
  }
  __syncthreads();

  int m = 0, failed = 0;
#pragma unroll 1
  for (int j = 0; j < kb; ++j) {
    const int buf = j & 1;
    if (warp == (j & 15)) {
      const T rowj = (j >> 4) ? x[1] : x[0];  // g~[j][lane]
      const T gjj = shfl_t(rowj, j);
      const int sj = s_spin[j];
      const double uj = s_u[j];
      // delta = e^{-2 lambda s} - 1, r = 1 + delta (1 - g~_jj), R = e^{2 lambda s} r^2
      const T delta = sj > 0 ? dpos : dneg;
      int dec = -2;
      if (!forced) {
        const float rf = fmaf(sj > 0 ? dposf : dnegf, 1.f - MM::hi(gjj), 1.f);
        const float Rf = (sj > 0 ? eposf : enegf) * rf * rf;
        const float uf = (float)uj;
        if (Rf > 0.f && Rf < 1e30f) {
          if (uf < Rf * (1.f - 1e-5f)) dec = 1;
          else if (uf > Rf * (1.f + 1e-5f)) dec = 0;
        }
      }
      const T r = MM::mad(delta, one - gjj, one);
      if (dec == -2) {
        const T R = (sj > 0 ? epos : eneg) * r * r;
        if (!MM::positive(R) || !MM::finite(R))
          dec = -1;
        else if (forced)
          dec = s_forced[j] ? 1 : 0;
        else
          dec = MM::positive(R - MM::from(uj)) ? 1 : 0;  // accept iff u < R
      }
      s_row[buf][lane] = rowj;
      if (lane == 0) {
        s_dec[buf] = dec;
        if (dec > 0) {
          const T cj = MM::div(delta, r);
          s_c[buf] = cj;
          s_P[m] = j;
          s_dinv[m] = MM::div(one, delta);
          s_cinv[m] = cj;
          s_spin[j] = -sj;
        }
      }
    }
    __syncthreads();
    const int dec = s_dec[buf];
    if (dec < 0) {
      failed = 1;
      break;
    }
    if (dec == 0) continue;
    // trailing update g~[i][v] += c g~[j][v] g~[i][j] for the rows i > j of
    // this warp (columns v <= j are done with and take harmless values)
    const T cg = s_c[buf] * s_row[buf][lane];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = warp + 16 * q;
      const T xi = shfl_t(x[q], j);
      if (i > j) x[q] = MM::mad(cg, xi, x[q]);
    }
    ++m;
  }
  if (tid < kb) s[a.s0 + tid] = (int8_t)s_spin[tid];

  // Gamma = (Delta^{-1} + I - G[P,P])^{-1} by in-place Gauss-Jordan, P in order
  {
    double g0[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = warp + 16 * q;
      g0[q] = (i < m && lane < m) ? gin(s_P[i], s_P[lane]) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = warp + 16 * q;
      x[q] = (i < m && lane < m) ? (i == lane ? one + s_dinv[i] : zero) - MM::from(g0[q]) : zero;
    }
  }
#pragma unroll 1
  for (int p = 0; p < m; ++p) {
    const int buf = p & 1;
    const T pinv = s_cinv[p];
    if (warp == (p & 15)) {
      const T xp = (p >> 4) ? x[1] : x[0];
      const T nr = (lane == p) ? pinv : xp * pinv;
      if (p >> 4)
        x[1] = nr;
      else
        x[0] = nr;
      s_row[buf][lane] = nr;
    }
    __syncthreads();
    const T rp = s_row[buf][lane];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = warp + 16 * q;
      const T f = shfl_t(x[q], p);
      if (i < m && i != p) x[q] = (lane == p) ? -(f * pinv) : MM::mad(-f, rp, x[q]);
    }
  }

  // alpha[r][P_q] = Gamma[q][r], beta[r][P_r] = 1 (row stride K); the rest zero
  for (int e = tid; e < a.K * a.K; e += kMetroCta) {
    alpha_out[e] = 0.0;
    beta_out[e] = 0.0;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int i = warp + 16 * q;
    if (i < m && lane < m) alpha_out[lane * a.K + s_P[i]] = MM::to(x[q]);
  }
  if (tid < m) beta_out[tid * a.K + s_P[tid]] = 1.0;
  if (a.perm && tid < a.K) a.perm[tid] = tid < m ? s_P[tid] : -1;
  if (tid == 0) {
    *accept_count = m;
    if (failed) *status = 1;
    if (total) atomicAdd(total, (unsigned long long)m);
  }
}

template <int NC, typename T>
static cudaError_t launch_metro_t(const MetroArgs &a, const void *g, bool g_f32, int8_t *s,
                                  const uint8_t *forced, double *alpha, double *beta, int *accept_count,
                                  int *status, unsigned long long *total, cudaStream_t st,
                                  int reserve_smem) {
  // reserve_smem > the block's own need claims that much shared memory so
  // that no CTA of a concurrently running kernel shares the SM; the kernel's
  // static shared memory (under 3 KB) comes on top
  const size_t need = (size_t)2 * NC * (NC + 1) * sizeof(T);
  size_t smem = need;
  if ((size_t)reserve_smem > smem) smem = std::min<size_t>((size_t)reserve_smem, 224 * 1024);
  const void *fn = (const void *)metropolis_block_kernel<NC, T>;
  cudaError_t e = ensure_smem_attr(fn, (int)std::max<size_t>(smem, 200 * 1024));
  if (e != cudaSuccess) return e;
  DQ_KSCOPE(KF_METRO, st);
  metropolis_block_kernel<NC, T><<<1, 4 * NC, smem, st>>>(a, g, g_f32 ? 1 : 0, s, forced, alpha, beta,
                                                          accept_count, status, total);
  return cudaGetLastError();
}

// the 16-warp form of the block (kb <= 32)
template <typename T>
static cudaError_t launch_metro_cta(const MetroArgs &a, const void *g, bool g_f32, int8_t *s,
                                    const uint8_t *forced, double *alpha, double *beta, int *accept_count,
                                    int *status, unsigned long long *total, cudaStream_t st, int reserve_smem) {
  const size_t smem = reserve_smem > 0 ? std::min<size_t>((size_t)reserve_smem, 224 * 1024) : 0;
  const void *fn = (const void *)metropolis_cta_kernel<T>;
  if (smem > 0) {
    cudaError_t e = ensure_smem_attr(fn, (int)smem);
    if (e != cudaSuccess) return e;
  }
  DQ_KSCOPE(KF_METRO, st);
  metropolis_cta_kernel<T><<<1, kMetroCta, smem, st>>>(a, g, g_f32 ? 1 : 0, s, forced, alpha, beta, accept_count,
                                                      status, total);
  return cudaGetLastError();
}

cudaError_t launch_metropolis(const MetroArgs &a, const void *g, bool g_f32, int8_t *s,
                              const uint8_t *forced, double *alpha, double *beta, int *accept_count,
                              int *status, unsigned long long *total, cudaStream_t st, bool df,
                              int reserve_smem) {
  if (a.kb < 1 || a.kb > 64 || a.kb > a.K) return cudaErrorInvalidValue;
  const bool wide = a.kb > 32;
  if (!wide)
    return df ? launch_metro_cta<df64>(a, g, g_f32, s, forced, alpha, beta, accept_count, status, total, st,
                                       reserve_smem)
              : launch_metro_cta<double>(a, g, g_f32, s, forced, alpha, beta, accept_count, status, total, st,
                                         reserve_smem);
  if (df)
    return wide ? launch_metro_t<64, df64>(a, g, g_f32, s, forced, alpha, beta, accept_count, status, total, st, reserve_smem)
                : launch_metro_t<32, df64>(a, g, g_f32, s, forced, alpha, beta, accept_count, status, total, st, reserve_smem);
  return wide ? launch_metro_t<64, double>(a, g, g_f32, s, forced, alpha, beta, accept_count, status, total, st, reserve_smem)
              : launch_metro_t<32, double>(a, g, g_f32, s, forced, alpha, beta, accept_count, status, total, st, reserve_smem);
}

// ----------------------------------------------------------------- A = G[:,S] alpha
// A[i][mm] = sum_{u < kb} Gcol[i][u] alpha[mm][u] for mm < m, zero for m <= mm < K.
// FP64 arithmetic; output T (double / float) or, for the double-float flush,
// a (hi, lo) FP32 pair.
template <typename T, typename TA>
__global__ void __launch_bounds__(256)
    amat_kernel(int N, int K, int kb, int ldc, const T *__restrict__ Gcol,
                const double *__restrict__ alpha, int lda, const int *__restrict__ accept_count,
                TA *__restrict__ A) {
  const int m = accept_count ? *accept_count : kb;
  const int rows_per = 256 / K;
  const int i = blockIdx.x * rows_per + threadIdx.x / K;
  const int mm = threadIdx.x % K;
  if (i >= N) return;
  double v = 0.0;
  if (mm < m) {
    const T *gc = Gcol + (size_t)i * ldc;
    const double *ar = alpha + (size_t)mm * lda;
    for (int u = 0; u < kb; ++u) v = fma((double)gc[u], ar[u], v);
  }
  if constexpr (std::is_same<TA, float2>::value)
    A[(size_t)i * K + mm] = split_df_bits(v);
  else
    A[(size_t)i * K + mm] = (TA)v;
}

// ----------------------------------------------------------------- rank-m flush
// G[:, J] -= A B_J, B_J = [beta_m] (E_S - Grow)[:, J], one CTA per stripe J
// of SW consecutive columns covering all N rows, so B_J (K x SW) is formed
// once. Thread (rsub, col) owns column j0 + col and rows rsub, rsub + 256/SW,
// ...; it keeps its column of B in registers and streams G once (read,
// subtract, write). The epilogue gathers the next block's rows / columns.
//   T  = storage type of G (double or float)
//   DF = FP64-accurate product on the FP32 units: A and B as (hi, lo) FP32
//        pairs, each MAC an exact FP32 product plus cross terms, accumulated
//        with TwoSum (12 FP32 operations); T must be double.
__device__ __forceinline__ void df_mac(float ah, float al, float bh, float bl, float &sh, float &sl) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  const float t = sh + p;
  const float z = t - sh;
  const float err = (sh - (t - z)) + (p - z);
  sh = t;
  sl += err + e;
}

template <typename T, int K, int SW, bool DF>
__global__ void __launch_bounds__(256)
    flush_kernel(FlushArgs a, T *__restrict__ G, const void *__restrict__ A_,
                 const T *__restrict__ Grow, const double *__restrict__ beta,
                 const int *__restrict__ accept_count, T *__restrict__ Gcol_next,
                 T *__restrict__ Grow_next) {
  constexpr int RSTEP = 256 / SW;
  __shared__ double Bsh[K][SW];
  const int tid = threadIdx.x, col = tid % SW, rsub = tid / SW;
  const int N = a.N;
  const int j0 = blockIdx.x * SW, j = j0 + col;
  const bool jok = j < N;
  const int m = accept_count ? *accept_count : a.kb;

  // B_J[mm][c] = beta[mm][j - s0] (j in S) - sum_u beta[mm][u] Grow[u][j]
  if (m > 0) {
    for (int e = tid; e < K * SW; e += 256) {
      const int mm = e / SW, c = e % SW, jj = j0 + c;
      double w = 0.0;
      if (jj < N && mm < m) {
        const int js = jj - a.s0;
        if (js >= 0 && js < a.kb) w = beta[mm * a.ldb + js];
        for (int u = 0; u < a.kb; ++u) w = fma(-beta[mm * a.ldb + u], (double)Grow[(size_t)u * N + jj], w);
      }
      Bsh[mm][c] = w;
    }
  }
  __syncthreads();

  using WT = typename std::conditional<DF, float, T>::type;
  WT bh[K], bl[DF ? K : 1];
#pragma unroll
  for (int p = 0; p < K; ++p) {
    const double w = (m > 0) ? Bsh[p][col] : 0.0;
    if constexpr (DF) {
      const float2 sp = split_df_bits(w);
      bh[p] = sp.x;
      bl[p] = sp.y;
    } else {
      bh[p] = (T)w;
    }
  }
  if (!jok) return;

  for (int i = rsub; i < N; i += RSTEP) {
    T acc = T(0);
    if (m > 0) {
      if constexpr (DF) {
        const float4 *ap = reinterpret_cast<const float4 *>(static_cast<const float2 *>(A_) + (size_t)i * K);
        float sh = 0.f, sl = 0.f;
#pragma unroll
        for (int p = 0; p < K; p += 2) {
          if (p < m) {
            const float4 v = ap[p >> 1];
            df_mac(v.x, v.y, bh[p], bl[p], sh, sl);
            df_mac(v.z, v.w, bh[p + 1], bl[p + 1], sh, sl);
          }
        }
        acc = f2d_bits(sh) + f2d_bits(sl);
      } else {
        const T *ap = static_cast<const T *>(A_) + (size_t)i * K;
#pragma unroll
        for (int p = 0; p < K; p += 4) {
          if (p < m) {
            if constexpr (sizeof(T) == 4) {
              const float4 g4 = *reinterpret_cast<const float4 *>(ap + p);
              acc = fmaf(g4.x, bh[p], acc);
              acc = fmaf(g4.y, bh[p + 1], acc);
              acc = fmaf(g4.z, bh[p + 2], acc);
              acc = fmaf(g4.w, bh[p + 3], acc);
            } else {
              const double2 g0 = *reinterpret_cast<const double2 *>(ap + p);
              const double2 g1 = *reinterpret_cast<const double2 *>(ap + p + 2);
              acc = fma(g0.x, bh[p], acc);
              acc = fma(g0.y, bh[p + 1], acc);
              acc = fma(g1.x, bh[p + 2], acc);
              acc = fma(g1.y, bh[p + 3], acc);
            }
          }
        }
      }
    }
    T *gp = G + (size_t)i * N + j;
    const T val = *gp - acc;
    if (m > 0) *gp = val;
    if (a.nkb > 0) {
      const int it = i - a.ns0, jt = j - a.ns0;
      if (it >= 0 && it < a.nkb) Grow_next[(size_t)it * N + j] = val;
      if (jt >= 0 && jt < K) Gcol_next[(size_t)i * K + jt] = (jt < a.nkb) ? val : T(0);
    }
  }
}

// ----------------------------------------------------------------- tiled double-float flush
// A (N x K pairs, as amat_kernel) and
//   B[mm][j] = beta[mm][j - s0] [j in S] - sum_w beta[mm][w] Grow[w][j]
// (K x N pairs, rows mm >= m zero) of the double-float flush in one launch,
// both accumulated in double-float arithmetic on the FP32 units: blocks
// [0, nblk_a) form A, the rest B (one column per thread, one mm per block row).
template <int K>
__global__ void __launch_bounds__(256)
    amat_bmat_df_kernel(FlushArgs a, const double *__restrict__ Gcol,
                        const double *__restrict__ alpha, const double *__restrict__ Grow,
                        const double *__restrict__ beta, const int *__restrict__ accept_count,
                        float2 *__restrict__ A, float2 *__restrict__ B, int nblk_a) {
  const int N = a.N, tid = threadIdx.x;
  const int m = accept_count ? *accept_count : a.kb;
  if ((int)blockIdx.x < nblk_a) {
    constexpr int rows_per = 256 / K;
    const int i = blockIdx.x * rows_per + tid / K, mm = tid % K;
    if (i >= N) return;
    df64 v(0.f, 0.f);
    if (mm < m) {
      const double *gc = Gcol + (size_t)i * a.ldc;
      const double *ar = alpha + (size_t)mm * a.lda;
      for (int u = 0; u < a.kb; ++u) v = df_from(gc[u]) * df_from(ar[u]) + v;
    }
    A[(size_t)i * K + mm] = make_float2(v.hi, v.lo);
  } else {
    const int nbj = (N + 255) / 256;
    const int b = blockIdx.x - nblk_a, mm = b / nbj;
    const int j = (b % nbj) * 256 + tid;
    if (j >= N) return;
    df64 w(0.f, 0.f);
    if (mm < m) {
      const int js = j - a.s0;
      if (js >= 0 && js < a.kb) w = df_from(beta[mm * a.ldb + js]);
      for (int u = 0; u < a.kb; ++u) w = w - df_from(beta[mm * a.ldb + u]) * df_from(Grow[(size_t)u * N + j]);
    }
    B[(size_t)mm * N + j] = make_float2(w.hi, w.lo);
  }
}

// G[i0:i0+64, j0:j0+64] -= A B with A (N x K) and B (K x N) as FP32 pairs:
// one 64 x 64 tile per CTA, 256 threads, a 4 x 4 block of outputs per thread
// (rows 4 ty .. 4 ty + 3, columns 4 tx .. 4 tx + 3), operands staged once in
// shared memory (A transposed, row stride 66 pairs). Abuf holds A (N x K
// pairs) followed by B (K x N pairs). Each MAC is the
// double-float product of df_mac; the epilogue subtracts hi + lo from the
// FP64 G and gathers the next block's rows / columns as the stripe kernel does.
constexpr int kDfTile = 64, kDfLdA = 66;

template <int K>
__global__ void __launch_bounds__(256)
    flush_df_tile_kernel(FlushArgs a, double *__restrict__ G, const float2 *__restrict__ A,
                         const float2 *__restrict__ B, const int *__restrict__ accept_count,
                         double *__restrict__ Gcol_next, double *__restrict__ Grow_next, int vec) {
  extern __shared__ __align__(16) float2 dsm[];
  float2 *As = dsm;                      // [K][kDfLdA]
  float2 *Bs = dsm + K * kDfLdA;         // [K][kDfTile]
  const int N = a.N, tid = threadIdx.x;
  const int i0 = blockIdx.y * kDfTile, j0 = blockIdx.x * kDfTile;
  const int ty = tid >> 4, tx = tid & 15;
  const int m = accept_count ? *accept_count : a.kb;
  const bool gather = a.nkb > 0 &&
                      ((i0 < a.ns0 + a.nkb && i0 + kDfTile > a.ns0) || (j0 < a.ns0 + K && j0 + kDfTile > a.ns0));
  if (m == 0 && !gather) return;
  if (m > 0) {
    for (int e = tid; e < kDfTile * K; e += 256) {
      const int r = e / K, k = e % K;
      const int i = i0 + r;
      As[k * kDfLdA + r] = (i < N && k < m) ? A[(size_t)i * K + k] : make_float2(0.f, 0.f);
    }
    for (int e = tid; e < kDfTile * K; e += 256) {
      const int k = e / kDfTile, c = e % kDfTile;
      const int j = j0 + c;
      Bs[k * kDfTile + c] = (j < N && k < m) ? B[(size_t)k * N + j] : make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  float sh[4][4], sl[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) sh[r][c] = sl[r][c] = 0.f;
  for (int k = 0; k < m; ++k) {
    const float4 a01 = *reinterpret_cast<const float4 *>(&As[k * kDfLdA + 4 * ty]);
    const float4 a23 = *reinterpret_cast<const float4 *>(&As[k * kDfLdA + 4 * ty + 2]);
    const float4 b01 = *reinterpret_cast<const float4 *>(&Bs[k * kDfTile + 4 * tx]);
    const float4 b23 = *reinterpret_cast<const float4 *>(&Bs[k * kDfTile + 4 * tx + 2]);
    const float ah[4] = {a01.x, a01.z, a23.x, a23.z}, al[4] = {a01.y, a01.w, a23.y, a23.w};
    const float bh[4] = {b01.x, b01.z, b23.x, b23.z}, bl[4] = {b01.y, b01.w, b23.y, b23.w};
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) df_mac(ah[r], al[r], bh[c], bl[c], sh[r][c], sl[r][c]);
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + 4 * ty + r;
    if (i >= N) continue;
    const int jb = j0 + 4 * tx;
    double v[4];
    if (vec && jb + 3 < N) {
      const double2 g0 = *reinterpret_cast<const double2 *>(&G[(size_t)i * N + jb]);
      const double2 g1 = *reinterpret_cast<const double2 *>(&G[(size_t)i * N + jb + 2]);
      v[0] = g0.x; v[1] = g0.y; v[2] = g1.x; v[3] = g1.y;
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) v[c] = (jb + c < N) ? G[(size_t)i * N + jb + c] : 0.0;
    }
    if (m > 0) {
#pragma unroll
      for (int c = 0; c < 4; ++c) v[c] -= f2d_bits(sh[r][c]) + f2d_bits(sl[r][c]);
      if (vec && jb + 3 < N) {
        *reinterpret_cast<double2 *>(&G[(size_t)i * N + jb]) = make_double2(v[0], v[1]);
        *reinterpret_cast<double2 *>(&G[(size_t)i * N + jb + 2]) = make_double2(v[2], v[3]);
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (jb + c < N) G[(size_t)i * N + jb + c] = v[c];
      }
    }
    if (gather) {
      const int it = i - a.ns0;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = jb + c;
        if (j >= N) continue;
        const int jt = j - a.ns0;
        if (it >= 0 && it < a.nkb) Grow_next[(size_t)it * N + j] = v[c];
        if (jt >= 0 && jt < K) Gcol_next[(size_t)i * K + jt] = (jt < a.nkb) ? v[c] : 0.0;
      }
    }
  }
}

template <int K>
static cudaError_t launch_update_df_tiled(const FlushArgs &a, double *G, void *Abuf,
                                          const double *Grow, const double *beta, const int *acc,
                                          double *Gcol_next, double *Grow_next, cudaStream_t st) {
  // A and B (pairs) were formed by amat_bmat_df_kernel
  const float2 *A = static_cast<const float2 *>(Abuf);
  const float2 *B = static_cast<const float2 *>(Abuf) + (size_t)a.N * K;
  (void)Grow;
  (void)beta;
  const int smem = (int)((size_t)K * (kDfLdA + kDfTile) * sizeof(float2));
  cudaError_t e = ensure_smem_attr((const void *)flush_df_tile_kernel<K>, smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((a.N + kDfTile - 1) / kDfTile, (a.N + kDfTile - 1) / kDfTile);
  DQ_KSCOPE(KF_FLUSH, st);
  add_work(KF_FLUSH, 2.0 * a.N * (double)a.N * a.kb,
           (2.0 * a.N * (double)a.N + 2.0 * a.N * (double)a.kb) * sizeof(double));
  // 16-byte vector access to G only where every row start is 16-byte aligned
  const int vec = (a.N % 2 == 0) && ((reinterpret_cast<uintptr_t>(G) & 15) == 0);
  flush_df_tile_kernel<K><<<grid, 256, smem, st>>>(a, G, A, B, acc, Gcol_next, Grow_next, vec);
  return cudaGetLastError();
}

template <typename T, int K, bool DF>
static cudaError_t launch_amat_K(const FlushArgs &a, const T *Gcol, const T *Grow,
                                 const double *alpha, const double *beta, const int *acc,
                                 void *Abuf, cudaStream_t st) {
  const int rows_per = 256 / K;
  DQ_KSCOPE(KF_BLOCKAUX, st);
  add_work(KF_BLOCKAUX, 2.0 * a.N * (double)a.kb * a.kb, 8.0 * a.N * (double)(a.kb + K));
  if constexpr (DF) {
    // A and B of the double-float flush together
    add_work(KF_BLOCKAUX, 2.0 * K * (double)a.N * a.kb, 8.0 * a.N * (double)(a.kb + K));
    const int nblk_a = (a.N + rows_per - 1) / rows_per, nblk_b = ((a.N + 255) / 256) * K;
    float2 *A = static_cast<float2 *>(Abuf);
    amat_bmat_df_kernel<K><<<nblk_a + nblk_b, 256, 0, st>>>(a, Gcol, alpha, Grow, beta, acc, A,
                                                            A + (size_t)a.N * K, nblk_a);
  } else
    amat_kernel<T, T><<<(a.N + rows_per - 1) / rows_per, 256, 0, st>>>(
        a.N, K, a.kb, a.ldc, Gcol, alpha, a.lda, acc, static_cast<T *>(Abuf));
  return cudaGetLastError();
}

template <typename T, int K, bool DF>
static cudaError_t launch_update_K(const FlushArgs &a, T *G, const void *Abuf, const T *Grow,
                                   const double *beta, const int *acc, T *Gcol_next, T *Grow_next,
                                   cudaStream_t st) {
  constexpr int SW = 4;
  const int grid = (a.N + SW - 1) / SW;
  DQ_KSCOPE(KF_FLUSH, st);
  // rank-m update of the N x N G, m = accepted flips (<= kb): 2 N^2 m flops,
  // counted at m = kb (an upper bound; the kernel skips the unused terms);
  // G read and written once, A read once
  add_work(KF_FLUSH, 2.0 * a.N * (double)a.N * a.kb,
           (2.0 * a.N * (double)a.N + (double)a.N * a.kb) * sizeof(T));
  flush_kernel<T, K, SW, DF><<<grid, 256, 0, st>>>(a, G, Abuf, Grow, beta, acc, Gcol_next, Grow_next);
  return cudaGetLastError();
}

#define DQ_K_SWITCH(K, CALL) \
  switch (K) {               \
    case 4: { constexpr int KK = 4; return CALL; }   \
    case 8: { constexpr int KK = 8; return CALL; }   \
    case 16: { constexpr int KK = 16; return CALL; } \
    case 32: { constexpr int KK = 32; return CALL; } \
    case 64: { constexpr int KK = 64; return CALL; } \
    default: return cudaErrorInvalidValue;           \
  }

template <typename T>
cudaError_t launch_amat(int K, const FlushArgs &a, const T *Gcol, const T *Grow,
                        const double *alpha, const double *beta, const int *acc, void *Abuf,
                        bool df, cudaStream_t st) {
  if constexpr (std::is_same<T, double>::value) {
    if (df)
      DQ_K_SWITCH(K, (launch_amat_K<double, KK, true>(a, Gcol, Grow, alpha, beta, acc, Abuf, st)))
  }
  DQ_K_SWITCH(K, (launch_amat_K<T, KK, false>(a, Gcol, Grow, alpha, beta, acc, Abuf, st)))
}

template <typename T>
cudaError_t launch_flush_update(int K, const FlushArgs &a, T *G, const void *Abuf, const T *Grow,
                                const double *beta, const int *acc, T *Gcol_next, T *Grow_next,
                                bool df, cudaStream_t st) {
  if constexpr (std::is_same<T, double>::value) {
    if (df)
      DQ_K_SWITCH(K, (launch_update_df_tiled<KK>(a, G, const_cast<void *>(Abuf), Grow, beta, acc,
                                                 Gcol_next, Grow_next, st)))
  }
  DQ_K_SWITCH(K, (launch_update_K<T, KK, false>(a, G, Abuf, Grow, beta, acc, Gcol_next, Grow_next,
                                                st)))
}
#undef DQ_K_SWITCH

template <typename T>
cudaError_t launch_flush(int K, const FlushArgs &a, T *G, const T *Gcol, const T *Grow,
                         const double *alpha, const double *beta, const int *acc, void *Abuf,
                         T *Gcol_next, T *Grow_next, bool df, cudaStream_t st) {
  cudaError_t e = launch_amat<T>(K, a, Gcol, Grow, alpha, beta, acc, Abuf, df, st);
  if (e != cudaSuccess) return e;
  return launch_flush_update<T>(K, a, G, Abuf, Grow, beta, acc, Gcol_next, Grow_next, df, st);
}

// ----------------------------------------------------------------- look-ahead block
// g' = G'[S', S'] of the next block S' = [ns0, ns0 + nkb) after the pending
// flush of the current block, from the pre-flush G:
//   g'[u][v] = G[i][j] - sum_m A[i][m] B[m][j],  i = ns0 + u, j = ns0 + v,
//   B[m][j] = -sum_w beta[m][w] Grow[w][j]   (j is outside the current block),
// the same entries the flush writes, in FP64. It lets the next block's
// Metropolis run while the flush streams G. One CTA per column v.
template <typename T, bool DFA>
__global__ void __launch_bounds__(64)
    lookahead_g_kernel(FlushArgs a, int K, const T *__restrict__ G, const void *__restrict__ A_,
                       const T *__restrict__ Grow, const double *__restrict__ beta,
                       const int *__restrict__ accept_count, double *__restrict__ gnext) {
  __shared__ double bcol[64];
  const int v = blockIdx.x, tid = threadIdx.x;
  const int N = a.N, j = a.ns0 + v;
  const int m = accept_count ? *accept_count : a.kb;
  for (int mm = tid; mm < 64; mm += blockDim.x) {
    double w = 0.0;
    if (mm < m)
      for (int u = 0; u < a.kb; ++u) w = fma(-beta[mm * a.ldb + u], (double)Grow[(size_t)u * N + j], w);
    bcol[mm] = w;
  }
  __syncthreads();
  for (int u = tid; u < a.nkb; u += blockDim.x) {
    const int i = a.ns0 + u;
    double val = (double)G[(size_t)i * N + j];
    for (int mm = 0; mm < m; ++mm) {
      double av;
      if constexpr (DFA) {
        const float2 p = static_cast<const float2 *>(A_)[(size_t)i * K + mm];
        av = (double)p.x + (double)p.y;
      } else {
        av = (double)static_cast<const T *>(A_)[(size_t)i * K + mm];
      }
      val = fma(-av, bcol[mm], val);
    }
    gnext[u * a.nkb + v] = val;
  }
}

template <typename T>
cudaError_t launch_lookahead_g(int K, const FlushArgs &a, const T *G, const void *Abuf, bool df,
                               const T *Grow, const double *beta, const int *acc, double *gnext,
                               cudaStream_t st) {
  if (a.nkb < 1 || a.nkb > 64 || K > 64) return cudaErrorInvalidValue;
  DQ_KSCOPE(KF_BLOCKAUX, st);
  add_work(KF_BLOCKAUX, 2.0 * a.nkb * (double)K * (a.kb + a.nkb), 8.0 * a.nkb * (double)(a.kb + a.nkb));
  if (df && std::is_same<T, double>::value)
    lookahead_g_kernel<T, true><<<a.nkb, 64, 0, st>>>(a, K, G, Abuf, Grow, beta, acc, gnext);
  else
    lookahead_g_kernel<T, false><<<a.nkb, 64, 0, st>>>(a, K, G, Abuf, Grow, beta, acc, gnext);
  return cudaGetLastError();
}
template cudaError_t launch_lookahead_g<double>(int, const FlushArgs &, const double *, const void *,
                                                bool, const double *, const double *, const int *,
                                                double *, cudaStream_t);
template cudaError_t launch_lookahead_g<float>(int, const FlushArgs &, const float *, const void *,
                                               bool, const float *, const double *, const int *,
                                               double *, cudaStream_t);
template cudaError_t launch_amat<double>(int, const FlushArgs &, const double *, const double *,
                                         const double *, const double *, const int *, void *, bool,
                                         cudaStream_t);
template cudaError_t launch_amat<float>(int, const FlushArgs &, const float *, const float *,
                                        const double *, const double *, const int *, void *, bool,
                                        cudaStream_t);
template cudaError_t launch_flush_update<double>(int, const FlushArgs &, double *, const void *,
                                                 const double *, const double *, const int *,
                                                 double *, double *, bool, cudaStream_t);
template cudaError_t launch_flush_update<float>(int, const FlushArgs &, float *, const void *,
                                                const float *, const double *, const int *, float *,
                                                float *, bool, cudaStream_t);
template cudaError_t launch_flush<double>(int, const FlushArgs &, double *, const double *,
                                          const double *, const double *, const double *,
                                          const int *, void *, double *, double *, bool,
                                          cudaStream_t);
template cudaError_t launch_flush<float>(int, const FlushArgs &, float *, const float *,
                                         const float *, const double *, const double *,
                                         const int *, void *, float *, float *, bool,
                                         cudaStream_t);

}  // namespace dq
