// Delayed-update Metropolis over one time slice.
//
// Sites are proposed in index order in blocks S of k consecutive sites. For a
// block, every quantity the sequential Sherman-Morrison updates need lies in
// the k x k sub-block g = G[S,S] (submatrix form of the delayed update): the
// current diagonal G~_jj, the restricted columns/rows of the accepted updates,
// and two coefficient recursions alpha, beta such that after the block
//     G' = G - G[:,S] Gamma (I - G)[S,:],   Gamma = sum_m alpha_m beta_m^T,
// which is exactly the product of the sequential rank-one updates (Woodbury).
// The block's serial loop runs in one CTA in FP64 (ratios and bookkeeping);
// the flush is one rank-k product over the whole N x N G in the working
// precision, and its epilogue gathers G[:,S'] and G[S',:] of the next block.
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
  gather_block_kernel<T><<<grid, 256, 0, st>>>(N, s0, kb, K, G, Gcol, Grow);
  return cudaGetLastError();
}
template cudaError_t launch_gather<double>(int, int, int, int, const double *, double *, double *,
                                           cudaStream_t);
template cudaError_t launch_gather<float>(int, int, int, int, const float *, float *, float *,
                                          cudaStream_t);

// ----------------------------------------------------------------- Metropolis block

// One CTA of K threads (K = 32 or 64 rounded up from kb). Thread u owns
// block-local site u. Shared: g (kb x (kb+1)), and per accepted flip m the
// restricted update column As[m][*] = (delta/r) G~[S, j], row
// Bs[m][*] = e_j - G~[j, S], and the coefficient vectors al[m][*], be[m][*].
template <typename TG>
__global__ void metropolis_block_kernel(MetroArgs a, const TG *__restrict__ g, int8_t *s,
                                        const uint8_t *__restrict__ forced, double *Gamma,
                                        int *accept_count, int *status,
                                        unsigned long long *total) {
  extern __shared__ __align__(16) double sm[];
  const int kb = a.kb, u = threadIdx.x;
  const int ldg = kb + 1;
  double *gs = sm;                    // kb * ldg
  double *As = gs + kb * ldg;         // kb * kb  [m][u]
  double *Bs = As + kb * kb;          // [m][u]
  double *al = Bs + kb * kb;          // [m][u]
  double *be = al + kb * kb;          // [m][u]
  // decision and coefficient of site j, double-buffered by the parity of j:
  // a rejected site has no second barrier, so the slot written at j + 2 must
  // differ from the one still being read at j
  __shared__ int s_dec[2];
  __shared__ double s_coef[2];

  for (int e = u; e < kb * kb; e += blockDim.x) {
    const int r = e / kb, c = e % kb;
    gs[r * ldg + c] = (double)g[(size_t)r * a.ld_g + c];
  }
  double dtil = 0.0, urand = 0.0;
  int si = 1;
  if (u < kb) {
    const uint4 r = philox4x32_10(make_uint4((uint32_t)(a.s0 + u), (uint32_t)a.slice0, a.c2, a.c3),
                                  a.k0, a.k1);
    urand = uniform53(r.x, r.y);
    si = (int)s[a.s0 + u];
  }
  __syncthreads();
  if (u < kb) dtil = gs[u * ldg + u];

  const double e2l = a.e2l, em2l = a.em2l;
  int m = 0;
  for (int j = 0; j < kb; ++j) {
    if (u == j) {
      // delta = e^{-2 lambda s} - 1, r = 1 + delta (1 - G~_jj), R = e^{2 lambda s} r^2
      const double delta = (si > 0 ? em2l : e2l) - 1.0;
      const double r = 1.0 + delta * (1.0 - dtil);
      const double R = (si > 0 ? e2l : em2l) * r * r;
      int dec;
      if (!(R > 0.0) || !isfinite(R)) {
        dec = -1;
      } else if (forced) {
        dec = forced[j] ? 1 : 0;
      } else {
        dec = (urand < R) ? 1 : 0;
      }
      s_dec[j & 1] = dec;
      s_coef[j & 1] = delta / r;
    }
    __syncthreads();
    const int dec = s_dec[j & 1];
    if (dec < 0) {
      if (u == 0) *status = 1;
      break;
    }
    if (dec) {
      const double c = s_coef[j & 1];
      if (u < kb) {
        double col = gs[u * ldg + j], row = gs[j * ldg + u];
        double alv = (u == j) ? 1.0 : 0.0, bev = alv;
        for (int mm = 0; mm < m; ++mm) {
          const double bj = Bs[mm * kb + j], aj = As[mm * kb + j];
          col -= As[mm * kb + u] * bj;
          row -= aj * Bs[mm * kb + u];
          alv -= al[mm * kb + u] * bj;
          bev += aj * be[mm * kb + u];
        }
        const double acol = c * col;
        const double brow = ((u == j) ? 1.0 : 0.0) - row;
        As[m * kb + u] = acol;
        Bs[m * kb + u] = brow;
        al[m * kb + u] = c * alv;
        be[m * kb + u] = bev;
        dtil -= acol * brow;
        if (u == j) {
          si = -si;
          s[a.s0 + u] = (int8_t)si;
        }
      }
      ++m;
      __syncthreads();
    }
  }
  // Gamma[u][w] = sum_m al[m][u] be[m][w]; full K x K, zero outside kb
  for (int e = u; e < a.K * a.K; e += blockDim.x) {
    const int r = e / a.K, c = e % a.K;
    double acc = 0.0;
    if (r < kb && c < kb)
      for (int mm = 0; mm < m; ++mm) acc += al[mm * kb + r] * be[mm * kb + c];
    Gamma[e] = acc;
  }
  if (u == 0) {
    *accept_count = m;
    if (total) atomicAdd(total, (unsigned long long)m);
  }
}

template <typename TG>
cudaError_t launch_metropolis(const MetroArgs &a, const TG *g, int8_t *s, const uint8_t *forced,
                              double *Gamma, int *accept_count, int *status,
                              unsigned long long *total, cudaStream_t st) {
  if (a.kb < 1 || a.kb > 64 || a.kb > a.K) return cudaErrorInvalidValue;
  const int threads = a.kb <= 32 ? 32 : 64;
  const size_t smem = (size_t)(a.kb * (a.kb + 1) + 4 * a.kb * a.kb) * sizeof(double);
  cudaError_t e = ensure_smem_attr((const void *)metropolis_block_kernel<TG>,
                                   (int)(5 * 64 * 65 * sizeof(double)));
  if (e != cudaSuccess) return e;
  metropolis_block_kernel<TG><<<1, threads, smem, st>>>(a, g, s, forced, Gamma, accept_count,
                                                         status, total);
  return cudaGetLastError();
}
template cudaError_t launch_metropolis<double>(const MetroArgs &, const double *, int8_t *,
                                               const uint8_t *, double *, int *, int *,
                                               unsigned long long *, cudaStream_t);
template cudaError_t launch_metropolis<float>(const MetroArgs &, const float *, int8_t *,
                                              const uint8_t *, double *, int *, int *,
                                              unsigned long long *, cudaStream_t);

// ----------------------------------------------------------------- rank-k flush
// G[:, J] -= Gcol * W_J,  W_J = Gamma (E_S - Grow)[:, J], one CTA per
// (32-column stripe J, row chunk). Lane = column of J; warp w owns rows
// i = r0 + w, r0 + w + 8, ... Each thread keeps its column of W_J (K values)
// in registers and streams G[i, j] once: read, subtract, write. The epilogue
// also gathers the next block (rows / columns S' = [ns0, ns0 + nkb)).

template <typename T, int K>
__global__ void __launch_bounds__(256)
    flush_kernel(FlushArgs a, T *__restrict__ G, const T *__restrict__ Gcol,
                 const T *__restrict__ Grow, const double *__restrict__ Gamma,
                 const int *__restrict__ accept_count, T *__restrict__ Gcol_next,
                 T *__restrict__ Grow_next) {
  __shared__ double Wsh[K][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int N = a.N;
  const int j = blockIdx.x * 32 + lane;
  const bool jok = j < N;
  const int m_acc = accept_count ? *accept_count : 1;

  // W_J[p][lane] = Gamma[p][j - s0] (if j in S) - sum_q Gamma[p][q] Grow[q][j]
  if (m_acc > 0) {
    for (int p = warp; p < K; p += 8) {
      double w = 0.0;
      if (jok && p < a.kb) {
        const int js = j - a.s0;
        if (js >= 0 && js < a.kb) w = Gamma[p * K + js];
        for (int q = 0; q < a.kb; ++q) w -= Gamma[p * K + q] * (double)Grow[(size_t)q * N + j];
      }
      Wsh[p][lane] = w;
    }
  }
  __syncthreads();
  T wreg[K];
#pragma unroll
  for (int p = 0; p < K; ++p) wreg[p] = (m_acc > 0) ? (T)Wsh[p][lane] : T(0);

  const int r0 = blockIdx.y * a.rows_per_cta;
  const int r1 = min(N, r0 + a.rows_per_cta);
  for (int i = r0 + warp; i < r1; i += 8) {
    if (!jok) continue;
    const T *gc = Gcol + (size_t)i * K;
    T acc = T(0);
    if (m_acc > 0) {
#pragma unroll
      for (int p = 0; p < K; p += 4) {
        if constexpr (sizeof(T) == 4) {
          const float4 g4 = *reinterpret_cast<const float4 *>(gc + p);
          acc = fmaf(g4.x, wreg[p], acc);
          acc = fmaf(g4.y, wreg[p + 1], acc);
          acc = fmaf(g4.z, wreg[p + 2], acc);
          acc = fmaf(g4.w, wreg[p + 3], acc);
        } else {
          const double2 g0 = *reinterpret_cast<const double2 *>(gc + p);
          const double2 g1 = *reinterpret_cast<const double2 *>(gc + p + 2);
          acc = fma(g0.x, wreg[p], acc);
          acc = fma(g0.y, wreg[p + 1], acc);
          acc = fma(g1.x, wreg[p + 2], acc);
          acc = fma(g1.y, wreg[p + 3], acc);
        }
      }
    }
    T *gp = G + (size_t)i * N + j;
    const T val = *gp - acc;
    if (m_acc > 0) *gp = val;
    if (a.nkb > 0) {
      const int it = i - a.ns0, jt = j - a.ns0;
      if (it >= 0 && it < a.nkb) Grow_next[(size_t)it * N + j] = val;
      if (jt >= 0 && jt < K) Gcol_next[(size_t)i * K + jt] = (jt < a.nkb) ? val : T(0);
    }
  }
}

template <typename T, int K>
static cudaError_t launch_flush_K(const FlushArgs &a0, T *G, const T *Gcol, const T *Grow,
                                  const double *Gamma, const int *acc, T *Gcol_next, T *Grow_next,
                                  cudaStream_t st) {
  FlushArgs a = a0;
  const int stripes = (a.N + 31) / 32;
  // enough CTAs to cover ~2 waves of 152 SMs
  int chunks = (304 + stripes - 1) / stripes;
  if (chunks < 1) chunks = 1;
  a.rows_per_cta = (a.N + chunks - 1) / chunks;
  a.rows_per_cta = ((a.rows_per_cta + 7) / 8) * 8;
  chunks = (a.N + a.rows_per_cta - 1) / a.rows_per_cta;
  dim3 grid(stripes, chunks);
  flush_kernel<T, K><<<grid, 256, 0, st>>>(a, G, Gcol, Grow, Gamma, acc, Gcol_next, Grow_next);
  // Gcol_next columns jt in [nkb, K) of rows not visited stay as they were:
  // the gather zero-fills them on allocation and after a ragged block.
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_flush(int K, const FlushArgs &a, T *G, const T *Gcol, const T *Grow,
                         const double *Gamma, const int *acc, T *Gcol_next, T *Grow_next,
                         cudaStream_t st) {
  switch (K) {
    case 4: return launch_flush_K<T, 4>(a, G, Gcol, Grow, Gamma, acc, Gcol_next, Grow_next, st);
    case 8: return launch_flush_K<T, 8>(a, G, Gcol, Grow, Gamma, acc, Gcol_next, Grow_next, st);
    case 16: return launch_flush_K<T, 16>(a, G, Gcol, Grow, Gamma, acc, Gcol_next, Grow_next, st);
    case 32: return launch_flush_K<T, 32>(a, G, Gcol, Grow, Gamma, acc, Gcol_next, Grow_next, st);
    case 64: return launch_flush_K<T, 64>(a, G, Gcol, Grow, Gamma, acc, Gcol_next, Grow_next, st);
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t launch_flush<double>(int, const FlushArgs &, double *, const double *,
                                          const double *, const double *, const int *, double *,
                                          double *, cudaStream_t);
template cudaError_t launch_flush<float>(int, const FlushArgs &, float *, const float *,
                                         const float *, const double *, const int *, float *,
                                         float *, cudaStream_t);

}  // namespace dq
