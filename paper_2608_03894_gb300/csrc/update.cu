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
#include <type_traits>

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
  DQ_KSCOPE(KF_OTHER, st);
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
  DQ_KSCOPE(KF_METRO, st);
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
// G[:, J] -= Gcol W_J, W_J = Gamma (E_S - Grow)[:, J], one CTA per stripe J
// of SW consecutive columns covering all N rows, so W_J (K x SW) is formed
// once. Thread (rsub, col) owns column j0 + col and rows rsub, rsub + 256/SW,
// ...; it keeps its column of W in registers and streams G once (read,
// subtract, write). The epilogue gathers the next block's rows / columns.
//   T  = storage type of G (double or float)
//   DF = FP64-accurate product on the FP32 units: Gcol holds (hi, lo) FP32
//        pairs, W is split in registers, each MAC is an exact FP32 product
//        plus cross terms accumulated with TwoSum (T must be double).
__device__ __forceinline__ void df_mac2(float ah, float al, float bh, float bl, float &sh, float &sl) {
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
    flush_kernel(FlushArgs a, T *__restrict__ G, const void *__restrict__ Gcol_,
                 const T *__restrict__ Grow, const double *__restrict__ Gamma,
                 const int *__restrict__ accept_count, void *__restrict__ Gcol_next_,
                 T *__restrict__ Grow_next) {
  constexpr int RSTEP = 256 / SW;
  __shared__ double Wsh[K][SW];
  const int tid = threadIdx.x, col = tid % SW, rsub = tid / SW;
  const int N = a.N;
  const int j0 = blockIdx.x * SW, j = j0 + col;
  const bool jok = j < N;
  const int m_acc = accept_count ? *accept_count : 1;

  if (m_acc > 0) {
    for (int e = tid; e < K * SW; e += 256) {
      const int p = e / SW, c = e % SW, jj = j0 + c;
      double w = 0.0;
      if (jj < N && p < a.kb) {
        const int js = jj - a.s0;
        if (js >= 0 && js < a.kb) w = Gamma[p * K + js];
        for (int q = 0; q < a.kb; ++q) w -= Gamma[p * K + q] * (double)Grow[(size_t)q * N + jj];
      }
      Wsh[p][c] = w;
    }
  }
  __syncthreads();

  using WT = typename std::conditional<DF, float, T>::type;
  WT wh[K], wl[DF ? K : 1];
#pragma unroll
  for (int p = 0; p < K; ++p) {
    const double w = (m_acc > 0) ? Wsh[p][col] : 0.0;
    if constexpr (DF) {
      wh[p] = (float)w;
      wl[p] = (float)(w - (double)wh[p]);
    } else {
      wh[p] = (T)w;
    }
  }
  if (!jok) return;

  for (int i = rsub; i < N; i += RSTEP) {
    T acc = T(0);
    if (m_acc > 0) {
      if constexpr (DF) {
        const float2 *gc = static_cast<const float2 *>(Gcol_) + (size_t)i * a.ldc;
        float sh = 0.f, sl = 0.f;
        if ((a.ldc & 1) == 0) {
#pragma unroll
          for (int p = 0; p < K; p += 2) {
            if (p < a.kb) {
              const float4 g = *reinterpret_cast<const float4 *>(gc + p);
              df_mac2(g.x, g.y, wh[p], wl[p], sh, sl);
              df_mac2(g.z, g.w, wh[p + 1], wl[p + 1], sh, sl);
            }
          }
        } else {
#pragma unroll
          for (int p = 0; p < K; ++p)
            if (p < a.kb) df_mac2(gc[p].x, gc[p].y, wh[p], wl[p], sh, sl);
        }
        acc = (double)sh + (double)sl;
      } else {
        const T *gc = static_cast<const T *>(Gcol_) + (size_t)i * a.ldc;
        if ((a.ldc & 3) == 0) {
          // 16-byte vector loads; a group straddling kb stays inside the row
          // (ldc >= kb rounded up to 4) and meets zero rows of W
#pragma unroll
          for (int p = 0; p < K; p += 4) {
            if (p < a.kb) {
              if constexpr (sizeof(T) == 4) {
                const float4 g4 = *reinterpret_cast<const float4 *>(gc + p);
                acc = fmaf(g4.x, wh[p], acc);
                acc = fmaf(g4.y, wh[p + 1], acc);
                acc = fmaf(g4.z, wh[p + 2], acc);
                acc = fmaf(g4.w, wh[p + 3], acc);
              } else {
                const double2 g0 = *reinterpret_cast<const double2 *>(gc + p);
                const double2 g1 = *reinterpret_cast<const double2 *>(gc + p + 2);
                acc = fma(g0.x, wh[p], acc);
                acc = fma(g0.y, wh[p + 1], acc);
                acc = fma(g1.x, wh[p + 2], acc);
                acc = fma(g1.y, wh[p + 3], acc);
              }
            }
          }
        } else {
#pragma unroll
          for (int p = 0; p < K; ++p)
            if (p < a.kb) acc = fma(gc[p], wh[p], acc);
        }
      }
    }
    T *gp = G + (size_t)i * N + j;
    const T val = *gp - acc;
    if (m_acc > 0) *gp = val;
    if (a.nkb > 0) {
      const int it = i - a.ns0, jt = j - a.ns0;
      if (it >= 0 && it < a.nkb) Grow_next[(size_t)it * N + j] = val;
      if (jt >= 0 && jt < K) {
        if constexpr (DF) {
          float2 *gn = static_cast<float2 *>(Gcol_next_) + (size_t)i * K + jt;
          if (jt < a.nkb) {
            const float h = (float)val;
            *gn = make_float2(h, (float)(val - (double)h));
          } else {
            *gn = make_float2(0.f, 0.f);
          }
        } else {
          static_cast<T *>(Gcol_next_)[(size_t)i * K + jt] = (jt < a.nkb) ? val : T(0);
        }
      }
    }
  }
}

template <typename T, int K, bool DF>
static cudaError_t launch_flush_K(const FlushArgs &a, T *G, const void *Gcol, const T *Grow,
                                  const double *Gamma, const int *acc, void *Gcol_next,
                                  T *Grow_next, cudaStream_t st) {
  constexpr int SW = 4;
  const int grid = (a.N + SW - 1) / SW;
  DQ_KSCOPE(KF_FLUSH, st);
  // rank-kb update of the N x N G: 2 N^2 kb flops (+ 2 kb^2 N for W); G read
  // and written once, Gcol and Grow read once
  add_work(KF_FLUSH, 2.0 * a.N * (double)a.N * a.kb + 2.0 * a.kb * (double)a.kb * a.N,
           (2.0 * a.N * (double)a.N + 2.0 * a.N * (double)a.kb) * sizeof(T));
  flush_kernel<T, K, SW, DF><<<grid, 256, 0, st>>>(a, G, Gcol, Grow, Gamma, acc, Gcol_next, Grow_next);
  return cudaGetLastError();
}

template <typename T, bool DF>
static cudaError_t launch_flush_any(int K, const FlushArgs &a, T *G, const void *Gcol, const T *Grow,
                                    const double *Gamma, const int *acc, void *Gcol_next, T *Grow_next,
                                    cudaStream_t st) {
  switch (K) {
    case 4: return launch_flush_K<T, 4, DF>(a, G, Gcol, Grow, Gamma, acc, Gcol_next, Grow_next, st);
    case 8: return launch_flush_K<T, 8, DF>(a, G, Gcol, Grow, Gamma, acc, Gcol_next, Grow_next, st);
    case 16: return launch_flush_K<T, 16, DF>(a, G, Gcol, Grow, Gamma, acc, Gcol_next, Grow_next, st);
    case 32: return launch_flush_K<T, 32, DF>(a, G, Gcol, Grow, Gamma, acc, Gcol_next, Grow_next, st);
    case 64: return launch_flush_K<T, 64, DF>(a, G, Gcol, Grow, Gamma, acc, Gcol_next, Grow_next, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_flush(int K, const FlushArgs &a, T *G, const T *Gcol, const T *Grow,
                         const double *Gamma, const int *acc, T *Gcol_next, T *Grow_next,
                         cudaStream_t st) {
  return launch_flush_any<T, false>(K, a, G, Gcol, Grow, Gamma, acc, Gcol_next, Grow_next, st);
}
template cudaError_t launch_flush<double>(int, const FlushArgs &, double *, const double *,
                                          const double *, const double *, const int *, double *,
                                          double *, cudaStream_t);
template cudaError_t launch_flush<float>(int, const FlushArgs &, float *, const float *,
                                         const float *, const double *, const int *, float *,
                                         float *, cudaStream_t);

cudaError_t launch_flush_df(int K, const FlushArgs &a, double *G, const float2 *Gcol,
                            const double *Grow, const double *Gamma, const int *acc,
                            float2 *Gcol_next, double *Grow_next, cudaStream_t st) {
  return launch_flush_any<double, true>(K, a, G, Gcol, Grow, Gamma, acc, Gcol_next, Grow_next, st);
}

// Gather for the double-float flush: Gcol as (hi, lo) FP32 pairs, Grow in FP64.
__global__ void gather_block_df_kernel(int N, int s0, int kb, int K, const double *__restrict__ G,
                                       float2 *__restrict__ Gcol, double *__restrict__ Grow) {
  const long total = (long)N * K;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e / K), t = (int)(e % K);
    float2 v = make_float2(0.f, 0.f);
    if (t < kb) {
      const double x = G[(size_t)i * N + s0 + t];
      const float h = (float)x;
      v = make_float2(h, (float)(x - (double)h));
    }
    Gcol[e] = v;
  }
  const long total2 = (long)kb * N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total2;
       e += (long)gridDim.x * blockDim.x) {
    const int t = (int)(e / N), j = (int)(e % N);
    Grow[e] = G[(size_t)(s0 + t) * N + j];
  }
}

cudaError_t launch_gather_df(int N, int s0, int kb, int K, const double *G, float2 *Gcol,
                             double *Grow, cudaStream_t st) {
  const long work = (long)N * K;
  int grid = (int)((work + 255) / 256);
  if (grid > 4096) grid = 4096;
  if (grid < 1) grid = 1;
  DQ_KSCOPE(KF_OTHER, st);
  gather_block_df_kernel<<<grid, 256, 0, st>>>(N, s0, kb, K, G, Gcol, Grow);
  return cudaGetLastError();
}

}  // namespace dq
