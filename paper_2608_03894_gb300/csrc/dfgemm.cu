// FP64-accurate GEMM on the FP32 units ("double-float" arithmetic).
//
// On GB300 the FP64 pipe runs at 1/64 of the FP32 rate. Every FP64 operand
// is split once into an unevaluated pair hi + lo of FP32 numbers
// (hi = fl32(x), lo = fl32(x - hi)), and each multiply-accumulate is done as
//     p + e = a_hi * b_hi           exactly (e from an FMA)
//     e    += a_hi * b_lo + a_lo * b_hi
//     (s_hi, err) = TwoSum(s_hi, p) ; s_lo += err + e
// (Dekker's product split via FMA and Knuth's TwoSum), 12 FP32 operations
// per MAC, relative accuracy ~2^-46 per dot product of length K << 2^20.
// The FP32 exponent range is assumed for the operands (all stabilisation
// GEMMs act on orthogonal or pivot-bounded factors; the large and small
// scales D are applied in FP64 outside the product).
#include "linalg.cuh"

namespace dq {

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

__global__ void split_df_kernel(const double *__restrict__ X, int rows, int cols, int ld,
                                float2 *__restrict__ out) {
  const long total = (long)rows * cols;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e / cols), j = (int)(e % cols);
    const double v = X[(size_t)i * ld + j];
    const float h = (float)v;
    out[e] = make_float2(h, (float)(v - (double)h));
  }
}

// C = alpha diag(rs) op(A) op(B) diag(cs) + beta C with A, B given as split
// pairs (packed, A: (TA ? K x M : M x K), B: (TB ? N x K : K x N)).
template <bool TA, bool TB>
__global__ void __launch_bounds__(256)
    dfgemm_kernel(int M, int N, int K, double alpha, const float2 *__restrict__ A,
                  const float2 *__restrict__ B, double beta, double *__restrict__ C, int ldc,
                  const double *__restrict__ rs, const double *__restrict__ cs, int klen,
                  double *__restrict__ part) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ float2 As[BK][BM + 1];
  __shared__ float2 Bs[BK][BN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kbeg = blockIdx.z * klen;
  const int kend = min(K, kbeg + klen);
  const int lda = TA ? M : K, ldb = TB ? K : N;
  float sh[4][4], sl[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) sh[i][j] = sl[i][j] = 0.f;

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
      float2 v = make_float2(0.f, 0.f);
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
      float2 v = make_float2(0.f, 0.f);
      if (gn < N && gk < kend) v = TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) df_mac(a[i].x, a[i].y, b[j].x, b[j].y, sh[i][j], sl[i][j]);
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
      const double acc = (double)sh[i][j] + (double)sl[i][j];
      const double v = alpha * r * acc * (cs ? cs[gn] : 1.0);
      double *cp = C + (size_t)gm * ldc + gn;
      if (part)
        part[((size_t)blockIdx.z * M + gm) * N + gn] = v;
      else
        *cp = (beta != 0.0) ? v + beta * (*cp) : v;
    }
  }
}

static thread_local float2 *t_ws = nullptr;
static thread_local size_t t_ws_elems = 0;
static thread_local bool t_df = false;

void set_df_workspace(float2 *ws, size_t elems) {
  t_ws = ws;
  t_ws_elems = elems;
}
void set_gemm_df(bool on) { t_df = on; }
bool gemm_df() { return t_df && t_ws != nullptr; }

static int grid_for_df(long work) {
  long g = (work + 255) / 256;
  if (g > 8192) g = 8192;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t dfgemm(bool ta, bool tb, int M, int N, int K, double alpha, const double *A, int lda,
                   const double *B, int ldb, double beta, double *C, int ldc, const double *rs,
                   const double *cs, cudaStream_t st, int splitk, int tiles_target) {
  const size_t na = (size_t)M * K, nbn = (size_t)K * N;
  if (na + nbn > t_ws_elems) return cudaErrorInvalidValue;
  float2 *As = t_ws, *Bs = t_ws + na;
  {
    DQ_KSCOPE(KF_SLICE, st);
    if (!ta)
      split_df_kernel<<<grid_for_df((long)na), 256, 0, st>>>(A, M, K, lda, As);
    else
      split_df_kernel<<<grid_for_df((long)na), 256, 0, st>>>(A, K, M, lda, As);
  }
  {
    DQ_KSCOPE(KF_SLICE, st);
    if (!tb)
      split_df_kernel<<<grid_for_df((long)nbn), 256, 0, st>>>(B, K, N, ldb, Bs);
    else
      split_df_kernel<<<grid_for_df((long)nbn), 256, 0, st>>>(B, N, K, ldb, Bs);
  }
  const int tiles = ((M + 63) / 64) * ((N + 63) / 64);
  if (splitk <= 0) {
    splitk = 1;
    if (tiles < tiles_target) {
      splitk = (tiles_target + tiles - 1) / tiles;
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
    dfgemm_kernel<false, false><<<grid, 256, 0, st>>>(M, N, K, alpha, As, Bs, beta, C, ldc, rs, cs, klen, part);
  else if (ta && !tb)
    dfgemm_kernel<true, false><<<grid, 256, 0, st>>>(M, N, K, alpha, As, Bs, beta, C, ldc, rs, cs, klen, part);
  else if (!ta && tb)
    dfgemm_kernel<false, true><<<grid, 256, 0, st>>>(M, N, K, alpha, As, Bs, beta, C, ldc, rs, cs, klen, part);
  else
    dfgemm_kernel<true, true><<<grid, 256, 0, st>>>(M, N, K, alpha, As, Bs, beta, C, ldc, rs, cs, klen, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !part) return e;
  return splitk_reduce(part, splitk, M, N, beta, C, ldc, st);
}

}  // namespace dq
