// Cholesky factorisation with the inverse factor, and CholeskyQR2, for the
// UDV stabilisation of the mixed-precision sweep.
//
// The stabilisation (not in the paper; standard DQMC practice) needs an
// orthogonal-triangular factorisation X = Q R of an N x N product with
// graded columns every n_stab slices. In mixed precision the products run as
// FP64-accurate digit-slice GEMMs on the tensor cores, and a Householder QR,
// whose panels are a serial column loop on the FP64 pipe, dominates. Here the
// factorisation is CholeskyQR2 (Fukaya, Nakatsukasa, Yanagisawa, Yamamoto
// 2014): W = X^T X = R1^T R1, Q1 = X R1^{-1}, then once more on Q1, giving
// Q = Q1 R2^{-1} and R = R2 R1. It is orthogonal to working precision for
// cond(X) up to ~1e7; the pre-pivoted stack products and the scale-separated
// matrix of the Green's function recomputation stay well inside that.
//
// The Cholesky factor and its inverse are computed by recursion on the
// leading half: [A11 A12; . A22] -> R11, R12 = R11^{-T} A12, A22 - R12^T R12
// -> R22, and R^{-1}_12 = -R11^{-1} R12 R22^{-1}; blocks of at most 64
// columns are factorised and inverted by one CTA in shared memory, in FP64.
// Every other operation is a GEMM (dgemm: the digit-slice GEMM in mixed
// precision for the large blocks, FP64 below 256).
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "linalg.cuh"

namespace dq {

constexpr int kCholLeaf = 64;

// A (n x n, n <= 64, upper triangle read) = R^T R: R to A's upper triangle,
// zeros below; Ri = R^{-1} (upper, zeros below). A non-positive or non-finite
// pivot sets *status = 1 (the factor is then garbage; the sweep reports it).
__global__ void __launch_bounds__(256)
    chol_leaf_kernel(double *__restrict__ A, int lda, double *__restrict__ Ri, int ldr, int n,
                     int *status) {
  __shared__ double a[kCholLeaf][kCholLeaf + 1];
  __shared__ double x[kCholLeaf][kCholLeaf + 1];
  __shared__ double dinv[kCholLeaf];
  const int tid = threadIdx.x;
  for (int e = tid; e < kCholLeaf * kCholLeaf; e += 256) {
    const int r = e / kCholLeaf, c = e % kCholLeaf;
    a[r][c] = (r < n && c < n && c >= r) ? A[(size_t)r * lda + c] : 0.0;
    x[r][c] = 0.0;
  }
  __syncthreads();
  // right-looking Cholesky on the upper triangle
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      double d = a[j][j];
      if (!(d > 0.0) || !isfinite(d)) {
        *status = 1;
        d = 1.0;
      }
      const double s = sqrt(d);
      a[j][j] = s;
      dinv[j] = 1.0 / s;
    }
    __syncthreads();
    const double si = dinv[j];
    for (int c = j + 1 + tid; c < n; c += 256) a[j][c] *= si;
    __syncthreads();
    const int m = n - j - 1;
    for (int e = tid; e < m * m; e += 256) {
      const int r = j + 1 + e / m, c = j + 1 + e % m;
      if (c >= r) a[r][c] = fma(-a[j][r], a[j][c], a[r][c]);
    }
    __syncthreads();
  }
  // X = R^{-1}: column c by back substitution, four threads per column
  // (the dot products split over them), every lane running all 64 rows so
  // that the shuffles stay warp-uniform
  {
    const int c = tid >> 2, q = tid & 3;
    for (int i = kCholLeaf - 1; i >= 0; --i) {
      double part = 0.0;
      const bool act = (c < n) && (i <= c);
      if (act)
        for (int k = i + 1 + q; k <= c; k += 4) part = fma(a[i][k], x[k][c], part);
      part += __shfl_xor_sync(0xffffffffu, part, 1);
      part += __shfl_xor_sync(0xffffffffu, part, 2);
      if (act && q == 0) x[i][c] = ((i == c ? 1.0 : 0.0) - part) * dinv[i];
      __syncwarp();
    }
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += 256) {
    const int r = e / n, c = e % n;
    A[(size_t)r * lda + c] = (c >= r) ? a[r][c] : 0.0;
    Ri[(size_t)r * ldr + c] = (c >= r) ? x[r][c] : 0.0;
  }
}

// FP64 FMA for small blocks (the digit-slice GEMM's operand splitting does
// not pay below a few hundred), the dispatching dgemm above.
static cudaError_t gemm_blk(bool ta, bool tb, int M, int N, int K, double alpha, const double *A,
                            int lda, const double *B, int ldb, double beta, double *C, int ldc,
                            cudaStream_t st) {
  if (M <= 256 && N <= 256 && K <= 256)
    return dgemm_fp64(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, nullptr, nullptr, st);
  return dgemm(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, nullptr, nullptr, st);
}

static cudaError_t copy_block(const double *src, int lds, double *dst, int ldd, int rows, int cols,
                              cudaStream_t st) {
  return cudaMemcpy2DAsync(dst, (size_t)ldd * sizeof(double), src, (size_t)lds * sizeof(double),
                           (size_t)cols * sizeof(double), rows, cudaMemcpyDeviceToDevice, st);
}

// Recursion; Ri's strictly lower blocks must already be zero.
static cudaError_t chol_inv_rec(double *A, int lda, double *Ri, int ldr, double *Wk, int ldw, int n,
                                int *status, cudaStream_t st) {
  if (n <= kCholLeaf) {
    DQ_KSCOPE(KF_QRPANEL, st);
    add_work(KF_QRPANEL, 2.0 * n * (double)n * n / 3.0, 3.0 * 8.0 * n * (double)n);
    chol_leaf_kernel<<<1, 256, 0, st>>>(A, lda, Ri, ldr, n, status);
    return cudaGetLastError();
  }
  const int nl = (n + kCholLeaf - 1) / kCholLeaf;
  const int n1 = (nl / 2) * kCholLeaf, n2 = n - n1;
  double *A12 = A + n1, *A21 = A + (size_t)n1 * lda, *A22 = A21 + n1;
  double *R12i = Ri + n1, *R22i = Ri + (size_t)n1 * ldr + n1;
  double *W12 = Wk + n1, *W22 = Wk + (size_t)n1 * ldw + n1;
  cudaError_t e = chol_inv_rec(A, lda, Ri, ldr, Wk, ldw, n1, status, st);
  if (e != cudaSuccess) return e;
  // R12 = R11^{-T} A12 (into the scratch, then A12)
  if ((e = gemm_blk(true, false, n1, n2, n1, 1.0, Ri, ldr, A12, lda, 0.0, W12, ldw, st)) != cudaSuccess)
    return e;
  if ((e = copy_block(W12, ldw, A12, lda, n1, n2, st)) != cudaSuccess) return e;
  if ((e = cudaMemset2DAsync(A21, (size_t)lda * sizeof(double), 0, (size_t)n1 * sizeof(double), n2, st)) !=
      cudaSuccess)
    return e;
  // Schur complement A22 - R12^T R12
  if ((e = gemm_blk(true, false, n2, n2, n1, -1.0, W12, ldw, W12, ldw, 1.0, A22, lda, st)) != cudaSuccess)
    return e;
  if ((e = chol_inv_rec(A22, lda, R22i, ldr, W22, ldw, n2, status, st)) != cudaSuccess) return e;
  // R^{-1}_12 = -R11^{-1} (R12 R22^{-1})
  if ((e = gemm_blk(false, false, n1, n2, n2, 1.0, W12, ldw, R22i, ldr, 0.0, R12i, ldr, st)) != cudaSuccess)
    return e;
  if ((e = gemm_blk(false, false, n1, n2, n1, -1.0, Ri, ldr, R12i, ldr, 0.0, W12, ldw, st)) != cudaSuccess)
    return e;
  return copy_block(W12, ldw, R12i, ldr, n1, n2, st);
}

cudaError_t chol_inv(double *A, int lda, double *Ri, int ldr, double *Wk, int ldw, int n, int *status,
                     cudaStream_t st) {
  cudaError_t e =
      cudaMemset2DAsync(Ri, (size_t)ldr * sizeof(double), 0, (size_t)n * sizeof(double), n, st);
  if (e != cudaSuccess) return e;
  return chol_inv_rec(A, lda, Ri, ldr, Wk, ldw, n, status, st);
}

// W += s I with s = c tr(W): one CTA, the trace summed in a fixed order.
__global__ void __launch_bounds__(256) shift_diag_kernel(double *W, int n, int ld, double c) {
  __shared__ double red[256];
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) t += W[(size_t)i * ld + i];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double sft = c * red[0];
  for (int i = threadIdx.x; i < n; i += 256) W[(size_t)i * ld + i] += sft;
}

cudaError_t shift_diag(double *W, int n, int ld, double c, cudaStream_t st) {
  DQ_KSCOPE(KF_STABAUX, st);
  shift_diag_kernel<<<1, 256, 0, st>>>(W, n, ld, c);
  return cudaGetLastError();
}

cudaError_t cholqr2(const double *X, int n, double *Q, double *R, double *Q1, double *W, double *Ri,
                    double *Wk, int *status, cudaStream_t st) {
  cudaError_t e;
  // pass 1: W = X^T X = R1^T R1, Q1 = X R1^{-1}; R1 is kept in R
  if ((e = dgemm(true, false, n, n, n, 1.0, X, n, X, n, 0.0, R, n, nullptr, nullptr, st)) != cudaSuccess)
    return e;
  if ((e = chol_inv(R, n, Ri, n, Wk, n, n, status, st)) != cudaSuccess) return e;
  if ((e = dgemm(false, false, n, n, n, 1.0, X, n, Ri, n, 0.0, Q1, n, nullptr, nullptr, st)) != cudaSuccess)
    return e;
  // pass 2: W = Q1^T Q1 = R2^T R2, Q = Q1 R2^{-1}, R = R2 R1
  if ((e = dgemm(true, false, n, n, n, 1.0, Q1, n, Q1, n, 0.0, W, n, nullptr, nullptr, st)) != cudaSuccess)
    return e;
  if ((e = chol_inv(W, n, Ri, n, Wk, n, n, status, st)) != cudaSuccess) return e;
  if ((e = dgemm(false, false, n, n, n, 1.0, Q1, n, Ri, n, 0.0, Q, n, nullptr, nullptr, st)) != cudaSuccess)
    return e;
  if ((e = dgemm(false, false, n, n, n, 1.0, W, n, R, n, 0.0, Wk, n, nullptr, nullptr, st)) != cudaSuccess)
    return e;
  return cudaMemcpyAsync(R, Wk, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice, st);
}

}  // namespace dq
