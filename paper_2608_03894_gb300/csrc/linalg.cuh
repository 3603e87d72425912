// FP64 dense linear algebra for the UDV stabilisation (row-major storage).
#pragma once

#include "common.cuh"

namespace dq {

// C = alpha diag(rs) op(A) op(B) diag(cs) + beta C; rs/cs may be NULL.
// A is M x K (lda) or, transposed, K x M; B is K x N (ldb) or N x K.
// splitk > 1 splits K over CTAs: each split writes its partial product to the
// calling thread's split-K workspace and one more kernel sums the splits in a
// fixed order (results do not depend on CTA scheduling). Without a workspace
// large enough for splits * M * N doubles the GEMM runs unsplit.
// While set_gemm_df(true) is in effect for the calling thread (and a
// workspace is bound), dgemm runs as dfgemm: FP64 in and out, FP64-accurate
// products computed on the FP32 units from (hi, lo) FP32 pairs.
cudaError_t dgemm(bool ta, bool tb, int M, int N, int K, double alpha, const double *A, int lda,
                  const double *B, int ldb, double beta, double *C, int ldc, const double *rs,
                  const double *cs, cudaStream_t st, int splitk = 0);
// dgemm without the fast-variant dispatch: always FP64 FMA.
cudaError_t dgemm_fp64(bool ta, bool tb, int M, int N, int K, double alpha, const double *A,
                       int lda, const double *B, int ldb, double beta, double *C, int ldc,
                       const double *rs, const double *cs, cudaStream_t st, int splitk = 0);
cudaError_t dfgemm(bool ta, bool tb, int M, int N, int K, double alpha, const double *A, int lda,
                   const double *B, int ldb, double beta, double *C, int ldc, const double *rs,
                   const double *cs, cudaStream_t st, int splitk, int tiles_target);
void set_df_workspace(float2 *ws, size_t elems);  // >= max over calls of M*K + K*N pairs
void set_gemm_df(bool on);
bool gemm_df();

// FP64-accurate GEMM from exact 7-bit digit slices on the bf16 tensor cores
// (see ozgemm.cu). While set_gemm_oz(true) is in effect for the calling thread
// (and a workspace is bound), dgemm runs as ozgemm.
cudaError_t ozgemm(bool ta, bool tb, int M, int N, int K, double alpha, const double *A, int lda,
                   const double *B, int ldb, double beta, double *C, int ldc, const double *rs,
                   const double *cs, cudaStream_t st);
size_t oz_workspace_bytes(int M, int N, int K);
void set_oz_workspace(void *ws, size_t bytes, int *exps, size_t nexp);  // exps: >= M + N ints
void set_gemm_oz(bool on);
// While set (calling thread), the Householder panels of qr_factor run their
// column loop in double-float arithmetic (mixed precision).
void set_qr_panel_df(bool on);
// For the calling thread in digit-slice mode, the two small products of each
// block reflector: gram = 0 the Gram matrix V^T V as a digit-slice GEMM, 1 by
// a parallel FP64 kernel, 2 by a parallel double-float kernel; tw = 0 op(T) W
// as a digit-slice GEMM, 1 by a parallel FP64 kernel, 2 by a column-scaled
// double-float kernel.
void set_reflector_modes(int gram, int tw);
bool gemm_oz();
// While set_gemm_oz_tc(true) is in effect for the calling thread, the
// digit-slice products run on tcgen05 (tensor memory accumulators) instead of
// the warp-level mma.sync kernel. oz_tc_timed_out: whether a bounded wait of
// that kernel gave up since the library was loaded (synchronises the stream).
void set_gemm_oz_tc(bool on, bool force = false);  // force: every shape (else M, N, K >= 256)
bool oz_tc_timed_out(cudaStream_t st);

// Call sites of the stabilisation GEMMs. The fast FP64-accurate variants
// (double-float, digit slices) are accurate relative to the largest entries
// of a row / column, not per term; the mask selects the sites where they are
// used (bit s = site s), the others stay FP64 FMA.
enum GemmSite {
  GS_QR_UPDATE = 0,  // trailing update of a Householder QR
  GS_FORM_Q,         // explicit Q
  GS_T_UPDATE,       // T_new = R'' P^T T_old (graded R'')
  GS_UU,             // U_r^T U_l
  GS_TT,             // T_r T_l^T
  GS_QRM,            // trailing updates of the QR of the scale-separated matrix
  GS_APPLY_QT,       // Q^T B in the solve
  GS_TRSM,           // block triangular solve
  GS_FINAL,          // G = U_l Z
  GS_CHOLQR,         // CholeskyQR2: Gram matrices, Cholesky recursion, Q and R products
  GS_COUNT
};
void set_gemm_site(int site);
void set_gemm_site_mask(unsigned mask);
// sites (within the site mask) that use the double-float GEMM even while the
// digit-slice GEMM is on (needs a double-float workspace)
void set_gemm_df_site_mask(unsigned mask);
cudaError_t scale_matrix(double *C, int M, int N, int ldc, double beta, cudaStream_t st);

// Split-K workspace of the calling host thread (doubles); splitk_ws_doubles()
// covers every split the GEMMs here choose by themselves.
void set_splitk_workspace(double *ws, size_t n);
size_t splitk_ws_doubles();
// The partial-product buffer for `splits` splits of an M x N output, or NULL
// when splits <= 1 or the bound workspace is too small.
double *splitk_partials(int splits, int M, int N);
// C = beta C + sum_{z < splits} part[z] (fixed order), part dense M x N per split.
cudaError_t splitk_reduce(const double *part, int splits, int M, int N, double beta, double *C,
                          int ldc, cudaStream_t st);

// Householder QR workspace for an n x n matrix: V (unit lower trapezoidal,
// explicit; panel p in columns p..p+nb), tau, the compact-WY factor T of each
// panel (nb x nb, upper triangular), GEMM scratch W / W2 (nb x n) and the
// panel Gram matrix, and the inverses of the nb x nb diagonal blocks of R.
struct QRWork {
  int n = 0, nb = 0, ctas = 8;
  double *V = nullptr, *tau = nullptr, *W = nullptr, *W2 = nullptr, *Gram = nullptr;
  double *T = nullptr;     // (n/nb + 1) blocks of nb x nb
  double *Rinv = nullptr;  // (n/nb + 1) blocks of nb x nb
};
int qr_panel_width(int n);
size_t qr_work_doubles(int n);
void qr_work_bind(QRWork &w, int n, double *mem);

// In-place QR A = Q R (R in the upper triangle of A, V in QRWork).
cudaError_t qr_factor(double *A, int n, QRWork &w, cudaStream_t st);
// Q (explicit) into Qout (n x n).
cudaError_t qr_form_q(double *Qout, int n, QRWork &w, cudaStream_t st);
// B <- Q^T B for B n x ncols (ld ldb).
cudaError_t qr_apply_qt(double *B, int n, int ncols, int ldb, QRWork &w, cudaStream_t st);
// Z = R^{-1} B (R upper triangular in A's upper triangle), B destroyed; Z n x ncols.
cudaError_t qr_solve_r(const double *A, int n, double *B, double *Z, int ncols, QRWork &w,
                       cudaStream_t st);

// Cholesky A = R^T R of the symmetric positive definite n x n matrix A (upper
// triangle read, ld lda): R to A's upper triangle (zeros below), R^{-1} to Ri
// (upper, zeros below, ld ldr). Wk: n x n scratch (ld ldw). A non-positive
// pivot sets *status = 1 (device int).
cudaError_t chol_inv(double *A, int lda, double *Ri, int ldr, double *Wk, int ldw, int n, int *status,
                     cudaStream_t st);
// W += c tr(W) I (the shift of a shifted Cholesky QR pass; tr(W) >= ||X||_2^2
// for W = X^T X).
cudaError_t shift_diag(double *W, int n, int ld, double c, cudaStream_t st);
// CholeskyQR2 of the n x n X (row-major, ld n): Q (n x n) and R (n x n upper,
// zeros below) with X = Q R. Scratch Q1, W, Ri, Wk: n x n each; none may alias
// X, Q or R. X is only read.
cudaError_t cholqr2(const double *X, int n, double *Q, double *R, double *Q1, double *W, double *Ri,
                    double *Wk, int *status, cudaStream_t st);

// ---- elementwise / small helpers
cudaError_t set_identity(double *A, int n, int ld, cudaStream_t st);
cudaError_t set_value(double *x, long n, double v, cudaStream_t st);
// out[i*n + j] = in[j*ld + i] * rs[i]   (scaled transpose; rs may be NULL)
cudaError_t transpose_scale(const double *in, int ld, double *out, int n, const double *rs,
                            cudaStream_t st);
// X[i, j] *= rs[i] (rs NULL skips) and *= cs[j]
cudaError_t scale_rows_cols(double *X, int n, int ld, const double *rs, const double *cs,
                            cudaStream_t st);
// norms[j] = ||X[:, j]|| * D[j]
cudaError_t column_norms_scaled(const double *X, int n, const double *D, double *norms,
                                cudaStream_t st);
// perm = argsort(-key) (stable, one CTA), n <= 8192
cudaError_t argsort_desc(const double *key, int n, int *perm, cudaStream_t st);
// out[:, c] = X[:, perm[c]] ; dP[c] = D[perm[c]] ; Trow[c, :] = T[perm[c], :]
cudaError_t permute_udv(const double *X, const double *D, const double *T, const int *perm, int n,
                        double *Xp, double *Dp, double *Tp, cudaStream_t st);
// After QR of Xp: D_new[i] = |R_ii| Dp[i];  R''[i,j] = R_ij Dp[j] / D_new[i] (j >= i), 0 below.
cudaError_t udv_diag_and_scale(double *R, int n, const double *Dp, double *Dnew, cudaStream_t st);
// out = max |A - B| over n x n (A fp64, B float or double); result written to *out (device)
cudaError_t max_abs_diff_f64(const double *A, const double *B, int n, double *out, cudaStream_t st);
cudaError_t max_abs_diff_f32(const double *A, const float *B, int n, double *out, cudaStream_t st);
cudaError_t convert_f64_to_f32(const double *A, float *B, long n, cudaStream_t st);
cudaError_t convert_f32_to_f64(const float *A, double *B, long n, cudaStream_t st);
// dmax = max(D, 1), dmin = min(D, 1), and their reciprocals where needed
cudaError_t split_scales(const double *D, int n, double *dmax_inv, double *dmin, cudaStream_t st);

}  // namespace dq
