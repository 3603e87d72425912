// Launch interfaces of the hot-path kernels (propagation, delayed update,
// measurement), shared by the engine and the operator entry points.
#pragma once

#include "common.cuh"
#include "df64.cuh"

namespace dq {

// ---- FFT propagator (prop_f32.cu / prop_f64.cu)
cudaError_t launch_prop_f64(int L, int side, const double *X, double *Y, int nvec, int ld,
                            const cpx<double> *E, const double *pre, const double *post,
                            const double *vscale, cudaStream_t st);
cudaError_t launch_prop_f32(int L, int side, const float *X, float *Y, int nvec, int ld,
                            const cpx<float> *E, const float *pre, const float *post,
                            const float *vscale, cudaStream_t st);

// FP64 operand, double-float arithmetic (prop_df.cu); E: (hi, lo) FP32 pairs
cudaError_t launch_prop_df(int L, int side, const double *X, double *Y, int nvec, int ld,
                           const cpx<df64> *E, const double *pre, const double *post,
                           const double *vscale, cudaStream_t st);

// ---- delayed update (update.cu)
template <typename T>
cudaError_t launch_gather(int N, int s0, int kb, int K, const T *G, T *Gcol, T *Grow,
                          cudaStream_t st);

// One delayed-update block: decisions, flips in s, and the coefficient
// vectors alpha (rows m' < m, row stride K) and beta of the accepted flips;
// g = G[S,S] (double, or float when g_f32).
struct MetroArgs {
  int N, s0, kb, K;
  int ld_g;              // row stride of g = G[S, S]
  double e2l, em2l;      // e^{2 lambda}, e^{-2 lambda} (host-computed)
  uint32_t k0, k1;       // Philox key (seed)
  uint32_t c2, c3;       // counter words 2 (2*sweep + pass) and 3 (chain | domain << 24)
  int slice0;            // counter word 1 (0-based slice)
  int *perm = nullptr;   // k <= 32: if set, the accepted sites (block-relative, in order), -1 after
};
// Decisions and Woodbury coefficients of one block (see update.cu), in FP64
// or (df) double-float arithmetic. reserve_smem: shared memory to claim
// (bytes, <= 224 KB) so that the block has its SM to itself while another
// kernel runs concurrently; 0 = its need.
cudaError_t launch_metropolis(const MetroArgs &a, const void *g, bool g_f32, int8_t *s,
                              const uint8_t *forced, double *alpha, double *beta, int *accept_count,
                              int *status, unsigned long long *total, cudaStream_t st,
                              bool df = false, int reserve_smem = 0);

struct FlushArgs {
  int N, s0, kb;   // current block
  int ns0, nkb;    // next block (nkb = 0: none)
  int rows_per_cta;
  int ldc;         // row stride of Gcol (>= kb); the next-block Gcol uses stride K
  int ldb;         // row stride of beta
  int lda;         // row stride of alpha
};
// G <- G - (Gcol alpha^T)(beta (E_S - Grow)): the A kernel then the rank-m
// flush. Abuf: N x K scratch (T), or, when df, 2 N K float2 pairs (A, then B).
// df = FP64-accurate double-float product on the FP32 units (T = double only).
template <typename T>
cudaError_t launch_flush(int K, const FlushArgs &a, T *G, const T *Gcol, const T *Grow,
                         const double *alpha, const double *beta, const int *acc, void *Abuf,
                         T *Gcol_next, T *Grow_next, bool df, cudaStream_t st);

// The two halves of launch_flush: A = Gcol alpha^T into Abuf (and, when df,
// the B factor after it), then the rank-m update of G (with the next block's
// gather when a.nkb > 0).
template <typename T>
cudaError_t launch_amat(int K, const FlushArgs &a, const T *Gcol, const T *Grow,
                        const double *alpha, const double *beta, const int *acc, void *Abuf,
                        bool df, cudaStream_t st);
template <typename T>
cudaError_t launch_flush_update(int K, const FlushArgs &a, T *G, const void *Abuf, const T *Grow,
                                const double *beta, const int *acc, T *Gcol_next, T *Grow_next,
                                bool df, cudaStream_t st);
// Look-ahead: the next block's G'[S', S'] (a.nkb x a.nkb doubles, row stride
// a.nkb) after the pending flush, from the pre-flush G, A (Abuf) and beta.
template <typename T>
cudaError_t launch_lookahead_g(int K, const FlushArgs &a, const T *G, const void *Abuf, bool df,
                               const T *Grow, const double *beta, const int *acc, double *gnext,
                               cudaStream_t st);

// The FP64-accurate flush on tcgen05 (flush_tc.cu), delay rank K = 32
// (a.kb, a.nkb <= 32; row strides ldc = lda = ldb = 32): the A and B factors
// as digit tiles in ws (flush_tc_workspace_bytes, 256-byte aligned, zeroed
// once before first use), then G <- G - A B^T with the next block's gather
// into Gcol_next (N x 32) / Grow_next (a.nkb x N). flush_tc_timed_out:
// whether a bounded wait of the flush kernel gave up (synchronises st).
size_t flush_tc_workspace_bytes(int N);
cudaError_t launch_flush_tc(const FlushArgs &a, double *G, const double *Gcol, const double *Grow,
                            const double *alpha, const double *beta, const int *acc, void *ws,
                            double *Gcol_next, double *Grow_next, cudaStream_t st);
bool flush_tc_timed_out(cudaStream_t st);
// The two launches of launch_flush_tc: the digit tiles (and, when Anext is
// not NULL, the next block's rows of A as double-float pairs, Anext[i * 32 +
// r] for a.ns0 <= i < a.ns0 + a.nkb, for the look-ahead), then the update.
// With perm (the accepted sites of the block, as the Metropolis block writes
// them; beta then has its selector form), the tiles kernel skips the scan of
// the coefficients and, given G (pre-flush) and gnext, also writes the next
// block's G'[S', S'] (a.nkb x a.nkb, row stride a.nkb).
cudaError_t launch_flush_tc_prep(const FlushArgs &a, const double *Gcol, const double *Grow, const double *alpha,
                                 const double *beta, const int *acc, void *ws, float2 *Anext, cudaStream_t st,
                                 const int *perm = nullptr, const double *G = nullptr, double *gnext = nullptr);
cudaError_t launch_flush_tc_update(const FlushArgs &a, double *G, const int *acc, void *ws, double *Gcol_next,
                                   double *Grow_next, cudaStream_t st);

// ---- measurement (measure.cu)
struct MeasTables {
  const double *pc, *ps;    // e^{i Q r} for Q = Gamma + dk
  const double *wgc, *wgs;  // CDW weights at Gamma
  const double *wkc, *wks;  // CDW weights at K (nullptr if absent)
  const int *nbr;           // 4 neighbours per site (with repeats for tiny tori)
};
constexpr int kMeasRaw = 10;
cudaError_t launch_measure(const double *G, int N, const MeasTables &t, double *raw, double thop,
                           double *obs, cudaStream_t st);

// ---- shared-memory opt-in, once per (kernel, device)
cudaError_t ensure_smem_attr(const void *func, int bytes);

}  // namespace dq
