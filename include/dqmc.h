/*
 * dqmc.h -- C ABI of the GB300 kagome DQMC time-slice sweep.
 *
 * Method: finite-temperature determinant QMC for the attractive Hubbard model
 * (Eq. 1 of arXiv 2608.03894, U < 0 is attraction) on an L x L-cell kagome
 * torus with N = 3 L^2 sites. The hot path per imaginary-time slice is
 *   (1) the kinetic propagator products e^{-dtau K} G and G e^{+dtau K}, done
 *       as 2D FFTs over cells per sublattice, a per-momentum 3x3 block multiply
 *       and inverse FFTs (Sec. II, Eq. 2-6);
 *   (2) the diagonal e^{V(s)} scaling of the Ising Hubbard-Stratonovich field;
 *   (3) the Metropolis sweep over the slice with delayed updates: k rank-one
 *       Sherman-Morrison corrections accumulated and flushed as one rank-k
 *       product (the delayed-update scheme the paper combines with its FFT
 *       propagation, Sec. II last paragraph and Sec. III);
 *   (4) periodic FP64 UDV (QR) stabilisation and recomputation of G.
 *
 * Conventions (all calls):
 *   - Site index i = (x1*L + x2)*3 + a, a in {A,B,C} (Kronecker order of Eq. 3).
 *   - G_ij = <c_i c_j^+> of one spin species, N x N, ROW-MAJOR, FP64 on the
 *     host side of this ABI.
 *   - Ising field s[l-1][i] in {-1,+1}, int8, M x N slice-major, M = beta/dtau.
 *   - U uses the paper's sign: U <= 0; U > 0 is rejected (DQMC_EINVAL).
 *   - Interaction in particle-hole symmetric form U (n_up - 1/2)(n_dn - 1/2);
 *     mu = -1 puts the U = 0 Fermi level at the Dirac point (rho = 2/3).
 *   - Random numbers: Philox4x32-10, key = seed, counter = (site, slice-1,
 *     2*sweep + pass, chain | domain << 24); one draw per proposal.
 *   - Every call returns a dqmc_status; on failure dqmc_last_error() returns a
 *     thread-local message. No C++ exception crosses this boundary.
 *   - Host buffers passed in are owned by the caller and only read or written
 *     during the call. Device memory the library allocates is owned by the
 *     context and freed by dqmc_destroy.
 *   - After DQMC_ECUDA or DQMC_ETIMEOUT a context is poisoned: every later
 *     call except dqmc_destroy returns DQMC_ESTATE.
 */
#ifndef DQMC_GB300_H
#define DQMC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dqmc_ctx dqmc_ctx;

typedef enum {
  DQMC_OK = 0,
  DQMC_EINVAL = 1,    /* bad argument (size, sign of U, unsupported L, null pointer) */
  DQMC_ENOMEM = 2,    /* device or host allocation failed, or the host refused another
                         resource (no C++ exception crosses this interface) */
  DQMC_ECUDA = 3,     /* a CUDA runtime call or kernel failed */
  DQMC_ENUMERIC = 4,  /* non-positive or non-finite acceptance ratio, drift above the hard limit */
  DQMC_ETIMEOUT = 5,  /* a bounded device wait gave up */
  DQMC_ESTATE = 6     /* context poisoned by an earlier failure, or call out of order */
} dqmc_status;

/* Binned means and errors of the equal-time estimators (Sec. III and IV):
 *   S_pair_G  = S_Pair(Gamma), S_pair_dk = S_Pair(Gamma + dk), dk = b1/L,
 *     symmetric definition (1/N) sum_ij e^{iQ(r_i - r_j)} <D_i^+ D_j + D_j D_i^+>;
 *   phi2_G, phi2_K = <phi^+ phi>(Q) of the CDW field
 *     phi(Q) = (1/N) sum_cells e^{iQR}(n_A + w n_B + w^2 n_C), w = e^{2 pi i/3};
 *     phi2_K is NaN when 3 does not divide L (no K point on the mesh);
 *   density = (2/N) sum_x (1 - G_xx), ekin = (2/N) sum_ij K_ij (delta_ij - G_ji).
 * Derived with a jackknife over bins: R_pair = 1 - S(Gamma+dk)/S(Gamma),
 * P = sqrt(S(Gamma)/N), D_G = sqrt(phi2_G), D_K = sqrt(phi2_K). */
typedef struct {
  double S_pair_G, S_pair_dk, phi2_G, phi2_K, density, ekin; /* means */
  double err[6];                                             /* standard errors over bins */
  long n_samples;                                            /* measurements accumulated */
  long n_bins;
  double R_pair, R_pair_err, P, P_err, D_G, D_K;
} dqmc_obs;

/* Run statistics. */
#define DQMC_KERNEL_FAMILIES 10

typedef struct {
  long sweeps;           /* sweeps done since create/load */
  long proposed;         /* Metropolis proposals (2 N M per sweep) */
  long accepted;
  double max_drift;      /* max |G_wrapped - G_fresh| at stabilisation points */
  double last_drift;     /* same, over the last sweep only */
  double ms_wrap, ms_update, ms_stab, ms_measure; /* device time per phase (timing >= 1) */
  /* device time and launch count per kernel family (timing = 2): 0 FFT
   * propagation, 1 Metropolis block, 2 rank-k flush, 3 stabilisation GEMMs,
   * 4 QR panels and Cholesky diagonal blocks, 5 measurement, 6 other small kernels, 7 operand splitting of
   * the emulated GEMMs, 8 delayed-update helpers (gathers, A/B factors,
   * look-ahead block), 9 stabilisation helpers (T factors, triangular
   * inverses, pivoting, scaling) */
  double ms_kernel[DQMC_KERNEL_FAMILIES];
  long n_kernel[DQMC_KERNEL_FAMILIES];
  /* algorithmic work per family (any timing): flops of the operation and
   * bytes of one read of its inputs plus one write of its outputs */
  double flops_kernel[DQMC_KERNEL_FAMILIES];
  double bytes_kernel[DQMC_KERNEL_FAMILIES];
  unsigned long long launches; /* kernel launches issued for this context (any timing) */
} dqmc_stats;

/* ------------------------------------------------------------------ context API */

/* Validate parameters and create a context for one Markov chain on the current
 * CUDA device. L >= 1 from the supported set {1,2,3,4,6,8,12,16,24,36}; beta/dtau
 * a positive integer (1e-9); U <= 0. Device memory is allocated lazily on the
 * first call that needs it, so dqmc_set_option / dqmc_set_stream /
 * dqmc_set_allocator / dqmc_set_field may follow. Initial field: Philox
 * (domain 1), s = +1 iff the low bit of word 0 is set. Returns DQMC_EINVAL on a
 * bad argument. */
dqmc_status dqmc_create(int L, double beta, double dtau, double U, double mu, uint64_t seed,
                        dqmc_ctx **out);

/* Options (numbers):
 *   "k"          delay rank (4, 8, 16, 32 or 64; default 32);
 *   "n_stab"     slices between UDV refreshes (default 10);
 *   "precision"  0 = plain FP64 (default);
 *                1 = mixed: FP64 data; rank-m flush as FP64-accurate
 *                    digit slices on the tcgen05 tensor cores at k = 32 (see
 *                    "flush_tc"), else in double-float arithmetic (FP32
 *                    pairs, ~2^-47) on the FP32 units; FFT
 *                    propagation in FP64 (see "df_prop"); stabilisation
 *                    products as exact digit slices on the bf16 tensor
 *                    cores, except the two small products of each block
 *                    reflector (FP64 kernels, see "refl_gram", "refl_tw");
 *                    Metropolis decisions and Woodbury coefficients in
 *                    double-float (see "df_metro"); Householder panels and
 *                    triangular inverses in FP64;
 *                2 = plain FP32 propagation and flush, which drifts by
 *                    1e-3..1e-1 per refresh interval (for comparison);
 *   "chain"      Philox chain id;
 *   "timing"     1 = per-phase CUDA-event timers, 2 = also per kernel family
 *                (the events cost time: time throughput with 0);
 *   "site_offsets" 1 = S_Pair phases use site positions R + tau_a, 0 = cells;
 *   "bin"        measurements per bin (default 10);
 *   "drift_limit" hard limit on the refresh drift (default 1e-3 -> DQMC_ENUMERIC);
 *   "pipeline"   1 (default): the next delayed-update block's Metropolis runs on
 *                a second stream beside the current flush; 0: everything on the
 *                context's stream, one kernel after another (the same decisions;
 *                for profilers that serialise launches);
 *   "metro_reserve" shared memory in bytes (0..229376, default 204800) that the
 *                Metropolis block of the next delayed-update block claims while
 *                it runs beside the current flush, so that it has an SM to
 *                itself; 0 = only what it needs;
 * mixed precision only (1 = double-float, 0 = native FP64 for that step):
 *   "df_flush"   rank-m flush as double-float products (default 1);
 *   "flush_tc"   with df_flush = 1 and k = 32: the flush as digit slices on
 *                tcgen05 (dqmc_op_flush_tc), whose digit-tile kernel also
 *                forms the next block's look-ahead rows; with "pipeline" = 1
 *                the next block's Metropolis runs on the second stream beside
 *                the flush (default 1; 0 = the double-float flush); a bounded
 *                wait of its kernel that gives up makes dqmc_sweep return
 *                DQMC_ETIMEOUT;
 *   "df_prop"    FFT propagation in double-float arithmetic (default 0: the
 *                propagation is ~4% of a sweep, and its rounding, applied to
 *                the whole G every slice, dominated the double-float drift at
 *                L = 36: 1.1e-6 against 4.5e-7 with FP64 propagation);
 *   "df_metro"   Metropolis decisions, the tracked k x k block and the
 *                Woodbury coefficients in double-float arithmetic (default 1;
 *                0 = FP64, whose serial chain is ~8x slower on this part);
 *   "df_panel"   Householder panel column loop (dot products and row
 *                updates) in double-float arithmetic on columns scaled by
 *                powers of two, reflector scalars in FP64 (default 0: the
 *                panel is bound by barrier latency, not by the FP64 pipe, and
 *                this gains ~2% of an L = 24 sweep for ~2x the drift);
 *   "refl_gram"  with stab_gemm = 2: the Gram matrix V^T V of each block
 *                reflector of the QR, whose digit-slice GEMM leaves most of
 *                the GPU idle: 0 = digit slices, 1 = a parallel FP64 kernel
 *                (default), 2 = a parallel double-float kernel (its error costs
 *                the reflectors' orthogonality: L = 36 drift above 1e-6);
 *   "refl_tw"    with stab_gemm = 2: op(T) W of each block reflector:
 *                0 = digit slices, 1 = a parallel FP64 kernel (default;
 *                ~3% faster per L = 24 sweep than 0), 2 = a column-scaled
 *                double-float kernel (as fast as 1, but it drifts to ~1e-6
 *                at L = 24 and 1.9e-6 at L = 36 over a few sweeps);
 *   "stab_gemm"  stabilisation GEMMs: 0 = FP64, 1 = double-float, 2 = exact
 *                7-bit digit slices on the bf16 tensor cores (default 2);
 *   "tc_gemm"    with stab_gemm = 2: 1 (default) = the digit-slice products
 *                with M, N, K >= 256 on tcgen05 (tensor-memory accumulators),
 *                the skinny ones on warp-level mma.sync; 0 = all on mma.sync;
 *                a bounded wait of the tcgen05 kernel that gives up makes
 *                dqmc_sweep return DQMC_ETIMEOUT;
 *   "gemm_sites" 32-bit mask of the stabilisation GEMM call sites that use the
 *                stab_gemm variant (default all);
 *   "gemm_df_sites" with stab_gemm = 2: mask of those sites that use the
 *                double-float GEMM instead (default 0). Site bits: 0 QR trailing
 *                update, 1 explicit Q, 2 T update, 3 U_r^T U_l, 4 T_r T_l^T,
 *                5 QR of the scale-separated matrix, 6 Q^T B, 7 triangular
 *                solve, 8 final product, 9 CholeskyQR2 (Gram matrices,
 *                Cholesky recursion, Q and R products).
 *   "stab_qr"    orthogonal-triangular factorisation of the stabilisation:
 *                0 = Householder QR (panels on one thread-block cluster),
 *                1 = CholeskyQR2 for the stack products and shifted
 *                CholeskyQR3 for the scale-separated matrix (all but 64 x 64
 *                diagonal blocks as GEMMs; slower than Householder with the
 *                present GEMMs, and its Gram matrix loses definiteness on
 *                the L = 36 stacks), 0 (default) = Householder, -1 =
 *                CholeskyQR in mixed precision only. dqmc_green always uses
 *                Householder QR. A non-positive Cholesky pivot makes
 *                dqmc_sweep return DQMC_ENUMERIC.
 * "k", "n_stab", "precision", "chain", "df_flush", "flush_tc", "df_prop", "df_metro",
 * "stab_gemm", "stab_qr" and "gemm_df_sites" are accepted only before the first sweep;
 * later they return DQMC_ESTATE. */
dqmc_status dqmc_set_option(dqmc_ctx *ctx, const char *key, double value);

/* Launch every kernel of this context on the given cudaStream_t (e.g. the
 * current PyTorch stream). NULL = the legacy default stream. */
dqmc_status dqmc_set_stream(dqmc_ctx *ctx, void *cuda_stream);

/* Route device allocations through the caller (e.g. PyTorch's caching
 * allocator). alloc(bytes, user) returns a device pointer or NULL; release(ptr,
 * user) frees it. Must be called before the first allocation (DQMC_ESTATE
 * otherwise). */
dqmc_status dqmc_set_allocator(dqmc_ctx *ctx, void *(*alloc)(size_t, void *),
                               void (*release)(void *, void *), void *user);

/* n_sweeps sweeps: an up pass l = 1..M (wrap, then propose all N sites of slice
 * l in index order) and a down pass l = M..1 (propose, then unwrap); G is
 * recomputed from the UDV stacks every n_stab slices. measure != 0 accumulates
 * the estimators at every up-pass stabilisation point (fresh FP64 G). The call
 * returns when the work is done (it synchronises the stream). */
dqmc_status dqmc_sweep(dqmc_ctx *ctx, int n_sweeps, int measure);

/* G(tau_slice), 0 <= slice <= M, recomputed from scratch in FP64 from the
 * current field (QR chain over all slices; does not touch the running state).
 * G_out: host, N*N doubles, row-major, caller-owned. */
dqmc_status dqmc_green(dqmc_ctx *ctx, int slice, double *G_out);

/* The running (wrapped/updated) G at the current slice, converted to FP64.
 * G_out: host N*N doubles; *slice receives the current slice index. */
dqmc_status dqmc_get_running_green(dqmc_ctx *ctx, double *G_out, int *slice);

/* Binned means/errors accumulated so far (see dqmc_obs). */
dqmc_status dqmc_measure(dqmc_ctx *ctx, dqmc_obs *out);

/* Statistics (see dqmc_stats). */
dqmc_status dqmc_get_stats(dqmc_ctx *ctx, dqmc_stats *out);

/* Copy the field out (M*N int8) or in. Setting a field rebuilds the stacks
 * and G at tau = 0 (values other than +-1 -> DQMC_EINVAL). Setting the field
 * the chain already holds at tau = 0 (e.g. the one dqmc_get_field returned
 * after a sweep) is detected on the device and keeps the running G and the
 * stacks as they are. */
dqmc_status dqmc_get_field(dqmc_ctx *ctx, int8_t *s_out);
dqmc_status dqmc_set_field(dqmc_ctx *ctx, const int8_t *s);

/* Replay (forced flips through the fast path), for measuring |dG| against an
 * exact G. Starting from the fresh G at tau = 0 of the current field, runs the
 * up pass l = 1..slice exactly as dqmc_sweep does (wrap, delayed-update blocks
 * of rank k in the context's precision, UDV refreshes at the checkpoints
 * before `slice`), except that every decision is forced: site i of slice l
 * flips iff its spin differs from target[(l-1)*N + i]. G_out (N*N doubles,
 * caller-owned host memory, row-major) receives the running G(tau_slice) of
 * the fast path, before any refresh at that slice. Afterwards slices
 * 1..slice of the field equal the target and the others are unchanged; the
 * stacks are rebuilt by the next call. The flips count as accepted proposals
 * in dqmc_stats. Sequential Sherman-Morrison / Woodbury update of Sec. II
 * with the wrap of Eq. 5-6. DQMC_EINVAL on NULL pointers, a slice outside
 * [1, M] or target values other than +-1. */
dqmc_status dqmc_replay(dqmc_ctx *ctx, const int8_t *target, int slice, double *G_out);

/* Checkpoint: parameters, the options k, n_stab, precision, chain,
 * site_offsets and bin, the field, the sweep counter, statistics and bins (the
 * other options keep the loading context's values). G is recomputed on load.
 * Binary file; DQMC_EINVAL if the file does not match the context's
 * (L, beta, dtau, U, mu) or cannot be opened. */
dqmc_status dqmc_save(dqmc_ctx *ctx, const char *path);
dqmc_status dqmc_load(dqmc_ctx *ctx, const char *path);

/* Batched independent chains (several Markov chains, of possibly different
 * L, sharing one GPU; the paper does not say how it used its cores, DQMC
 * usually parallelises over independent chains). dqmc_batch_create makes n
 * contexts from params, n rows of (L, beta, dtau, U, mu, seed) doubles (L and
 * seed integral), into the caller's array out[n]; chain i gets chain id i
 * and its own non-blocking CUDA stream (destroyed with the context). Each
 * context is then an ordinary one (options, measurements, fields, destroy).
 * On any failure every context made so far is destroyed, out[] is NULL and
 * the status of the failing chain is returned (DQMC_EINVAL for bad rows).
 * dqmc_batch_sweep runs n_sweeps sweeps on the n distinct contexts at once,
 * one host thread per chain, so that the kernels of different chains overlap
 * on the GPU; it returns when all are done, with the first failing chain's
 * status. */
dqmc_status dqmc_batch_create(int n, const double *params, dqmc_ctx **out);
dqmc_status dqmc_batch_sweep(dqmc_ctx **ctxs, int n, int n_sweeps, int measure);

/* Autotuner of the delay rank k and the refresh interval n_stab (the paper
 * fixes both by hand, Sec. II): for every candidate pair (ks[a], n_stabs[b])
 * a fresh chain of the given parameters, seed and precision (0 FP64, 1 mixed,
 * 2 FP32) runs `warmup` untimed sweeps, then `sweeps` sweeps timed with CUDA
 * events on a stream of its own; a pair whose max |G_wrapped - G_fresh| over
 * those sweeps exceeds drift_bar is not admissible. On success *k_best and
 * *n_stab_best get the admissible pair with the least time per sweep (the
 * first in candidate order on ties) and *sec_per_sweep its time; times (NULL
 * or nk * ns doubles, row a, column b) gets every pair's seconds per sweep,
 * -1 for a pair that is not admissible. The FFT tiling is not a knob: the
 * propagation kernel is specialised per L. Host pointers; the chains are
 * created and destroyed inside the call (device memory from cudaMalloc).
 * DQMC_EINVAL on empty candidate lists, a candidate < 1, warmup < 0,
 * sweeps < 1, drift_bar <= 0, a precision other than 0, 1, 2, NULL outputs,
 * a candidate the chain rejects, or when no pair is admissible; a failing
 * chain's status otherwise. */
dqmc_status dqmc_autotune(int L, double beta, double dtau, double U, double mu, uint64_t seed,
                          int precision, const int *ks, int nk, const int *n_stabs, int ns,
                          int warmup, int sweeps, double drift_bar, int *k_best, int *n_stab_best,
                          double *sec_per_sweep, double *times);

/* Message of the last failure on the calling host thread ("" if none); valid
 * until the thread's next failing call. */
const char *dqmc_last_error(void);
/* Synchronise the context's streams, free its device memory (through the
 * allocator callbacks when set) and the context. NULL is ignored. */
void dqmc_destroy(dqmc_ctx *ctx);

/* Library version string. */
const char *dqmc_version(void);

/* ------------------------------------------------------------------ operator API
 * Stateless steps of the hot path on caller-owned DEVICE memory, launched on
 * the given stream (NULL = legacy default stream). They validate sizes and
 * pointers, return DQMC_EINVAL on misuse, and report launch failures as
 * DQMC_ECUDA. They are what the parity tests call one step at a time. */

/* Eq. 5-6: kinetic propagator product with fused diagonal scalings.
 *   side 0 (left, acts on the N-long columns of X):
 *     Y = diag(post) e^{scale K} diag(pre) X diag(vscale)
 *   side 1 (right, acts on the N-long rows of X):
 *     Y = diag(vscale) X diag(pre) e^{scale K} diag(post)
 * X, Y: N x nvec (side 0) or nvec x N (side 1) row-major with leading dimension
 * ld >= (side 0 ? nvec : N); Y may alias X. pre/post: length N or NULL;
 * vscale: length nvec or NULL. _f64: double data and vectors, _f32: float,
 * _df: double data and vectors, computed in double-float arithmetic (pairs of
 * FP32, ~2^-47 relative) on the FP32 units. The 3x3 momentum blocks
 * e^{scale H(k)} are built on the host in FP64 (cached per (L, scale)). */
dqmc_status dqmc_op_propagate_f64(int L, double scale, int side, const double *X, double *Y,
                                  int nvec, int ld, const double *pre, const double *post,
                                  const double *vscale, void *stream);
dqmc_status dqmc_op_propagate_df(int L, double scale, int side, const double *X, double *Y,
                                 int nvec, int ld, const double *pre, const double *post,
                                 const double *vscale, void *stream);
dqmc_status dqmc_op_propagate_f32(int L, double scale, int side, const float *X, float *Y,
                                  int nvec, int ld, const float *pre, const float *post,
                                  const float *vscale, void *stream);

/* Delayed-update block (one CTA, FP64 bookkeeping; the delayed update the
 * paper combines with its FFT propagation): propose the kb <= 64 sites
 * S = [site0, site0+kb) of slice `slice1` (1-based) in order, given
 * g = G[S,S] (kb x kb, row-major, ld_g, device FP64), the field row s (N int8,
 * device, flipped in place on accept), lambda, the Philox key/counter words.
 * Writes accept_count[0] = m and alpha, beta (kb x kb, row-major FP64, device):
 * rows 0..m-1 hold the coefficient vectors of the accepted flips in order, the
 * other rows zero, such that the m sequential Sherman-Morrison updates equal
 *   G' = G - (G[:,S] alpha^T) (beta (E_S - G[S,:]))
 * with E_S the kb x N selector of S: alpha^T beta is the Woodbury matrix
 * Gamma = (Delta^{-1} + I - G[P,P])^{-1} of the accepted sites P (row r of
 * beta selects the r-th accepted site, row r of alpha is column r of Gamma).
 * Non-positive or non-finite ratios set *status = 1 and stop. forced != NULL
 * (kb bytes) replaces the decision. */
dqmc_status dqmc_op_metropolis_block(int N, int site0, int kb, const double *g, int ld_g,
                                     int8_t *s, double lambda, uint64_t seed, uint32_t chain,
                                     uint32_t sweep_pass, int slice1, const uint8_t *forced,
                                     double *alpha, double *beta, int *accept_count, int *status,
                                     void *stream);
/* The same block with the decision arithmetic (the tracked k x k block, the
 * ratios) and the Woodbury coefficients in double-float arithmetic (FP32
 * pairs, ~2^-47) on the FP32 units: the mixed precision mode's Metropolis.
 * Same arguments, outputs and errors as dqmc_op_metropolis_block. */
dqmc_status dqmc_op_metropolis_block_df(int N, int site0, int kb, const double *g, int ld_g,
                                        int8_t *s, double lambda, uint64_t seed, uint32_t chain,
                                        uint32_t sweep_pass, int slice1, const uint8_t *forced,
                                        double *alpha, double *beta, int *accept_count, int *status,
                                        void *stream);

/* Rank-m flush of one block: G <- G - (Gcol alpha^T)(beta (E_S - Grow)), with
 * Gcol = G[:,S] (N x kb, ld kb) and Grow = G[S,:] (kb x N, ld N) taken before
 * the update, alpha/beta/accept_count as written by dqmc_op_metropolis_block
 * (device). G: N x N row-major (ld N), device. The N x kb factor A lives in
 * scratch memory that the call allocates and frees on the stream.
 * _f64: FP64 arithmetic; _df: FP64 storage, FP64-accurate double-float
 * product on the FP32 units; _f32: FP32 G. */
dqmc_status dqmc_op_flush_f64(int N, int site0, int kb, double *G, const double *Gcol,
                              const double *Grow, const double *alpha, const double *beta,
                              const int *accept_count, void *stream);
dqmc_status dqmc_op_flush_df(int N, int site0, int kb, double *G, const double *Gcol,
                             const double *Grow, const double *alpha, const double *beta,
                             const int *accept_count, void *stream);
dqmc_status dqmc_op_flush_f32(int N, int site0, int kb, float *G, const float *Gcol,
                              const float *Grow, const double *alpha, const double *beta,
                              const int *accept_count, void *stream);
/* The same flush, FP64 G, with the product on the tcgen05 tensor cores:
 * the N x kb factors A = Gcol alpha^T and B^T = beta (E_S - Grow) in
 * double-float arithmetic, cut into seven 8-bit digits per entry (row-wise
 * power-of-two scaling) and multiplied digit pair by digit pair (28 pairs,
 * exact FP32 accumulation in tensor memory), the levels combined exactly in
 * integers and subtracted from G in FP64: FP64-accurate like _df. The mixed
 * precision sweep's flush at delay rank 32. Requires kb <= 32 (else
 * DQMC_EINVAL); scratch (~0.9 KB per row of G) is allocated and freed on the
 * stream. A bounded wait inside the kernel that gives up returns
 * DQMC_ETIMEOUT with G unchanged in the tiles it covers. */
dqmc_status dqmc_op_flush_tc(int N, int site0, int kb, double *G, const double *Gcol,
                             const double *Grow, const double *alpha, const double *beta,
                             const int *accept_count, void *stream);

/* dqmc_op_flush_f64 without any device allocation. The paper has no
 * counterpart: it is a deployment variant of dqmc_op_flush_f64 (above) for
 * callers that cannot allocate. Same arguments, semantics and FP64 result, but
 * the N x K scratch for the factor A (K = kb rounded up to a power of two >= 4)
 * is a fixed device array compiled into the library: 248,832 doubles (1.9 MiB),
 * enough for N <= 3888 (L = 36) at K = 64. Larger N * K -> DQMC_EINVAL, before
 * any launch. For callers that cannot allocate device memory during the call:
 * a process that has handed all device memory to its own pool or caching
 * allocator up front (a cudaMallocAsync here could fail or grow a pool that
 * must stay fixed), and host code that must not block on the device
 * (cudaFree synchronises). The first call on a device resolves the array's
 * device address (cudaGetSymbolAddress, with that device current) and keeps it
 * for the life of the process; make that first call before any stream capture,
 * and do not use the entry point on a device after cudaDeviceReset there (the
 * kept address would belong to the destroyed context). Nothing has to start at zero: every
 * scratch entry is written before it is read. The one array is shared by all
 * calls on a device, so overlapping calls (several streams or host threads at
 * once) race; serialise them. */
dqmc_status dqmc_op_flush_f64_noalloc(int N, int site0, int kb, double *G, const double *Gcol,
                                      const double *Grow, const double *alpha, const double *beta,
                                      const int *accept_count, void *stream);

/* FP64 GEMM of the stabilisation, C = alpha op(A) op(B) + beta C (row-major,
 * device), op = transpose when ta / tb. mode 0: FP64 FMA; 1: FP64-accurate
 * double-float product on the FP32 units; 2: FP64-accurate product from exact
 * 7-bit digit slices on the bf16 tensor cores (Ozaki-style error-free
 * splitting; the stabilisation of the mixed precision mode uses it), warp-level
 * mma.sync; 3: the same digit slices on tcgen05 with tensor-memory
 * accumulators.
 * Modes 1-2 allocate their operand workspace on the stream. */
dqmc_status dqmc_op_gemm_f64(int mode, int ta, int tb, int M, int N, int K, double alpha,
                             const double *A, int lda, const double *B, int ldb, double beta,
                             double *C, int ldc, void *stream);

/* Trial orbitals of the projector (zero-temperature) variant, Sec. II: an
 * orthonormal real basis of the lowest n_occ eigenstates of
 * K + eps diag(+1, 0, -1) (sublattices A, B, C; t = 1), the filling being
 * rho = 2 n_occ / N. eps splits the Dirac-point degeneracy of the closed shell
 * at rho = 2/3 when 3 | L (1e-4 is the reading used here); 0 is allowed when
 * the shell is closed without it. Host-only (no device work): P_out is a
 * caller-owned host buffer of N * n_occ doubles, row-major (site index
 * (x1 L + x2) 3 + a), built from the momentum blocks of Eq. 4. Open shell (the
 * n_occ-th and next level closer than 1e-9, or a pair k, -k split) or
 * 1 <= n_occ < N violated -> DQMC_EINVAL. */
dqmc_status dqmc_op_trial_state(int L, int n_occ, double eps, double *P_out);

/* Full-momentum maps of the two order-parameter correlators of Sec. III and
 * IV from one FP64 G (N x N row-major, device, N = 3 L^2): for every mesh
 * momentum Q = m1 b1 / L + m2 b2 / L, S_out[m1 * L + m2] = S_Pair(Q) (the
 * symmetric pair structure factor, site positions R + tau_a when
 * site_offsets != 0, else cell positions) and phi2_out[m1 * L + m2] =
 * <phi^+ phi>(Q) (the CDW field with the sublattice phases 1, w, w^2, cell
 * positions); the same definitions as dqmc_obs, at every Q. S_out and
 * phi2_out: host arrays of L^2 doubles, caller-owned. One pass over G bins
 * the correlations by sublattice pair and cell difference, then a Fourier
 * sum per Q. Allocates its scratch on the stream and synchronises it.
 * DQMC_EINVAL for an unsupported L or NULL pointers. */
dqmc_status dqmc_op_measure_fullq(int L, const double *G, int site_offsets, double *S_out,
                                  double *phi2_out, void *stream);

/* Equal-time estimator sums from one FP64 G (N x N row-major, device): writes
 * out[6] (host) = S_pair_G, S_pair_dk, phi2_G, phi2_K, density, ekin, with the
 * same definitions and phase conventions as dqmc_obs (site_offsets as the
 * option). Synchronises the stream. */
dqmc_status dqmc_op_measure(int L, const double *G, int site_offsets, double *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DQMC_GB300_H */
