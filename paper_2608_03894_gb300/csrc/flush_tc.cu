// The rank-m flush of the delayed update on the 5th-generation tensor cores,
// FP64-accurate (mixed precision, delay rank K = 32).
//
// The flush is G <- G - A B^T with the N x K factors
//     A[i][r] = sum_u G[i, S_u] alpha[r][u],
//     B[j][r] = beta[r][j - s0] [j in S] - sum_u beta[r][u] G[S_u, j]
// (update.cu states the Woodbury form they come from). Both are formed in
// double-float arithmetic (as for the double-float flush), then every row of
// A and of B is scaled by a power of two, 2^ex, so that its entries lie in
// (-1, 1), and each entry is cut into seven signed 8-bit digits (the
// error-free splitting of Ozaki, Ogita, Oishi and Rump, 2012; integer
// operations on the bits, balanced digits in [-128, 128], exact in bf16):
//     x = 2^ex sum_{p=1..7} x_p 2^{-7-8(p-1)}   (+ a tail below 2^-55 2^ex).
// Then
//     (A B^T)_ij = 2^{ex_i+ex_j} sum_{l=2..} 2^{-14-8(l-2)} D_l[i][j],
//     D_l = sum_{p+q=l} sum_r a_p[i][r] b_q[j][r],
// keeping the 28 digit pairs with p + q <= 8 (what is dropped weighs less
// than ~2^-48 of max|A_i| max|B_j| in the worst case, far less in practice;
// the double-float flush is good to ~K 2^-47 of the same). Every D_l is a sum
// of at most 7 * 32 products of 8-bit integers, below 2^22, so the bf16
// tensor-core MMA with FP32 accumulation computes it exactly.
//
// Kernels:
//   flush_tc_prep_kernel  one warp per row of A or B (lane = r): the
//       double-float row, its exponent (warp maximum), the digits, written
//       into the tile images the flush kernel copies (see below);
//   flush_tc_kernel       one CTA per 128 columns x 32 rows of G. The MMA's M
//       side is G's columns (the B digits), its N side G's rows (the A
//       digits), so that tensor-memory lane = column and a warp's 32 lanes
//       read and write 32 consecutive entries of a row of G (coalesced). One
//       thread bulk-copies the CTA's two digit tiles (56 KB + 14 KB, one
//       cp.async.bulk each) and issues the 56 MMAs (28 pairs x two K halves
//       of 16) into seven level accumulators of 32 tensor-memory columns; the
//       eight warps then read their lanes' levels (two warps per lane
//       quarter, 16 rows each), combine them exactly into one int64
//       (weights 2^{8(7-l)}, level 8 rounded in), convert that to FP64 with
//       integer operations and subtract it from G (one FP64 add per entry),
//       and gather the next block's rows and columns of the new G.
//       Two CTAs share an SM (256 tensor-memory columns and 70 KB of shared
//       memory each), so one's epilogue overlaps the other's MMAs.
// One thread waits for the copies and the MMAs (bounded, suspending in
// hardware) while the others sleep in a CTA barrier; a wait that gives up
// sets a device flag (flush_tc_timed_out), skips the update and frees the
// tensor memory.
#include <cuda_bf16.h>
#include <stdint.h>

#include "df64.cuh"
#include "kernels.cuh"
#include "linalg.cuh"
#include "tc05.cuh"

namespace dq {

constexpr int FT_K = 32;                       // delay rank (two K halves of 16)
constexpr int FT_M = 128, FT_N = 32;           // G columns x G rows per CTA
constexpr int FT_ND = 7;                       // digits per value
constexpr int FT_LMAX = 8;                     // levels 2..8
constexpr int FT_USLAB = FT_M * 16 * 2;        // bytes of one (digit, K half) tile of the M side
constexpr int FT_VSLAB = FT_N * 16 * 2;
constexpr int FT_UTILE = FT_ND * 2 * FT_USLAB;  // 57344
constexpr int FT_VTILE = FT_ND * 2 * FT_VSLAB;  // 14336
constexpr int FT_SMEM = FT_UTILE + FT_VTILE + 64;
constexpr int FT_TMEM = 256;
constexpr uint32_t FT_IDESC = tc5::idesc_bf16(FT_M, FT_N);

__device__ int g_flush_tc_timeout = 0;

size_t flush_tc_workspace_bytes(int N) {
  const size_t tu = (size_t)(N + FT_M - 1) / FT_M, tv = (size_t)(N + FT_N - 1) / FT_N;
  return tu * FT_UTILE + tv * FT_VTILE + 2 * sizeof(int) * ((size_t)N + FT_M);
}

// x * 2^(55 - ex) truncated toward zero, for a double-float x with |x| < 2^ex
__device__ __forceinline__ long long fixed55_part(float f, int ex) {
  const unsigned int b = (unsigned int)__float_as_int(f);
  const int ef = (int)((b >> 23) & 0xff);
  if (ef == 0 && (b & 0x7fffff) == 0) return 0;
  const long long mant = (long long)((b & 0x7fffff) | (ef ? 0x800000u : 0u));
  const int sh = (ef ? ef : 1) - 150 + 55 - ex;  // value = mant 2^(ef - 150)
  long long v;
  if (sh >= 0)
    v = mant << sh;  // < 2^55 since |f| < 2^ex
  else
    v = (sh > -64) ? (mant >> -sh) : 0;
  return (b >> 31) ? -v : v;
}

__device__ __forceinline__ unsigned short digit_bf16(int d) {
  return __bfloat16_as_ushort(__float2bfloat16_rn((float)d));  // |d| <= 128: exact
}

// Rows [0, N) of A are warps 0 .. N-1 of the first nblk_a CTAs (eight warps
// each), rows of B the warps after them. The CTA stages alpha (A rows) or
// beta (B rows) transposed in shared memory as double-float values; lane u
// converts the row's u-th input once and broadcasts it.
__global__ void __launch_bounds__(256)
    flush_tc_prep_kernel(FlushArgs a, const double *__restrict__ Gcol, const double *__restrict__ alpha,
                         const double *__restrict__ Grow, const double *__restrict__ beta,
                         const int *__restrict__ accept_count, unsigned short *__restrict__ Ud,
                         unsigned short *__restrict__ Vd, int *__restrict__ eU, int *__restrict__ eV,
                         int nblk_a, float2 *__restrict__ Anext, const int *__restrict__ perm,
                         const double *__restrict__ G, double *__restrict__ gnext) {
  __shared__ df64 sc[FT_K][FT_K + 1];  // sc[u][r] = coefficient [r][u]
  __shared__ int s_sel[FT_K];          // B rows: the column of row r's single 1 (-1: none)
  __shared__ int s_nz[FT_K], s_nnz, s_general;  // A rows: the columns with a nonzero coefficient
  const int N = a.N, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m = accept_count ? *accept_count : a.kb;
  const bool isa = (int)blockIdx.x < nblk_a;
  const int row = (isa ? (int)blockIdx.x : (int)blockIdx.x - nblk_a) * 8 + warp;
  // this warp's row inputs, read before the coefficients are staged: lane u
  // holds G[row, s0 + u] (A rows) or G[s0 + u, row] (B rows)
  double gin = 0.0;
  if (row < N && lane < a.kb) gin = isa ? Gcol[(size_t)row * a.ldc + lane] : Grow[(size_t)lane * N + row];
  {
    const double *coef = isa ? alpha : beta;
    const int ld = isa ? a.lda : a.ldb;
    if (threadIdx.x == 0) {
      s_nnz = 0;
      s_general = 0;
    }
    // with the accepted sites given, beta is a selector (not staged) and
    // alpha's nonzero columns are those sites
    if (isa || !perm)
      for (int e = threadIdx.x; e < FT_K * FT_K; e += 256) {
        const int r = e / FT_K, u = e % FT_K;
        sc[u][r] = (r < m && u < a.kb) ? df_from(coef[r * ld + u]) : df64(0.f, 0.f);
      }
    if (perm && threadIdx.x < FT_K) {
      const int t = (int)threadIdx.x < m ? perm[threadIdx.x] : -1;
      s_sel[threadIdx.x] = t;
      s_nz[threadIdx.x] = t < 0 ? 0 : t;
    }
    __syncthreads();
    if (perm) {
      if (threadIdx.x == 0) s_nnz = m;
    } else if (warp == 0) {
      // column u of the coefficients holds a nonzero (A), or row r = lane is a
      // selector: one entry equal to 1, the rest 0 (B)
      bool nz = false;
      int sel = -1, ones = 0, other = 0;
      for (int t = 0; t < FT_K; ++t) {
        const df64 cu = sc[lane][t], cr = sc[t][lane];  // coefficient [t][lane], coefficient [lane][t]
        nz = nz || cu.hi != 0.f;
        if (cr.hi == 1.f && cr.lo == 0.f) {
          ++ones;
          sel = t;
        } else if (cr.hi != 0.f) {
          ++other;
        }
      }
      if (isa) {
        const unsigned msk = __ballot_sync(0xffffffffu, nz);
        if (nz) s_nz[__popc(msk & ((1u << lane) - 1u))] = lane;
        if (lane == 0) s_nnz = __popc(msk);
      } else {
        s_sel[lane] = (lane < m) ? sel : -1;
        if (__any_sync(0xffffffffu, lane < m && (ones != 1 || other != 0))) s_general = 1;
      }
    }
  }
  __syncthreads();
  if (row >= N) return;
  const int r = lane;
  const df64 gu = df_from(gin);
  df64 x(0.f, 0.f);
  if (isa) {
    for (int k = 0; k < s_nnz; ++k) {
      const int u = s_nz[k];
      const df64 gv(__shfl_sync(0xffffffffu, gu.hi, u), __shfl_sync(0xffffffffu, gu.lo, u));
      x = gv * sc[u][r] + x;
    }
  } else if (!s_general) {
    // B[j][r] = [j = s0 + t_r] - G[s0 + t_r][j] with t_r the selected column
    const int t = s_sel[r];
    const df64 gt(__shfl_sync(0xffffffffu, gu.hi, t & 31), __shfl_sync(0xffffffffu, gu.lo, t & 31));
    if (t >= 0) x = (row == a.s0 + t ? df64(1.f, 0.f) : df64(0.f, 0.f)) - gt;
  } else {
    const int js = row - a.s0;
    if (js >= 0 && js < a.kb) x = sc[js][r];
    for (int u = 0; u < a.kb; ++u) {
      const df64 gv(__shfl_sync(0xffffffffu, gu.hi, u), __shfl_sync(0xffffffffu, gu.lo, u));
      x = x - sc[u][r] * gv;
    }
  }
  // the next block's rows of A (double-float pairs, row stride 32) for the look-ahead
  if (isa && Anext && row - a.ns0 >= 0 && row - a.ns0 < a.nkb) Anext[(size_t)row * FT_K + r] = make_float2(x.hi, x.lo);
  // ... or the look-ahead itself: G'[i][j] = G[i][j] + sum_q A[i][q] G[S_{P_q}][j] for the
  // next block's rows i and columns j (beta's row q selects P_q; j is outside this block)
  if (isa && perm && gnext && row - a.ns0 >= 0 && row - a.ns0 < a.nkb) {
    df64 acc(0.f, 0.f);
    for (int q = 0; q < m; ++q) {
      const df64 aq(__shfl_sync(0xffffffffu, x.hi, q), __shfl_sync(0xffffffffu, x.lo, q));
      const double gq = lane < a.nkb ? Grow[(size_t)s_sel[q] * N + a.ns0 + lane] : 0.0;
      acc = aq * df_from(gq) + acc;
    }
    if (lane < a.nkb)
      gnext[(size_t)(row - a.ns0) * a.nkb + lane] = G[(size_t)row * N + a.ns0 + lane] + df_to(acc);
  }
  // row exponent: |x| < 2^ex for every entry (|hi| + |lo| < 2^(e(hi) + 1))
  const unsigned int hb = (unsigned int)__float_as_int(x.hi);
  const int ef = (hb & 0x7fffffff) ? (int)((hb >> 23) & 0xff) : 0;
  const int efmax = __reduce_max_sync(0xffffffffu, ef);
  const int ex = efmax - 126;
  long long y = fixed55_part(x.hi, ex) + fixed55_part(x.lo, ex);
  int d[FT_ND];
#pragma unroll
  for (int p = FT_ND - 1; p >= 1; --p) {
    d[p] = (int)(((y + 128) & 255) - 128);
    y = (y - d[p]) >> 8;
  }
  d[0] = (int)y;
  const int s = r >> 4, k = r & 15;
  if (isa) {
    unsigned short *t = Vd + (size_t)(row / FT_N) * (FT_VTILE / 2);
#pragma unroll
    for (int p = 0; p < FT_ND; ++p) t[(p * 2 + s) * (FT_VSLAB / 2) + tc5::swz(row % FT_N, k)] = digit_bf16(d[p]);
    if (lane == 0) eV[row] = ex;
  } else {
    unsigned short *t = Ud + (size_t)(row / FT_M) * (FT_UTILE / 2);
#pragma unroll
    for (int p = 0; p < FT_ND; ++p) t[(p * 2 + s) * (FT_USLAB / 2) + tc5::swz(row % FT_M, k)] = digit_bf16(d[p]);
    if (lane == 0) eU[row] = ex;
  }
}

// an FP32 holding an integer of magnitude < 2^22, as an int (exact)
__device__ __forceinline__ int f2i_small(float v) {
  return __float_as_int(v + 12582912.0f) - 0x4B400000;  // 1.5 * 2^23
}

// I * 2^s as an FP64 value (|I| < 2^62), with integer operations and no
// branch: normalise |I| so that its leading one is bit 63, keep 53 bits,
// round half up on the bit below, and add the rounded significand (implicit
// bit included) to the biased exponent minus one, so that a carry out of the
// significand moves into the exponent. Zero and results below the normal
// range give zero.
__device__ __forceinline__ double i64_scaled_to_double(long long I, int s) {
  const unsigned long long sign = (unsigned long long)I & 0x8000000000000000ull;
  const unsigned long long a = I < 0 ? 0ull - (unsigned long long)I : (unsigned long long)I;
  const int lz = __clzll((long long)a);
  const unsigned long long t = a << (lz & 63);
  const unsigned long long mant = (t >> 11) + ((t >> 10) & 1ull);
  const long long be1 = 1085 - lz + s;  // biased exponent of 2^(63 - lz + s), minus one
  const unsigned long long bits = sign | (((unsigned long long)be1 << 52) + mant);
  return (a == 0ull || be1 < 0) ? 0.0 : __longlong_as_double((long long)bits);
}

// the update of one entry from its seven level sums D_2 .. D_8 (exact FP32
// integers): I = sum_{l<=7} D_l 2^{8(7-l)} + round(D_8 / 256), then
// I 2^(ex_i + ex_j - 54)
__device__ __forceinline__ double level_update(const float (&v)[FT_LMAX - 1][8], int c, int s) {
  const int h = f2i_small(v[0][c]) * 256 + f2i_small(v[1][c]);   // D_2 2^8 + D_3
  const int mm = f2i_small(v[2][c]) * 256 + f2i_small(v[3][c]);  // D_4 2^8 + D_5
  const int lo = f2i_small(v[4][c]) * 256 + f2i_small(v[5][c]) + f2i_small(v[6][c] * (1.0f / 256.0f));
  const long long I = (long long)h * 4294967296ll + (long long)mm * 65536ll + (long long)lo;
  return i64_scaled_to_double(I, s);
}

// 256 threads: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (the
// tile's columns) for rows 16 (w / 4) .. + 15 of the tile.
constexpr int FT_THREADS = 256;

__global__ void __launch_bounds__(FT_THREADS, 2)
    flush_tc_kernel(FlushArgs a, double *__restrict__ G, const unsigned short *__restrict__ Ud,
                    const unsigned short *__restrict__ Vd, const int *__restrict__ eU,
                    const int *__restrict__ eV, const int *__restrict__ accept_count,
                    double *__restrict__ Gcol_next, double *__restrict__ Grow_next) {
  extern __shared__ __align__(1024) unsigned char fsm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = a.N;
  const int j0 = blockIdx.x * FT_M, i0 = blockIdx.y * FT_N;
  const uint32_t sU = tc5::smem_u32(fsm), sV = sU + FT_UTILE;
  unsigned char *ctl = fsm + FT_UTILE + FT_VTILE;
  const uint32_t mb_load = tc5::smem_u32(ctl), mb_mma = mb_load + 8;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(ctl + 16);
  volatile int *abort = reinterpret_cast<volatile int *>(ctl + 20);
  const int m = accept_count ? *accept_count : a.kb;

  if (tid == 0) {
    tc5::mbar_init(mb_load, 1);
    tc5::mbar_init(mb_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    *abort = 0;
  }
  if (warp == 0) tc5::alloc(tslot, FT_TMEM);
  tc5::fence_before();
  __syncthreads();
  tc5::fence_after();
  const uint32_t tbase = *tslot;

  if (tid == 0 && m > 0) {
    tc5::mbar_expect_tx(mb_load, FT_UTILE + FT_VTILE);
    tc5::bulk_copy(sU, Ud + (size_t)blockIdx.x * (FT_UTILE / 2), FT_UTILE, mb_load);
    tc5::bulk_copy(sV, Vd + (size_t)blockIdx.y * (FT_VTILE / 2), FT_VTILE, mb_load);
  }
  const int q4 = warp & 3, ib = i0 + 16 * (warp >> 2);
  const int j = j0 + 32 * q4 + lane;
  const bool jok = j < N;
  // the first 8 rows of this thread's column, read while the copies and MMAs run
  double gv[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) gv[c] = (jok && ib + c < N) ? G[(size_t)(ib + c) * N + j] : 0.0;

  bool issued = false;
  if (tid == 0 && m > 0) {
    if (tc5::mbar_sleep_wait(mb_load, 0, abort)) {
      issued = true;
      tc5::fence_after();
      const int nh = m > 16 ? 2 : 1;  // K halves holding accepted flips
#pragma unroll 1
      for (int l = 2; l <= FT_LMAX; ++l) {
        uint32_t acc = 0;
#pragma unroll 1
        for (int p = 1; p < l; ++p) {
          const int q = l - p;
          if (p > FT_ND || q > FT_ND) continue;
          for (int h = 0; h < nh; ++h) {
            tc5::mma(tbase + (uint32_t)((l - 2) * FT_N), tc5::desc(sU + ((p - 1) * 2 + h) * FT_USLAB),
                     tc5::desc(sV + ((q - 1) * 2 + h) * FT_VSLAB), FT_IDESC, acc);
            acc = 1;
          }
        }
      }
      tc5::commit(mb_mma);
      tc5::mbar_sleep_wait(mb_mma, 0, abort);
      tc5::fence_before();
    }
  }
  // the other threads sleep in the barrier while the one thread waits for the MMAs
  __syncthreads();
  if (!*abort) {
    tc5::fence_after();
    const uint32_t trow = tbase + ((uint32_t)(32 * q4) << 16) + (uint32_t)(ib - i0);
    const int sj = (jok ? eU[j] : 0) - 54;
    // the tiles that hold rows or columns of the next block also gather them
    const bool cta_gather = a.nkb > 0 && ((i0 < a.ns0 + a.nkb && i0 + FT_N > a.ns0) ||
                                          (j0 < a.ns0 + FT_K && j0 + FT_M > a.ns0));
    double *gp = G + (size_t)ib * N + j;
#pragma unroll
    for (int c0 = 0; c0 < 16; c0 += 8) {
      float v[FT_LMAX - 1][8];
      if (m > 0) {
#pragma unroll
        for (int l = 0; l < FT_LMAX - 1; ++l) tc5::ld8(trow + (uint32_t)(l * FT_N + c0), v[l]);
      }
      int se[8];
      double gn[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        se[c] = (ib + c0 + c < N) ? eV[ib + c0 + c] : 0;
        if (c0 == 0) gn[c] = (jok && ib + 8 + c < N) ? G[(size_t)(ib + 8 + c) * N + j] : 0.0;
      }
      if (m > 0) tc5::wait_ld();
      const int nr = min(8, N - (ib + c0));  // rows of this chunk inside G
      if (jok && m > 0) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          if (c < nr) {
            gv[c] -= level_update(v, c, sj + se[c]);
            gp[(size_t)(c0 + c) * N] = gv[c];
          }
        }
      }
      if (cta_gather && jok) {
        const bool gcol = j >= a.ns0 && j < a.ns0 + FT_K;
        const int jt = j - a.ns0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int i = ib + c0 + c;
          if (c >= nr) continue;
          const int it = i - a.ns0;
          if (it >= 0 && it < a.nkb) Grow_next[(size_t)it * N + j] = gv[c];
          if (gcol) Gcol_next[(size_t)i * FT_K + jt] = (jt < a.nkb) ? gv[c] : 0.0;
        }
      }
      if (c0 == 0) {
#pragma unroll
        for (int c = 0; c < 8; ++c) gv[c] = gn[c];
      }
    }
  }
  tc5::fence_before();
  if (__syncthreads_or(*abort)) {
    // give MMAs already issued a bounded time to finish before the tensor
    // memory goes: a second commit completes the barrier's next phase once
    // they are done
    if (tid == 0) {
      if (issued) {
        volatile int *never = abort + 1;  // a flag nothing sets: the wait runs to its own limit at most
        *never = 0;
        tc5::commit(mb_mma);
        tc5::mbar_sleep_wait(mb_mma, 1, never);
      }
      atomicExch(&g_flush_tc_timeout, 1);
    }
    __syncthreads();
  }
  if (warp == 0) {
    tc5::fence_after();
    tc5::dealloc(tbase, FT_TMEM);
  }
}

cudaError_t launch_flush_tc_prep(const FlushArgs &a, const double *Gcol, const double *Grow, const double *alpha,
                                 const double *beta, const int *acc, void *ws, float2 *Anext, cudaStream_t st,
                                 const int *perm, const double *G, double *gnext) {
  if (a.kb < 1 || a.kb > FT_K || a.nkb > FT_K) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return cudaErrorInvalidValue;
  const int N = a.N;
  const size_t tu = (size_t)(N + FT_M - 1) / FT_M, tv = (size_t)(N + FT_N - 1) / FT_N;
  unsigned short *Ud = static_cast<unsigned short *>(ws);
  unsigned short *Vd = Ud + tu * (FT_UTILE / 2);
  int *eU = reinterpret_cast<int *>(Vd + tv * (FT_VTILE / 2));
  int *eV = eU + N + FT_M;
  DQ_KSCOPE(KF_BLOCKAUX, st);
  add_work(KF_BLOCKAUX, 4.0 * N * (double)FT_K * a.kb, 8.0 * N * (double)(2 * a.kb + 2 * FT_K));
  const int nblk = (N + 7) / 8;
  flush_tc_prep_kernel<<<2 * nblk, 256, 0, st>>>(a, Gcol, alpha, Grow, beta, acc, Ud, Vd, eU, eV, nblk, Anext,
                                                 perm, G, gnext);
  return cudaGetLastError();
}

cudaError_t launch_flush_tc_update(const FlushArgs &a, double *G, const int *acc, void *ws, double *Gcol_next,
                                   double *Grow_next, cudaStream_t st) {
  if (a.kb < 1 || a.kb > FT_K || a.nkb > FT_K) return cudaErrorInvalidValue;
  const int N = a.N;
  const size_t tu = (size_t)(N + FT_M - 1) / FT_M, tv = (size_t)(N + FT_N - 1) / FT_N;
  unsigned short *Ud = static_cast<unsigned short *>(ws);
  unsigned short *Vd = Ud + tu * (FT_UTILE / 2);
  int *eU = reinterpret_cast<int *>(Vd + tv * (FT_VTILE / 2));
  int *eV = eU + N + FT_M;
  DQ_KSCOPE(KF_FLUSH, st);
  add_work(KF_FLUSH, 2.0 * N * (double)N * a.kb, 2.0 * N * (double)N * sizeof(double));
  cudaError_t e = ensure_smem_attr((const void *)flush_tc_kernel, FT_SMEM);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)tu, (unsigned)tv);
  flush_tc_kernel<<<grid, FT_THREADS, FT_SMEM, st>>>(a, G, Ud, Vd, eU, eV, acc, Gcol_next, Grow_next);
  return cudaGetLastError();
}

cudaError_t launch_flush_tc(const FlushArgs &a, double *G, const double *Gcol, const double *Grow,
                            const double *alpha, const double *beta, const int *acc, void *ws,
                            double *Gcol_next, double *Grow_next, cudaStream_t st) {
  cudaError_t e = launch_flush_tc_prep(a, Gcol, Grow, alpha, beta, acc, ws, nullptr, st);
  if (e != cudaSuccess) return e;
  return launch_flush_tc_update(a, G, acc, ws, Gcol_next, Grow_next, st);
}

bool flush_tc_timed_out(cudaStream_t st) {
  int v = 0;
  if (cudaMemcpyFromSymbolAsync(&v, g_flush_tc_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return false;
  if (cudaStreamSynchronize(st) != cudaSuccess) return false;
  return v != 0;
}

}  // namespace dq
