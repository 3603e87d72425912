// FP64-accurate GEMM on the bf16 tensor cores by exact slicing (the
// error-free splitting of Ozaki, Ogita, Oishi and Rump, 2012).
//
// op(A) (M x K) and op(B) (K x N) are scaled per row / per column by powers of
// two, E_i and F_j, so that every entry lies in (-1, 1), and each entry is cut
// into 9 signed 7-bit digits:  a = 2^E_i sum_{p=1..9} a_p 2^{-7p} (+ a tail
// below 2^-63), a_p integers in [-127, 127], exactly representable in bf16.
// Then
//     (op(A) op(B))_ij = 2^{E_i+F_j} sum_{p,q} 2^{-7(p+q)} sum_k a_p[i,k] b_q[k,j],
// keeping the 45 digit pairs with p + q <= 10 (the dropped ones, and the
// truncated tails, weigh less than about K 2^-63 max|row| max|column|: FP64
// rounding level for K up to a few thousand). Each inner sum over a K-chunk
// of 64 is a sum of products of 7-bit integers, < 9 * 64 * 127^2 < 2^24 per
// level, so the bf16 tensor-core MMA with FP32 accumulation computes it
// exactly. Levels l = p + q in 2..7 fold into one exact int64 accumulator
// (weights 2^{7(7-l)}), levels 8..10 into an FP32 accumulator; the FP64
// result is formed once per output.
//
// Tensor paths: warp-level mma.sync m16n8k16 bf16 for every shape, and for
// products with M, N, K >= 256 a tcgen05 kernel (tensor-memory accumulators,
// bulk-copy staging) further down.
#include <cuda_bf16.h>
#include <stdint.h>

#include "kernels.cuh"
#include "linalg.cuh"
#include "tc05.cuh"

namespace dq {

constexpr int OZ_S = 9;       // digits per value (63 bits)
constexpr int OZ_KC = 64;      // K chunk
constexpr int OZ_BM = 64, OZ_BN = 64;

// exponent field (biased) of |x|; 0 for zero / subnormal
__device__ __forceinline__ int exp_field(double x) {
  return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ff);
}

// One operand of the slicing: the vectors are the rows of op(A) / the columns
// of op(B); `vec_is_row` says whether the storage row index or the storage
// column index is the vector index.
struct OzOperand {
  const double *X;
  int rows, cols, ld, vec_is_row;
  int *emax;             // per vector: maximum exponent field
  int nvec, Kp;
  unsigned short *out;   // digit planes [p][v][k], or with `blocked` [p][k / 16][v][k % 16]
  int blocked;
};

// Both slicing passes work on tiles of 32 vectors x 64 positions along K,
// over both operands in one launch (A's tiles first). A tile is read in
// storage order (rows of op(A) are contiguous when !ta, columns of op(B) are
// strided when !tb: either way the reads are coalesced).
constexpr int OZ_TV = 32, OZ_TK = 64;

__device__ __forceinline__ int oz_tiles(const OzOperand &o) {
  return ((o.nvec + OZ_TV - 1) / OZ_TV) * (o.Kp / OZ_TK);
}

// x of element (v, k) of the tile, in shared memory tile[v][k]
__device__ __forceinline__ void oz_load_tile(const OzOperand &o, int v0, int k0, double (*tile)[OZ_TK + 1]) {
  const int K = o.vec_is_row ? o.cols : o.rows;
  for (int e = threadIdx.x; e < OZ_TV * OZ_TK; e += blockDim.x) {
    int v, k;
    if (o.vec_is_row) {
      v = e / OZ_TK;
      k = e % OZ_TK;
    } else {
      k = e / OZ_TV;
      v = e % OZ_TV;
    }
    double x = 0.0;
    if (v0 + v < o.nvec && k0 + k < K)
      x = o.vec_is_row ? o.X[(size_t)(v0 + v) * o.ld + k0 + k] : o.X[(size_t)(k0 + k) * o.ld + v0 + v];
    tile[v][k] = x;
  }
}

// Maximum exponent field per vector (emax must start at 0).
__global__ void __launch_bounds__(256) oz_maxexp_kernel(OzOperand a, OzOperand b) {
  __shared__ double tile[OZ_TV][OZ_TK + 1];
  __shared__ int mx[OZ_TV];
  const int ta = oz_tiles(a);
  const bool isa = (int)blockIdx.x < ta;
  const OzOperand &o = isa ? a : b;
  const int t = isa ? blockIdx.x : blockIdx.x - ta;
  const int ktiles = o.Kp / OZ_TK;
  const int v0 = (t / ktiles) * OZ_TV, k0 = (t % ktiles) * OZ_TK;
  if (threadIdx.x < OZ_TV) mx[threadIdx.x] = 0;
  oz_load_tile(o, v0, k0, tile);
  __syncthreads();
  // 8 threads per vector, 8 positions each
  const int v = threadIdx.x / 8, part = threadIdx.x % 8;
  int m = 0;
#pragma unroll
  for (int q = 0; q < OZ_TK / 8; ++q) m = max(m, exp_field(tile[v][part * (OZ_TK / 8) + q]));
  atomicMax(&mx[v], m);
  __syncthreads();
  if (threadIdx.x < OZ_TV && v0 + threadIdx.x < o.nvec && mx[threadIdx.x] > 0)
    atomicMax(&o.emax[v0 + threadIdx.x], mx[threadIdx.x]);
}

__device__ __forceinline__ unsigned short int_to_bf16_bits(int d) {
  if (d == 0) return 0;
  const unsigned int s = d < 0 ? 0x8000u : 0u;
  const unsigned int a = (unsigned int)(d < 0 ? -d : d);   // 1..127
  const int msb = 31 - __clz(a);                             // 0..6
  const unsigned int mant = (a << (7 - msb)) & 0x7f;         // 7 mantissa bits, exact
  return (unsigned short)(s | ((unsigned int)(msb + 127) << 7) | mant);
}

// Digits of element (v, k) of the vectors, written to out[p][v][k] (bf16, row
// length Kp, zero padded); the vector's exponent is emax[v]. Integer
// operations only; the tile is staged in shared memory and the planes are
// written along k (coalesced).
__global__ void __launch_bounds__(256) oz_slice_kernel(OzOperand a, OzOperand b) {
  __shared__ double tile[OZ_TV][OZ_TK + 1];
  const int ta = oz_tiles(a);
  const bool isa = (int)blockIdx.x < ta;
  const OzOperand &o = isa ? a : b;
  const int t = isa ? blockIdx.x : blockIdx.x - ta;
  const int ktiles = o.Kp / OZ_TK;
  const int v0 = (t / ktiles) * OZ_TV, k0 = (t % ktiles) * OZ_TK;
  oz_load_tile(o, v0, k0, tile);
  __syncthreads();
  const size_t plane = (size_t)o.nvec * o.Kp;
  for (int e = threadIdx.x; e < OZ_TV * OZ_TK; e += blockDim.x) {
    const int v = e / OZ_TK, k = e % OZ_TK;
    if (v0 + v >= o.nvec) continue;
    const double x = tile[v][k];
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int ef = (int)((bits >> 52) & 0x7ff);
    unsigned long long F = 0;
    if (ef != 0 && ef != 0x7ff) {
      const unsigned long long m53 = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
      // |x| / 2^{E} with E = emax - 1022 as a fixed-point number with 7 S = 63
      // fraction bits (m53 < 2^53, shift <= 10)
      const int sh = ef - o.emax[v0 + v] + (7 * OZ_S - 53);
      F = sh >= 0 ? (m53 << sh) : (sh > -64 ? (m53 >> (-sh)) : 0ull);
    }
    const int neg = (int)(bits >> 63);
    const int kk = k0 + k, vv = v0 + v;
    // blocked: [p][k / 16][v][16] with the two 8-position halves of a row
    // swapped on rows 4..7 of every 8 (the 32-byte swizzle the tcgen05 kernel's
    // descriptors expect, so that one bulk copy per plane lands ready)
    unsigned short *dst = o.blocked
                              ? o.out + ((size_t)(kk >> 4) * o.nvec + vv) * 16 +
                                    ((((kk & 15) >> 3) ^ ((vv >> 2) & 1)) << 3) + (kk & 7)
                              : o.out + (size_t)vv * o.Kp + kk;
#pragma unroll
    for (int p = 1; p <= OZ_S; ++p) {
      int d = (int)((F >> (7 * OZ_S - 7 * p)) & 127ull);
      if (neg) d = -d;
      dst[(size_t)(p - 1) * plane] = int_to_bf16_bits(d);
    }
  }
}

__device__ __forceinline__ void ldmatrix_x4(unsigned (&r)[4], const void *p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// C = alpha diag(rs) (op(A) op(B)) diag(cs) + beta C from the digit planes.
// CTA tile 64 x 64, 8 warps (warp tile 16 x 32 = 4 MMA n-tiles). The 9 digit
// planes of the A and B tiles are staged in shared memory 32 positions of K
// at a time, double-buffered with cp.async: the next sub-chunk is in flight
// while the MMAs of the current one run. Register blocking: per 16-wide k
// step a warp loads the fragments of all 9 A planes once (36 registers) and,
// plane by plane, the B fragments of its 4 n-tiles; every digit pair (p, q)
// with p + q <= 10 is one MMA into the accumulator of its level l = p + q
// (9 levels x 16 FP32 live), 0.15 ldmatrix per MMA. After every 64 positions
// of K the exact level sums are folded: levels 2..7 into an int64
// accumulator (weight 2^{7(7-l)}), 8..10 into FP32; the epilogue forms
// (I + F) 2^{-49} 2^{E_i + F_j} once per output (split K: partial products, summed in order).
constexpr int OZ_SC = 32;           // staging sub-chunk of K
constexpr int OZ_LDS = OZ_SC + 8;   // padded smem row (bf16): 80 B, conflict-free ldmatrix
constexpr int OZ_BUF = OZ_S * (OZ_BM + OZ_BN) * OZ_LDS;  // one buffer, bf16 elements

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// Planes p of rows m0.. of A and n0.. of B, positions k0..k0+31, into buffer
// sbuf ([A: p][64][OZ_LDS], then [B: q][64][OZ_LDS]); rows beyond M / N are
// zero. Every global address is 16-byte aligned (Kp and k0 multiples of 32,
// 8 bf16 per copy) and so is every shared one (80-byte rows).
__device__ __forceinline__ void oz_stage(unsigned short *sbuf, const unsigned short *Ad,
                                         const unsigned short *Bd, int M, int N, int Kp, int m0,
                                         int n0, int k0, size_t aplane, size_t bplane) {
  unsigned short *As = sbuf, *Bs = sbuf + OZ_S * OZ_BM * OZ_LDS;
  for (int e = threadIdx.x; e < OZ_S * OZ_BM * (OZ_SC / 8); e += blockDim.x) {
    const int p = e / (OZ_BM * (OZ_SC / 8));
    const int rem = e % (OZ_BM * (OZ_SC / 8));
    const int r = rem / (OZ_SC / 8), c8 = rem % (OZ_SC / 8);
    unsigned short *da = As + (p * OZ_BM + r) * OZ_LDS + c8 * 8;
    unsigned short *db = Bs + (p * OZ_BN + r) * OZ_LDS + c8 * 8;
    if (m0 + r < M)
      cp_async16(da, Ad + p * aplane + (size_t)(m0 + r) * Kp + k0 + c8 * 8);
    else
      *reinterpret_cast<uint4 *>(da) = make_uint4(0, 0, 0, 0);
    if (n0 + r < N)
      cp_async16(db, Bd + p * bplane + (size_t)(n0 + r) * Kp + k0 + c8 * 8);
    else
      *reinterpret_cast<uint4 *>(db) = make_uint4(0, 0, 0, 0);
  }
}

__global__ void __launch_bounds__(256)
    oz_gemm_rb_kernel(int M, int N, int Kp, const unsigned short *__restrict__ Ad,
                      const unsigned short *__restrict__ Bd, const int *__restrict__ ea,
                      const int *__restrict__ eb, double alpha, double beta, double *__restrict__ C,
                      int ldc, const double *__restrict__ rs, const double *__restrict__ cs,
                      int kchunks, double *__restrict__ part) {
  extern __shared__ __align__(16) unsigned short osm[];  // two buffers of OZ_BUF
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;               // 4 x 2 warps
  const int m0 = blockIdx.y * OZ_BM, n0 = blockIdx.x * OZ_BN;
  const size_t aplane = (size_t)M * Kp, bplane = (size_t)N * Kp;

  long long I[4][4];
  float F[4][4];
#pragma unroll
  for (int t = 0; t < 4; ++t)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      I[t][r] = 0;
      F[t][r] = 0.f;
    }
  float acc[OZ_S][4][4];  // level l = p + q at index l - 2

  // split K: this CTA takes chunks [z * kchunks, (z + 1) * kchunks) of 64
  const int kbeg = blockIdx.z * kchunks * OZ_KC;
  const int kend = min(Kp, kbeg + kchunks * OZ_KC);
  const int nsub = (kend - kbeg) / OZ_SC;  // even: Kp is a multiple of 64
  if (nsub > 0) oz_stage(osm, Ad, Bd, M, N, Kp, m0, n0, kbeg, aplane, bplane);
  cp_async_commit();
  for (int it = 0; it < nsub; ++it) {
    if (it + 1 < nsub) {
      oz_stage(osm + ((it + 1) & 1) * OZ_BUF, Ad, Bd, M, N, Kp, m0, n0, kbeg + (it + 1) * OZ_SC,
               aplane, bplane);
      cp_async_commit();
      cp_async_wait_one();
    } else {
      cp_async_wait_all();
    }
    __syncthreads();
    const unsigned short *As = osm + (it & 1) * OZ_BUF;
    const unsigned short *Bs = As + OZ_S * OZ_BM * OZ_LDS;
    if ((it & 1) == 0) {
#pragma unroll
      for (int l = 0; l < OZ_S; ++l)
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
          for (int r = 0; r < 4; ++r) acc[l][t][r] = 0.f;
    }
#pragma unroll 1
    for (int ks = 0; ks < OZ_SC; ks += 16) {
      unsigned a[OZ_S][4];
#pragma unroll
      for (int p = 0; p < OZ_S; ++p)
        ldmatrix_x4(a[p], As + ((p * OZ_BM) + wm * 16 + (lane & 15)) * OZ_LDS + ks + (lane >> 4) * 8);
#pragma unroll
      for (int q = 0; q < OZ_S; ++q) {
        unsigned b[2][4];
#pragma unroll
        for (int t2 = 0; t2 < 2; ++t2) {
          const int nrow = t2 * 16 + ((lane >> 4) << 3) + (lane & 7);
          const int kof = ((lane >> 3) & 1) * 8;
          ldmatrix_x4(b[t2], Bs + ((q * OZ_BN) + wn * 32 + nrow) * OZ_LDS + ks + kof);
        }
#pragma unroll
        for (int p = 0; p + q <= OZ_S - 1; ++p) {  // digit indices p+1, q+1: level p + q + 2 <= OZ_S + 1
#pragma unroll
          for (int t2 = 0; t2 < 2; ++t2) {
            mma_bf16(acc[p + q][2 * t2], a[p], b[t2][0], b[t2][1]);
            mma_bf16(acc[p + q][2 * t2 + 1], a[p], b[t2][2], b[t2][3]);
          }
        }
      }
    }
    if (it & 1) {
      // fold the exact level sums of 64 positions (level l = idx + 2): 2..7 into
      // int64 with weight 2^{7(7-l)}, 8..10 into FP32 with weight 2^{-7(l-7)}
#pragma unroll
      for (int idx = 0; idx < OZ_S; ++idx) {
        const int l = idx + 2;
        if (l <= 7) {
          const int shift = 7 * (7 - l);
#pragma unroll
          for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int r = 0; r < 4; ++r) I[t][r] += ((long long)__float2int_rn(acc[idx][t][r])) << shift;
        } else {
          const float w = __int_as_float((127 - 7 * (l - 7)) << 23);
#pragma unroll
          for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int r = 0; r < 4; ++r) F[t][r] = fmaf(acc[idx][t][r], w, F[t][r]);
        }
      }
    }
    // the buffer just read is the target of the next iteration's prefetch
    __syncthreads();
  }
  const int g = lane >> 2, c2 = (lane & 3) * 2;
#pragma unroll
  for (int t = 0; t < 4; ++t)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = m0 + wm * 16 + g + ((r >> 1) << 3);
      const int j = n0 + wn * 32 + t * 8 + c2 + (r & 1);
      if (i >= M || j >= N) continue;
      const double dot = ((double)I[t][r] + (double)F[t][r]);
      const int e2 = (ea[i] - 1022) + (eb[j] - 1022) - 49;
      double v = ldexp(dot, e2) * alpha;
      if (rs) v *= rs[i];
      if (cs) v *= cs[j];
      double *cp = C + (size_t)i * ldc + j;
      if (part)
        part[((size_t)blockIdx.z * M + i) * N + j] = v;
      else
        *cp = (beta != 0.0) ? v + beta * (*cp) : v;
    }
}

// ====================================================================== tcgen05 path
// The same digit-slice product on the 5th-generation tensor cores: bf16
// tcgen05.mma (kind::f16, FP32 accumulate) with the accumulators in tensor
// memory, fed from the digit planes the slicing kernel wrote.
//
// CTA tile 128 x 48 (M x N), 192 threads, K in stages of 16 positions, four
// stage buffers in shared memory: the 9 planes of the A tile (128 x 16 bf16)
// and of the B tile (48 x 16), K-major with 32-byte rows in the 32-byte
// swizzle (8-row groups of 256 B: stride byte offset 256). The slicing kernel
// writes the planes blocked by 16 positions of K and already swizzled, so a
// plane's rows of one stage are one contiguous run that a single bulk copy
// (cp.async.bulk, completing on the slot's mbarrier by byte count) moves.
// One thread issues the copies up to four stages ahead; another issues the
// 45 MMAs of a stage (digit pairs p + q <= 10) as soon as its copies have
// landed; a slot is refilled once the MMAs that read it have completed
// (tcgen05.commit on one mbarrier per slot).
// Tensor memory: 512 columns; level l = p + q (2..10) accumulates in columns
// 48 (l - 2) .. 48 (l - 2) + 47, lane = output row. Every 128 positions of K
// (eight stages) the sums of levels 2..6 are exact integers below 2^24 (a
// level has at most 5 digit pairs: 5 * 128 * 127^2 < 2^24); the four fold
// warps wait for the MMAs, load their rows of those levels (tcgen05.ld
// 32x32b: warp w reads lanes 32 w .. 32 w + 31) and fold them into an exact
// int64 accumulator
// (weights 2^{7(6-l)}); the next period's first MMA of each of these levels
// overwrites (enable-input-d false). Levels 7..10 keep accumulating in FP32
// over the whole K (their rounding stays below 2^-53 of the level-2 sum) and
// are read once. Measured on this part: an M128 x N48 x K16 bf16 MMA issues
// every 46 cycles (N = 256: 128 cycles, 2.4 PFLOP/s over the 152 SMs).
//
// Every wait on an mbarrier is bounded; a wait that gives up sets a device
// flag (read by oz_tc_timed_out) and the CTA stops issuing work, drains its
// copies, frees its tensor memory and returns.
constexpr int TC_BM = 128, TC_BN = 48, TC_BK = 16, TC_NS = 4;
constexpr int TC_A_PLANE = TC_BM * TC_BK * 2, TC_B_PLANE = TC_BN * TC_BK * 2;
constexpr int TC_DIG = OZ_S * (TC_A_PLANE + TC_B_PLANE);                 // 50688 B per stage
constexpr int TC_SMEM = TC_NS * TC_DIG + 128;                            // + mbarriers, TMEM address, abort flag
constexpr int TC_TMEM_COLS = 512;
constexpr uint32_t TC_IDESC = tc5::idesc_bf16(TC_BM, TC_BN);
constexpr int TC_FOLD = 8;  // stages per fold of the exact levels (128 positions)

__device__ int g_oz_tc_timeout = 0;

// Stage `st` (positions k0 .. k0 + 15) of the digit planes into slot b by one
// thread: per plane, the 128 rows of the A tile and the 48 of the B tile are
// contiguous 32-byte rows of the blocked plane layout (already in the 32-byte
// swizzle), two bulk copies (cp.async.bulk) completing on the slot's mbarrier
// with the byte count. Rows beyond M / N are not copied: the slot keeps stale
// rows there, which feed only output rows / columns that are never stored.
__device__ __forceinline__ uint32_t tc_stage_bytes(int M, int N, int m0, int n0) {
  const int ra = min(TC_BM, M - m0), rb = min(TC_BN, N - n0);
  return (uint32_t)(OZ_S * (ra + rb) * 32);
}
__device__ __forceinline__ void tc_stage_bulk(uint32_t sdig, int b, uint32_t mbar, const unsigned short *Ad,
                                              const unsigned short *Bd, int M, int N, int m0, int n0, int k0,
                                              size_t aplane, size_t bplane) {
  const int ra = min(TC_BM, M - m0), rb = min(TC_BN, N - n0);
  const uint32_t stage = sdig + b * TC_DIG;
  const size_t kb = (size_t)(k0 >> 4);
  tc5::mbar_expect_tx(mbar, tc_stage_bytes(M, N, m0, n0));
#pragma unroll 1
  for (int p = 0; p < OZ_S; ++p) {
    tc5::bulk_copy(stage + p * TC_A_PLANE, Ad + p * aplane + (kb * M + m0) * 16, (uint32_t)ra * 32, mbar);
    tc5::bulk_copy(stage + OZ_S * TC_A_PLANE + p * TC_B_PLANE, Bd + p * bplane + (kb * N + n0) * 16, (uint32_t)rb * 32,
              mbar);
  }
}

// Warp roles (192 threads): warps 0-3 fold and write the output (TMEM lane
// quarters 0-3), warp 4 lane 0 issues the MMAs, warp 5 lane 0 the bulk
// copies. They hand over through mbarriers only, never a CTA-wide barrier
// inside the K loop, so the MMA thread (which blocks while the tensor pipe's
// queue is full) never holds up the copies:
//   full[b]  (expect_tx)      the bulk copies of the stage in slot b landed
//   empty[b] (tcgen05.commit) the MMAs that read slot b completed
//   acc      (tcgen05.commit) the MMAs up to a fold point completed
//   freed    (4 arrivals)     one per fold warp, after its tensor-memory loads
constexpr int TC_THREADS = 192;
constexpr int TC_COPY0 = 160;  // the copy thread (warp 5, lane 0)

__global__ void __launch_bounds__(TC_THREADS, 1)
    oz_gemm_tc_kernel(int M, int N, int Kp, const unsigned short *__restrict__ Ad,
                      const unsigned short *__restrict__ Bd, const int *__restrict__ ea,
                      const int *__restrict__ eb, double alpha, double beta, double *__restrict__ C,
                      int ldc, const double *__restrict__ rs, const double *__restrict__ cs,
                      int kstages, double *__restrict__ part) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * TC_BN;
  const size_t aplane = (size_t)M * Kp, bplane = (size_t)N * Kp;
  const uint32_t sdig = tc5::smem_u32(tsm);
  // mbarriers: full[4], empty[4], acc, freed; then the TMEM address and the abort flag
  unsigned char *ctl = tsm + TC_NS * TC_DIG;
  const uint32_t mb = tc5::smem_u32(ctl);
  const uint32_t mb_full = mb, mb_empty = mb + 8 * TC_NS, mb_acc = mb + 16 * TC_NS, mb_freed = mb_acc + 8;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(ctl + 16 * TC_NS + 16);
  volatile int *abort = reinterpret_cast<volatile int *>(ctl + 16 * TC_NS + 20);

  if (tid == 0) {
    for (int bb = 0; bb < TC_NS; ++bb) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb_full + 8 * bb));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb_empty + 8 * bb));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb_acc));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;\n" ::"r"(mb_freed));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    *abort = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tc5::smem_u32(tslot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tbase = *tslot;

  // split K: this CTA takes stages [z kstages, (z + 1) kstages) of 16 positions
  const int sbeg = blockIdx.z * kstages;
  const int nst = max(0, min(Kp / TC_BK, sbeg + kstages) - sbeg);
  const int nfold = (nst + TC_FOLD - 1) / TC_FOLD;

  if (tid == TC_COPY0) {
    // ---- copier: stage st into slot st % 4 once the MMAs of stage st - 4 are done
    for (int st = 0; st < nst; ++st) {
      const int b = st % TC_NS;
      if (st >= TC_NS && !tc5::mbar_wait_or_abort(mb_empty + 8 * b, ((st / TC_NS) - 1) & 1, abort)) break;
      tc_stage_bulk(sdig, b, mb_full + 8 * b, Ad, Bd, M, N, m0, n0, (sbeg + st) * TC_BK, aplane, bplane);
    }
  } else if (tid == 128) {
    // ---- MMA issuer
    for (int st = 0; st < nst; ++st) {
      const int b = st % TC_NS;
      if (!tc5::mbar_wait_or_abort(mb_full + 8 * b, (st / TC_NS) & 1, abort)) break;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint64_t ad0 = tc5::desc(sdig + b * TC_DIG), bd0 = tc5::desc(sdig + b * TC_DIG + OZ_S * TC_A_PLANE);
      // a new fold period overwrites the exact levels: the previous fold must have read them
      const bool restart = (st % TC_FOLD) == 0;
      if (st > 0 && restart) {
        if (!tc5::mbar_wait_or_abort(mb_freed, ((st / TC_FOLD) - 1) & 1, abort)) break;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      }
      // exact levels 2..6 restart every TC_FOLD stages, 7..10 only at the first
#pragma unroll 1
      for (int p = 0; p < OZ_S; ++p)
#pragma unroll 1
        for (int q = 0; p + q <= OZ_S - 1; ++q) {
          const uint32_t accf = (restart && p == 0 && (q <= 4 || st == 0)) ? 0u : 1u;
          tc5::mma(tbase + (uint32_t)((p + q) * TC_BN), ad0 + (uint64_t)((p * TC_A_PLANE) >> 4),
                 bd0 + (uint64_t)((q * TC_B_PLANE) >> 4), TC_IDESC, accf);
        }
      tc5::commit(mb_empty + 8 * b);
      if ((st % TC_FOLD) == TC_FOLD - 1 || st == nst - 1) tc5::commit(mb_acc);
    }
  }

  // ---- folds and output: warps 0-3, lane quarter = warp
  const int i = m0 + warp * 32 + lane;
  if (warp < 4) {
    long long I[TC_BN];
#pragma unroll
    for (int c = 0; c < TC_BN; ++c) I[c] = 0;
    const uint32_t trow = tbase + ((uint32_t)(warp * 32) << 16);
    bool ok = true;
    for (int f = 0; f < nfold && ok; ++f) {
      // lane 0 polls and the warp follows its verdict, so the aligned
      // tensor-memory loads stay warp-uniform
      int okw = lane == 0 ? (int)tc5::mbar_sleep_wait(mb_acc, f & 1, abort) : 0;
      ok = __shfl_sync(0xffffffffu, okw, 0) != 0;
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
      for (int idx = 0; idx < 5; ++idx) {
        const int l = idx + 2;
#pragma unroll
        for (int ch = 0; ch < TC_BN / 16; ++ch) {
          float v[16];
          tc5::ld16(trow + (uint32_t)(idx * TC_BN + ch * 16), v);
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
          for (int c = 0; c < 16; ++c) I[ch * 16 + c] += ((long long)__float2int_rn(v[c])) << (7 * (6 - l));
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) tc5::mbar_arrive(mb_freed);
    }
    // levels 7..10 (weights 2^{-7(l-6)}) are read once, 16 columns at a time
    // (the last fold waited for every MMA), and the outputs formed:
    // (I + F) 2^{-42} 2^{E_i + F_j}
    if (ok && nst > 0) {
      const bool row_ok = i < M;
      const double r = (rs && row_ok) ? rs[i] * alpha : alpha;
#pragma unroll
      for (int ch = 0; ch < TC_BN / 16; ++ch) {
        float F[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) F[c] = 0.f;
#pragma unroll
        for (int idx = 5; idx < OZ_S; ++idx) {
          const float w = __int_as_float((127 - 7 * (idx - 4)) << 23);
          float v[16];
          tc5::ld16(trow + (uint32_t)(idx * TC_BN + ch * 16), v);
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
          for (int c = 0; c < 16; ++c) F[c] = fmaf(v[c], w, F[c]);
        }
        if (row_ok) {
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const int j = n0 + ch * 16 + c;
            if (j >= N) continue;
            const double dot = (double)I[ch * 16 + c] + (double)F[c];
            const int e2 = (ea[i] - 1022) + (eb[j] - 1022) - 42;
            double v = ldexp(dot, e2) * r;
            if (cs) v *= cs[j];
            double *cp = C + (size_t)i * ldc + j;
            if (part)
              part[((size_t)blockIdx.z * M + i) * N + j] = v;
            else
              *cp = (beta != 0.0) ? v + beta * (*cp) : v;
          }
        }
      }
    } else if (!*abort && nst == 0 && i < M) {
      // an empty K range: the product is zero
      for (int c = 0; c < TC_BN; ++c) {
        const int j = n0 + c;
        if (j >= N) break;
        double *cp = C + (size_t)i * ldc + j;
        if (part)
          part[((size_t)blockIdx.z * M + i) * N + j] = 0.0;
        else
          *cp = (beta != 0.0) ? beta * (*cp) : 0.0;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  if (__syncthreads_or(*abort)) {
    // give the MMAs already issued a bounded time to finish before the tensor memory goes
    if (tid == 128) {
      volatile int *never = abort + 1;  // a flag nothing sets: the drain runs to its own limit
      *never = 0;
      tc5::commit(mb_acc);
      tc5::mbar_wait_or_abort(mb_acc, nfold & 1, never);
      atomicExch(&g_oz_tc_timeout, 1);
    }
    __syncthreads();
  }
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tbase), "r"(TC_TMEM_COLS));
  }
}

static thread_local bool t_oz_tc = false, t_oz_tc_force = false;
void set_gemm_oz_tc(bool on, bool force) {
  t_oz_tc = on;
  t_oz_tc_force = on && force;
}

bool oz_tc_timed_out(cudaStream_t st) {
  int v = 0;
  if (cudaMemcpyFromSymbolAsync(&v, g_oz_tc_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return false;
  if (cudaStreamSynchronize(st) != cudaSuccess) return false;
  return v != 0;
}

static thread_local unsigned short *t_ozws = nullptr;
static thread_local size_t t_ozws_bytes = 0;
static thread_local int *t_ozexp = nullptr;
static thread_local size_t t_ozexp_n = 0;
static thread_local bool t_oz = false;

void set_gemm_oz(bool on) { t_oz = on; }
bool gemm_oz() { return t_oz && t_ozws != nullptr; }

void set_oz_workspace(void *ws, size_t bytes, int *exps, size_t nexp) {
  t_ozws = static_cast<unsigned short *>(ws);
  t_ozws_bytes = bytes;
  t_ozexp = exps;
  t_ozexp_n = nexp;
}

size_t oz_workspace_bytes(int M, int N, int K) {
  const size_t Kp = (size_t)((K + OZ_KC - 1) / OZ_KC) * OZ_KC;
  return (size_t)OZ_S * ((size_t)M + N) * Kp * sizeof(unsigned short);
}


cudaError_t ozgemm(bool ta, bool tb, int M, int N, int K, double alpha, const double *A, int lda,
                   const double *B, int ldb, double beta, double *C, int ldc, const double *rs,
                   const double *cs, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const int Kp = ((K + OZ_KC - 1) / OZ_KC) * OZ_KC;
  if (oz_workspace_bytes(M, N, K) > t_ozws_bytes || (size_t)(M + N) > t_ozexp_n)
    return cudaErrorInvalidValue;
  unsigned short *Ad = t_ozws, *Bd = t_ozws + (size_t)OZ_S * M * Kp;
  int *ea = t_ozexp, *eb = t_ozexp + M;
  cudaError_t e = cudaMemsetAsync(t_ozexp, 0, (size_t)(M + N) * sizeof(int), st);
  if (e != cudaSuccess) return e;
  // op(A) rows: storage rows when !ta (M x K), storage columns when ta (K x M);
  // op(B) columns: storage columns when !tb (K x N), storage rows when tb (N x K)
  // the tcgen05 kernel reads the planes blocked by 16 positions of K: one
  // stage of one plane is then a contiguous run of 16-position rows
  // tcgen05 tiles are 128 x 48: the skinny products of the QR panels (64
  // rows) run faster on the mma.sync kernel's 64 x 64 tiles
  const bool tc = t_oz_tc && (t_oz_tc_force || (M >= 256 && N >= 256 && K >= 256));
  const OzOperand oa{A, ta ? K : M, ta ? M : K, lda, ta ? 0 : 1, ea, M, Kp, Ad, tc ? 1 : 0};
  const OzOperand ob{B, tb ? N : K, tb ? K : N, ldb, tb ? 1 : 0, eb, N, Kp, Bd, tc ? 1 : 0};
  const int stiles = ((M + OZ_TV - 1) / OZ_TV + (N + OZ_TV - 1) / OZ_TV) * (Kp / OZ_TK);
  {
    DQ_KSCOPE(KF_SLICE, st);
    oz_maxexp_kernel<<<stiles, 256, 0, st>>>(oa, ob);
  }
  {
    DQ_KSCOPE(KF_SLICE, st);
    oz_slice_kernel<<<stiles, 256, 0, st>>>(oa, ob);
  }
  const int BM = tc ? TC_BM : OZ_BM, BN = tc ? TC_BN : OZ_BN;
  const int smem = tc ? TC_SMEM : 2 * OZ_BUF * (int)sizeof(unsigned short);  // two staging buffers
  e = ensure_smem_attr(tc ? (const void *)oz_gemm_tc_kernel : (const void *)oz_gemm_rb_kernel, smem);
  if (e != cudaSuccess) return e;
  // one CTA per SM (shared memory); split K when the tiles do not fill the GPU
  const int tiles = ((N + BN - 1) / BN) * ((M + BM - 1) / BM);
  // K is split in chunks of 64 positions (the tcgen05 kernel counts stages of 16)
  const int nchunks = Kp / OZ_KC;
  int splits = 1;
  if (tiles < 152) {
    splits = (152 + tiles - 1) / tiles;
    const int maxs = (nchunks + 1) / 2;  // at least two chunks per split
    if (splits > maxs) splits = maxs;
    if (splits < 1) splits = 1;
  }
  int kchunks = (nchunks + splits - 1) / splits;
  splits = (nchunks + kchunks - 1) / kchunks;
  double *part = splitk_partials(splits, M, N);
  if (splits > 1 && !part) {
    splits = 1;
    kchunks = nchunks;
  }
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, splits);
  DQ_KSCOPE(KF_GEMM, st);
  add_work(KF_GEMM, 2.0 * M * (double)N * K,
           8.0 * ((double)M * K + (double)K * N + (beta != 0.0 ? 2.0 : 1.0) * (double)M * N));
  if (tc)
    oz_gemm_tc_kernel<<<grid, TC_THREADS, smem, st>>>(M, N, Kp, Ad, Bd, ea, eb, alpha, beta, C, ldc, rs, cs,
                                              kchunks * (OZ_KC / TC_BK), part);
  else
    oz_gemm_rb_kernel<<<grid, 256, smem, st>>>(M, N, Kp, Ad, Bd, ea, eb, alpha, beta, C, ldc, rs, cs,
                                              kchunks, part);
  e = cudaGetLastError();
  if (e != cudaSuccess || !part) return e;
  return splitk_reduce(part, splits, M, N, beta, C, ldc, st);
}

}  // namespace dq
