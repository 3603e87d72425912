// Kinetic propagator product e^{scale K} X by the three steps of Eq. 6:
// per vector (a column of X for the left product, a row for the right
// product) and per sublattice, a 2D FFT over the L x L cells, a 3x3 block
// multiply per momentum, and the inverse 2D FFT.
//
// One CTA owns VT vectors. Their N = 3 L^2 values go to shared memory once,
// the five transform passes run there (each thread holds a whole line in
// registers), and the result goes back to HBM once: each launch reads and
// writes every element of X exactly once, the minimum for this product.
//
// Shared layout: complex slot ((a*L + x1)*H + k2)*VT + v, H = L/2 + 1, the
// vector index v fastest so that the VT lanes touching one line position
// hit consecutive banks. Real input sits packed in the same slots before the
// first pass (x2 = 2q, 2q+1 -> real/imag of slot q).
//   P1: along x2, real -> half spectrum (k2 < H)      [lines (a, x1, v)]
//   P2: along x1, forward                              [lines (a, k2, v)]
//   P3: 3x3 block multiply E(k1, k2)                   [items (k1, k2, v)]
//   P4: along x1, inverse                              [lines (a, k2, v)]
//   P5: along x2, half spectrum -> real (Hermitian completion)
#pragma once

#include "fft.cuh"
#include "kernels.cuh"

namespace dq {

// Storage type of the operand in HBM for compute type T: double-float
// (df64) computes on FP64 data, the others store what they compute.
template <typename T> struct PropStore { using type = T; };
template <> struct PropStore<df64> { using type = double; };

template <typename T, typename S> __device__ __forceinline__ T ld_val(S x) {
  if constexpr (std::is_same<T, df64>::value) return df_from(x);
  else return x;
}
template <typename S, typename T> __device__ __forceinline__ S st_val(T x) {
  if constexpr (std::is_same<T, df64>::value) return df_to(x);
  else return x;
}

template <typename T, int L> struct PropCfg {
  static constexpr int H = L / 2 + 1;
  static constexpr int N = 3 * L * L;
  static constexpr int kSlotsPerVec = 3 * L * H;
  static constexpr int kBytesPerVec = kSlotsPerVec * (int)sizeof(cpx<T>);
  // vectors per CTA: a power of two up to 16 (f32) / 8 (f64) that keeps the
  // tile within ~100 KB so that two CTAs fit on an SM
  static constexpr int vt_cap() {
    int v = sizeof(T) == 4 ? 16 : 8;
    while (v > 1 && v * kBytesPerVec > 100 * 1024) v >>= 1;
    return v;
  }
  static constexpr int VT = vt_cap();
  static constexpr int kSmem = VT * kBytesPerVec;
  static constexpr int kThreads = 256;
};

template <typename T, int L, int SIDE>
__global__ void __launch_bounds__(256)
    prop_kernel(const typename PropStore<T>::type *__restrict__ X,
                typename PropStore<T>::type *__restrict__ Y, int nvec, int ld,
                const cpx<T> *__restrict__ E, const typename PropStore<T>::type *__restrict__ pre,
                const typename PropStore<T>::type *__restrict__ post,
                const typename PropStore<T>::type *__restrict__ vscale) {
  using C = PropCfg<T, L>;
  using S = typename PropStore<T>::type;
  constexpr int H = C::H, N = C::N, VT = C::VT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T> *buf = reinterpret_cast<cpx<T> *>(smem_raw);
  T *rbuf = reinterpret_cast<T *>(smem_raw);
  const int v0 = blockIdx.x * VT;
  const int nv = min(VT, nvec - v0);
  const int tid = threadIdx.x;

  // ---- load (with the optional pre scaling along the vector)
  if constexpr (SIDE == 0) {
    for (int w = tid; w < N * VT; w += blockDim.x) {
      const int v = w % VT, i = w / VT;
      T val = T(0);
      if (v < nv) {
        val = ld_val<T, S>(X[(size_t)i * ld + v0 + v]);
        if (pre) val *= ld_val<T, S>(pre[i]);
      }
      const int a = i % 3, cell = i / 3, x2 = cell % L, x1 = cell / L;
      rbuf[2 * (((a * L + x1) * H + (x2 >> 1)) * VT + v) + (x2 & 1)] = val;
    }
  } else {
    for (int w = tid; w < N * VT; w += blockDim.x) {
      const int j = w % N, v = w / N;
      T val = T(0);
      if (v < nv) {
        val = ld_val<T, S>(X[(size_t)(v0 + v) * ld + j]);
        if (pre) val *= ld_val<T, S>(pre[j]);
      }
      const int a = j % 3, cell = j / 3, x2 = cell % L, x1 = cell / L;
      rbuf[2 * (((a * L + x1) * H + (x2 >> 1)) * VT + v) + (x2 & 1)] = val;
    }
  }
  __syncthreads();

  // ---- P1: along x2, real -> half spectrum
  for (int w = tid; w < 3 * L * VT; w += blockDim.x) {
    const int v = w % VT, line = w / VT;
    cpx<T> *p = buf + (size_t)line * H * VT + v;
    T re[L], im[L];
#pragma unroll
    for (int q = 0; q < (L + 1) / 2; ++q) {
      const cpx<T> z = p[q * VT];
      re[2 * q] = z.x;
      if (2 * q + 1 < L) re[2 * q + 1] = z.y;
    }
#pragma unroll
    for (int x = 0; x < L; ++x) im[x] = T(0);
    RegFFT<T, L, -1>::run(re, im);
#pragma unroll
    for (int k = 0; k < H; ++k) p[k * VT] = mkc(re[k], im[k]);
  }
  __syncthreads();

  // ---- P2: along x1, forward
  for (int w = tid; w < 3 * H * VT; w += blockDim.x) {
    const int v = w % VT, r = w / VT;
    const int a = r / H, k2 = r % H;
    cpx<T> *p = buf + ((size_t)a * L * H + k2) * VT + v;
    T re[L], im[L];
#pragma unroll
    for (int x = 0; x < L; ++x) {
      const cpx<T> z = p[x * H * VT];
      re[x] = z.x;
      im[x] = z.y;
    }
    RegFFT<T, L, -1>::run(re, im);
#pragma unroll
    for (int x = 0; x < L; ++x) p[x * H * VT] = mkc(re[x], im[x]);
  }
  __syncthreads();

  // ---- P3: per-momentum 3x3 block
  for (int w = tid; w < L * H * VT; w += blockDim.x) {
    const int v = w % VT, kk = w / VT;
    const cpx<T> *e = E + kk * 9;
    cpx<T> in[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) in[a] = buf[((size_t)a * L * H + kk) * VT + v];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T sr = T(0), si = T(0);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const cpx<T> m = e[a * 3 + b];
        sr += m.x * in[b].x - m.y * in[b].y;
        si += m.x * in[b].y + m.y * in[b].x;
      }
      buf[((size_t)a * L * H + kk) * VT + v] = mkc(sr, si);
    }
  }
  __syncthreads();

  // ---- P4: along x1, inverse
  for (int w = tid; w < 3 * H * VT; w += blockDim.x) {
    const int v = w % VT, r = w / VT;
    const int a = r / H, k2 = r % H;
    cpx<T> *p = buf + ((size_t)a * L * H + k2) * VT + v;
    T re[L], im[L];
#pragma unroll
    for (int x = 0; x < L; ++x) {
      const cpx<T> z = p[x * H * VT];
      re[x] = z.x;
      im[x] = z.y;
    }
    RegFFT<T, L, +1>::run(re, im);
#pragma unroll
    for (int x = 0; x < L; ++x) p[x * H * VT] = mkc(re[x], im[x]);
  }
  __syncthreads();

  // ---- P5: along x2, half spectrum -> real
  for (int w = tid; w < 3 * L * VT; w += blockDim.x) {
    const int v = w % VT, line = w / VT;
    cpx<T> *p = buf + (size_t)line * H * VT + v;
    T re[L], im[L];
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const cpx<T> z = p[k * VT];
      re[k] = z.x;
      im[k] = z.y;
    }
#pragma unroll
    for (int k = H; k < L; ++k) {
      re[k] = re[L - k];
      im[k] = -im[L - k];
    }
    RegFFT<T, L, +1>::run(re, im);
#pragma unroll
    for (int q = 0; q < (L + 1) / 2; ++q)
      p[q * VT] = mkc(re[2 * q], (2 * q + 1 < L) ? re[2 * q + 1] : T(0));
  }
  __syncthreads();

  // ---- store (with post scaling along the vector and the per-vector scale)
  if constexpr (SIDE == 0) {
    for (int w = tid; w < N * VT; w += blockDim.x) {
      const int v = w % VT, i = w / VT;
      if (v >= nv) continue;
      const int a = i % 3, cell = i / 3, x2 = cell % L, x1 = cell / L;
      T val = rbuf[2 * (((a * L + x1) * H + (x2 >> 1)) * VT + v) + (x2 & 1)];
      if (post) val *= ld_val<T, S>(post[i]);
      if (vscale) val *= ld_val<T, S>(vscale[v0 + v]);
      Y[(size_t)i * ld + v0 + v] = st_val<S, T>(val);
    }
  } else {
    for (int w = tid; w < N * VT; w += blockDim.x) {
      const int j = w % N, v = w / N;
      if (v >= nv) continue;
      const int a = j % 3, cell = j / 3, x2 = cell % L, x1 = cell / L;
      T val = rbuf[2 * (((a * L + x1) * H + (x2 >> 1)) * VT + v) + (x2 & 1)];
      if (post) val *= ld_val<T, S>(post[j]);
      if (vscale) val *= ld_val<T, S>(vscale[v0 + v]);
      Y[(size_t)(v0 + v) * ld + j] = st_val<S, T>(val);
    }
  }
}

// Host launcher for one L (templated) -- returns cudaError_t of the launch.
template <typename T, int L>
cudaError_t launch_prop_L(int side, const typename PropStore<T>::type *X,
                          typename PropStore<T>::type *Y, int nvec, int ld, const cpx<T> *E,
                          const typename PropStore<T>::type *pre,
                          const typename PropStore<T>::type *post,
                          const typename PropStore<T>::type *vscale, cudaStream_t st) {
  using C = PropCfg<T, L>;
  const int grid = (nvec + C::VT - 1) / C::VT;
  if (grid == 0) return cudaSuccess;
  DQ_KSCOPE(KF_PROP, st);
  // one read and one write of the N x nvec operand; flops per vector
  // 15 L^2 log2(L^2) + 36 L^2 (real-input FFTs both ways plus the 3x3 blocks)
  {
    const double L2 = (double)L * L;
    const double lg = L > 1 ? std::log2(L2) : 0.0;
    add_work(KF_PROP, (15.0 * L2 * lg + 36.0 * L2) * nvec,
             2.0 * C::N * (double)nvec * sizeof(typename PropStore<T>::type));
  }
  if (side == 0) {
    cudaError_t e = ensure_smem_attr((const void *)prop_kernel<T, L, 0>, C::kSmem);
    if (e != cudaSuccess) return e;
    prop_kernel<T, L, 0><<<grid, C::kThreads, C::kSmem, st>>>(X, Y, nvec, ld, E, pre, post, vscale);
  } else {
    cudaError_t e = ensure_smem_attr((const void *)prop_kernel<T, L, 1>, C::kSmem);
    if (e != cudaSuccess) return e;
    prop_kernel<T, L, 1><<<grid, C::kThreads, C::kSmem, st>>>(X, Y, nvec, ld, E, pre, post, vscale);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prop(int L, int side, const typename PropStore<T>::type *X,
                        typename PropStore<T>::type *Y, int nvec, int ld, const cpx<T> *E,
                        const typename PropStore<T>::type *pre,
                        const typename PropStore<T>::type *post,
                        const typename PropStore<T>::type *vscale, cudaStream_t st) {
  switch (L) {
#define DQ_PROP_CASE(LL) \
  case LL: return launch_prop_L<T, LL>(side, X, Y, nvec, ld, E, pre, post, vscale, st);
    DQ_PROP_CASE(1)
    DQ_PROP_CASE(2)
    DQ_PROP_CASE(3)
    DQ_PROP_CASE(4)
    DQ_PROP_CASE(6)
    DQ_PROP_CASE(8)
    DQ_PROP_CASE(12)
    DQ_PROP_CASE(16)
    DQ_PROP_CASE(24)
    DQ_PROP_CASE(36)
#undef DQ_PROP_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dq
