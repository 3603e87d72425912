// Register-resident mixed-radix FFT of compile-time length L.
//
// Each thread owns one line of L complex values in registers. The transform
// is the Stockham autosort formulation (natural-order output, no bit
// reversal): stage s with radix R reads x[j + r L/R], twiddles by
// W_{Ns R}^{(j mod Ns) r}, applies an R-point DFT and writes
// y[(j / Ns) Ns R + (j mod Ns) + r Ns], Ns being the product of the radices
// already applied. Every loop is unrolled, so all indices and twiddle
// exponents are compile-time constants and the twiddles become constant-bank
// operands of the FMAs.
//
// Twiddles are computed at compile time from their Taylor series after an
// exact octant reduction of the rational angle 2 pi p / q.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "df64.cuh"

namespace dq {

constexpr double kPi = 3.14159265358979323846264338327950288;

constexpr double taylor_sin(double x) {
  double t = x, s = x;
  for (int n = 1; n < 16; ++n) {
    t *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
    s += t;
  }
  return s;
}

constexpr double taylor_cos(double x) {
  double t = 1.0, s = 1.0;
  for (int n = 1; n < 16; ++n) {
    t *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
    s += t;
  }
  return s;
}

struct CosSin {
  double c, s;
};

// cos and sin of 2 pi p / q. The angle is split into an octant o and a
// remainder; the series is only ever evaluated on [0, pi/4].
constexpr CosSin sincos2pi(long p, long q) {
  p %= q;
  if (p < 0) p += q;
  const long P = 8 * p;
  const long o = P / q;
  const long rem = P - o * q;
  double c = 0.0, s = 0.0;
  if ((o & 1) == 0) {
    const double phi = (kPi / 4.0) * (double)rem / (double)q;
    c = taylor_cos(phi);
    s = taylor_sin(phi);
  } else {
    const double psi = (kPi / 4.0) * (double)(q - rem) / (double)q;
    c = taylor_cos(psi);
    s = -taylor_sin(psi);
  }
  const long quarters = ((o & 1) == 0 ? o / 2 : (o + 1) / 2) % 4;
  for (long n = 0; n < quarters; ++n) {
    const double t = c;
    c = -s;
    s = t;
  }
  return CosSin{c, s};
}

// W_L^j = cos(2 pi j / L) + i sin(2 pi j / L), j = 0..L-1.
template <int L> struct TwTable {
  double c[L];
  double s[L];
  float cf[L];
  float sf[L];
  float cl[L];  // cf + cl = c to ~2^-48 (double-float twiddles)
  float sl[L];
  constexpr TwTable() : c(), s(), cf(), sf(), cl(), sl() {
    for (int j = 0; j < L; ++j) {
      const CosSin w = sincos2pi(j, L);
      c[j] = w.c;
      s[j] = w.s;
      cf[j] = (float)w.c;
      sf[j] = (float)w.s;
      cl[j] = (float)(w.c - (double)cf[j]);
      sl[j] = (float)(w.s - (double)sf[j]);
    }
  }
};

template <int L> __constant__ TwTable<L> kTw = TwTable<L>();

template <typename T, int L> struct Tw {
  static __device__ __forceinline__ T c(int e) {
    if constexpr (std::is_same<T, df64>::value) return df64(kTw<L>.cf[e], kTw<L>.cl[e]);
    else if constexpr (sizeof(T) == 8) return kTw<L>.c[e];
    else return kTw<L>.cf[e];
  }
  static __device__ __forceinline__ T s(int e) {
    if constexpr (std::is_same<T, df64>::value) return df64(kTw<L>.sf[e], kTw<L>.sl[e]);
    else if constexpr (sizeof(T) == 8) return kTw<L>.s[e];
    else return kTw<L>.sf[e];
  }
};

__host__ __device__ constexpr int pick_radix(int n) {
  if (n % 4 == 0) return (n % 8 == 0 && (n / 8) % 2 == 1) ? 8 : 4;
  if (n % 3 == 0) return 3;
  if (n % 2 == 0) return 2;
  int p = 5;
  while (n % p) ++p;
  return p;
}

// R-point DFT in place, sign DIR (-1 forward, +1 inverse). Generic radices
// take their roots of unity from the length-L table (R divides L).
template <typename T, int R, int DIR, int L>
__device__ __forceinline__ void dft_small(T (&vr)[R], T (&vi)[R]) {
  if constexpr (R == 1) {
    return;
  } else if constexpr (R == 2) {
    const T ar = vr[0] + vr[1], ai = vi[0] + vi[1];
    vr[1] = vr[0] - vr[1];
    vi[1] = vi[0] - vi[1];
    vr[0] = ar;
    vi[0] = ai;
  } else if constexpr (R == 3) {
    constexpr double h = 0.86602540378443864676372317075294;  // sqrt(3)/2
    const T sr = vr[1] + vr[2], si = vi[1] + vi[2];
    const T dr = vr[1] - vr[2], di = vi[1] - vi[2];
    const T tr = vr[0] - T(0.5) * sr, ti = vi[0] - T(0.5) * si;
    vr[0] += sr;
    vi[0] += si;
    const T hd_r = T(DIR * h) * di, hd_i = T(DIR * h) * dr;
    vr[1] = tr - hd_r;
    vi[1] = ti + hd_i;
    vr[2] = tr + hd_r;
    vi[2] = ti - hd_i;
  } else if constexpr (R == 4) {
    const T s0r = vr[0] + vr[2], s0i = vi[0] + vi[2];
    const T d0r = vr[0] - vr[2], d0i = vi[0] - vi[2];
    const T s1r = vr[1] + vr[3], s1i = vi[1] + vi[3];
    const T d1r = vr[1] - vr[3], d1i = vi[1] - vi[3];
    // i*DIR*(d1) = DIR*(-d1i, d1r)
    vr[0] = s0r + s1r;
    vi[0] = s0i + s1i;
    vr[2] = s0r - s1r;
    vi[2] = s0i - s1i;
    if constexpr (DIR < 0) {
      vr[1] = d0r + d1i;
      vi[1] = d0i - d1r;
      vr[3] = d0r - d1i;
      vi[3] = d0i + d1r;
    } else {
      vr[1] = d0r - d1i;
      vi[1] = d0i + d1r;
      vr[3] = d0r + d1i;
      vi[3] = d0i - d1r;
    }
  } else if constexpr (R == 8) {
    T er[4] = {vr[0], vr[2], vr[4], vr[6]}, ei[4] = {vi[0], vi[2], vi[4], vi[6]};
    T orr[4] = {vr[1], vr[3], vr[5], vr[7]}, oi[4] = {vi[1], vi[3], vi[5], vi[7]};
    dft_small<T, 4, DIR, L>(er, ei);
    dft_small<T, 4, DIR, L>(orr, oi);
    constexpr double r2 = 0.70710678118654752440084436210485;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      T wr = orr[m], wi = oi[m];
      if (m == 1) {  // (1 + i DIR)/sqrt2
        wr = T(r2) * (orr[1] - T(DIR) * oi[1]);
        wi = T(r2) * (oi[1] + T(DIR) * orr[1]);
      } else if (m == 2) {  // i DIR
        wr = -T(DIR) * oi[2];
        wi = T(DIR) * orr[2];
      } else if (m == 3) {  // (-1 + i DIR)/sqrt2
        wr = T(r2) * (-orr[3] - T(DIR) * oi[3]);
        wi = T(r2) * (-oi[3] + T(DIR) * orr[3]);
      }
      vr[m] = er[m] + wr;
      vi[m] = ei[m] + wi;
      vr[m + 4] = er[m] - wr;
      vi[m + 4] = ei[m] - wi;
    }
  } else {
    T outr[R], outi[R];
#pragma unroll
    for (int m = 0; m < R; ++m) {
      T ar = vr[0], ai = vi[0];
#pragma unroll
      for (int q = 1; q < R; ++q) {
        const int e = ((q * m) % R) * (L / R);
        const T c = Tw<T, L>::c(e), s = T(DIR) * Tw<T, L>::s(e);
        ar += vr[q] * c - vi[q] * s;
        ai += vr[q] * s + vi[q] * c;
      }
      outr[m] = ar;
      outi[m] = ai;
    }
#pragma unroll
    for (int m = 0; m < R; ++m) {
      vr[m] = outr[m];
      vi[m] = outi[m];
    }
  }
}

template <typename T, int L, int DIR> struct RegFFT {
  static __device__ __forceinline__ void run(T (&re)[L], T (&im)[L]) { stage<1>(re, im); }

  template <int Ns>
  static __device__ __forceinline__ void stage(T (&re)[L], T (&im)[L]) {
    if constexpr (Ns < L) {
      constexpr int R = pick_radix(L / Ns);
      T ore[L], oim[L];
#pragma unroll
      for (int j = 0; j < L / R; ++j) {
        const int k = j % Ns;
        T vr[R], vi[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const T xr = re[j + r * (L / R)], xi = im[j + r * (L / R)];
          const int e = (k * r * (L / (Ns * R))) % L;
          if (e == 0) {
            vr[r] = xr;
            vi[r] = xi;
          } else {
            const T c = Tw<T, L>::c(e), s = T(DIR) * Tw<T, L>::s(e);
            vr[r] = xr * c - xi * s;
            vi[r] = xr * s + xi * c;
          }
        }
        dft_small<T, R, DIR, L>(vr, vi);
        const int idx = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          ore[idx + r * Ns] = vr[r];
          oim[idx + r * Ns] = vi[r];
        }
      }
#pragma unroll
      for (int i = 0; i < L; ++i) {
        re[i] = ore[i];
        im[i] = oim[i];
      }
      stage<Ns * R>(re, im);
    }
  }
};

}  // namespace dq
