// Host-side kagome momentum blocks (Eq. 4) and their exponentials.
#include "lattice_host.h"

#include <algorithm>
#include <cmath>

namespace dq {

// A(x)-B(x), A(x)-B(x+e2), A(x)-C(x), A(x)-C(x+e1), B(x)-C(x), B(x)-C(x+e1-e2):
// the six bonds per cell of the Kronecker form of Eq. 3.
const Bond kKagomeBonds[6] = {{0, 1, 0, 0}, {0, 1, 0, 1}, {0, 2, 0, 0},
                              {0, 2, 1, 0}, {1, 2, 0, 0}, {1, 2, 1, -1}};

void kagome_block(int L, int m1, int m2, double t, cd H[3][3]) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) H[a][b] = 0.0;
  const double two_pi = 6.283185307179586476925286766559;
  for (const Bond &bd : kKagomeBonds) {
    // exact reduction of the phase 2 pi (m1 d1 + m2 d2) / L before cos/sin
    long p = ((long)m1 * bd.d1 + (long)m2 * bd.d2) % L;
    if (p < 0) p += L;
    const double ang = two_pi * (double)p / (double)L;
    const cd ph(std::cos(ang), std::sin(ang));
    H[bd.a][bd.b] += -t * ph;
    H[bd.b][bd.a] += -t * std::conj(ph);
  }
}

static void mul3(const cd A[3][3], const cd B[3][3], cd C[3][3]) {
  cd T[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cd s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[i][k] * B[k][j];
      T[i][j] = s;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C[i][j] = T[i][j];
}

void expm3(const cd A[3][3], cd E[3][3]) {
  double norm = 0.0;
  for (int i = 0; i < 3; ++i) {
    double r = 0.0;
    for (int j = 0; j < 3; ++j) r += std::abs(A[i][j]);
    norm = std::fmax(norm, r);
  }
  int sq = 0;
  while (norm > 0.25) {
    norm *= 0.5;
    ++sq;
  }
  const double f = std::ldexp(1.0, -sq);
  cd X[3][3], term[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      X[i][j] = A[i][j] * f;
      E[i][j] = (i == j) ? 1.0 : 0.0;
      term[i][j] = E[i][j];
    }
  // ||X|| <= 1/4: 20 terms reach far below double rounding
  for (int n = 1; n <= 20; ++n) {
    mul3(term, X, term);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        term[i][j] /= (double)n;
        E[i][j] += term[i][j];
      }
  }
  for (int s = 0; s < sq; ++s) mul3(E, E, E);
}

std::vector<cd> block_exp_table(int L, double scale, double t) {
  const int Hh = L / 2 + 1;
  std::vector<cd> out((size_t)L * Hh * 9);
  const double norm = 1.0 / ((double)L * (double)L);
  for (int m1 = 0; m1 < L; ++m1)
    for (int m2 = 0; m2 < Hh; ++m2) {
      cd H[3][3], A[3][3], E[3][3];
      kagome_block(L, m1, m2, t, H);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) A[a][b] = scale * H[a][b];
      expm3(A, E);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) out[((size_t)m1 * Hh + m2) * 9 + a * 3 + b] = E[a][b] * norm;
    }
  return out;
}

}  // namespace dq

namespace dq {

// Eigen-decomposition of a 3 x 3 Hermitian matrix by cyclic Jacobi sweeps:
// each step first turns A_pq real by a phase on index q, then zeroes it with
// a real plane rotation. Q accumulates the unitary: A_in = Q diag(w) Q^H.
void eigh3(const cd A_in[3][3], double w[3], cd Q[3][3]) {
  cd A[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      A[i][j] = A_in[i][j];
      Q[i][j] = (i == j) ? 1.0 : 0.0;
    }
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, scale = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) (i == j ? scale : off) += std::norm(A[i][j]);
    if (off <= 1e-34 * (scale + 1e-300)) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        const double g = std::abs(A[p][q]);
        if (g == 0.0) continue;
        // phase: column q times conj(e), row q times e, e = A_pq / |A_pq|
        const cd e = A[p][q] / g;
        for (int i = 0; i < 3; ++i) A[i][q] *= std::conj(e);
        for (int j = 0; j < 3; ++j) A[q][j] *= e;
        for (int i = 0; i < 3; ++i) Q[i][q] *= std::conj(e);
        // real rotation zeroing the (now real) A_pq = g
        const double app = A[p][p].real(), aqq = A[q][q].real();
        const double theta = (aqq - app) / (2.0 * g);
        const double tt = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(tt * tt + 1.0), sn = tt * c;
        for (int i = 0; i < 3; ++i) {  // columns p, q
          const cd ap = A[i][p], aq = A[i][q];
          A[i][p] = c * ap - sn * aq;
          A[i][q] = sn * ap + c * aq;
        }
        for (int j = 0; j < 3; ++j) {  // rows p, q
          const cd ap = A[p][j], aq = A[q][j];
          A[p][j] = c * ap - sn * aq;
          A[q][j] = sn * ap + c * aq;
        }
        for (int i = 0; i < 3; ++i) {
          const cd qp = Q[i][p], qq = Q[i][q];
          Q[i][p] = c * qp - sn * qq;
          Q[i][q] = sn * qp + c * qq;
        }
      }
  }
  for (int i = 0; i < 3; ++i) w[i] = A[i][i].real();
}

int trial_orbitals(int L, int n_occ, double eps, double t, double gap_min, std::vector<double> &P) {
  const int N = 3 * L * L;
  if (L < 1 || n_occ < 1 || n_occ >= N) return 1;
  const double two_pi = 6.283185307179586476925286766559;
  // one entry per real level group: a self-conjugate momentum (one state) or
  // a pair k, -k (two states of equal energy)
  struct Level {
    double e;
    int m1, m2, b, count;
  };
  std::vector<Level> lv;
  std::vector<double> W((size_t)L * L * 3);
  std::vector<cd> U((size_t)L * L * 9);
  for (int m1 = 0; m1 < L; ++m1)
    for (int m2 = 0; m2 < L; ++m2) {
      cd H[3][3], Qk[3][3];
      kagome_block(L, m1, m2, t, H);
      H[0][0] += eps;
      H[2][2] -= eps;
      double w[3];
      eigh3(H, w, Qk);
      const size_t kk = (size_t)m1 * L + m2;
      for (int b = 0; b < 3; ++b) {
        W[kk * 3 + b] = w[b];
        for (int a = 0; a < 3; ++a) U[kk * 9 + a * 3 + b] = Qk[a][b];
      }
      const int c1 = (L - m1) % L, c2 = (L - m2) % L;
      const bool self = (c1 == m1 && c2 == m2);
      if (!self && std::make_pair(m1, m2) > std::make_pair(c1, c2)) continue;  // partner lists the pair
      for (int b = 0; b < 3; ++b) lv.push_back({w[b], m1, m2, b, self ? 1 : 2});
    }
  std::stable_sort(lv.begin(), lv.end(), [](const Level &x, const Level &y) { return x.e < y.e; });
  // take whole levels up to n_occ states; the cut must fall between levels
  // at least gap_min apart (a pair k, -k is never split)
  int taken = 0;
  size_t nl = 0;
  while (nl < lv.size() && taken < n_occ) taken += lv[nl++].count;
  if (taken != n_occ) return 2;
  if (nl < lv.size() && lv[nl].e - lv[nl - 1].e < gap_min) return 2;
  P.assign((size_t)N * n_occ, 0.0);
  int col = 0;
  for (size_t q = 0; q < nl; ++q) {
    const Level &v = lv[q];
    const size_t kk = (size_t)v.m1 * L + v.m2;
    // phi(x, a) = u_a e^{i k.x} / L; self-conjugate k: real up to a global
    // phase (fixed so that the largest component is real); a pair gives
    // sqrt2 Re phi and sqrt2 Im phi
    cd u[3];
    int amax = 0;
    for (int a = 0; a < 3; ++a) {
      u[a] = U[kk * 9 + a * 3 + v.b];
      if (std::abs(u[a]) > std::abs(u[amax])) amax = a;
    }
    if (v.count == 1) {
      const cd ph = std::conj(u[amax]) / std::abs(u[amax]);
      for (int a = 0; a < 3; ++a) u[a] *= ph;
    }
    const double f = (v.count == 1) ? 1.0 / L : std::sqrt(2.0) / L;
    for (int x1 = 0; x1 < L; ++x1)
      for (int x2 = 0; x2 < L; ++x2) {
        long pidx = ((long)v.m1 * x1 + (long)v.m2 * x2) % L;
        const double ang = two_pi * (double)pidx / (double)L;
        const cd e(std::cos(ang), std::sin(ang));
        for (int a = 0; a < 3; ++a) {
          const cd phi = f * u[a] * e;
          const size_t i = ((size_t)x1 * L + x2) * 3 + a;
          P[i * n_occ + col] = phi.real();
          if (v.count == 2) P[i * n_occ + col + 1] = phi.imag();
        }
      }
    col += v.count;
  }
  return 0;
}

}  // namespace dq
