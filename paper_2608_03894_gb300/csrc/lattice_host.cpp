// Host-side kagome momentum blocks (Eq. 4) and their exponentials.
#include "lattice_host.h"

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
