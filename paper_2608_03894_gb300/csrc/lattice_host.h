// Host-side kagome tables: momentum blocks of the kinetic matrix (Eq. 4) and
// their exponentials, built in FP64.
#pragma once

#include <complex>
#include <vector>

namespace dq {

using cd = std::complex<double>;

// Nearest-neighbour bonds of the kagome torus in the index order of Eq. 3:
// sublattice a of cell x is bonded to sublattice b of cell x + (d1, d2).
struct Bond {
  int a, b, d1, d2;
};
extern const Bond kKagomeBonds[6];

// H(k)_{ab} = sum over bonds of -t e^{i k.d} (and the Hermitian partner), for
// reduced momentum k = 2 pi (m1, m2) / L. With the forward transform
// v~(k) = sum_x e^{-i k.x} v(x), (K v)~(k) = H(k) v~(k).
void kagome_block(int L, int m1, int m2, double t, cd H[3][3]);

// exp(A) of a 3x3 complex matrix by scaling and squaring of the Taylor series.
void expm3(const cd A[3][3], cd E[3][3]);

// Table E[(m1*Hh + m2)*9 + a*3 + b] = exp(scale H(k))_{ab} / L^2 for m1 in
// [0, L), m2 in [0, Hh), Hh = L/2 + 1: the half spectrum the real-input FFT
// keeps; 1/L^2 is the normalisation of the inverse 2D transform.
std::vector<cd> block_exp_table(int L, double scale, double t = 1.0);

// Eigen-decomposition A = Q diag(w) Q^H of a 3 x 3 Hermitian matrix (Jacobi).
void eigh3(const cd A[3][3], double w[3], cd Q[3][3]);

// Trial orbitals of projector QMC: an orthonormal real basis P (N x n_occ,
// row-major, site index (x1 L + x2) 3 + a) of the lowest n_occ eigenstates of
// K + eps diag(+1, 0, -1 by sublattice), built from the momentum blocks
// H(k) + eps diag(1, 0, -1): one Bloch state per self-conjugate momentum,
// the real and imaginary parts of u(k) e^{i k.x} for each pair k, -k.
// Returns 0, 1 (bad arguments) or 2 (open shell: the cut at n_occ falls
// inside a degenerate level, gap < gap_min, or splits a pair k, -k).
int trial_orbitals(int L, int n_occ, double eps, double t, double gap_min, std::vector<double> &P);

}  // namespace dq
