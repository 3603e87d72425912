"""Equal-time observables by Wick's theorem (test infrastructure; see package header).

For one HS field both spin species share the same G_ij = <c_i c_j^+>, so

  <Delta_i^+ Delta_j>  = (delta_ij - G_ji)^2,   Delta_i^+ = c+_{i up} c+_{i dn}
  <Delta_j Delta_i^+>  = G_ji^2
  <n_x n_y>            = 4 (1 - G_xx)(1 - G_yy) + 2 (delta_xy - G_yx) G_xy,  n = n_up + n_dn

Observables (all Sec. III / IV of the paper):
  S_Pair(Q) = (1/N) sum_ij e^{i Q (r_i - r_j)} <Delta_i^+ Delta_j + Delta_j Delta_i^+>
      (the symmetric definition the paper adopts in Sec. III),
  <phi^+ phi>(Q),  phi(Q) = (1/N) sum_cells e^{i Q R} (n_A + w n_B + w^2 n_C),  w = e^{2 pi i/3}
      (Sec. IV; normalised by the number of sites N as printed),
  density rho = (2/N) sum_x (1 - G_xx),
  kinetic energy per site (2/N) sum_ij K_ij (delta_ij - G_ji).
Derived: R_Pair = 1 - S(Gamma + dk)/S(Gamma), P = sqrt(S(Gamma)/N), D(Q) = sqrt(<phi^+ phi>(Q)).
Full-momentum maps (all Q of the mesh) evaluate the same two definitions at
every Q.
"""

import numpy as np

from . import lattice, lattices

OMEGA = np.exp(2j * np.pi / 3.0)


def pair_structure_factor(G, phase):
    """S_Pair for the site phases phase_i = e^{i Q r_i}; real part (the
    imaginary part of a single-field estimate averages to zero)."""
    N = G.shape[0]
    X = (np.eye(N) - G.T) ** 2 + G.T ** 2        # X_ij for the pair (i, j)
    return float(np.real(phase @ X @ phase.conj())) / N


def cdw_weights(L1, L2, m1, m2):
    """w_x = e^{i Q R_cell(x)} w^{a(x)} (cell positions: the sublattice
    phases of Sec. IV carry the intra-cell structure)."""
    ph = lattice.momentum_phase(m1, m2, L1, L2, with_offsets=False)
    sub = np.tile(OMEGA ** np.arange(3), L1 * L2)
    return ph * sub


def density_correlation(G):
    """<n_x n_y> matrix."""
    N = G.shape[0]
    d = 1.0 - np.diag(G)
    return 4.0 * np.outer(d, d) + 2.0 * (np.eye(N) - G.T) * G


def cdw_correlator(G, w):
    """<phi^+ phi>(Q) = (1/N^2) sum_xy conj(w_x) w_y <n_x n_y>."""
    N = G.shape[0]
    return float(np.real(w.conj() @ density_correlation(G) @ w)) / N ** 2


def density(G):
    return 2.0 * float(np.sum(1.0 - np.diag(G))) / G.shape[0]


def kinetic_energy(G, K):
    N = G.shape[0]
    return 2.0 * float(np.sum(K * (np.eye(N) - G.T))) / N


class Observables:
    """The six equal-time estimators for one torus."""

    NAMES = ("S_pair_G", "S_pair_dk", "phi2_G", "phi2_K", "density", "ekin")

    def __init__(self, L1, L2=None, K=None, site_offsets=True, lattice_name="kagome"):
        if L2 is None:
            L2 = L1
        self.L1, self.L2 = L1, L2
        self.lattice = lattice_name
        if lattice_name == "kagome":
            self.N = 3 * L1 * L2
            self.K = K if K is not None else lattice.kinetic_matrix(L1, L2)
            self.ph_G = lattice.momentum_phase(0, 0, L1, L2, site_offsets)
            self.ph_dk = lattice.momentum_phase(1 % L1, 0, L1, L2, site_offsets)
            self.w_G = cdw_weights(L1, L2, 0, 0)
            kp = lattice.dirac_point(L1) if L1 == L2 else None
            self.w_K = cdw_weights(L1, L2, kp[0], kp[1]) if kp is not None else None
        else:
            # other lattices: the pair structure factor, density and kinetic
            # energy; the three-sublattice CDW order parameter is kagome's
            self.N = lattices.SITES_PER_CELL[lattice_name] * L1 * L2
            self.K = K if K is not None else lattices.kinetic(lattice_name, L1, L2)
            self.ph_G = lattices.momentum_phase(lattice_name, 0, 0, L1, L2, site_offsets)
            self.ph_dk = lattices.momentum_phase(lattice_name, 1 % L1, 0, L1, L2, site_offsets)
            self.w_G = self.w_K = None

    def __call__(self, G):
        return {
            "S_pair_G": pair_structure_factor(G, self.ph_G),
            "S_pair_dk": pair_structure_factor(G, self.ph_dk),
            "phi2_G": cdw_correlator(G, self.w_G) if self.w_G is not None else float("nan"),
            "phi2_K": cdw_correlator(G, self.w_K) if self.w_K is not None else float("nan"),
            "density": density(G),
            "ekin": kinetic_energy(G, self.K),
        }


def pair_structure_factor_all(G, L1, L2=None, site_offsets=True):
    """S_Pair(Q) at every mesh momentum Q = m1 b1 / L1 + m2 b2 / L2 (array
    indexed [m1, m2]), each by the definition above."""
    if L2 is None:
        L2 = L1
    S = np.zeros((L1, L2))
    for m1 in range(L1):
        for m2 in range(L2):
            S[m1, m2] = pair_structure_factor(G, lattice.momentum_phase(m1, m2, L1, L2, site_offsets))
    return S


def cdw_correlator_all(G, L1, L2=None):
    """<phi^+ phi>(Q) at every mesh momentum (array indexed [m1, m2])."""
    if L2 is None:
        L2 = L1
    P = np.zeros((L1, L2))
    for m1 in range(L1):
        for m2 in range(L2):
            P[m1, m2] = cdw_correlator(G, cdw_weights(L1, L2, m1, m2))
    return P


def derived(S_G, S_dk, phi2_G, phi2_K, N):
    """R_Pair, P, D(Gamma), D(K) from the means (Sec. III, IV)."""
    return {
        "R_pair": 1.0 - S_dk / S_G,
        "P": float(np.sqrt(S_G / N)),
        "D_G": float(np.sqrt(phi2_G)),
        "D_K": float(np.sqrt(phi2_K)) if np.isfinite(phi2_K) else float("nan"),
    }


def jackknife(samples, fn):
    """Delete-one jackknife over bins: returns (estimate, error) of fn(mean)."""
    x = np.asarray(samples, dtype=float)
    n = len(x)
    full = fn(x.mean(axis=0))
    if n < 2:
        return full, float("nan")
    loo = np.array([fn((x.sum(axis=0) - x[i]) / (n - 1)) for i in range(n)])
    err = np.sqrt((n - 1) / n * np.sum((loo - loo.mean()) ** 2))
    return full, float(err)
