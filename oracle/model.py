"""Model, HS decoupling and slice propagators (test infrastructure; see package header).

Hamiltonian. Eq. 1 (Sec. II) with the paper's sign: U < 0 is attraction. We
take the interaction in particle-hole symmetric form,
    H = sum_{ij,s} c+_{is} K_ij c_{js} - mu sum_{i,s} n_{is} + U sum_i (n_up - 1/2)(n_dn - 1/2),
which differs from Eq. 1 by mu -> mu - U/2 and a constant; with it mu = -1
puts the U = 0 Fermi level at the Dirac point (-t), i.e. rho = 2/3.

Trotter / HS (the paper fixes neither; this is the standard charge-channel
reading for U <= 0, sign-free because both spins see the same field):
    e^{-dtau U (n_up - 1/2)(n_dn - 1/2)} = (1/2) e^{-dtau |U| / 4} sum_{s=+-1} e^{lambda s (n_up + n_dn - 1)},
    cosh(lambda) = e^{dtau |U| / 2}.
Weight of a field s_{i,l}: prod_{i,l} e^{-lambda s_{il}} det(I + B_M ... B_1)^2, with
    B_l = e^{V_l} e^{-dtau K},   (e^{V_l})_ii = e^{lambda s_{il} + dtau mu}.
"""

import numpy as np

from . import lattice as lattice_mod
from . import lattices


class Model:
    """Parameters plus dense propagators for one kagome torus."""

    def __init__(self, L, beta, dtau, U, mu, t=1.0, L2=None, lattice="kagome"):
        if U > 0:
            raise ValueError("U > 0 (repulsive) has a sign problem in the charge channel; U <= 0 only")
        M = beta / dtau
        if abs(M - round(M)) > 1e-9 or round(M) < 1:
            raise ValueError("beta / dtau must be a positive integer")
        self.L1 = int(L)
        self.L2 = int(L if L2 is None else L2)
        self.beta, self.dtau, self.U, self.mu, self.t = float(beta), float(dtau), float(U), float(mu), float(t)
        self.M = int(round(M))
        self.lattice = lattice
        self.N = lattices.SITES_PER_CELL[lattice] * self.L1 * self.L2
        self.lam = float(np.arccosh(np.exp(self.dtau * abs(self.U) / 2.0)))
        self.K = (lattice_mod.kinetic_matrix(self.L1, self.L2, self.t) if lattice == "kagome"
                  else lattices.kinetic(lattice, self.L1, self.L2, self.t))
        w, V = np.linalg.eigh(self.K)
        self.eps, self.Vk = w, V
        self.expK = (V * np.exp(-self.dtau * w)) @ V.T      # e^{-dtau K}
        self.expKinv = (V * np.exp(self.dtau * w)) @ V.T    # e^{+dtau K}

    def expV(self, s_slice):
        """Diagonal of e^{V_l} for one slice of the field."""
        return np.exp(self.lam * np.asarray(s_slice, dtype=np.float64) + self.dtau * self.mu)

    def B(self, s_slice):
        """B_l = e^{V_l} e^{-dtau K}."""
        return self.expV(s_slice)[:, None] * self.expK

    def Binv(self, s_slice):
        """B_l^{-1} = e^{+dtau K} e^{-V_l}."""
        return self.expKinv / self.expV(s_slice)[None, :]

    def BT(self, s_slice):
        """B_l^T = e^{-dtau K} e^{V_l} (K is symmetric)."""
        return self.expK * self.expV(s_slice)[None, :]

    def log_boson_weight(self, field):
        """log prod_{i,l} e^{-lambda s_il}."""
        return -self.lam * float(np.sum(field))

    def hs_constant(self):
        """C in e^{-dtau U(n_up-1/2)(n_dn-1/2)} = C sum_s e^{lambda s (n-1)}."""
        return 0.5 * np.exp(-self.dtau * abs(self.U) / 4.0)

    def green_free(self):
        """U = 0 closed form G = (1 + e^{-beta (K - mu)})^{-1} via the spectrum of K
        (Fermi function per eigenvalue; numerically safe for any beta)."""
        x = self.beta * (self.eps - self.mu)
        occ_hole = 0.5 * (1.0 + np.tanh(x / 2.0))      # 1/(1+e^{-x})
        return (self.Vk * occ_hole) @ self.Vk.T

    def ekin_free(self):
        """Free-fermion kinetic energy per site, both spins: (2/N) sum_n eps_n f(eps_n - mu)."""
        f = 0.5 * (1.0 - np.tanh(self.beta * (self.eps - self.mu) / 2.0))
        return 2.0 * float(np.sum(self.eps * f)) / self.N

    def density_free(self):
        f = 0.5 * (1.0 - np.tanh(self.beta * (self.eps - self.mu) / 2.0))
        return 2.0 * float(np.sum(f)) / self.N
