"""Exact Fock-space references on tiny tori (test infrastructure; see package header).

* ``ED``: exact thermal averages of the particle-hole symmetric Hamiltonian
  (see ``model``) in the full 4^N-dimensional Fock space, block-diagonalised
  by (N_up, N_dn).
* ``trotter``: the same averages for the Trotterised density matrix
  (e^{-dtau (U_hat - mu N_hat)} e^{-dtau K_hat})^M, the operator that the
  discrete HS sum reproduces exactly; the observable sits at tau = 0 = beta,
  the slice at which G = (I + B_M ... B_1)^{-1} is evaluated.
* ``brute_force_hs``: the sum over all 2^{NM} Ising fields of
  prod e^{-lambda s} det(I + B_M ... B_1)^2 and the weighted Wick estimators.

Identity pinned by the tests (no statistics):
  Tr[(e^{-dtau(U_hat - mu N_hat)} e^{-dtau K_hat})^M] = C^{NM} sum_s w_s,
  C = (1/2) e^{-dtau |U| / 4},
and every Wick estimator averaged with w_s equals the Fock-space trace.
Spin up and down are independent species; with all up modes ordered before
all down modes, every same-species bilinear c+_{i s} c_{j s} is
(h_ij (x) 1) or (1 (x) h_ij) -- the Jordan-Wigner strings cancel -- and the
pair operator Delta_i^+ Delta_j = (c+_{i dn} c_{j dn})(c+_{i up} c_{j up})
is h_ij (x) h_ij.
"""

import itertools

import numpy as np
import scipy.linalg as sla

from . import measure


def single_species_hops(N):
    """h[i][j] = c_i^+ c_j on the 2^N single-species Fock space (bit i of the
    basis index is mode i; Jordan-Wigner sign counts occupied modes below)."""
    dim = 1 << N

    def annihilate(i, b):
        if not (b >> i) & 1:
            return None, 0
        sign = -1 if bin(b & ((1 << i) - 1)).count("1") % 2 else 1
        return b ^ (1 << i), sign

    def create(i, b):
        if (b >> i) & 1:
            return None, 0
        sign = -1 if bin(b & ((1 << i) - 1)).count("1") % 2 else 1
        return b | (1 << i), sign

    h = [[np.zeros((dim, dim)) for _ in range(N)] for _ in range(N)]
    for i in range(N):
        for j in range(N):
            for b in range(dim):
                b1, s1 = annihilate(j, b)
                if b1 is None:
                    continue
                b2, s2 = create(i, b1)
                if b2 is None:
                    continue
                h[i][j][b2, b] += s1 * s2
    return h


class Sectors:
    """(N_up, N_dn) sectors of the two-species Fock space for a model."""

    def __init__(self, model, obs=None):
        self.model = model
        N = model.N
        self.N = N
        h = single_species_hops(N)
        dim = 1 << N
        pop = np.array([bin(b).count("1") for b in range(dim)])
        self.idx = [np.nonzero(pop == n)[0] for n in range(N + 1)]
        self.h = [[[h[i][j][np.ix_(self.idx[n], self.idx[n])] for j in range(N)] for i in range(N)]
                  for n in range(N + 1)]
        K = model.K
        self.k = [sum(K[i, j] * self.h[n][i][j] for i in range(N) for j in range(N) if K[i, j] != 0.0)
                  if len(self.idx[n]) else np.zeros((0, 0)) for n in range(N + 1)]
        self.bits = [np.array([[(b >> i) & 1 for i in range(N)] for b in self.idx[n]], dtype=float)
                     for n in range(N + 1)]
        self.obs = obs if obs is not None else measure.Observables(model.L1, model.L2, K,
                                                                   lattice_name=getattr(model, "lattice", "kagome"))

    def _kin(self, nu, nd):
        ku, kd = self.k[nu], self.k[nd]
        return np.kron(ku, np.eye(len(kd))) + np.kron(np.eye(len(ku)), kd)

    def _pot_diag(self, nu, nd):
        """Diagonal of U sum_i (n_up - 1/2)(n_dn - 1/2) - mu N_hat."""
        m = self.model
        bu, bd = self.bits[nu], self.bits[nd]
        uu = (bu - 0.5)[:, None, :] * (bd - 0.5)[None, :, :]
        return (m.U * uu.sum(axis=2) - m.mu * (nu + nd)).reshape(-1)

    def _ops(self, nu, nd):
        """Observable operators in the sector, matching measure.Observables."""
        N = self.N
        hu, hd = self.h[nu], self.h[nd]
        Iu, Id = np.eye(len(self.idx[nu])), np.eye(len(self.idx[nd]))
        ops = {}

        def pair(phase):
            S = 0.0
            for i in range(N):
                for j in range(N):
                    c = phase[i] * np.conj(phase[j])
                    d = 1.0 if i == j else 0.0
                    S = S + c * (np.kron(hu[i][j], hd[i][j])
                                 + np.kron(d * Iu - hu[i][j], d * Id - hd[i][j]))
            return S / N

        ops["S_pair_G"] = pair(self.obs.ph_G)
        ops["S_pair_dk"] = pair(self.obs.ph_dk)
        nvec = (self.bits[nu][:, None, :] + self.bits[nd][None, :, :]).reshape(-1, N)  # n_x per basis state

        def cdw(w):
            if w is None:
                return None
            phi = nvec @ w / N
            return np.diag(np.abs(phi) ** 2)

        ops["phi2_G"] = cdw(self.obs.w_G)
        ops["phi2_K"] = cdw(self.obs.w_K)
        ops["density"] = np.diag(nvec.sum(axis=1) / N)
        ops["ekin"] = self._kin(nu, nd) * (1.0 / N)
        return ops

    def sectors(self):
        for nu in range(self.N + 1):
            for nd in range(self.N + 1):
                yield nu, nd

    def exact(self, beta=None):
        """Exact thermal averages <O> = Tr[O e^{-beta H}] / Z."""
        m = self.model
        beta = m.beta if beta is None else beta
        data = []
        emin = np.inf
        for nu, nd in self.sectors():
            H = self._kin(nu, nd) + np.diag(self._pot_diag(nu, nd))
            w, V = np.linalg.eigh(H)
            emin = min(emin, w.min())
            data.append((nu, nd, w, V))
        Z = 0.0
        acc = {k: 0.0 for k in measure.Observables.NAMES}
        for nu, nd, w, V in data:
            p = np.exp(-beta * (w - emin))
            Z += p.sum()
            ops = self._ops(nu, nd)
            for k, O in ops.items():
                if O is None:
                    continue
                Od = np.einsum('ai,ab,bi->i', V.conj(), O, V)
                acc[k] += float(np.real(np.sum(p * Od)))
        out = {k: v / Z for k, v in acc.items()}
        if self.obs.w_K is None:
            out["phi2_K"] = float("nan")
        if self.obs.w_G is None:
            out["phi2_G"] = float("nan")
        return out, Z, emin

    def trotter(self, M=None, with_green=False):
        """Averages and Z for rho_T = (e^{-dtau(U_hat - mu N_hat)} e^{-dtau K_hat})^M.
        ``with_green`` adds "G": the matrix <c_i c_j^+> = delta_ij - <c_j^+ c_i>
        (spin up), a one-body observable commuting with neither factor."""
        m = self.model
        M = m.M if M is None else M
        dtau = m.beta / M
        Z = 0.0
        acc = {k: 0.0 for k in measure.Observables.NAMES}
        Gacc = np.zeros((self.N, self.N))
        for nu, nd in self.sectors():
            ku, kd = self.k[nu], self.k[nd]
            Eu = sla.expm(-dtau * ku) if len(ku) else ku
            Ed = sla.expm(-dtau * kd) if len(kd) else kd
            X = np.exp(-dtau * self._pot_diag(nu, nd))[:, None] * np.kron(Eu, Ed)
            rho = np.linalg.matrix_power(X, M)
            Z += np.trace(rho)
            for k, O in self._ops(nu, nd).items():
                if O is None:
                    continue
                acc[k] += float(np.real(np.trace(O @ rho)))
            if with_green:
                Id = np.eye(len(self.idx[nd]))
                for i in range(self.N):
                    for j in range(self.N):
                        hop = np.kron(self.h[nu][j][i], Id)      # c+_j c_i, spin up
                        Gacc[i, j] -= float(np.real(np.trace(hop @ rho)))
        out = {k: v / Z for k, v in acc.items()}
        if self.obs.w_K is None:
            out["phi2_K"] = float("nan")
        if self.obs.w_G is None:
            out["phi2_G"] = float("nan")
        if with_green:
            out["G"] = np.eye(self.N) + Gacc / float(np.real(Z))
        return out, float(np.real(Z))


    def _green_up(self, left, right, norm, nu, nd):
        """<c_i c_j^+> (spin up) = delta_ij - <c_j^+ c_i> between two sector vectors."""
        Id = np.eye(len(self.idx[nd]))
        G = np.eye(self.N)
        for i in range(self.N):
            for j in range(self.N):
                G[i, j] -= float(left @ (np.kron(self.h[nu][j][i], Id) @ right)) / norm
        return G

    def _expect(self, left, right, n, with_green):
        norm = float(left @ right)
        out = {}
        for k, O in self._ops(n, n).items():
            out[k] = float("nan") if O is None else float(np.real(left @ (O @ right))) / norm
        if with_green:
            out["G"] = self._green_up(left, right, norm, n, n)
        return out, norm

    def slater(self, P):
        """Fock vector (one species, sector n = P.shape[1]) of the Slater
        determinant of P's columns: the unique ground state of
        -sum_ij (P P^T)_ij c+_i c_j with n particles (energy -n, gap 1)."""
        n = P.shape[1]
        Pp = P @ P.T
        H = -sum(Pp[i, j] * self.h[n][i][j] for i in range(self.N) for j in range(self.N))
        w, V = np.linalg.eigh(H)
        if len(w) > 1 and w[1] - w[0] < 0.5:
            raise ValueError("P does not define a unique Slater determinant")
        return V[:, 0]

    def pqmc(self, P, l, M=None, with_green=False):
        """Projector averages <Psi_T| X^{M-l} O X^l |Psi_T> / <Psi_T| X^M |Psi_T>,
        X = e^{-dtau(U_hat - mu N_hat)} e^{-dtau K_hat}, |Psi_T> the Slater
        determinant of P for both species (sector (n, n), n = N_occ); the
        observable sits at slice l, where G(tau_l) = I - R (L R)^{-1} L."""
        m = self.model
        M = m.M if M is None else M
        dtau = m.beta / M
        n = P.shape[1]
        psi1 = self.slater(P)
        psi = np.kron(psi1, psi1)
        E = sla.expm(-dtau * self.k[n])
        X = np.exp(-dtau * self._pot_diag(n, n))[:, None] * np.kron(E, E)
        right = psi.copy()
        for _ in range(l):
            right = X @ right
        left = psi.copy()
        for _ in range(M - l):
            left = X.T @ left
        return self._expect(left, right, n, with_green)

    def ground(self, n, with_green=False):
        """Ground-state averages of H in the (n, n) sector (exact diagonalisation)."""
        H = self._kin(n, n) + np.diag(self._pot_diag(n, n))
        w, V = np.linalg.eigh(H)
        if len(w) > 1 and w[1] - w[0] < 1e-9:
            raise ValueError("degenerate ground state in the (n, n) sector")
        v = V[:, 0]
        out, _ = self._expect(v, v, n, with_green)
        return out, float(w[0])


def brute_force_hs(model, obs=None, with_green=False):
    """Sum over all 2^{N M} Ising fields: returns (weighted Wick averages,
    sum_s w_s). Weight w_s = prod e^{-lambda s} det(I + B_M ... B_1)^2.
    ``with_green`` adds the weighted average "G" of G = (I + B_M...B_1)^{-1}."""
    N, M = model.N, model.M
    obs = obs if obs is not None else measure.Observables(model.L1, model.L2, model.K,
                                                          lattice_name=getattr(model, "lattice", "kagome"))
    Wsum = 0.0
    acc = {k: 0.0 for k in measure.Observables.NAMES}
    Gacc = np.zeros((N, N))
    I = np.eye(N)
    for bits in itertools.product((1, -1), repeat=N * M):
        field = np.array(bits, dtype=np.int8).reshape(M, N)
        P = I
        for l in range(1, M + 1):
            P = model.B(field[l - 1]) @ P
        A = I + P
        w = np.exp(model.log_boson_weight(field)) * np.linalg.det(A) ** 2
        G = np.linalg.inv(A)
        vals = obs(G)
        Wsum += w
        Gacc += w * G
        for k in acc:
            acc[k] += w * vals[k]
    out = {k: v / Wsum for k, v in acc.items()}
    if with_green:
        out["G"] = Gacc / Wsum
    return out, Wsum


def field_weights(model):
    """Exact normalised weight of every field (for histogram tests), keyed by
    the field's bit pattern (row-major s[l-1, i], +1 -> 1)."""
    N, M = model.N, model.M
    I = np.eye(N)
    ws = {}
    for bits in itertools.product((1, -1), repeat=N * M):
        field = np.array(bits, dtype=np.int8).reshape(M, N)
        P = I
        for l in range(1, M + 1):
            P = model.B(field[l - 1]) @ P
        ws[bits] = np.exp(model.log_boson_weight(field)) * np.linalg.det(I + P) ** 2
    tot = sum(ws.values())
    return {k: v / tot for k, v in ws.items()}
