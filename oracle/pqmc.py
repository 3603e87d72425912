"""Projector (zero-temperature) DQMC, the paper's own method (test
infrastructure; see package header).

Sec. II: the ground state is projected out of a trial Slater determinant
built from the lowest N_occ eigenstates of K; the filling is
rho = 2 N_occ / N, and the projection length beta = M dtau is split into the
same slices B_l = e^{V_l} e^{-dtau K} as the finite-temperature chain.

With P (N x N_occ, orthonormal columns) the trial orbitals of one spin
species, and for a fixed field,
    R = B(tau_l, 0) P = B_l ... B_1 P,      L = P^T B(beta, tau_l) = P^T B_M ... B_{l+1},
    weight  w(s) = prod e^{-lambda s} det(L R)^2,
    G(tau_l) = I - R (L R)^{-1} L,          G_ij = <c_i c_j^+>
(the mixed estimator of two Slater determinants obeys Wick's theorem with
this G). Replacing R by R X and L by Y L for invertible X, Y leaves G
unchanged, so only the column spaces of R and L^T matter: with orthonormal
bases Q_R of span(R) and Q_L of span(L^T),
    G = I - Q_R (Q_L^T Q_R)^{-1} Q_L^T,
and the stacks keep only Q factors, re-orthonormalised by a QR after every
slice. Flipping s_il multiplies R by (I + delta e_i e_i^T) and gives the same
ratio 1 + delta (1 - G_ii) and the same rank-one update of G as the
finite-temperature chain (Sherman-Morrison on L R), so the sweep, the
proposals and the Philox streams are those of ``dqmc.Chain``.

Readings (the paper gives no formulas for these):
* trial state: the lowest N_occ eigenvectors of K + eps diag(+1, 0, -1)
  (sublattices A, B, C), eps = 1e-4 t by default. At rho = 2/3 with 3 | L the
  N_occ-th level of K is degenerate (the Dirac points sit on the momentum
  mesh); the small sublattice potential splits it, so that span(P) is unique.
  A filling whose shell is still open raises ValueError.
* the measurement slice is the checkpoint closest to beta / 2 on the up pass.
"""

import itertools

import numpy as np

from . import dqmc, measure
from .model import Model


def trial_state(model, n_occ, eps=1e-4, gap_min=1e-9):
    """P: the lowest n_occ eigenvectors of K + eps diag(sublattice pattern +1, 0, -1)."""
    N = model.N
    if not 1 <= n_occ < N:
        raise ValueError("need 1 <= n_occ < N")
    pattern = np.tile(np.array([1.0, 0.0, -1.0]), N // 3)
    w, V = np.linalg.eigh(model.K + eps * np.diag(pattern))
    if w[n_occ] - w[n_occ - 1] < gap_min:
        raise ValueError(f"open shell: levels {n_occ - 1} and {n_occ} are degenerate "
                         f"({w[n_occ - 1]:.12f}, {w[n_occ]:.12f})")
    return V[:, :n_occ].copy()


def orthonormal(A):
    """Orthonormal basis of the column space of A (reduced Householder QR)."""
    Q, _ = np.linalg.qr(A)
    return Q


class OrthStack:
    """Orthonormal basis Q of span(A_k ... A_1 P), re-orthonormalised after
    every left multiplication."""

    def __init__(self, P):
        self.Q = orthonormal(P)

    def copy(self):
        o = OrthStack.__new__(OrthStack)
        o.Q = self.Q.copy()
        return o

    def left_multiply(self, A):
        self.Q = orthonormal(A @ self.Q)
        return self


def green_from_bases(QR, QL):
    """G = I - Q_R (Q_L^T Q_R)^{-1} Q_L^T."""
    N = QR.shape[0]
    return np.eye(N) - QR @ np.linalg.solve(QL.T @ QR, QL.T)


def green_direct(model, P, field, l):
    """G(tau_l) = I - R (L R)^{-1} L with R = B_l ... B_1 P and
    L = P^T B_M ... B_{l+1}, formed without stabilisation (small beta only)."""
    R = P.copy()
    for m in range(1, l + 1):
        R = model.B(field[m - 1]) @ R
    Lm = P.T.copy()
    for m in range(model.M, l, -1):
        Lm = Lm @ model.B(field[m - 1])
    return np.eye(model.N) - R @ np.linalg.solve(Lm @ R, Lm)


def right_basis(model, P, field, l):
    """Q_R: orthonormal basis of span(B_l ... B_1 P), QR after every slice."""
    s = OrthStack(P)
    for m in range(1, l + 1):
        s.left_multiply(model.B(field[m - 1]))
    return s


def left_basis(model, P, field, l):
    """Q_L: orthonormal basis of span(B_{l+1}^T ... B_M^T P), QR after every slice."""
    s = OrthStack(P)
    for m in range(model.M, l, -1):
        s.left_multiply(model.BT(field[m - 1]))
    return s


def green_stable(model, P, field, l):
    """Stabilised G(tau_l) from the two orthonormal bases."""
    return green_from_bases(right_basis(model, P, field, l).Q, left_basis(model, P, field, l).Q)


def log_weight(model, P, field):
    """log w(s) = -lambda sum s + 2 log |det(P^T B(beta, 0) P)| (the sign of
    det(L R) squares away)."""
    R = P.copy()
    for m in range(1, model.M + 1):
        R = model.B(field[m - 1]) @ R
    sign, logdet = np.linalg.slogdet(P.T @ R)
    return model.log_boson_weight(field) + 2.0 * logdet


class PQMCChain(dqmc.Chain):
    """The finite-temperature ``dqmc.Chain`` sweep with the projector G: stacks
    of orthonormal N x N_occ bases instead of UDV products, measurements at
    the checkpoint closest to beta / 2."""

    def __init__(self, L, beta, dtau, U, mu, seed, n_occ, n_stab=10, chain=0, eps=1e-4, t=1.0,
                 L2=None, field=None, site_offsets=True):
        self.P = trial_state(Model(L, beta, dtau, U, mu, t=t, L2=L2), n_occ, eps)
        self.n_occ = int(n_occ)
        super().__init__(L, beta, dtau, U, mu, seed, n_stab=n_stab, chain=chain, t=t, L2=L2,
                         field=field, site_offsets=site_offsets)
        half = self.M / 2.0
        self.c_meas = min(range(self.C + 1), key=lambda c: (abs(self.tau[c] - half), self.tau[c]))

    def _chunk_right(self, u, c):
        for l in range(self.tau[c - 1] + 1, self.tau[c] + 1):
            u.left_multiply(self.model.B(self.field[l - 1]))
        return u

    def _chunk_left(self, u, c):
        for l in range(self.tau[c + 1], self.tau[c], -1):
            u.left_multiply(self.model.BT(self.field[l - 1]))
        return u

    def reset_green(self):
        self.left = [None] * (self.C + 1)
        self.right = [None] * (self.C + 1)
        self.left[self.C] = OrthStack(self.P)
        for c in range(self.C - 1, -1, -1):
            self.left[c] = self._chunk_left(self.left[c + 1].copy(), c)
        self.right[0] = OrthStack(self.P)
        self.G = green_from_bases(self.right[0].Q, self.left[0].Q)
        self.slice = 0

    def _refresh(self, c):
        G_fresh = green_from_bases(self.right[c].Q, self.left[c].Q)
        self.max_drift = max(self.max_drift, float(np.max(np.abs(G_fresh - self.G))))
        self.G = G_fresh

    def _measure_at(self, c):
        return c == self.c_meas

    def green_fresh(self, l):
        return green_stable(self.model, self.P, self.field, l)


def brute_force(model, P, l, obs=None, with_green=False):
    """Sum over all 2^{N M} Ising fields of w(s) times the Wick estimators of
    G_s(tau_l) (``green_direct``), divided by sum_s w(s) (tiny systems only)."""
    N, M = model.N, model.M
    obs = obs if obs is not None else measure.Observables(model.L1, model.L2, model.K)
    Wsum = 0.0
    acc = {k: 0.0 for k in measure.Observables.NAMES}
    Gacc = np.zeros((N, N))
    for bits in itertools.product((1, -1), repeat=N * M):
        field = np.array(bits, dtype=np.int8).reshape(M, N)
        w = float(np.exp(log_weight(model, P, field)))
        G = green_direct(model, P, field, l)
        vals = obs(G)
        Wsum += w
        Gacc += w * G
        for k in acc:
            acc[k] += w * vals[k]
    out = {k: v / Wsum for k, v in acc.items()}
    if with_green:
        out["G"] = Gacc / Wsum
    return out, Wsum


def field_weights(model, P):
    """Exact normalised weight of every field, keyed by its bit pattern
    (row-major s[l-1, i], +1 -> 1)."""
    N, M = model.N, model.M
    lw = {}
    for bits in itertools.product((1, -1), repeat=N * M):
        field = np.array(bits, dtype=np.int8).reshape(M, N)
        lw[bits] = log_weight(model, P, field)
    mx = max(lw.values())
    ws = {k: np.exp(v - mx) for k, v in lw.items()}
    tot = sum(ws.values())
    return {k: v / tot for k, v in ws.items()}
