"""Equal-time Green's function from scratch (test infrastructure; see package header).

G(tau_l) = (I + B_l ... B_1 B_M ... B_{l+1})^{-1},  G_ij = <c_i c_j^+>.

Two routes:
* ``green_direct``: form the product and invert (only for small beta, where
  the product is well conditioned);
* ``green_udv``: the product split at tau_l into B(tau_l, 0) = U_r D_r T_r and
  B(beta, tau_l) = T_l D_l U_l, each kept in UDV form by a column-pivoted QR
  after every slice, and combined by the scale-separated inversion
      G = U_l^T (D_l^max)^{-1} [ (D_r^max)^{-1} U_r^T U_l^T (D_l^max)^{-1}
                                + D_r^min T_r T_l D_l^min ]^{-1} (D_r^max)^{-1} U_r^T
  with D^max = max(D, 1), D^min = min(D, 1) (Loh and Gubernatis; the paper
  does not specify its stabilisation).
"""

import numpy as np
import scipy.linalg as sla


class UDV:
    """Represents the matrix U diag(D) T with U orthogonal."""

    def __init__(self, N):
        self.U = np.eye(N)
        self.D = np.ones(N)
        self.T = np.eye(N)

    def copy(self):
        o = UDV.__new__(UDV)
        o.U, o.D, o.T = self.U.copy(), self.D.copy(), self.T.copy()
        return o

    def left_multiply(self, A):
        """Replace U D T by A U D T, re-factorised by a column-pivoted QR of
        (A U) D:  (A U D) P = Q R  ->  U' = Q, D' = |diag R|, T' = D'^{-1} R P^T T."""
        X = (A @ self.U) * self.D[None, :]
        Q, R, piv = sla.qr(X, pivoting=True)
        d = np.abs(np.diag(R))
        Rn = R / d[:, None]
        # (Rn P^T) T : column j of Rn belongs to original column piv[j]
        RP = np.empty_like(Rn)
        RP[:, piv] = Rn
        T = RP @ self.T
        self.U, self.D, self.T = Q, d, T
        return self

    def matrix(self):
        return (self.U * self.D[None, :]) @ self.T


def right_chain(model, field, l, every=1):
    """B(tau_l, 0) = B_l ... B_1 in UDV form, a QR after every ``every`` slices
    (the products of up to ``every`` slices are formed densely in between)."""
    u = UDV(model.N)
    X = None
    for m in range(1, l + 1):
        B = model.B(field[m - 1])
        X = B if X is None else B @ X
        if m % every == 0 or m == l:
            u.left_multiply(X)
            X = None
    return u


def left_chain(model, field, l, every=1):
    """B(beta, tau_l) = B_M ... B_{l+1}, kept as the UDV form of its transpose
    B_{l+1}^T ... B_M^T, so that B(beta, tau_l) = T^T D U^T; a QR after every
    ``every`` slices."""
    u = UDV(model.N)
    X = None
    cnt = 0
    for m in range(model.M, l, -1):
        Bt = model.BT(field[m - 1])
        X = Bt if X is None else Bt @ X
        cnt += 1
        if cnt % every == 0 or m == l + 1:
            u.left_multiply(X)
            X = None
    return u


def combine(right, left):
    """G from B(tau,0) = U_r D_r T_r and B(beta,tau)^T = U' D_l T' (so that
    B(beta,tau) = T'^T D_l U'^T, i.e. U_l^T = U', T_l = T'^T)."""
    Ur, Dr, Tr = right.U, right.D, right.T
    Ulp, Dl, Tlp = left.U, left.D, left.T
    Drmax, Drmin = np.maximum(Dr, 1.0), np.minimum(Dr, 1.0)
    Dlmax, Dlmin = np.maximum(Dl, 1.0), np.minimum(Dl, 1.0)
    Mmat = (Ur.T @ Ulp) / Drmax[:, None] / Dlmax[None, :] \
        + (Drmin[:, None] * (Tr @ Tlp.T)) * Dlmin[None, :]
    rhs = Ur.T / Drmax[:, None]
    Z = np.linalg.solve(Mmat, rhs)
    return (Ulp / Dlmax[None, :]) @ Z


def green_udv(model, field, l, every=1):
    """Stabilised G(tau_l) for slice index l in 0..M (a QR after every
    ``every`` slices on both sides; 1 is the reference)."""
    return combine(right_chain(model, field, l, every), left_chain(model, field, l, every))


def product_chain(model, field, l):
    """B_l ... B_1 B_M ... B_{l+1} as a plain dense product."""
    P = np.eye(model.N)
    for m in range(l, 0, -1):
        P = P @ model.B(field[m - 1])
    for m in range(model.M, l, -1):
        P = P @ model.B(field[m - 1])
    return P


def green_direct(model, field, l):
    """Unstabilised G(tau_l) = (I + B_l...B_1 B_M...B_{l+1})^{-1} (small beta only)."""
    return np.linalg.inv(np.eye(model.N) + product_chain(model, field, l))
