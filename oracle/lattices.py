"""The other composite lattices of the paper's appendix (test infrastructure;
see package header): the triangular lattice (one site per cell, 1 x 1
momentum blocks) and the honeycomb lattice (two sites per cell, 2 x 2
blocks). Site index i = (x1*L2 + x2)*n + a with n sites per cell, the same
order as the kagome lattice of Eq. 3.

Each kinetic matrix is built twice, from its Kronecker form (Appendix A, the
triangular and honeycomb equations, with hopping -t as for the kagome matrix
of Sec. II) and from planar geometry (nearest-neighbour pairs on the torus),
so that the two pin each other; the textbook band structures pin both.
"""

import numpy as np

from .lattice import shift_matrix

# triangular: Bravais vectors with the three bond directions a1, a2, a1 + a2
# (unit length), one site per cell
TRI_A1 = np.array([1.0, 0.0])
TRI_A2 = np.array([-0.5, np.sqrt(3.0) / 2.0])
# honeycomb: Bravais vectors at 60 degrees, B = A + (0, 1/sqrt 3); A(x) is
# bonded to B(x), B(x + e1) and B(x + e2) at distance 1/sqrt 3
HON_A1 = np.array([0.5, -np.sqrt(3.0) / 2.0])
HON_A2 = np.array([-0.5, -np.sqrt(3.0) / 2.0])
HON_TAU = np.array([[0.0, 0.0], [0.0, 1.0 / np.sqrt(3.0)]])

SITES_PER_CELL = {"kagome": 3, "triangular": 1, "honeycomb": 2}
# sublattice offsets in units of (A1, A2): honeycomb B = A + (0, 1/sqrt 3) = A - (A1 + A2) / 3
TAU_FRAC = {"triangular": np.zeros((1, 2)), "honeycomb": np.array([[0.0, 0.0], [-1.0 / 3.0, -1.0 / 3.0]])}


def momentum_phase(lattice, m1, m2, L1, L2=None, with_offsets=True):
    """e^{i Q . r_i} for Q = m1 b1 / L1 + m2 b2 / L2 on the triangular or
    honeycomb torus (site positions R + tau_a, or cell positions R)."""
    if L2 is None:
        L2 = L1
    tau = TAU_FRAC[lattice]
    n = len(tau)
    ph = np.zeros(n * L1 * L2, dtype=complex)
    for x1 in range(L1):
        for x2 in range(L2):
            for a in range(n):
                f = np.array([x1, x2], dtype=float) + (tau[a] if with_offsets else 0.0)
                ph[(x1 * L2 + x2) * n + a] = np.exp(2j * np.pi * (m1 * f[0] / L1 + m2 * f[1] / L2))
    return ph


def triangular_kinetic(L1, L2=None, t=1.0):
    """K = -t [I (x) K_s + K_s (x) I + K_s (x) K_s + h.c.] (Appendix A,
    triangular lattice) on an L1 x L2 torus."""
    if L2 is None:
        L2 = L1
    K1, K2 = shift_matrix(L1), shift_matrix(L2)
    I1, I2 = np.eye(L1), np.eye(L2)
    X = np.kron(I1, K2) + np.kron(K1, I2) + np.kron(K1, K2)
    return -t * (X + X.T)


def honeycomb_kinetic(L1, L2=None, t=1.0):
    """K = -t [(I (x) I + I (x) K_s + K_s (x) I) (x) delta + h.c.] (Appendix A,
    honeycomb lattice), delta the 2 x 2 matrix with its single one at (2, 1):
    sublattice B <- A."""
    if L2 is None:
        L2 = L1
    K1, K2 = shift_matrix(L1), shift_matrix(L2)
    I1, I2 = np.eye(L1), np.eye(L2)
    delta = np.zeros((2, 2))
    delta[1, 0] = 1.0
    X = np.kron(np.kron(I1, I2) + np.kron(I1, K2) + np.kron(K1, I2), delta)
    return -t * (X + X.T)


def kinetic(lattice, L1, L2=None, t=1.0):
    if lattice == "triangular":
        return triangular_kinetic(L1, L2, t)
    if lattice == "honeycomb":
        return honeycomb_kinetic(L1, L2, t)
    raise ValueError(f"unknown lattice {lattice!r}")


def site_positions(lattice, L1, L2=None):
    if L2 is None:
        L2 = L1
    if lattice == "triangular":
        a1, a2, tau = TRI_A1, TRI_A2, np.zeros((1, 2))
    elif lattice == "honeycomb":
        a1, a2, tau = HON_A1, HON_A2, HON_TAU
    else:
        raise ValueError(f"unknown lattice {lattice!r}")
    n = len(tau)
    r = np.zeros((n * L1 * L2, 2))
    for x1 in range(L1):
        for x2 in range(L2):
            for a in range(n):
                r[(x1 * L2 + x2) * n + a] = x1 * a1 + x2 * a2 + tau[a]
    return r, a1, a2


def kinetic_from_geometry(lattice, L1, L2=None, t=1.0, tol=1e-9):
    """-t times the number of torus images at which two sites sit at the
    nearest-neighbour distance (1 triangular, 1/sqrt 3 honeycomb)."""
    if L2 is None:
        L2 = L1
    r, a1, a2 = site_positions(lattice, L1, L2)
    dnn = 1.0 if lattice == "triangular" else 1.0 / np.sqrt(3.0)
    N = len(r)
    K = np.zeros((N, N))
    images = [n1 * L1 * a1 + n2 * L2 * a2 for n1 in (-1, 0, 1) for n2 in (-1, 0, 1)]
    for i in range(N):
        for j in range(N):
            if i == j:
                continue
            d = r[j] - r[i]
            cnt = sum(1 for im in images if abs(np.linalg.norm(d + im) - dnn) < tol)
            K[i, j] = -t * cnt
    return K


def triangular_band(k1, k2, t=1.0):
    """Textbook triangular band: -2t (cos k1 + cos k2 + cos(k1 + k2))."""
    return -2.0 * t * (np.cos(k1) + np.cos(k2) + np.cos(k1 + k2))


def honeycomb_bands(k1, k2, t=1.0):
    """Textbook honeycomb bands: +-t |1 + e^{i k1} + e^{i k2}|."""
    f = abs(1.0 + np.exp(1j * k1) + np.exp(1j * k2))
    return np.array([-t * f, t * f])
