"""Kagome lattice for the oracle (test infrastructure; see package header).

Index order. The Kronecker form of Eq. 3 (Sec. II) puts the first cell
coordinate slowest and the sublattice fastest, so site i = (x1*L2 + x2)*3 + a
with a in {A=0, B=1, C=2}.

Two independent constructions of K are provided so that each pins the other:
``kinetic_matrix`` follows Eq. 3 term by term with numpy Kronecker products;
``kinetic_from_geometry`` places the sites in the plane and connects every
pair at nearest-neighbour distance on the torus.
"""

import numpy as np

# Bravais vectors and sublattice offsets of a kagome lattice whose bonds are
# exactly the ones Eq. 3 lists (A(x)-B(x), A(x)-B(x+e2), A(x)-C(x),
# A(x)-C(x+e1), B(x)-C(x), B(x)-C(x+e1-e2)); nearest-neighbour distance 1/2.
A1 = np.array([1.0, 0.0])
A2 = np.array([0.5, np.sqrt(3.0) / 2.0])
TAU = np.array([[0.0, 0.0], -A2 / 2.0, -A1 / 2.0])
# the same offsets in units of (A1, A2)
TAU_FRAC = np.array([[0.0, 0.0], [0.0, -0.5], [-0.5, 0.0]])


def shift_matrix(L):
    """K_s of Eq. 3: the L x L circulant one-step translation, with ones on
    the first subdiagonal and in the top-right corner, so K_s e_j = e_{j+1 mod L}.
    For L=1 the corner entry is the only one: K_s = [1]."""
    Ks = np.zeros((L, L))
    for j in range(L):
        Ks[(j + 1) % L, j] += 1.0
    return Ks


def intra_cell_matrices():
    """delta_a, delta_b, delta_c of Eq. 3: single ones at (2,1), (3,1), (3,2)
    (one-based), i.e. B<-A, C<-A, C<-B."""
    da = np.zeros((3, 3))
    db = np.zeros((3, 3))
    dc = np.zeros((3, 3))
    da[1, 0] = 1.0
    db[2, 0] = 1.0
    dc[2, 1] = 1.0
    return da, db, dc


def kinetic_matrix(L1, L2=None, t=1.0):
    """Spinless kinetic matrix K of Eq. 3 (Sec. II) on an L1 x L2-cell torus:

        K = -t [ I (x) (I + K_s) (x) d_a + (I + K_s) (x) I (x) d_b
                 + (I (x) I + K_s (x) K_s^T) (x) d_c + h.c. ]

    K_ij = -t for nearest neighbours (text under Eq. 1); a bond that the
    Kronecker form lists twice (L=1, or the 2x1 six-site cluster) adds.
    The paper writes L1 = L2 = L; the rectangular case is oracle-only."""
    if L2 is None:
        L2 = L1
    I1, I2 = np.eye(L1), np.eye(L2)
    K1, K2 = shift_matrix(L1), shift_matrix(L2)
    da, db, dc = intra_cell_matrices()
    X = (np.kron(np.kron(I1, I2 + K2), da)
         + np.kron(np.kron(I1 + K1, I2), db)
         + np.kron(np.kron(I1, I2) + np.kron(K1, K2.T), dc))
    return -t * (X + X.T)


def site_positions(L1, L2=None):
    """Planar positions r_i = x1*A1 + x2*A2 + tau_a (index order above)."""
    if L2 is None:
        L2 = L1
    r = np.zeros((3 * L1 * L2, 2))
    for x1 in range(L1):
        for x2 in range(L2):
            for a in range(3):
                r[(x1 * L2 + x2) * 3 + a] = x1 * A1 + x2 * A2 + TAU[a]
    return r


def kinetic_from_geometry(L1, L2=None, t=1.0, tol=1e-9):
    """K from geometry alone: -t times the number of torus images at which two
    sites sit at the nearest-neighbour distance 1/2. Independent of Eq. 3."""
    if L2 is None:
        L2 = L1
    r = site_positions(L1, L2)
    N = len(r)
    K = np.zeros((N, N))
    images = [n1 * L1 * A1 + n2 * L2 * A2 for n1 in (-1, 0, 1) for n2 in (-1, 0, 1)]
    for i in range(N):
        for j in range(N):
            if i == j:
                continue
            d = r[j] - r[i]
            cnt = sum(1 for im in images if abs(np.linalg.norm(d + im) - 0.5) < tol)
            K[i, j] = -t * cnt
    return K


def kagome_bands(k1, k2, t=1.0):
    """Textbook kagome bands for nearest-neighbour hopping -t, at reduced
    momentum (k1, k2) (phases e^{i k . x} with x in units of A1, A2):
    a flat band at +2t and -t (1 +/- sqrt(1 + 8 cos(k1/2) cos(k2/2) cos((k1-k2)/2)))."""
    c = np.cos(k1 / 2) * np.cos(k2 / 2) * np.cos((k1 - k2) / 2)
    root = np.sqrt(max(0.0, 1.0 + 8.0 * c))
    return np.sort(np.array([-t * (1 + root), -t * (1 - root), 2.0 * t]))


def fourier_matrix(L):
    """Unitary one-dimensional DFT matrix F_{x,m} = e^{2 pi i x m / L} / sqrt(L).
    Eq. 2 uses F^dagger on the left and Eq. 4 writes F K_s F^dagger; either
    orientation diagonalises the circulant K_s, we take this one."""
    x = np.arange(L)
    return np.exp(2j * np.pi * np.outer(x, x) / L) / np.sqrt(L)


def block_diagonal_form(K, L1, L2=None, n=3):
    """Lambda of Eq. 2: [(F^dag)^{(x)2} (x) I_n] K [F^{(x)2} (x) I_n], dense.
    Returns the full matrix (to check it is block diagonal) and the
    (L1*L2, n, n) stack of its diagonal blocks indexed by (m1*L2 + m2)."""
    if L2 is None:
        L2 = L1
    F = np.kron(np.kron(fourier_matrix(L1), fourier_matrix(L2)), np.eye(n))
    Lam = F.conj().T @ K @ F
    blocks = np.array([Lam[q * n:(q + 1) * n, q * n:(q + 1) * n] for q in range(L1 * L2)])
    return Lam, blocks


def expm_hermitian(H, scale):
    """exp(scale * H) for a Hermitian (or real symmetric) H by eigendecomposition."""
    w, V = np.linalg.eigh(H)
    return (V * np.exp(scale * w)) @ V.conj().T


def propagate_fft_form(blocks, scale, Mat, L1, L2=None, n=3):
    """exp(scale*K) @ Mat by the three steps of Eq. 6 (Sec. II): Fourier
    transform every column per sublattice, multiply each momentum's n x n block
    exp(scale*Lambda_k), transform back. numpy's fft2 is the unnormalised
    forward transform, sqrt(L1 L2) F^dagger per axis pair, and ifft2 undoes it,
    so the normalisations of Eq. 6 cancel."""
    if L2 is None:
        L2 = L1
    N = n * L1 * L2
    cols = Mat.shape[1]
    E = np.array([expm_hermitian(b, scale) for b in blocks])  # (L1*L2, n, n)
    v = Mat.reshape(L1, L2, n, cols)
    vt = np.fft.fft2(v, axes=(0, 1))                         # step 1
    vt = vt.reshape(L1 * L2, n, cols)
    wt = np.einsum('qab,qbc->qac', E, vt)                    # step 2
    w = np.fft.ifft2(wt.reshape(L1, L2, n, cols), axes=(0, 1))  # step 3
    return w.reshape(N, cols).real


def momentum_phase(m1, m2, L1, L2=None, with_offsets=True):
    """e^{i Q . r_i} for Q = m1 b1/L1 + m2 b2/L2 (b_i . A_j = 2 pi delta_ij).
    ``with_offsets`` uses site positions R + tau_a, otherwise cell positions R."""
    if L2 is None:
        L2 = L1
    ph = np.zeros(3 * L1 * L2, dtype=complex)
    for x1 in range(L1):
        for x2 in range(L2):
            for a in range(3):
                f = np.array([x1, x2], dtype=float)
                if with_offsets:
                    f = f + TAU_FRAC[a]
                ph[(x1 * L2 + x2) * 3 + a] = np.exp(2j * np.pi * (m1 * f[0] / L1 + m2 * f[1] / L2))
    return ph


def dirac_point(L, t=1.0, tol=1e-9):
    """Reduced momentum (m1, m2) of the K point: the first mesh point (in
    lexicographic order) where the two dispersive bands touch at -t. None if
    the L x L mesh has no such point (3 does not divide L)."""
    for m1 in range(L):
        for m2 in range(L):
            e = kagome_bands(2 * np.pi * m1 / L, 2 * np.pi * m2 / L, t)
            if abs(e[0] + t) < tol and abs(e[1] + t) < tol:
                return (m1, m2)
    return None
