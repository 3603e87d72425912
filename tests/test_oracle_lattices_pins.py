"""Pins of the other composite lattices of the appendix (``oracle.lattices``,
CPU only): the Kronecker forms equal the geometric nearest-neighbour
construction, their spectra are the textbook bands, the Fourier transform
block-diagonalises them into 1 x 1 (triangular) and 2 x 2 (honeycomb) blocks,
and the three-step FFT propagator product of Eq. 6 equals the dense
exponential."""

import numpy as np
import pytest

from oracle import lattice, lattices


@pytest.mark.parametrize("lat", ["triangular", "honeycomb"])
@pytest.mark.parametrize("L1,L2", [(3, 3), (4, 4), (5, 3), (6, 6)])
def test_kronecker_form_matches_geometry(lat, L1, L2):
    K = lattices.kinetic(lat, L1, L2)
    assert np.array_equal(K, K.T)
    assert np.max(np.abs(K - lattices.kinetic_from_geometry(lat, L1, L2))) == 0.0
    coord = {"triangular": 6, "honeycomb": 3}[lat]
    assert np.allclose(-K.sum(axis=1), coord)


@pytest.mark.parametrize("L", [1, 2, 3, 4, 6, 12])
def test_triangular_spectrum_is_the_textbook_band(L):
    K = lattices.triangular_kinetic(L)
    ks = 2 * np.pi * np.arange(L) / L
    want = np.sort([lattices.triangular_band(k1, k2) for k1 in ks for k2 in ks])
    assert np.max(np.abs(np.linalg.eigvalsh(K) - want)) < 1e-12


@pytest.mark.parametrize("L", [1, 2, 3, 4, 6, 12])
def test_honeycomb_spectrum_is_the_textbook_bands(L):
    K = lattices.honeycomb_kinetic(L)
    ks = 2 * np.pi * np.arange(L) / L
    want = np.sort(np.concatenate([lattices.honeycomb_bands(k1, k2) for k1 in ks for k2 in ks]))
    assert np.max(np.abs(np.linalg.eigvalsh(K) - want)) < 1e-12
    # Dirac points on the mesh when 3 | L: zero modes, two per valley
    if L % 3 == 0:
        assert np.sum(np.abs(want) < 1e-12) == 4


@pytest.mark.parametrize("lat,n", [("triangular", 1), ("honeycomb", 2)])
@pytest.mark.parametrize("L", [3, 4])
def test_fourier_conjugation_is_block_diagonal(lat, n, L):
    K = lattices.kinetic(lat, L)
    Lam, blocks = lattice.block_diagonal_form(K, L, L, n=n)
    off = Lam.copy()
    for q in range(L * L):
        off[q * n:(q + 1) * n, q * n:(q + 1) * n] = 0.0
    assert np.max(np.abs(off)) < 1e-12
    for b in blocks:
        assert np.max(np.abs(b - b.conj().T)) < 1e-12


@pytest.mark.parametrize("lat,n", [("triangular", 1), ("honeycomb", 2)])
@pytest.mark.parametrize("L,sign", [(3, -1), (4, -1), (4, +1), (6, -1)])
def test_fft_form_equals_dense_exponential(lat, n, L, sign):
    K = lattices.kinetic(lat, L)
    N = K.shape[0]
    X = np.random.default_rng(L).standard_normal((N, 7))
    _, blocks = lattice.block_diagonal_form(K, L, L, n=n)
    got = lattice.propagate_fft_form(blocks, sign * 0.1, X, L, L, n=n)
    want = lattice.expm_hermitian(K, sign * 0.1) @ X
    assert np.max(np.abs(got - want)) < 1e-12


def test_planted_mistakes_are_caught():
    """A dropped K_s (x) K_s term (square lattice) or a wrong intra-cell entry
    fails the geometric and spectral pins."""
    L = 4
    K1 = lattice.shift_matrix(L)
    I = np.eye(L)
    X = np.kron(I, K1) + np.kron(K1, I)
    square = -(X + X.T)
    assert np.max(np.abs(square - lattices.kinetic_from_geometry("triangular", L, L))) > 0.5
    delta = np.zeros((2, 2))
    delta[0, 1] = 1.0
    Y = np.kron(np.kron(I, I) + np.kron(I, K1) + np.kron(K1.T, I), delta)
    wrong = -(Y + Y.T)
    assert np.max(np.abs(wrong - lattices.kinetic_from_geometry("honeycomb", L, L))) > 0.5
