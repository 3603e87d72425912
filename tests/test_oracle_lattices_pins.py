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


# ---------------------------------------------------------------- the chain on other lattices
from oracle import dqmc, fock, green, measure, model  # noqa: E402

_OBS = ("S_pair_G", "S_pair_dk", "density", "ekin")


@pytest.mark.parametrize("lat,L1,L2,M", [("triangular", 2, 2, 1), ("triangular", 2, 2, 2),
                                         ("triangular", 3, 1, 2), ("honeycomb", 2, 1, 1),
                                         ("honeycomb", 1, 1, 3)])
def test_hs_sum_equals_fock_trotter(lat, L1, L2, M):
    """On the triangular and honeycomb tori the sum over all Ising fields of
    prod e^{-lambda s} det(I + B_M ... B_1)^2 reproduces the Fock-space
    Trotter trace, and its weighted Wick estimators the Fock-space averages."""
    m = model.Model(L1, 0.1 * M, 0.1, -4.0, -0.5, L2=L2, lattice=lat)
    bf, W = fock.brute_force_hs(m)
    tr, Z = fock.Sectors(m).trotter()
    assert abs(Z / (m.hs_constant() ** (m.N * m.M) * W) - 1.0) < 1e-12
    for k in _OBS:
        assert abs(bf[k] - tr[k]) < 1e-12 * max(1.0, abs(tr[k])), k
    assert np.isnan(bf["phi2_G"]) and np.isnan(tr["phi2_G"])


@pytest.mark.parametrize("lat", ["triangular", "honeycomb"])
def test_u0_closed_form_other_lattices(lat):
    m = model.Model(4, 8.0, 0.1, 0.0, -0.5, lattice=lat)
    f = np.ones((m.M, m.N), dtype=np.int8)
    for l in (0, 37, m.M):
        assert np.max(np.abs(green.green_udv(m, f, l) - m.green_free())) < 1e-10


def test_chain_samples_exact_field_distribution_honeycomb():
    """Two sites (one honeycomb cell), M = 3: 64 fields; the field histogram
    after each sweep matches the exact weights (chi^2)."""
    import scipy.stats as sst
    ch = dqmc.Chain(1, 0.3, 0.1, -4.0, -0.5, seed=7, n_stab=1, lattice="honeycomb")
    probs = fock.field_weights(ch.model)
    keys = list(probs.keys())
    index = {k: n for n, k in enumerate(keys)}
    counts = np.zeros(len(keys))
    n = 6000
    for _ in range(n):
        ch.sweep()
        counts[index[tuple(int(x) for x in ch.field.reshape(-1))]] += 1
    p = np.array([probs[k] for k in keys])
    expected = n * p
    ok = expected > 5
    chi2 = np.sum((counts[ok] - expected[ok]) ** 2 / expected[ok])
    dof = ok.sum() - 1
    assert chi2 < 2.0 * sst.chi2.ppf(0.999, dof), (chi2, dof)


def test_observables_on_other_lattices_use_their_own_geometry():
    """S_Pair phases follow the lattice's site positions: with offsets the
    honeycomb Gamma + dk phase of sublattice B differs from the cell phase by
    e^{i 2 pi (-1/3) / L}."""
    L = 3
    ph = lattices.momentum_phase("honeycomb", 1, 0, L, L, True)
    pc = lattices.momentum_phase("honeycomb", 1, 0, L, L, False)
    assert abs(ph[1] / pc[1] - np.exp(2j * np.pi * (-1.0 / 3.0) / L)) < 1e-14
    assert abs(ph[0] - pc[0]) < 1e-14
    obs = measure.Observables(L, lattice_name="triangular")
    assert obs.N == L * L and obs.w_G is None
