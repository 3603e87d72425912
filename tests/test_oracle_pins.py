"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: the paper's equations, a
textbook closed form, an independent construction, a library routine, an exact
identity in Fock space, or published known-answer vectors.
"""

import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.stats as sst

from oracle import dqmc, fock, green, lattice, measure, model, philox
from dqmc_inputs import random_field, random_matrix


# ---------------------------------------------------------------- lattice (Eq. 2-6)
@pytest.mark.parametrize("L", [1, 2, 3, 4, 5, 6])
def test_eq3_kronecker_matches_geometry(L):
    """Eq. 3 built with Kronecker products equals the kagome graph built from
    planar positions (bonds at distance 1/2 on the torus, repeated bonds add)."""
    K = lattice.kinetic_matrix(L)
    assert np.array_equal(K, lattice.kinetic_from_geometry(L))
    assert np.array_equal(K, K.T)
    assert np.all(np.diag(K) == 0)
    # coordination 4: each row sums to -4t whatever L
    assert np.allclose(K.sum(axis=1), -4.0)


def test_eq3_rectangular_six_site_cluster():
    K = lattice.kinetic_matrix(2, 1)
    assert K.shape == (6, 6)
    assert np.array_equal(K, lattice.kinetic_from_geometry(2, 1))


@pytest.mark.parametrize("L", [1, 3, 4, 6, 12])
def test_spectrum_matches_textbook_bands(L):
    """eig(K) equals the kagome bands 2t, -t(1 +- sqrt(1 + 8 c1 c2 c3)) on the
    L x L momentum mesh; trace zero; flat band degeneracy L^2 + 1."""
    K = lattice.kinetic_matrix(L)
    w = np.sort(np.linalg.eigvalsh(K))
    ref = np.sort(np.concatenate([lattice.kagome_bands(2 * np.pi * a / L, 2 * np.pi * b / L)
                                  for a in range(L) for b in range(L)]))
    assert np.max(np.abs(w - ref)) < 1e-12
    assert abs(np.trace(K)) == 0.0
    assert np.sum(np.abs(w - 2.0) < 1e-9) == (L * L + 1 if L > 1 else 2)
    assert abs(w[0] + 4.0) < 1e-12        # band bottom at Gamma


def test_gamma_point_and_dirac_point():
    e = lattice.kagome_bands(0.0, 0.0)
    assert np.allclose(e, [-4.0, 2.0, 2.0])
    assert lattice.dirac_point(12) == (4, 8)
    e = lattice.kagome_bands(2 * np.pi / 3, 4 * np.pi / 3)
    assert np.allclose(e, [-1.0, -1.0, 2.0])
    assert lattice.dirac_point(4) is None and lattice.dirac_point(16) is None


@pytest.mark.parametrize("L", [3, 4])
def test_eq2_fourier_conjugation_is_block_diagonal(L):
    K = lattice.kinetic_matrix(L)
    Lam, blocks = lattice.block_diagonal_form(K, L)
    mask = np.kron(np.eye(L * L), np.ones((3, 3)))
    assert np.max(np.abs(Lam * (1 - mask))) < 1e-12
    # every block is Hermitian and its eigenvalues are the bands at that k
    for q, b in enumerate(blocks):
        m1, m2 = divmod(q, L)
        assert np.allclose(b, b.conj().T, atol=1e-13)
        ref = lattice.kagome_bands(2 * np.pi * m1 / L, 2 * np.pi * m2 / L)
        assert np.allclose(np.sort(np.linalg.eigvalsh(b)), ref, atol=1e-12)


@pytest.mark.parametrize("L,sign", [(3, -1), (4, -1), (4, +1), (6, -1)])
def test_eq6_fft_form_equals_dense_exponential(L, sign):
    """e^{-+dtau K} M by the three steps of Eq. 6 equals the dense exponential
    to 1e-12 (the identity the paper's method rests on)."""
    K = lattice.kinetic_matrix(L)
    _, blocks = lattice.block_diagonal_form(K, L)
    X = random_matrix(3 * L * L, 11, seed=L)
    ref = lattice.expm_hermitian(K, sign * 0.1) @ X
    got = lattice.propagate_fft_form(blocks, sign * 0.1, X, L)
    assert np.max(np.abs(got - ref)) < 1e-12


def test_dense_exponential_matches_pade():
    m = model.Model(4, 1.0, 0.1, -4.0, -1.0)
    assert np.max(np.abs(sla.expm(-0.1 * m.K) - m.expK)) < 1e-13
    assert np.max(np.abs(sla.expm(0.1 * m.K) - m.expKinv)) < 1e-13


# ---------------------------------------------------------------- Philox
def test_philox_known_answer_vectors(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = philox.philox4x32_10(*r[:6])
        assert [int(x) for x in out] == r[6:]


def test_philox_uniforms_are_uniform():
    u = philox.metropolis_uniforms(seed=1, chain=0, sweep=0, pas=0, slice1=1, n_sites=200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    hist, _ = np.histogram(u, bins=100, range=(0, 1))
    chi2 = np.sum((hist - 2000.0) ** 2 / 2000.0)
    assert chi2 < sst.chi2.ppf(0.9999, 99)


def test_initial_field_is_balanced_and_seeded():
    f1 = philox.initial_field(1, 0, 20, 48)
    f2 = philox.initial_field(2, 0, 20, 48)
    assert set(np.unique(f1)) == {-1, 1}
    assert abs(f1.mean()) < 0.1
    assert not np.array_equal(f1, f2)


# ---------------------------------------------------------------- HS / Trotter (exact)
@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_hs_sum_equals_fock_trotter_three_sites(M):
    """Sum over all 2^{3M} Ising fields of prod e^{-lambda s} det(I+B...B)^2
    equals Tr[(e^{-dtau(U-mu N)} e^{-dtau K})^M] / C^{NM} in the 64-dim Fock
    space, and the weighted Wick estimators equal the Fock-space traces."""
    m = model.Model(1, 0.1 * M, 0.1, -4.0, -1.0)
    bf, W = fock.brute_force_hs(m)
    tr, Z = fock.Sectors(m).trotter()
    assert abs(Z / (m.hs_constant() ** (m.N * m.M) * W) - 1.0) < 1e-12
    for k in measure.Observables.NAMES:
        if k == "phi2_K":
            continue
        assert abs(bf[k] - tr[k]) < 1e-12 * max(1.0, abs(tr[k])), k


def test_hs_sum_equals_fock_trotter_six_sites():
    m = model.Model(2, 0.2, 0.1, -3.0, -0.5, L2=1)
    bf, W = fock.brute_force_hs(m, with_green=True)
    tr, Z = fock.Sectors(m).trotter(with_green=True)
    # the averaged one-body G pins the order of the Trotter factors in B_l
    assert np.max(np.abs(bf["G"] - tr["G"])) < 1e-12
    assert abs(Z / (m.hs_constant() ** (m.N * m.M) * W) - 1.0) < 1e-12
    for k in ("S_pair_G", "S_pair_dk", "phi2_G", "density", "ekin"):
        assert abs(bf[k] - tr[k]) < 1e-12 * max(1.0, abs(tr[k])), k


def test_trotter_converges_to_exact_diagonalisation_as_dtau_squared():
    m = model.Model(1, 1.0, 0.1, -4.0, -1.0)
    sec = fock.Sectors(m)
    ex, _, _ = sec.exact()
    errs = {}
    for M in (8, 16, 32):
        tr, _ = sec.trotter(M)
        errs[M] = {k: abs(tr[k] - ex[k]) for k in ("S_pair_G", "density", "ekin", "phi2_G")}
    for k in errs[8]:
        r1 = errs[8][k] / errs[16][k]
        r2 = errs[16][k] / errs[32][k]
        assert 3.5 < r1 < 4.5 and 3.8 < r2 < 4.2, (k, r1, r2)
    # Richardson extrapolation to dtau -> 0 lands on ED (residual O(dtau^4))
    tr32, _ = sec.trotter(32)
    tr64, _ = sec.trotter(64)
    for k in errs[8]:
        extrap = (4 * tr64[k] - tr32[k]) / 3
        assert abs(extrap - ex[k]) < 5e-6, k


def test_ed_six_site_free_limit():
    """U = 0: exact diagonalisation equals the free-fermion closed form."""
    m = model.Model(2, 1.5, 0.1, 0.0, -1.0, L2=1)
    ex, _, _ = fock.Sectors(m).exact()
    assert abs(ex["density"] - m.density_free()) < 1e-12
    assert abs(ex["ekin"] - m.ekin_free()) < 1e-12


# ---------------------------------------------------------------- G from scratch
def test_udv_matches_direct_inversion_small_beta():
    m = model.Model(4, 1.0, 0.1, -4.0, -1.0)
    f = random_field(m.M, m.N, 3)
    for l in (0, 1, 5, 10):
        for every in (1, 3):
            assert np.max(np.abs(green.green_udv(m, f, l, every) - green.green_direct(m, f, l))) < 1e-12


def test_udv_stabilisation_interval_does_not_change_g_large_beta():
    """A QR after every 8 slices (dense 8-slice products in between) gives the
    same G as a QR after every slice at beta = 24, where the unstabilised
    product is far out of reach of FP64."""
    m = model.Model(4, 24.0, 0.1, -4.0, -1.0)
    f = random_field(m.M, m.N, 4)
    for l in (0, 100, 240):
        assert np.max(np.abs(green.green_udv(m, f, l, 8) - green.green_udv(m, f, l))) < 1e-10


@pytest.mark.parametrize("L,beta", [(4, 24.0), (6, 36.0)])
def test_u0_closed_form_large_beta(L, beta):
    """U = 0: every slice propagator is e^{dtau mu} e^{-dtau K}, so the
    stabilised G must equal (1 + e^{-beta(K - mu)})^{-1} for any field."""
    m = model.Model(L, beta, 0.1, 0.0, -1.0)
    f = random_field(m.M, m.N, 5)
    G = green.green_udv(m, f, m.M // 3)
    assert np.max(np.abs(G - m.green_free())) < 1e-12


def test_u0_free_energy_and_density():
    m = model.Model(6, 10.0, 0.1, 0.0, -1.0)
    G = m.green_free()
    assert abs(measure.kinetic_energy(G, m.K) - m.ekin_free()) < 1e-12
    assert abs(measure.density(G) - m.density_free()) < 1e-12
    # Dirac filling at mu = -1: the lowest band is full, rho -> 2/3
    m2 = model.Model(6, 60.0, 0.1, 0.0, -1.0)
    assert abs(m2.density_free() - 2.0 / 3.0) < 0.02


def test_wick_estimators_equal_fock_traces_for_a_single_field():
    """For ONE field, <O> = Tr[O B_M..B_1]/Tr[B_M..B_1] in Fock space equals the
    Wick estimator of O built from G = (I + B_M...B_1)^{-1}."""
    m = model.Model(1, 0.3, 0.1, -4.0, -1.0)
    f = random_field(m.M, m.N, 9)
    sec = fock.Sectors(m)
    G = green.green_direct(m, f, 0)
    want = measure.Observables(1, 1, m.K)(G)
    # one-body operator product in Fock space: exp(V n) per spin and e^{-dtau K_hat}
    acc = {k: 0.0 for k in want}
    Ztot = 0.0
    for nu, nd in sec.sectors():
        ku, kd = sec.k[nu], sec.k[nd]
        if len(ku) == 0 or len(kd) == 0:
            continue
        E = np.kron(sla.expm(-m.dtau * ku), sla.expm(-m.dtau * kd))
        nvec = (sec.bits[nu][:, None, :] + sec.bits[nd][None, :, :]).reshape(-1, m.N)
        P = np.eye(len(E))
        for l in range(1, m.M + 1):
            v = m.lam * f[l - 1].astype(float) + m.dtau * m.mu
            P = (np.exp(nvec @ v)[:, None] * E) @ P
        Ztot += np.trace(P)
        for k, O in sec._ops(nu, nd).items():
            if O is not None:
                acc[k] += float(np.real(np.trace(O @ P)))
    for k in ("S_pair_G", "phi2_G", "density", "ekin"):
        assert abs(acc[k] / Ztot - want[k]) < 1e-12, k


# ---------------------------------------------------------------- updates and the chain
def test_sherman_morrison_matches_scratch_after_every_flip():
    ch = dqmc.Chain(2, 0.5, 0.1, -4.0, -1.0, seed=3, n_stab=5)
    m = ch.model
    l = 1
    ch.G = m.B(ch.field[0]) @ ch.G @ m.Binv(ch.field[0])
    forced = np.zeros(ch.N, dtype=bool)
    for i in range(ch.N):
        forced[:] = False
        forced[i] = True
        ch.update_slice(l, 0, forced)
        ref = green.green_direct(m, ch.field, l)
        assert np.max(np.abs(ch.G - ref)) < 1e-12


def test_delayed_rank_k_form_equals_sequential_updates():
    """Woodbury: k sequential rank-one updates equal one rank-k update
    G - G[:,S] D (I + (I-G)_SS D)^{-1} (I-G)[S,:] (the delayed form the paper
    combines with its FFT propagation)."""
    ch = dqmc.Chain(2, 0.5, 0.1, -4.0, -1.0, seed=4, n_stab=5)
    G0 = ch.G.copy()
    N = ch.N
    S = [0, 2, 3, 7, 9]
    delta = np.array([ch._delta[int(ch.field[0, i])] for i in S])
    forced = np.zeros(N, dtype=bool)
    forced[S] = True
    ch.update_slice(1, 0, forced)
    I = np.eye(N)
    D = np.diag(delta)
    Gam = D @ np.linalg.inv(np.eye(len(S)) + (I - G0)[np.ix_(S, S)] @ D)
    Gw = G0 - G0[:, S] @ Gam @ (I - G0)[S, :]
    assert np.max(np.abs(ch.G - Gw)) < 1e-12


def test_chain_refresh_agrees_with_running_green():
    ch = dqmc.Chain(4, 2.0, 0.1, -4.0, -1.0, seed=1, n_stab=10)
    ch.run(2)
    assert ch.max_drift < 1e-8
    assert np.max(np.abs(ch.G - ch.green_fresh(0))) < 1e-12
    assert 0.2 < ch.accepted / ch.proposed < 0.95


def test_markov_chain_samples_exact_field_distribution():
    """N = 3, M = 2: 64 fields. The histogram of the field after each sweep
    matches the exact normalised weights (chi^2, thinned)."""
    ch = dqmc.Chain(1, 0.2, 0.1, -4.0, -1.0, seed=7, n_stab=1)
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
    # sweeps are close to independent here; allow a factor 2 for autocorrelation
    assert chi2 < 2.0 * sst.chi2.ppf(0.999, dof), (chi2, dof)


def test_mc_means_match_brute_force_within_errors():
    ch = dqmc.Chain(1, 0.2, 0.1, -4.0, -1.0, seed=11, n_stab=1)
    bf, _ = fock.brute_force_hs(ch.model)
    ch.run(100)
    ch.samples = []
    ch.run(3000, measure_obs=True)
    b = ch.bins(50)
    for j, k in enumerate(measure.Observables.NAMES):
        if k == "phi2_K":
            continue
        mean, err = b[:, j].mean(), b[:, j].std(ddof=1) / math.sqrt(len(b))
        assert abs(mean - bf[k]) < 4.5 * err + 1e-12, (k, mean, bf[k], err)


# ---------------------------------------------------------------- planted mistakes
def test_planted_mistakes_are_caught(monkeypatch):
    """Plant plausible mistakes in the oracle and check a pin fails for each."""
    m = model.Model(1, 0.2, 0.1, -4.0, -1.0)

    def identity_holds(mm):
        bf, W = fock.brute_force_hs(mm, with_green=True)
        tr, Z = fock.Sectors(mm).trotter(with_green=True)
        okZ = abs(Z / (mm.hs_constant() ** (mm.N * mm.M) * W) - 1.0) < 1e-9
        okO = all(abs(bf[k] - tr[k]) < 1e-9 for k in ("S_pair_G", "density", "ekin", "phi2_G"))
        okG = np.max(np.abs(bf["G"] - tr["G"])) < 1e-9
        return okZ and okO and okG

    assert identity_holds(m)
    # 1) wrong sign of the bosonic factor
    monkeypatch.setattr(model.Model, "log_boson_weight", lambda self, f: self.lam * float(np.sum(f)))
    assert not identity_holds(m)
    monkeypatch.undo()
    # 2) Trotter factors in the other order, B = e^{-dtau K} e^{V}: Z and every
    #    observable commuting with the potential are blind to it; the averaged
    #    one-body G on the six-site cluster is not
    m6 = model.Model(2, 0.2, 0.1, -3.0, -0.5, L2=1)
    tr6, _ = fock.Sectors(m6).trotter(with_green=True)
    monkeypatch.setattr(model.Model, "B", lambda self, s: self.expK * self.expV(s)[None, :])
    bf6, _ = fock.brute_force_hs(m6, with_green=True)
    monkeypatch.undo()
    assert np.max(np.abs(bf6["G"] - tr6["G"])) > 1e-7
    # 3) lambda from cosh(lambda) = e^{dtau |U|} (factor 2 dropped)
    m_bad = model.Model(1, 0.2, 0.1, -4.0, -1.0)
    m_bad.lam = float(np.arccosh(np.exp(m_bad.dtau * 4.0)))
    assert not identity_holds(m_bad)
    # 4) the conventional pair structure factor <D_i^+ D_j + h.c.> in place of
    #    the symmetric definition the paper adopts (Sec. III)
    bf, _ = fock.brute_force_hs(m6)
    assert abs(bf["S_pair_G"] - tr6["S_pair_G"]) < 1e-12

    def conventional(G, phase):
        N = G.shape[0]
        X = (np.eye(N) - G.T) ** 2 + (np.eye(N) - G) ** 2
        return float(np.real(phase @ X @ phase.conj())) / N
    monkeypatch.setattr(measure, "pair_structure_factor", conventional)
    bf2, _ = fock.brute_force_hs(m6)
    monkeypatch.undo()
    assert abs(bf2["S_pair_G"] - tr6["S_pair_G"]) > 1e-6
