"""Pins of the projector (zero-temperature) oracle, ``oracle.pqmc`` (CPU only).

Each pin ties the oracle to something outside itself: the spectrum of K (the
trial state), the exact Fock-space projection with the Slater determinant of
the trial orbitals (the sum over all Hubbard-Stratonovich fields), exact
diagonalisation in the fixed-particle-number sector (the projection limit),
the U = 0 closed form, the unstabilised formula, and the exact field
distribution (the Markov chain). A planted-mistake test checks that these pins
catch plausible errors."""

import math

import numpy as np
import pytest
import scipy.stats as sst

from oracle import fock, measure, model, pqmc
from dqmc_inputs import random_field

OBS = [k for k in measure.Observables.NAMES if k != "phi2_K"]


# ---------------------------------------------------------------- trial state
def test_trial_state_splits_the_dirac_shell_at_two_thirds_filling():
    """At rho = 2/3 with 3 | L the N_occ-th level of K is the Dirac point -t,
    degenerate with the level above; the sublattice term splits it. P spans the
    lowest N_occ eigenvectors of K + eps diag(1, 0, -1)."""
    m = model.Model(3, 2.0, 0.1, -4.0, -1.0)
    n = m.N // 3
    w = np.linalg.eigvalsh(m.K)
    assert abs(w[n - 1] + 1.0) < 1e-12 and abs(w[n] + 1.0) < 1e-12
    with pytest.raises(ValueError):
        pqmc.trial_state(m, n, eps=0.0)
    P = pqmc.trial_state(m, n)
    assert 2 * n / m.N == pytest.approx(2.0 / 3.0)
    assert np.max(np.abs(P.T @ P - np.eye(n))) < 1e-12
    Kp = m.K + 1e-4 * np.diag(np.tile([1.0, 0.0, -1.0], m.N // 3))
    wp, Vp = np.linalg.eigh(Kp)
    # same subspace as the lowest n eigenvectors: projectors agree
    assert np.max(np.abs(P @ P.T - Vp[:, :n] @ Vp[:, :n].T)) < 1e-10
    # the occupied energy stays within O(eps) of the lowest band of K
    assert abs(np.sum(wp[:n]) - np.sum(w[:n])) < 1e-3


def test_trial_state_at_a_closed_shell_is_an_eigenbasis_of_k():
    """L = 4 (3 does not divide L): at rho = 2/3 the lowest band is a closed
    shell of K itself, and eps = 0 gives exact eigenvectors."""
    m = model.Model(4, 2.0, 0.1, -4.0, -1.0)
    n = m.N // 3
    P = pqmc.trial_state(m, n, eps=0.0)
    KP = m.K @ P
    assert np.max(np.abs(KP - P @ (P.T @ KP))) < 1e-12


# ---------------------------------------------------------------- exact projection
@pytest.mark.parametrize("M", [2, 3, 4])
def test_hs_sum_equals_fock_projection_three_sites(M):
    """Sum over all 2^{3M} fields of prod e^{-lambda s} det(L R)^2 times the
    Wick estimators of G = I - R (L R)^{-1} L equals
    <Psi_T| X^{M-l} O X^l |Psi_T> / <Psi_T| X^M |Psi_T> in Fock space, at the
    first, middle and last slice (rho = 2/3: one particle per spin)."""
    m = model.Model(1, 0.1 * M, 0.1, -4.0, -1.0)
    P = pqmc.trial_state(m, 1, eps=0.0)
    sec = fock.Sectors(m)
    for l in sorted({0, M // 2, M}):
        bf, _ = pqmc.brute_force(m, P, l, with_green=True)
        fk, _ = sec.pqmc(P, l, with_green=True)
        for k in OBS:
            assert abs(bf[k] - fk[k]) < 1e-12 * max(1.0, abs(fk[k])), (l, k)
        assert np.max(np.abs(bf["G"] - fk["G"])) < 1e-12


def test_hs_sum_equals_fock_projection_six_sites():
    """Rectangular 2 x 1-cell torus (6 sites), two particles per spin, M = 2."""
    m = model.Model(2, 0.2, 0.1, -3.0, -1.0, L2=1)
    P = pqmc.trial_state(m, 2)
    bf, _ = pqmc.brute_force(m, P, 1, with_green=True)
    fk, _ = fock.Sectors(m).pqmc(P, 1, with_green=True)
    for k in OBS:
        assert abs(bf[k] - fk[k]) < 1e-11 * max(1.0, abs(fk[k])), k
    assert np.max(np.abs(bf["G"] - fk["G"])) < 1e-11


def test_projection_converges_to_the_ed_ground_state_as_dtau_squared():
    """Three sites, one particle per spin, U = -4: the projected averages at
    the middle slice approach the exact ground state of the (1, 1) sector as
    beta grows, and the remaining Trotter error falls as dtau^2."""
    errs = []
    for beta, dtau in ((12.0, 0.1), (12.0, 0.05), (12.0, 0.025), (16.0, 0.025)):
        m = model.Model(1, beta, dtau, -4.0, -1.0)
        P = pqmc.trial_state(m, 1, eps=0.0)
        sec = fock.Sectors(m)
        gs, _ = sec.ground(1)
        pj, _ = sec.pqmc(P, m.M // 2)
        errs.append(max(abs(pj[k] - gs[k]) for k in ("S_pair_G", "ekin", "density")))
    # projection converged (beta 12 -> 16 changes nothing), Trotter error ~ dtau^2
    assert abs(errs[3] - errs[2]) < 1e-9
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs
    assert errs[2] < 3e-3


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("L,n", [(2, 1), (4, 16)])
def test_u0_green_is_the_trial_projector(L, n):
    """At U = 0 (lambda = 0) span(P) is invariant under e^{-dtau K} when P is
    an eigenbasis of K, so G(tau) = I - P P^T at every slice."""
    m = model.Model(L, 3.0, 0.1, 0.0, -1.0)
    P = pqmc.trial_state(m, n, eps=0.0)
    f = random_field(m.M, m.N, seed=3)
    ref = np.eye(m.N) - P @ P.T
    for l in (0, 7, m.M):
        assert np.max(np.abs(pqmc.green_stable(m, P, f, l) - ref)) < 1e-12


def test_stabilised_green_matches_unstabilised_small_beta():
    m = model.Model(3, 2.0, 0.1, -4.0, -1.0)
    P = pqmc.trial_state(m, m.N // 3)
    f = random_field(m.M, m.N, seed=1)
    for l in (0, 1, 10, 19, 20):
        assert np.max(np.abs(pqmc.green_stable(m, P, f, l) - pqmc.green_direct(m, P, f, l))) < 1e-11


# ---------------------------------------------------------------- the chain
def test_sherman_morrison_matches_scratch_for_the_projector_green():
    """Forced flips through the chain's rank-one update reproduce the
    from-scratch projector G of the flipped field."""
    ch = pqmc.PQMCChain(2, 1.0, 0.1, -4.0, -1.0, seed=5, n_occ=4, n_stab=5)
    l = 3
    for m_ in range(1, l + 1):
        ch.G = ch.model.B(ch.field[m_ - 1]) @ ch.G @ ch.model.Binv(ch.field[m_ - 1])
    forced = np.zeros(ch.N, dtype=bool)
    forced[[0, 5, 7]] = True
    ch.update_slice(l, 0, forced)
    assert np.max(np.abs(ch.G - pqmc.green_stable(ch.model, ch.P, ch.field, l))) < 1e-11


def test_chain_refresh_agrees_with_running_green():
    ch = pqmc.PQMCChain(2, 2.0, 0.1, -4.0, -1.0, seed=3, n_occ=4, n_stab=5)
    ch.run(3)
    assert ch.max_drift < 1e-10
    assert np.max(np.abs(ch.G - ch.green_fresh(ch.slice))) < 1e-10


def test_chain_measures_at_the_middle_checkpoint():
    ch = pqmc.PQMCChain(1, 1.0, 0.1, -4.0, -1.0, seed=1, n_occ=1, n_stab=3)
    assert ch.tau[ch.c_meas] in (4, 6) and abs(ch.tau[ch.c_meas] - ch.M / 2) <= 1
    ch.run(2, measure_obs=True)
    assert len(ch.samples) == 2


def test_markov_chain_samples_exact_field_distribution():
    """N = 3, M = 2: 64 fields; the field histogram after each sweep matches
    the exact normalised weights prod e^{-lambda s} det(L R)^2 (chi^2)."""
    ch = pqmc.PQMCChain(1, 0.2, 0.1, -4.0, -1.0, seed=7, n_occ=1, n_stab=1, eps=0.0)
    probs = pqmc.field_weights(ch.model, ch.P)
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


def test_mc_means_match_the_exact_projection_within_errors():
    ch = pqmc.PQMCChain(1, 0.4, 0.1, -4.0, -1.0, seed=11, n_occ=1, n_stab=2, eps=0.0)
    ref, _ = fock.Sectors(ch.model).pqmc(ch.P, ch.tau[ch.c_meas])
    ch.run(100)
    ch.samples = []
    ch.run(3000, measure_obs=True)
    b = ch.bins(50)
    for j, k in enumerate(measure.Observables.NAMES):
        if k == "phi2_K":
            continue
        mean, err = b[:, j].mean(), b[:, j].std(ddof=1) / math.sqrt(len(b))
        assert abs(mean - ref[k]) < 5.0 * err + 1e-12, (k, mean, ref[k], err)


# ---------------------------------------------------------------- planted mistakes
def test_planted_mistakes_are_caught(monkeypatch):
    """Each plausible slip in the oracle is caught by one of the pins above."""
    m = model.Model(1, 0.3, 0.1, -4.0, -1.0)
    P = pqmc.trial_state(m, 1, eps=0.0)
    sec = fock.Sectors(m)
    fk, _ = sec.pqmc(P, 1, with_green=True)

    def pinned_ok():
        bf, _ = pqmc.brute_force(m, P, 1, with_green=True)
        return np.max(np.abs(bf["G"] - fk["G"])) < 1e-12 and all(
            abs(bf[k] - fk[k]) < 1e-12 * max(1.0, abs(fk[k])) for k in OBS)

    assert pinned_ok()
    # 1. weight det(L R) instead of det(L R)^2 (one spin species dropped)
    orig_lw = pqmc.log_weight
    monkeypatch.setattr(pqmc, "log_weight",
                        lambda mm, PP, f: mm.log_boson_weight(f) + np.linalg.slogdet(
                            PP.T @ np.linalg.multi_dot([mm.B(f[k]) for k in range(mm.M - 1, -1, -1)] + [PP]))[1])
    assert not pinned_ok()
    monkeypatch.setattr(pqmc, "log_weight", orig_lw)
    # 2. G = R (L R)^{-1} L instead of I - R (L R)^{-1} L
    orig_gd = pqmc.green_direct
    monkeypatch.setattr(pqmc, "green_direct", lambda mm, PP, f, l: np.eye(mm.N) - orig_gd(mm, PP, f, l))
    assert not pinned_ok()
    monkeypatch.setattr(pqmc, "green_direct", orig_gd)
    # 3. left stack built with B instead of B^T: the stabilised G leaves the direct one
    f = random_field(m.M, m.N, seed=2)
    good = np.max(np.abs(pqmc.green_stable(m, P, f, 1) - pqmc.green_direct(m, P, f, 1)))
    orig_lb = pqmc.left_basis

    def wrong_left(mm, PP, ff, l):
        s = pqmc.OrthStack(PP)
        for k in range(mm.M, l, -1):
            s.left_multiply(mm.B(ff[k - 1]))
        return s

    monkeypatch.setattr(pqmc, "left_basis", wrong_left)
    bad = np.max(np.abs(pqmc.green_stable(m, P, f, 1) - pqmc.green_direct(m, P, f, 1)))
    monkeypatch.setattr(pqmc, "left_basis", orig_lb)
    assert good < 1e-12 and bad > 1e-6
