"""Pins of the oracle's estimator conventions and error analysis.

The CDW field of Sec. IV carries the sublattice phases 1, w, w^2 (w = e^{2 pi
i/3}) on A, B, C and the phase e^{iQ.R} of the cell position R. The pins use
classical charge patterns: for a diagonal G with entries 0 or 1 every site is
empty or doubly occupied, <n_x n_y> factorises into n_x n_y, and
<phi^+ phi>(Q) = |(1/N) sum_x e^{iQ.R_x} w^{a_x} n_x|^2 is a sum that can be
done by hand. The jackknife pins use cases with a closed-form error: a linear
function (the textbook standard error of the mean), an exactly proportional
ratio (zero error) and nearly deterministic samples (first-order error
propagation).
"""

import math

import numpy as np
import pytest

from oracle import lattice, measure

L3_SITES = 27  # L = 3: N = 3 L^2


def classical_green(occupied):
    """Diagonal G for a charge pattern: G_xx = 0 on doubly occupied sites,
    1 on empty ones (G_ij = <c_i c_j^+> of one spin species)."""
    return np.diag(np.where(occupied, 0.0, 1.0))


def sqrt3_pattern(L=3):
    """One doubly occupied site per cell, sublattice a = (x2 - x1) mod 3.
    At K = (1, 2) every occupied site has Q.R + 2 pi a/3 = 2 pi (x1 + 2 x2 +
    x2 - x1)/3 = 2 pi x2, a multiple of 2 pi: the pattern is the
    sqrt3 x sqrt3 order locked to the Dirac point that Sec. IV probes."""
    occ = np.zeros(3 * L * L, dtype=bool)
    for x1 in range(L):
        for x2 in range(L):
            occ[(x1 * L + x2) * 3 + (x2 - x1) % 3] = True
    return occ


def test_dirac_point_of_the_three_cell_torus():
    # the K point of the L = 3 mesh is the reduced momentum (1, 2): the two
    # dispersive bands touch at -t there (textbook kagome bands)
    assert lattice.dirac_point(3) == (1, 2)
    e = lattice.kagome_bands(2 * np.pi / 3, 4 * np.pi / 3)
    assert np.allclose(e[:2], [-1.0, -1.0])


def test_cdw_correlator_of_the_sqrt3_pattern_by_hand():
    """Hand values for the sqrt3 x sqrt3 pattern on the L = 3 torus (N = 27,
    9 doubly occupied sites, n = 2 each):
      phi(K)     = (1/27) * 9 * 2 * 1            -> <phi^+ phi>(K) = (2/3)^2 = 4/9
      phi(Gamma) = (2/27) * 3 (1 + w + w^2) = 0  -> 0
      phi(K')    at K' = (2, 1): phases 2 pi (2 x1 + x2 + x2 - x1)/3 sum to 0 -> 0."""
    occ = sqrt3_pattern()
    G = classical_green(occ)
    wK = measure.cdw_weights(3, 3, 1, 2)
    wG = measure.cdw_weights(3, 3, 0, 0)
    wK2 = measure.cdw_weights(3, 3, 2, 1)
    assert measure.cdw_correlator(G, wK) == pytest.approx(4.0 / 9.0, abs=1e-14)
    assert measure.cdw_correlator(G, wG) == pytest.approx(0.0, abs=1e-14)
    assert measure.cdw_correlator(G, wK2) == pytest.approx(0.0, abs=1e-14)
    # the estimator the chain reports uses the same K
    obs = measure.Observables(3, site_offsets=True)
    got = obs(G)
    assert got["phi2_K"] == pytest.approx(4.0 / 9.0, abs=1e-14)
    assert got["phi2_G"] == pytest.approx(0.0, abs=1e-14)


def test_cdw_correlator_of_one_sublattice_by_hand():
    """All A sites doubly occupied, B and C empty: phi(Gamma) = (1/27) * 9 * 2
    = 2/3 (sublattice phase 1), phi(K) = 0 (the cell phases sum to zero)."""
    occ = np.zeros(L3_SITES, dtype=bool)
    occ[0::3] = True
    G = classical_green(occ)
    assert measure.cdw_correlator(G, measure.cdw_weights(3, 3, 0, 0)) == pytest.approx(4.0 / 9.0, abs=1e-14)
    assert measure.cdw_correlator(G, measure.cdw_weights(3, 3, 1, 2)) == pytest.approx(0.0, abs=1e-14)
    # B only: phi(Gamma) = (2/3) w, the same modulus
    occ = np.zeros(L3_SITES, dtype=bool)
    occ[1::3] = True
    assert measure.cdw_correlator(classical_green(occ), measure.cdw_weights(3, 3, 0, 0)) == \
        pytest.approx(4.0 / 9.0, abs=1e-14)


def test_cdw_correlator_of_the_uniform_half_filled_state():
    """G = I/2 (no correlations, one particle per site on average):
    <n_x n_y> = 1 for x != y and 3/2 on the diagonal, the sublattice phases
    sum to zero in every cell, so <phi^+ phi>(Gamma) = (1/N^2) (1/2) N = 1/(2N)."""
    N = L3_SITES
    G = 0.5 * np.eye(N)
    assert measure.cdw_correlator(G, measure.cdw_weights(3, 3, 0, 0)) == pytest.approx(1.0 / (2 * N), abs=1e-15)


def test_planted_phase_mistakes_fail_the_hand_values(monkeypatch):
    """Plausible mistakes in the CDW phases: conjugated sublattice phases
    (A, B, C -> 1, w^2, w), site positions R + tau_a in place of cell
    positions, and the sublattice phases dropped. Each changes the value of
    the sqrt3 x sqrt3 pattern at K."""
    G = classical_green(sqrt3_pattern())
    good = measure.cdw_correlator(G, measure.cdw_weights(3, 3, 1, 2))
    assert good == pytest.approx(4.0 / 9.0, abs=1e-14)

    def conj_sub(L1, L2, m1, m2):
        return lattice.momentum_phase(m1, m2, L1, L2, with_offsets=False) * \
            np.tile(np.conj(measure.OMEGA ** np.arange(3)), L1 * L2)

    def site_pos(L1, L2, m1, m2):
        return lattice.momentum_phase(m1, m2, L1, L2, with_offsets=True) * \
            np.tile(measure.OMEGA ** np.arange(3), L1 * L2)

    def no_sub(L1, L2, m1, m2):
        return lattice.momentum_phase(m1, m2, L1, L2, with_offsets=False)

    for bad in (conj_sub, site_pos, no_sub):
        monkeypatch.setattr(measure, "cdw_weights", bad)
        v = measure.cdw_correlator(G, measure.cdw_weights(3, 3, 1, 2))
        monkeypatch.undo()
        assert abs(v - 4.0 / 9.0) > 1e-3, bad.__name__


# ---------------------------------------------------------------- derived quantities (Sec. III)
def test_correlation_ratio_vanishes_without_pair_correlations():
    """Sec. III: R_Pair -> 0 when there is no pairing order. For G = I/2
    (infinite temperature) the pair correlation is purely local, S_Pair(Q) =
    1/2 at every Q, so R_Pair = 0 exactly and P = sqrt(1/(2N))."""
    L = 4
    N = 3 * L * L
    obs = measure.Observables(L)
    got = obs(0.5 * np.eye(N))
    assert got["S_pair_G"] == pytest.approx(0.5, abs=1e-14)
    assert got["S_pair_dk"] == pytest.approx(0.5, abs=1e-14)
    d = measure.derived(got["S_pair_G"], got["S_pair_dk"], got["phi2_G"], got["phi2_K"], N)
    assert d["R_pair"] == pytest.approx(0.0, abs=1e-14)
    assert d["P"] == pytest.approx(math.sqrt(1.0 / (2 * N)), rel=1e-14)
    assert math.isnan(d["D_K"])  # 3 does not divide L = 4: no K point


# ---------------------------------------------------------------- jackknife
def test_jackknife_of_a_linear_function_is_the_standard_error():
    """For fn linear, every delete-one estimate is a linear function of the
    sample, and the jackknife error equals |a| s / sqrt(n) exactly (s the
    sample standard deviation)."""
    rng = np.random.default_rng(5)
    x = rng.normal(3.0, 2.0, size=37)
    a, b = -2.5, 7.0
    est, err = measure.jackknife(x[:, None], lambda m: a * m[0] + b)
    assert est == pytest.approx(a * x.mean() + b, rel=1e-14)
    assert err == pytest.approx(abs(a) * x.std(ddof=1) / math.sqrt(len(x)), rel=1e-12)


def test_jackknife_of_an_exact_ratio_has_no_error():
    """Samples with S_dk = c S_G exactly: every delete-one ratio is c, so
    R_Pair = 1 - c with zero jackknife error."""
    rng = np.random.default_rng(6)
    sg = rng.uniform(1.0, 2.0, size=20)
    c = 0.3
    smp = np.stack([sg, c * sg], axis=1)
    est, err = measure.jackknife(smp, lambda m: 1.0 - m[1] / m[0])
    assert est == pytest.approx(1.0 - c, abs=1e-14)
    assert err < 1e-14


def test_jackknife_matches_first_order_error_propagation():
    """Nearly deterministic samples (relative spread 1e-7): the jackknife
    error of f(mean) equals the delta-method error sqrt(grad^T C grad / n) to
    O(spread), for R = 1 - y/x and P = sqrt(x / N)."""
    rng = np.random.default_rng(7)
    n, N = 400, 48
    x0, y0, eps = 1.7, 0.4, 1e-7
    z = rng.normal(size=(n, 2))
    smp = np.stack([x0 * (1 + eps * z[:, 0]), y0 * (1 + eps * (0.6 * z[:, 0] + 0.8 * z[:, 1]))], axis=1)
    C = np.cov(smp.T, ddof=1)
    mx, my = smp.mean(axis=0)
    g_r = np.array([my / mx ** 2, -1.0 / mx])
    g_p = np.array([0.5 / math.sqrt(mx * N), 0.0])
    _, er = measure.jackknife(smp, lambda m: 1.0 - m[1] / m[0])
    _, ep = measure.jackknife(smp, lambda m: math.sqrt(m[0] / N))
    assert er == pytest.approx(math.sqrt(g_r @ C @ g_r / n), rel=1e-5)
    assert ep == pytest.approx(math.sqrt(g_p @ C @ g_p / n), rel=1e-5)
