"""Pins of the full-momentum estimators (``measure.pair_structure_factor_all``,
``measure.cdw_correlator_all``; CPU only): they reduce to the Gamma, Gamma + dk
and K estimators, obey the momentum sum rules exactly, equal the Fock-space
traces of the pair and density operators for one field, and have the
symmetries of a real G."""

import numpy as np
import pytest
from scipy.linalg import expm, logm

from oracle import fock, lattice, measure, model
from dqmc_inputs import random_field


def _green(L, beta=1.0, seed=1, U=-4.0):
    from oracle import green
    m = model.Model(L, beta, 0.1, U, -1.0)
    f = random_field(m.M, m.N, seed=seed)
    return m, green.green_udv(m, f, m.M // 2)


@pytest.mark.parametrize("L", [3, 4])
def test_full_maps_reduce_to_the_single_momentum_estimators(L):
    m, G = _green(L)
    obs = measure.Observables(L)(G)
    S = measure.pair_structure_factor_all(G, L)
    P = measure.cdw_correlator_all(G, L)
    assert abs(S[0, 0] - obs["S_pair_G"]) < 1e-13
    assert abs(S[1 % L, 0] - obs["S_pair_dk"]) < 1e-13
    assert abs(P[0, 0] - obs["phi2_G"]) < 1e-13
    kp = lattice.dirac_point(L)
    if kp is not None:
        assert abs(P[kp] - obs["phi2_K"]) < 1e-13


@pytest.mark.parametrize("L", [2, 3, 4])
def test_momentum_sum_rules(L):
    """With cell positions, sum_Q e^{iQ(R_i - R_j)} = L^2 delta_{R_i R_j}:
    sum_Q S(Q) = (L^2/N) sum over same-cell pairs of the pair correlation, and
    sum_Q <phi^+ phi>(Q) = (L^2/N^2) sum over same-cell pairs of
    conj(w_a) w_b <n_x n_y>."""
    m, G = _green(L, seed=L)
    N = m.N
    S = measure.pair_structure_factor_all(G, L, site_offsets=False)
    X = (np.eye(N) - G.T) ** 2 + G.T ** 2
    same = np.kron(np.eye(L * L), np.ones((3, 3)))
    assert abs(S.sum() - L * L / N * np.sum(X * same)) < 1e-12
    P = measure.cdw_correlator_all(G, L)
    w = np.tile(measure.OMEGA ** np.arange(3), L * L)
    C = measure.density_correlation(G) * np.outer(w.conj(), w)
    assert abs(P.sum() - L * L / N ** 2 * float(np.real(np.sum(C * same)))) < 1e-12


def test_full_maps_equal_fock_traces_for_one_field():
    """Six-site (2 x 1-cell) torus, one field: every S(Q) and <phi^+ phi>(Q)
    of the mesh equals the trace of the corresponding operator with the
    single-field density matrix."""
    m = model.Model(2, 0.2, 0.1, -4.0, -1.0, L2=1)
    field = np.array([[1, -1, 1, 1, -1, -1], [-1, 1, 1, -1, 1, -1]], dtype=np.int8)
    I = np.eye(m.N)
    Bp = I
    for l in range(1, m.M + 1):
        Bp = m.B(field[l - 1]) @ Bp
    G = np.linalg.inv(I + Bp)
    S = measure.pair_structure_factor_all(G, 2, 1)
    P = measure.cdw_correlator_all(G, 2, 1)
    sec = fock.Sectors(m)
    for m1 in range(2):
        ph = lattice.momentum_phase(m1, 0, 2, 1, True)
        w = measure.cdw_weights(2, 1, m1, 0)
        num_S = num_P = Z = 0.0
        for nu, nd in sec.sectors():
            # single-field density matrix: exp(sum_ij (log Bp)_ij c+_i c_j) per
            # species (both species see the same one-body propagator Bp)
            hu, hd = sec.h[nu], sec.h[nd]
            Lg = np.real_if_close(logm(Bp))
            Au = sum(Lg[i, j] * hu[i][j] for i in range(m.N) for j in range(m.N)) if len(sec.idx[nu]) else None
            Ad = sum(Lg[i, j] * hd[i][j] for i in range(m.N) for j in range(m.N)) if len(sec.idx[nd]) else None
            Eu = expm(Au) if Au is not None else np.zeros((0, 0))
            Ed = expm(Ad) if Ad is not None else np.zeros((0, 0))
            rho = np.kron(Eu, Ed)
            Z += np.trace(rho)
            N_ = m.N
            Iu, Id = np.eye(len(sec.idx[nu])), np.eye(len(sec.idx[nd]))
            Sop = 0.0
            for i in range(N_):
                for j in range(N_):
                    cph = ph[i] * np.conj(ph[j])
                    d = 1.0 if i == j else 0.0
                    Sop = Sop + cph * (np.kron(hu[i][j], hd[i][j]) + np.kron(d * Iu - hu[i][j], d * Id - hd[i][j]))
            num_S += np.real(np.trace(Sop @ rho)) / N_
            nvec = (sec.bits[nu][:, None, :] + sec.bits[nd][None, :, :]).reshape(-1, N_)
            phi = nvec @ w / N_
            num_P += np.real(np.trace(np.diag(np.abs(phi) ** 2) @ rho))
        assert abs(num_S / np.real(Z) - S[m1, 0]) < 1e-10, m1
        assert abs(num_P / np.real(Z) - P[m1, 0]) < 1e-10, m1


def test_pair_structure_factor_is_even_for_a_real_green_function():
    """For real G, S(-Q) = S(Q) (cell positions). The CDW map has no such
    symmetry: its sublattice phases w^a pick a chirality (K and K' differ)."""
    L = 4
    m, G = _green(L, seed=5)
    S = measure.pair_structure_factor_all(G, L, site_offsets=False)
    for m1 in range(L):
        for m2 in range(L):
            assert abs(S[m1, m2] - S[(-m1) % L, (-m2) % L]) < 1e-12
