"""Statistical parity of the GPU Markov chain, the library's error analysis,
its failure paths and its run-to-run reproducibility, through the C ABI.

* The chain's binned means agree with the exact sum over all Hubbard-
  Stratonovich fields (3 sites, 2 slices) within their error bars, and with an
  independent oracle chain (other seed) on the smallest benchmark workload
  (L = 4, beta = 2, k = 8, refresh every 10 slices) within the combined error
  bars, for the Sec. III / IV estimators and the derived R_Pair and P.
* dqmc_measure's bin errors and jackknife errors equal the oracle's on the
  same samples (loaded from a checkpoint file).
* A drift above the hard limit ends the sweep with DQMC_ENUMERIC.
* Two runs of the same chain give bit-identical G and drift (no
  order-dependent reductions in the sweep).
"""

import ctypes as C
import math
import struct

import numpy as np
import pytest

from oracle import dqmc as odqmc
from oracle import fock
from oracle import measure as omeas

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NAMES = omeas.Observables.NAMES


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import build_library
    build_library()
    import paper_2608_03894_gb300 as p
    return p


def test_chain_means_match_the_exact_hs_sum(pkg):
    """N = 3, M = 2 (64 fields): the exact HS-sum expectation values against
    the GPU chain's binned means (bins of 100 measurements), 4.5 sigma."""
    par = dict(L=1, beta=0.2, dtau=0.1, U=-4.0, mu=-1.0)
    ch = odqmc.Chain(**par, seed=5, n_stab=1)
    exact, _ = fock.brute_force_hs(ch.model)
    with pkg.DQMC(**par, seed=5, k=4, n_stab=1, bin=100, precision="fp64") as d:
        d.sweep(100)
        d.sweep(3000, measure=True)
        got = d.measure()
    assert got["n_samples"] == 6000 and got["n_bins"] == 60
    for k in NAMES:
        if k == "phi2_K":
            assert math.isnan(got[k])  # 3 does not divide L = 1
            continue
        err = got["err"][k]
        assert err > 0
        assert abs(got[k] - exact[k]) < 4.5 * err + 1e-12, (k, got[k], exact[k], err)


def test_chain_statistics_match_an_independent_oracle_chain(pkg):
    """The smallest benchmark workload (L = 4, N = 48, beta = 2, M = 20, U = -4,
    mu = -1, k = 8, refresh every 10 slices): GPU chain seed 1 against oracle
    chain seed 2, 200 warm-up + 600 measured sweeps each, bins of 20
    measurements (10 sweeps). Every estimator and the jackknifed R_Pair and P
    agree within 4 combined standard errors."""
    par = dict(L=4, beta=2.0, dtau=0.1, U=-4.0, mu=-1.0)
    ref = odqmc.Chain(**par, seed=2, n_stab=10)
    ref.run(200)
    ref.samples = []
    ref.run(600, measure_obs=True)
    b = ref.bins(20)
    with pkg.DQMC(**par, seed=1, k=8, n_stab=10, bin=20, precision="fp64") as d:
        d.sweep(200)
        d.sweep(600, measure=True)
        got = d.measure()
    assert got["n_samples"] == len(ref.samples) == 1200
    for j, k in enumerate(NAMES):
        if k == "phi2_K":
            continue
        m_ref, e_ref = b[:, j].mean(), b[:, j].std(ddof=1) / math.sqrt(len(b))
        comb = math.hypot(got["err"][k], e_ref)
        assert abs(got[k] - m_ref) < 4.0 * comb, (k, got[k], m_ref, comb)
    N = 48
    r_ref, er = omeas.jackknife(b[:, :2], lambda m: 1.0 - m[1] / m[0])
    p_ref, ep = omeas.jackknife(b[:, :1], lambda m: math.sqrt(m[0] / N))
    assert abs(got["R_pair"] - r_ref) < 4.0 * math.hypot(got["R_pair_err"], er)
    assert abs(got["P"] - p_ref) < 4.0 * math.hypot(got["P_err"], ep)


def _checkpoint(L, beta, dtau, U, mu, seed, M, N, samples, bin_, k=4, n_stab=1):
    ns = len(samples)
    return (b"DQMCGB31" + struct.pack("<5d", L, beta, dtau, U, mu) + struct.pack("<Q", seed)
            + struct.pack("<7i", k, n_stab, 0, 0, 1, bin_, 0) + struct.pack("<3q", 0, 0, 0)
            + struct.pack("<d", 0.0) + bytes([1] * (M * N)) + struct.pack("<q", ns)
            + np.ascontiguousarray(samples, dtype="<f8").tobytes())


def test_library_error_analysis_equals_the_oracle_on_the_same_samples(pkg, tmp_path):
    """Samples loaded from a checkpoint: dqmc_measure's means, bin errors and
    jackknife errors of R_Pair and P equal the oracle's on the same bins."""
    rng = np.random.default_rng(3)
    ns, bin_ = 230, 10  # 23 bins
    x = np.empty((ns, 6))
    x[:, 0] = 1.5 + 0.2 * rng.standard_normal(ns)
    x[:, 1] = 0.4 * x[:, 0] + 0.05 * rng.standard_normal(ns)
    x[:, 2:] = rng.uniform(0.1, 1.0, size=(ns, 4))
    path = tmp_path / "ck.bin"
    path.write_bytes(_checkpoint(1, 0.2, 0.1, -4.0, -1.0, 1, 2, 3, x, bin_))
    with pkg.DQMC(1, 0.2, 0.1, -4.0, -1.0, seed=1, k=4, n_stab=1) as d:
        d.load(path)
        got = d.measure()
    nb = ns // bin_
    bins = x[:nb * bin_].reshape(nb, bin_, 6).mean(axis=1)
    assert got["n_samples"] == ns and got["n_bins"] == nb
    for j, k in enumerate(NAMES):
        assert got[k] == pytest.approx(x[:, j].mean(), rel=1e-13)
        assert got["err"][k] == pytest.approx(bins[:, j].std(ddof=1) / math.sqrt(nb), rel=1e-11)
    N = 3
    r_ref, er = omeas.jackknife(bins[:, :2], lambda m: 1.0 - m[1] / m[0])
    p_ref, ep = omeas.jackknife(bins[:, :1], lambda m: math.sqrt(m[0] / N))
    d_ref = omeas.derived(x[:, 0].mean(), x[:, 1].mean(), x[:, 2].mean(), x[:, 3].mean(), N)
    assert got["R_pair"] == pytest.approx(d_ref["R_pair"], rel=1e-12)
    assert got["P"] == pytest.approx(d_ref["P"], rel=1e-12)
    assert got["R_pair_err"] == pytest.approx(er, rel=1e-10)
    assert got["P_err"] == pytest.approx(ep, rel=1e-10)
    assert got["D_G"] == pytest.approx(math.sqrt(x[:, 2].mean()), rel=1e-13)


def test_drift_above_the_hard_limit_is_a_numeric_error(pkg):
    """drift_limit below any attainable drift: the first sweep returns
    DQMC_ENUMERIC and the message names the drift; the context stays usable."""
    from paper_2608_03894_gb300 import _lib
    lib = _lib.load()
    with pkg.DQMC(4, 1.0, 0.1, -4.0, -1.0, seed=1, k=8, n_stab=5, drift_limit=1e-30) as d:
        st = lib.dqmc_sweep(d.h, 1, 0)
        assert st == 4  # DQMC_ENUMERIC
        assert "drift" in lib.dqmc_last_error().decode()
        d.set_option("drift_limit", 1e-3)
        assert lib.dqmc_sweep(d.h, 1, 0) == 0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sweeps_are_reproducible_bit_for_bit(pkg, prec):
    """The same chain run twice (L = 12, one sweep, split-K GEMMs in the
    stabilisation): identical field, running G and drift."""
    par = dict(L=12, beta=4.0, dtau=0.1, U=-4.0, mu=-1.0)
    out = []
    for _ in range(2):
        with pkg.DQMC(**par, seed=3, k=32, n_stab=8, precision=prec) as d:
            d.sweep(1)
            G, _ = d.running_green()
            out.append((d.field, G, d.stats()["max_drift"]))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]
