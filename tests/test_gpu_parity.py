"""GPU parity of every hot-path step against the FP64 CPU oracle, through the C ABI.

Tolerances: FP64 kernels 1e-12 (single steps) and 1e-10 (whole sweeps /
from-scratch G), the bar the FP64 path is held to; FP32 propagation 2e-6
relative to max|Y| (a few FP32 roundings through log2(L^2) butterfly stages);
mixed-precision sweeps max |G_wrapped - G_fresh| <= 1e-6.
"""

import numpy as np
import pytest

from dqmc_inputs import random_field, random_green_like, random_matrix
from oracle import dqmc as odqmc
from oracle import green as ogreen
from oracle import lattice as olat
from oracle import measure as omeas
from oracle import model as omodel
from oracle import philox as ophilox

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import build_library
    build_library()
    import paper_2608_03894_gb300 as p
    return p


def dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


# ------------------------------------------------------------------ Eq. 5-6 propagation
@pytest.mark.parametrize("L", [1, 2, 3, 4, 6, 8, 12, 16, 24, 36])
@pytest.mark.parametrize("side", [0, 1])
def test_propagate_f64_matches_dense_exponential(pkg, L, side):
    N = 3 * L * L
    nvec = 37 if L > 2 else 5          # ragged against every tile width
    scale = -0.1 if side == 0 else 0.1
    X = random_matrix(N, nvec, seed=L) if side == 0 else random_matrix(nvec, N, seed=L)
    rng = np.random.default_rng(100 + L)
    pre, post = rng.uniform(0.5, 2.0, N), rng.uniform(0.5, 2.0, N)
    vs = rng.uniform(0.5, 2.0, nvec)
    E = olat.expm_hermitian(olat.kinetic_matrix(L), scale)
    if side == 0:
        ref = (post[:, None] * (E @ (pre[:, None] * X))) * vs[None, :]
    else:
        ref = vs[:, None] * (((X * pre[None, :]) @ E) * post[None, :])
    Y = pkg.ops.propagate(L, scale, side, dev(X), pre=dev(pre), post=dev(post), vscale=dev(vs))
    err = np.max(np.abs(Y.cpu().numpy() - ref))
    assert err < 1e-12 * max(1.0, np.max(np.abs(ref))), err


@pytest.mark.parametrize("L", [1, 2, 3, 4, 6, 8, 12, 16, 24, 36])
@pytest.mark.parametrize("side", [0, 1])
def test_propagate_double_float_matches_dense_exponential(pkg, L, side):
    """FP64 data, double-float arithmetic (FP32 pairs, ~2^-47 per operation):
    within 1e-13 of max |Y| after the log2(L^2) butterfly stages both ways."""
    N = 3 * L * L
    nvec = 37 if L > 2 else 5
    scale = -0.1 if side == 0 else 0.1
    X = random_matrix(N, nvec, seed=L) if side == 0 else random_matrix(nvec, N, seed=L)
    rng = np.random.default_rng(200 + L)
    pre, post = rng.uniform(0.5, 2.0, N), rng.uniform(0.5, 2.0, N)
    vs = rng.uniform(0.5, 2.0, nvec)
    E = olat.expm_hermitian(olat.kinetic_matrix(L), scale)
    if side == 0:
        ref = (post[:, None] * (E @ (pre[:, None] * X))) * vs[None, :]
    else:
        ref = vs[:, None] * (((X * pre[None, :]) @ E) * post[None, :])
    Y = pkg.ops.propagate(L, scale, side, dev(X), pre=dev(pre), post=dev(post), vscale=dev(vs), df=True)
    err = np.max(np.abs(Y.cpu().numpy() - ref))
    assert err < 1e-13 * max(1.0, np.max(np.abs(ref))), err


@pytest.mark.parametrize("L", [4, 12, 24, 36])
def test_propagate_f32(pkg, L):
    N = 3 * L * L
    X = random_matrix(N, 40, seed=7)
    E = olat.expm_hermitian(olat.kinetic_matrix(L), -0.1)
    ref = E @ X
    Y = pkg.ops.propagate(L, -0.1, 0, dev(X, torch.float32))
    err = np.max(np.abs(Y.double().cpu().numpy() - ref)) / np.max(np.abs(ref))
    assert err < 2e-6, err
    Xr = X.T.copy()
    Yr = pkg.ops.propagate(L, -0.1, 1, dev(Xr, torch.float32))
    err = np.max(np.abs(Yr.double().cpu().numpy() - Xr @ E)) / np.max(np.abs(ref))
    assert err < 2e-6, err


def test_propagate_in_place_and_identity(pkg):
    L = 6
    N = 3 * L * L
    X = dev(random_matrix(N, N, seed=3))
    Xc = X.clone()
    pkg.ops.propagate(L, -0.1, 0, X, Y=X)          # in place
    pkg.ops.propagate(L, 0.1, 0, X, Y=X)           # inverse
    assert torch.max(torch.abs(X - Xc)).item() < 1e-12
    Y = pkg.ops.propagate(L, 0.0, 1, Xc)           # e^{0} = I
    assert torch.max(torch.abs(Y - Xc)).item() < 1e-13


# ------------------------------------------------------------------ delayed update
def _oracle_slice_update(L, beta, U, G0, field, l, pas, seed, sweep):
    ch = odqmc.Chain(L, beta, 0.1, U, -1.0, seed=seed, n_stab=1000)
    ch.field = field.copy()
    ch.G = G0.copy()
    ch.sweeps_done = sweep
    ch.update_slice(l, pas)
    return ch.G, ch.field


@pytest.mark.parametrize("L,k,mode", [(2, 4, "f64"), (4, 8, "f64"), (4, 32, "f64"), (6, 64, "f64"),
                                      (6, 16, "f64"), (6, 7, "f64"), (4, 32, "df"), (6, 64, "df"),
                                      (6, 12, "df"), (4, 32, "tc"), (6, 32, "tc"), (6, 12, "tc"),
                                      (2, 5, "tc")])
def test_delayed_update_slice_matches_one_at_a_time(pkg, L, k, mode):
    """A whole slice of proposals by blocks of k (Metropolis block + rank-k
    flush) reproduces the oracle's one-at-a-time Sherman-Morrison sweep: same
    decisions from the same Philox stream, same G."""
    beta, U, seed, sweep, l, pas = 0.5, -4.0, 5, 3, 2, 1
    m = omodel.Model(L, beta, 0.1, U, -1.0)
    N = m.N
    field = random_field(m.M, N, seed=L)
    G0 = ogreen.green_direct(m, field, l)
    Gref, fref = _oracle_slice_update(L, beta, U, G0, field, l, pas, seed, sweep)

    G = dev(G0)
    s = dev(field[l - 1], torch.int8)
    for s0 in range(0, N, k):
        kb = min(k, N - s0)
        Gcol = G[:, s0:s0 + kb].contiguous()
        Grow = G[s0:s0 + kb, :].contiguous()
        g = G[s0:s0 + kb, s0:s0 + kb].contiguous()
        al, be, cnt, st = pkg.ops.metropolis_block(N, s0, kb, g, s, m.lam, seed, 0, 2 * sweep + pas, l,
                                                   df=(mode in ("df", "tc")))
        assert st == 0
        pkg.ops.flush(N, s0, kb, G, Gcol, Grow, al, be, cnt, mode=mode)
    assert np.array_equal(s.cpu().numpy(), fref[l - 1])
    assert np.max(np.abs(G.cpu().numpy() - Gref)) < (1e-12 if mode == "f64" else 1e-11)


@pytest.mark.parametrize("L,kb,site0", [(12, 32, 0), (12, 21, 100), (12, 32, 400), (24, 32, 864),
                                         (24, 9, 1719), (6, 32, 64), (36, 32, 3856)])
def test_tensor_core_flush_equals_the_fp64_flush(pkg, L, kb, site0):
    """One block's flush from the same Metropolis output (double-float block
    on a G-like matrix): the tcgen05 digit-slice flush against the FP64 flush,
    all N^2 entries, at N not a multiple of the 128-column tile and ragged
    blocks. The digit slices keep ~2^-55 of each row scale; the factors are
    formed in double-float (~2^-47), so 1e-13 absolute on |G| ~ 1."""
    N = 3 * L * L
    G0 = dev(random_green_like(N, L + kb))
    s = dev(random_field(1, N, seed=kb)[0], torch.int8)
    g = G0[site0:site0 + kb, site0:site0 + kb].contiguous()
    al, be, cnt, st = pkg.ops.metropolis_block(N, site0, kb, g, s, 0.7, 11, 0, 1, 1, df=True)
    assert st == 0 and int(cnt.item()) > 0
    Gcol = G0[:, site0:site0 + kb].contiguous()
    Grow = G0[site0:site0 + kb, :].contiguous()
    Gt, Gf = G0.clone(), G0.clone()
    pkg.ops.flush(N, site0, kb, Gt, Gcol, Grow, al, be, cnt, mode="tc")
    pkg.ops.flush(N, site0, kb, Gf, Gcol, Grow, al, be, cnt, mode="f64")
    upd = (Gf - G0).abs().max().item()
    assert upd > 1e-3  # the block changed G
    assert (Gt - Gf).abs().max().item() < 1e-13


def test_tensor_core_flush_sweeps_follow_the_double_float_flush(pkg):
    """Mixed precision at L = 12, k = 32: three sweeps with the tcgen05 flush
    and with the double-float flush give the same field and running G within
    the double-float rounding."""
    par = dict(L=12, beta=4.0, dtau=0.1, U=-4.0, mu=-1.0)
    out = []
    for tc in (1, 0):
        with pkg.DQMC(**par, seed=4, k=32, n_stab=8, precision="mixed") as d:
            d.set_option("flush_tc", tc)
            d.sweep(3)
            G, _ = d.running_green()
            out.append((d.field, G, d.stats()["max_drift"]))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.max(np.abs(out[0][1] - out[1][1])) < 1e-9
    assert out[0][2] < 1e-7


def test_forced_flips_and_fp32_flush(pkg):
    L, k = 4, 16
    m = omodel.Model(L, 0.5, 0.1, -4.0, -1.0)
    N = m.N
    field = random_field(m.M, N, seed=9)
    G0 = ogreen.green_direct(m, field, 1)
    forced = np.zeros(N, dtype=bool)
    forced[[0, 3, 5, 17, 18, 40, 47]] = True
    ch = odqmc.Chain(L, 0.5, 0.1, -4.0, -1.0, seed=1)
    ch.field, ch.G = field.copy(), G0.copy()
    ch.update_slice(1, 0, forced)
    G = dev(G0)
    G32 = dev(G0, torch.float32)
    s = dev(field[0], torch.int8)
    s32 = s.clone()
    for s0 in range(0, N, k):
        f = dev(forced[s0:s0 + k], torch.uint8)
        al, be, cnt, _ = pkg.ops.metropolis_block(N, s0, k, G[s0:s0 + k, s0:s0 + k].contiguous(), s, m.lam,
                                                  1, 0, 0, 1, forced=f)
        pkg.ops.flush(N, s0, k, G, G[:, s0:s0 + k].contiguous(), G[s0:s0 + k, :].contiguous(), al, be, cnt)
        g32 = G32[s0:s0 + k, s0:s0 + k].double().contiguous()
        al32, be32, cnt32, _ = pkg.ops.metropolis_block(N, s0, k, g32, s32, m.lam, 1, 0, 0, 1, forced=f)
        pkg.ops.flush(N, s0, k, G32, G32[:, s0:s0 + k].contiguous(), G32[s0:s0 + k, :].contiguous(),
                      al32, be32, cnt32)
    assert np.array_equal(s.cpu().numpy(), ch.field[0])
    assert np.max(np.abs(G.cpu().numpy() - ch.G)) < 1e-12
    assert np.max(np.abs(G32.double().cpu().numpy() - ch.G)) < 1e-5


# ------------------------------------------------------------------ measurement
@pytest.mark.parametrize("L,offsets", [(4, True), (6, True), (12, True), (12, False)])
def test_measure_matches_wick_estimators(pkg, L, offsets):
    N = 3 * L * L
    G = random_green_like(N, seed=L)
    obs = omeas.Observables(L, L, olat.kinetic_matrix(L), site_offsets=offsets)(G)
    got = pkg.ops.measure(L, dev(G), site_offsets=offsets)
    for key, v in obs.items():
        if np.isnan(v):
            assert np.isnan(got[key])
        else:
            assert abs(got[key] - v) < 1e-12 * max(1.0, abs(v)), key


# ------------------------------------------------------------------ whole context
@pytest.mark.parametrize("L,offsets", [(1, True), (2, True), (3, True), (3, False), (4, True), (6, False),
                                       (12, True)])
def test_full_momentum_maps_match_the_oracle(pkg, L, offsets):
    """S_Pair(Q) and <phi^+ phi>(Q) at every mesh momentum (Sec. III, IV)
    against the oracle's maps, each Q by its definition, on a G-like matrix;
    at Gamma, Gamma + dk and K they also equal the single-momentum kernel."""
    N = 3 * L * L
    G0 = random_green_like(N, 13 + L)
    S, P = pkg.ops.measure_fullq(L, dev(G0), site_offsets=offsets)
    Sref = omeas.pair_structure_factor_all(G0, L, site_offsets=offsets)
    Pref = omeas.cdw_correlator_all(G0, L)
    assert np.max(np.abs(S - Sref)) < 1e-12 * max(1.0, np.max(np.abs(Sref)))
    assert np.max(np.abs(P - Pref)) < 1e-12 * max(1.0, np.max(np.abs(Pref)))
    single = pkg.ops.measure(L, dev(G0), site_offsets=offsets)
    assert abs(S[0, 0] - single["S_pair_G"]) < 1e-12 and abs(P[0, 0] - single["phi2_G"]) < 1e-12
    assert abs(S[1 % L, 0] - single["S_pair_dk"]) < 1e-12
    if L % 3 == 0:
        assert abs(P[L // 3, 2 * L // 3] - single["phi2_K"]) < 1e-12


def test_green_from_scratch_fixed_field_L4(pkg):
    par = dict(L=4, beta=2.0, dtau=0.1, U=-4.0, mu=-1.0)
    m = omodel.Model(**par)
    f = random_field(m.M, m.N, seed=1)
    with pkg.DQMC(**par, seed=1, k=8, n_stab=10) as d:
        d.field = f
        for l in (0, 7, 10, 20):
            assert np.max(np.abs(d.green(l) - ogreen.green_udv(m, f, l))) < 1e-10


def test_green_from_scratch_fixed_field_L12(pkg):
    par = dict(L=12, beta=12.0, dtau=0.1, U=-4.0, mu=-1.0)
    m = omodel.Model(**par)
    f = random_field(m.M, m.N, seed=1)
    with pkg.DQMC(**par, seed=1, k=32, n_stab=10) as d:
        d.field = f
        for l in (0, 50):
            assert np.max(np.abs(d.green(l) - ogreen.green_udv(m, f, l))) < 1e-10


def test_block_reflector_product_options_match_the_oracle(pkg):
    """Mixed precision, L = 12, a forced-flip replay through three refreshes:
    every kernel choice for the two small products of each block reflector of
    the QR (the Gram matrix V^T V and op(T) W; 0 digit slices, 1 FP64, 2
    double-float) gives the running G of the oracle's replay, to 1e-9 with
    digit slices or FP64 and 1e-6 in double-float; the choices are live (their
    results are not all bit-identical)."""
    par = dict(L=12, beta=12.0, dtau=0.1, U=-4.0, mu=-1.0)
    m = omodel.Model(**par)
    f0 = random_field(m.M, m.N, seed=1)
    flip = np.random.default_rng(2).random((m.M, m.N)) < 0.1
    f1 = np.where(flip, -f0, f0).astype(np.int8)
    sl = 33
    ref = _oracle_replay(par, 10, f0, f1, sl)
    out = {}
    for gram, tw, tol in ((0, 0, 1e-9), (1, 0, 1e-9), (0, 1, 1e-9), (1, 1, 1e-9), (2, 2, 1e-6)):
        with pkg.DQMC(**par, seed=1, k=32, n_stab=10, precision="mixed") as d:
            d.set_option("refl_gram", gram)
            d.set_option("refl_tw", tw)
            d.field = f0
            G = d.replay(f1, sl)
        err = float(np.max(np.abs(G - ref.G)))
        print(f"refl_gram={gram} refl_tw={tw}: |G - G_oracle| {err:.2e}")
        assert err < tol
        out[(gram, tw)] = G
    assert not all(np.array_equal(out[(0, 0)], G) for G in out.values())


def test_u0_closed_form_on_gpu(pkg):
    par = dict(L=12, beta=12.0, dtau=0.1, U=0.0, mu=-1.0)
    m = omodel.Model(**par)
    with pkg.DQMC(**par, seed=3, k=32, n_stab=10) as d:
        assert np.max(np.abs(d.green(0) - m.green_free())) < 1e-10
        d.sweep(1)
        G, sl = d.running_green()
        assert sl == 0
        assert np.max(np.abs(G - m.green_free())) < 1e-10


@pytest.mark.parametrize("L,k,n_stab,beta,prec", [(4, 8, 10, 2.0, "fp64"), (6, 16, 5, 1.0, "fp64"),
                                                 (2, 4, 3, 0.7, "fp64"), (4, 8, 10, 2.0, "mixed"),
                                                 (6, 32, 5, 1.0, "mixed")])
def test_identical_field_history_20_sweeps(pkg, L, k, n_stab, beta, prec):
    """Fed the same Philox stream, the GPU chain makes exactly the oracle's
    decisions for 20 sweeps (fields bit-identical after every sweep) and its G
    stays within 1e-10 -- in FP64 and in the FP64-accurate mixed mode."""
    par = dict(L=L, beta=beta, dtau=0.1, U=-4.0, mu=-1.0)
    ref = odqmc.Chain(**par, seed=1, n_stab=n_stab)
    with pkg.DQMC(**par, seed=1, k=k, n_stab=n_stab, precision=prec) as d:
        assert np.array_equal(d.field, ref.field)
        for s in range(20):
            d.sweep(1)
            ref.sweep()
            assert np.array_equal(d.field, ref.field), f"sweep {s}"
        G, _ = d.running_green()
        assert np.max(np.abs(G - ref.G)) < 1e-10
        st = d.stats()
        assert st["accepted"] == ref.accepted and st["proposed"] == ref.proposed


def _oracle_replay(par, n_stab, f0, f1, sl):
    """The oracle's up pass to slice sl with the decisions forced towards f1:
    wraps, one-at-a-time updates, refreshes at the checkpoints before sl."""
    ch = odqmc.Chain(**par, seed=1, n_stab=n_stab, field=f0)
    m = ch.model
    c = 1
    for l in range(1, sl + 1):
        ch.G = m.B(ch.field[l - 1]) @ ch.G @ m.Binv(ch.field[l - 1])
        ch.update_slice(l, 0, forced=(ch.field[l - 1] != f1[l - 1]))
        if l == sl:
            break
        if l == ch.tau[c]:
            ch.right[c] = ch._chunk_right(ch.right[c - 1].copy(), c)
            ch._refresh(c)
            c += 1
    return ch


@pytest.mark.parametrize("L,beta,k,n_stab,prec,sl,tol", [
    (4, 2.0, 8, 10, "fp64", 13, 1e-10), (4, 2.0, 8, 10, "fp64", 20, 3e-9),
    (12, 12.0, 32, 10, "fp64", 33, 1e-10), (12, 12.0, 32, 10, "fp64", 40, 3e-9),
    (12, 12.0, 32, 10, "mixed", 33, 1e-9), (12, 12.0, 32, 10, "mixed", 40, 1e-8)])
def test_replay_matches_oracle_green(pkg, L, beta, k, n_stab, prec, sl, tol):
    """Forced flips of 10% of the sites of every slice (seeded), through the
    fast path (wraps, delayed blocks, refreshes): the running G at the slice
    equals the oracle's running G of the same replay, and both stay within the
    drift bound 1e-8 of the from-scratch G of the field. Three slices after a
    refresh the two agree to 1e-10 in FP64; at the end of a full interval each
    has accumulated its own drift (the two stabilise differently: pre-pivoted
    blocked QR here, column-pivoted QR in the oracle), hence 3e-9."""
    par = dict(L=L, beta=beta, dtau=0.1, U=-4.0, mu=-1.0)
    m = omodel.Model(**par)
    f0 = random_field(m.M, m.N, seed=1)
    flip = np.random.default_rng(2).random((m.M, m.N)) < 0.1
    f1 = np.where(flip, -f0, f0).astype(np.int8)
    with pkg.DQMC(**par, seed=1, k=k, n_stab=n_stab, precision=prec) as d:
        d.field = f0
        G = d.replay(f1, sl)
        f = d.field
        assert np.array_equal(f[:sl], f1[:sl]) and np.array_equal(f[sl:], f0[sl:])
        ref = _oracle_replay(par, n_stab, f0, f1, sl)
        assert np.array_equal(ref.field, f)
        fresh = ogreen.green_udv(m, f, sl)
        err, drift, drift_ref = (np.max(np.abs(G - ref.G)), np.max(np.abs(G - fresh)),
                                 np.max(np.abs(ref.G - fresh)))
        print(f"replay L={L} {prec} slice {sl}: |G-G_oracle| {err:.2e}, drift {drift:.2e}, "
              f"oracle drift {drift_ref:.2e}")
        assert err < tol
        assert drift < 1e-8 and drift_ref < 1e-8
        st = d.stats()
        assert st["accepted"] == int(np.count_nonzero(f0[:sl] != f1[:sl]))
        # the next sweep rebuilds the stacks from the new field (drift bar 1e-6)
        d.sweep(1)
        assert d.stats()["max_drift"] < 1e-6


def test_replay_mixed_vs_fp64_full_size_L24(pkg):
    """At the headline size (L = 24, N = 1728, M = 240, k = 32, n_stab = 8) the
    oracle's from-scratch G is out of reach of a test; there the mixed fast
    path is held to the FP64 fast path on the same replay (the FP64 path is
    oracle-pinned at L <= 12), at the slice ending the longest refresh
    interval, and to its own drift bound 1e-6."""
    par = dict(L=24, beta=24.0, dtau=0.1, U=-4.0, mu=-1.0)
    M, N = 240, 1728
    f0 = random_field(M, N, seed=1)
    flip = np.random.default_rng(2).random((M, N)) < 0.1
    f1 = np.where(flip, -f0, f0).astype(np.int8)
    out = {}
    for prec in ("fp64", "mixed"):
        with pkg.DQMC(**par, seed=1, k=32, n_stab=8, precision=prec) as d:
            d.field = f0
            out[prec] = d.replay(f1, 16)
            assert d.stats()["max_drift"] < 1e-6
    assert np.max(np.abs(out["mixed"] - out["fp64"])) < 1e-6


def test_green_from_scratch_full_size_L24_against_oracle(pkg):
    """At the headline size (L = 24, N = 1728, M = 240) the GPU's FP64
    from-scratch G at the middle slice of a random field equals the oracle's
    stabilised G (UDV chains with a QR every 8 slices, pinned against the
    per-slice chain) on every entry."""
    par = dict(L=24, beta=24.0, dtau=0.1, U=-4.0, mu=-1.0)
    m = omodel.Model(**par)
    f = random_field(m.M, m.N, seed=6)
    with pkg.DQMC(**par, seed=1, k=32, n_stab=8, precision="fp64") as d:
        d.field = f
        G = d.green(120)
    ref = ogreen.green_udv(m, f, 120, 8)
    err = float(np.max(np.abs(G - ref)))
    print(f"L=24 from-scratch G against the oracle: {err:.2e}")
    assert err < 1e-9


@pytest.mark.parametrize("k", [32, 64])
def test_largest_workload_L36_mixed_sweep_keeps_the_drift_bar(pkg, k):
    """The largest workload (L = 36, N = 3888, M = 360, n_stab = 8, mixed
    precision; k = 32 with the tensor-core flush, k = 64 with the double-float
    flush): one sweep keeps every refresh within |dG| <= 1e-6, the field stays
    +-1, and the acceptance is a proper fraction."""
    par = dict(L=36, beta=36.0, dtau=0.1, U=-4.0, mu=-1.0)
    with pkg.DQMC(**par, seed=1, k=k, n_stab=8, precision="mixed") as d:
        d.sweep(1)
        st = d.stats()
        print(f"L=36 mixed: max drift {st['max_drift']:.2e}, acceptance {st['accepted'] / st['proposed']:.3f}")
        assert 0 < st["max_drift"] <= 1e-6
        assert 0.0 < st["accepted"] / st["proposed"] < 1.0
        f = d.field
        assert f.shape == (360, 3888) and set(np.unique(f)) <= {-1, 1}


def test_batched_chains_equal_single_chains(pkg):
    """Chains of different sizes swept concurrently (own streams, one host
    thread each) make exactly the decisions they make alone."""
    params = [(4, 2.0, 0.1, -4.0, -1.0, 3), (6, 1.0, 0.1, -4.0, -1.0, 5), (4, 2.0, 0.1, -3.0, -1.0, 7)]
    with pkg.Batch(params, k=8, n_stab=5, precision="mixed") as b:
        b.sweep(3, measure=True)
        fields = [c.field for c in b.chains]
        nsamp = [c.measure()["n_samples"] for c in b.chains]
    for i, (L, beta, dtau, U, mu, seed) in enumerate(params):
        with pkg.DQMC(L, beta, dtau, U, mu, seed=seed, k=8, n_stab=5, precision="mixed", chain=i) as d:
            d.sweep(3, measure=True)
            assert np.array_equal(d.field, fields[i])
            assert d.measure()["n_samples"] == nsamp[i]


def test_autotuner_picks_the_fastest_admissible_pair(pkg):
    """dqmc_autotune at L = 4 (mixed): every candidate (k, n_stab) is timed,
    the returned pair is the fastest one within the drift bar, and a bar that
    no chain meets is reported as an error."""
    ks, ns = (4, 8, 16), (5, 10)
    r = pkg.autotune(4, 2.0, 0.1, -4.0, -1.0, seed=1, precision="mixed", ks=ks, n_stabs=ns,
                     warmup=1, sweeps=1, drift_bar=1e-6)
    assert set(r["table"]) == {(k, n) for k in ks for n in ns}
    adm = {p: t for p, t in r["table"].items() if t is not None}
    assert adm and all(t > 0 for t in adm.values())
    assert r["table"][(r["k"], r["n_stab"])] == min(adm.values()) == r["sec_per_sweep"]
    with pytest.raises(pkg.DQMCError):
        pkg.autotune(4, 2.0, 0.1, -4.0, -1.0, ks=(8,), n_stabs=(10,), drift_bar=1e-300)


@pytest.mark.parametrize("L,beta,k,n_stab,prec", [
    (1, 0.4, 4, 2, "fp64"),     # N = 3 (doubled bonds), one ragged block kb = 3 < K = 4
    (2, 0.1, 4, 1, "fp64"),     # M = 1: a single slice, refresh after every visit
    (3, 0.3, 8, 5, "fp64"),     # n_stab > M: one stack interval
    (1, 0.4, 4, 2, "mixed"),
    (3, 0.3, 8, 5, "mixed")])
def test_degenerate_sizes_match_oracle(pkg, L, beta, k, n_stab, prec):
    """Degenerate tori and intervals: identical decisions and G to the oracle."""
    par = dict(L=L, beta=beta, dtau=0.1, U=-4.0, mu=-1.0)
    ref = odqmc.Chain(**par, seed=2, n_stab=n_stab)
    with pkg.DQMC(**par, seed=2, k=k, n_stab=n_stab, precision=prec) as d:
        assert np.array_equal(d.field, ref.field)
        for s in range(5):
            d.sweep(1)
            ref.sweep()
            assert np.array_equal(d.field, ref.field), f"sweep {s}"
        G, _ = d.running_green()
        assert np.max(np.abs(G - ref.G)) < 1e-10
        m = omodel.Model(**par)
        assert np.max(np.abs(d.green(m.M) - ogreen.green_udv(m, d.field, m.M))) < 1e-10


def test_measurements_equal_oracle_samples(pkg):
    par = dict(L=4, beta=1.0, dtau=0.1, U=-4.0, mu=-1.0)
    ref = odqmc.Chain(**par, seed=2, n_stab=5)
    with pkg.DQMC(**par, seed=2, k=8, n_stab=5, bin=5) as d:
        d.sweep(10, measure=True)
        ref.run(10, measure_obs=True)
        got = d.measure()
        assert got["n_samples"] == len(ref.samples)
        for key in ("S_pair_G", "S_pair_dk", "phi2_G", "density", "ekin"):
            want = np.mean([smp[key] for smp in ref.samples])
            assert abs(got[key] - want) < 1e-10, key


def test_mixed_precision_drift_L12(pkg):
    par = dict(L=12, beta=12.0, dtau=0.1, U=-4.0, mu=-1.0)
    with pkg.DQMC(**par, seed=1, k=32, n_stab=10, precision="mixed") as d:
        d.sweep(2)
        st = d.stats()
        assert 0 < st["max_drift"] <= 1e-6, st["max_drift"]
        m = omodel.Model(**par)
        G, sl = d.running_green()
        Gf = ogreen.green_udv(m, d.field, sl)
        assert np.max(np.abs(G - Gf)) <= 1e-6


def test_plain_fp32_mode_runs_and_reports_its_drift(pkg):
    """Plain FP32 wraps and flushes are available as precision "fp32"; their
    rounding is amplified by cond(B_l) between refreshes, so the drift is far
    above FP64's. The test checks the mode runs and reports a finite drift."""
    par = dict(L=4, beta=2.0, dtau=0.1, U=-4.0, mu=-1.0)
    with pkg.DQMC(**par, seed=1, k=8, n_stab=10, precision="fp32", drift_limit=10.0) as d:
        d.sweep(1)
        drift = d.stats()["max_drift"]
        assert np.isfinite(drift) and drift > 1e-8


def test_checkpoint_resume_is_exact(pkg, tmp_path):
    par = dict(L=4, beta=1.0, dtau=0.1, U=-4.0, mu=-1.0)
    with pkg.DQMC(**par, seed=4, k=8, n_stab=5) as a:
        a.sweep(3)
        a.save(tmp_path / "ck.bin")
        a.sweep(3)
        fa = a.field
    with pkg.DQMC(**par, seed=99, k=8, n_stab=5) as b:
        b.load(tmp_path / "ck.bin")
        b.sweep(3)
        assert np.array_equal(b.field, fa)


def test_allocator_failure_reports_enomem(pkg):
    import ctypes as C
    from paper_2608_03894_gb300 import _lib
    lib = _lib.load()
    h = C.c_void_p()
    assert lib.dqmc_create(4, 1.0, 0.1, -4.0, -1.0, 1, C.byref(h)) == 0
    calls = []

    def bad_alloc(n, u):
        calls.append(n)
        return None

    a_cb, f_cb = _lib.ALLOC_FN(bad_alloc), _lib.FREE_FN(lambda p, u: None)
    assert lib.dqmc_set_allocator(h, a_cb, f_cb, None) == 0
    assert lib.dqmc_sweep(h, 1, 0) == 2  # DQMC_ENOMEM
    assert calls
    lib.dqmc_destroy(h)


# ------------------------------------------------------------------ FP64-accurate GEMM variants
@pytest.mark.parametrize("mode", ["f64", "df", "oz", "tc"])
@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
def test_gemm_variants_are_fp64_accurate(pkg, mode, ta, tb):
    """FP64 FMA, double-float and tensor-core digit-slice GEMMs against numpy
    FP64, normwise |C - C_ref| <= tol |op(A)||op(B)| + |C0|. Rows of op(A) and
    columns of op(B) carry scales over 2^+-20 (the digit slices are exact
    relative to the largest entry of each row of op(A) / column of op(B))."""
    rng = np.random.default_rng(3)
    M, N, K = 131, 77, 203                       # ragged against every tile
    opA = rng.standard_normal((M, K)) * np.exp2(rng.integers(-20, 20, size=(M, 1)))
    opB = rng.standard_normal((K, N)) * np.exp2(rng.integers(-20, 20, size=(1, N)))
    A = np.ascontiguousarray(opA.T) if ta else opA
    B = np.ascontiguousarray(opB.T) if tb else opB
    C0 = rng.standard_normal((M, N))
    ref = 0.7 * opA @ opB - 0.3 * C0
    C = dev(C0)
    pkg.ops.gemm(dev(A), dev(B), C, alpha=0.7, beta=-0.3, ta=ta, tb=tb, mode=mode)
    bound = np.abs(opA) @ np.abs(opB) + np.abs(C0)
    rel = np.max(np.abs(C.cpu().numpy() - ref) / bound)
    tol = {"f64": 1e-14, "df": 1e-13, "oz": 1e-14, "tc": 1e-14}[mode]
    assert rel < tol, rel
    # agreement with the FP64 FMA GEMM at the FP64 rounding level
    if mode != "f64":
        C64 = dev(C0)
        pkg.ops.gemm(dev(A), dev(B), C64, alpha=0.7, beta=-0.3, ta=ta, tb=tb, mode="f64")
        err = np.max(np.abs(C.cpu().numpy() - C64.cpu().numpy()) / bound)
        assert err < {"df": 1e-13, "oz": 2e-15, "tc": 2e-15}[mode], err


@pytest.mark.parametrize("M,N,K", [(1728, 1728, 1728), (64, 1664, 1664), (2, 2, 2), (130, 50, 66),
                                   (129, 49, 65)])
@pytest.mark.parametrize("ta,tb", [(False, False), (True, True), (True, False), (False, True)])
def test_tcgen05_digit_slice_gemm_matches_the_mma_sync_kernel(pkg, M, N, K, ta, tb):
    """The tcgen05 digit-slice GEMM (slicing fused into its producer, tensor-
    memory accumulators) against the mma.sync one on the stabilisation's
    shapes (square N^3 at L = 24, the skinny QR trailing update, degenerate,
    ragged against every tile and stage; odd leading dimensions take the
    mma.sync path), in every transpose combination: the two sum the same exact
    level sums, so they agree to the FP64 rounding of the final combination."""
    rng = np.random.default_rng(11)
    opA = rng.standard_normal((M, K)) * np.exp2(rng.integers(-20, 20, size=(M, 1)))
    opB = rng.standard_normal((K, N)) * np.exp2(rng.integers(-20, 20, size=(1, N)))
    A = np.ascontiguousarray(opA.T) if ta else opA
    B = np.ascontiguousarray(opB.T) if tb else opB
    C0 = rng.standard_normal((M, N))
    C1, C2 = dev(C0), dev(C0)
    pkg.ops.gemm(dev(A), dev(B), C1, alpha=0.7, beta=-0.3, ta=ta, tb=tb, mode="oz")
    pkg.ops.gemm(dev(A), dev(B), C2, alpha=0.7, beta=-0.3, ta=ta, tb=tb, mode="tc")
    bound = np.abs(opA) @ np.abs(opB) + np.abs(C0)
    assert np.max(np.abs(C1.cpu().numpy() - C2.cpu().numpy()) / bound) < 1e-15
    assert np.max(np.abs(C2.cpu().numpy() - (0.7 * opA @ opB - 0.3 * C0)) / bound) < 1e-14


def test_digit_slice_gemm_accuracy_is_relative_to_row_scale(pkg):
    """With a dynamic range along K, digit slices lose the entries far below
    the row maximum: the error is bounded by 2^-56 K max|row| max|col|, not by
    |A||B|. (This is why the stabilisation uses them only on its orthogonal-
    factor products.)"""
    rng = np.random.default_rng(5)
    M, N, K = 64, 64, 256
    A = rng.standard_normal((M, K)) * np.exp2(rng.integers(-30, 0, size=(1, K)))
    B = rng.standard_normal((K, N))
    C = pkg.ops.gemm(dev(A), dev(B), mode="oz")
    ref = A @ B
    rowmax = np.abs(A).max(axis=1, keepdims=True)
    colmax = np.abs(B).max(axis=0, keepdims=True)
    assert np.max(np.abs(C.cpu().numpy() - ref) / (rowmax * colmax)) < K * 2.0 ** -55


def test_set_field_to_the_current_state_keeps_g(pkg):
    """Setting the field the chain is already in is a no-op (the running G is
    kept bit for bit); a different field is installed and G rebuilt from it
    (equal to the oracle's from-scratch G at slice 0)."""
    par = dict(L=4, beta=2.0, dtau=0.1, U=-4.0, mu=-1.0)
    m = omodel.Model(**par)
    with pkg.DQMC(**par, seed=1, k=8, n_stab=10, precision="fp64") as d:
        d.sweep(1)
        G0, sl0 = d.running_green()
        f = d.field
        d.field = f
        G1, sl1 = d.running_green()
        assert sl0 == sl1 == 0 and np.array_equal(G0, G1)
        f2 = f.copy()
        f2[0, 0] = -f2[0, 0]
        d.field = f2
        G2, sl2 = d.running_green()
        assert sl2 == 0 and np.array_equal(d.field, f2)
        assert np.max(np.abs(G2 - ogreen.green_udv(m, f2, 0))) < 1e-10
        d.sweep(1)
        assert d.stats()["max_drift"] < 1e-6


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_single_stream_mode_is_bit_identical(pkg, prec):
    """pipeline = 0 (the next block's Metropolis on the context's own stream,
    before the flush) takes the same decisions as the two-stream pipeline and
    gives the same G bit for bit (every reduction has a fixed order). In
    mixed precision at k = 32 this is the tensor-core flush path."""
    par = dict(L=12, beta=2.0, dtau=0.1, U=-4.0, mu=-1.0)
    out = {}
    for pl in (1, 0):
        with pkg.DQMC(**par, seed=4, k=32, n_stab=10, precision=prec) as d:
            d.set_option("pipeline", pl)
            d.sweep(2)
            out[pl] = (d.field, d.running_green()[0])
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
