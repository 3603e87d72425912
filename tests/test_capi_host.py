"""Host-side checks of the C ABI: the library builds, loads without a GPU,
exports every function include/dqmc.h declares, and validates arguments
before touching the device."""

import ctypes as C
import os
import re

import pytest

from conftest import ROOT, build_library


@pytest.fixture(scope="module")
def lib():
    build_library()
    from paper_2608_03894_gb300 import _lib
    return _lib.load()


def header_functions():
    txt = open(os.path.join(ROOT, "include", "dqmc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dqmc_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("dqmc_create", "dqmc_sweep", "dqmc_green", "dqmc_measure", "dqmc_destroy",
                     "dqmc_op_propagate_f64", "dqmc_op_flush_f32", "dqmc_op_metropolis_block"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol(lib):
    from paper_2608_03894_gb300 import _lib
    assert set(header_functions()) == set(_lib.SIGNATURES)


def test_version(lib):
    assert b"sm_103a" in lib.dqmc_version()


def _create(lib, L=4, beta=2.0, dtau=0.1, U=-4.0, mu=-1.0, seed=1):
    h = C.c_void_p()
    st = lib.dqmc_create(L, beta, dtau, U, mu, seed, C.byref(h))
    return st, h


@pytest.mark.parametrize("args,why", [
    (dict(U=4.0), "U"), (dict(L=5), "unsupported L"), (dict(L=0), "unsupported L"),
    (dict(beta=1.05), "integer"), (dict(dtau=0.0), "positive"), (dict(mu=float("nan")), "finite"),
])
def test_create_rejects_bad_parameters(lib, args, why):
    st, h = _create(lib, **args)
    assert st == 1  # DQMC_EINVAL
    assert why in lib.dqmc_last_error().decode()
    assert not h.value


def test_create_and_destroy_without_gpu_work(lib):
    st, h = _create(lib)
    assert st == 0 and h.value
    assert lib.dqmc_set_option(h, b"k", 16.0) == 0
    assert lib.dqmc_set_option(h, b"k", 7.0) == 1
    assert lib.dqmc_set_option(h, b"precision", 2.0) == 0
    assert lib.dqmc_set_option(h, b"precision", 3.0) == 1
    assert lib.dqmc_set_option(h, b"timing", 5.0) == 1
    assert lib.dqmc_set_option(h, b"nonsense", 1.0) == 1
    assert lib.dqmc_set_option(h, b"n_stab", 0.0) == 1
    assert lib.dqmc_set_option(h, b"drift_limit", -1.0) == 1
    assert lib.dqmc_set_option(h, None, 1.0) == 1
    # options of the stabilisation and the Metropolis block
    assert lib.dqmc_set_option(h, b"stab_qr", 1.0) == 0
    assert lib.dqmc_set_option(h, b"stab_qr", -1.0) == 0
    assert lib.dqmc_set_option(h, b"stab_qr", 2.0) == 1
    assert lib.dqmc_set_option(h, b"tc_gemm", 0.0) == 0
    assert lib.dqmc_set_option(h, b"df_metro", 0.0) == 0
    assert lib.dqmc_set_option(h, b"flush_tc", 0.0) == 0
    assert lib.dqmc_set_option(h, b"refl_gram", 2.0) == 0
    assert lib.dqmc_set_option(h, b"refl_gram", 3.0) == 1
    assert lib.dqmc_set_option(h, b"refl_tw", 2.0) == 0
    assert lib.dqmc_set_option(h, b"refl_tw", 3.0) == 1
    assert lib.dqmc_set_option(h, b"df_panel", 1.0) == 0
    assert lib.dqmc_set_option(h, b"metro_reserve", 224 * 1024 + 1.0) == 1
    lib.dqmc_destroy(h)


def test_null_arguments(lib):
    assert lib.dqmc_create(4, 2.0, 0.1, -4.0, -1.0, 1, None) == 1
    assert lib.dqmc_sweep(None, 1, 0) == 1
    st, h = _create(lib)
    assert lib.dqmc_sweep(h, -1, 0) == 1
    assert lib.dqmc_green(h, 0, None) == 1
    assert lib.dqmc_green(h, 999, C.c_void_p(1)) == 1   # slice out of range, checked first
    assert lib.dqmc_replay(h, None, 1, C.c_void_p(1)) == 1
    assert lib.dqmc_replay(h, C.c_void_p(1), 0, C.c_void_p(1)) == 1    # slice outside [1, M]
    assert lib.dqmc_replay(h, C.c_void_p(1), 21, C.c_void_p(1)) == 1
    lib.dqmc_destroy(h)


def test_field_values_other_than_plus_minus_one_are_refused_on_the_host(lib):
    """dqmc_set_field / dqmc_replay check every value before any device work."""
    st, h = _create(lib)
    M, N = 20, 48
    bad = (C.c_int8 * (M * N))(*([1] * (M * N - 1) + [2]))
    G = (C.c_double * 1)()
    assert lib.dqmc_set_field(h, bad) == 1
    assert "+1 or -1" in lib.dqmc_last_error().decode()
    assert lib.dqmc_replay(h, bad, 3, G) == 1
    assert "+1 or -1" in lib.dqmc_last_error().decode()
    lib.dqmc_destroy(h)


def test_operator_argument_validation(lib):
    # rejected on the host before any launch
    assert lib.dqmc_op_propagate_f64(5, -0.1, 0, C.c_void_p(16), C.c_void_p(16), 1, 1, None, None, None, None) == 1
    assert lib.dqmc_op_propagate_f64(4, -0.1, 2, C.c_void_p(16), C.c_void_p(16), 1, 1, None, None, None, None) == 1
    assert lib.dqmc_op_propagate_f64(4, -0.1, 1, C.c_void_p(16), C.c_void_p(16), 1, 10, None, None, None, None) == 1
    p = C.c_void_p(16)
    assert lib.dqmc_op_flush_f64(48, 40, 16, p, p, p, p, p, p, None) == 1      # site0 + kb > N
    assert lib.dqmc_op_flush_df(48, 0, 65, p, p, p, p, p, p, None) == 1        # kb > 64
    assert lib.dqmc_op_flush_f32(48, 0, 8, p, p, p, None, p, p, None) == 1     # null alpha
    assert lib.dqmc_op_flush_tc(48, 0, 33, p, p, p, p, p, p, None) == 1        # kb > 32
    assert lib.dqmc_op_flush_tc(48, 40, 16, p, p, p, p, p, p, None) == 1       # site0 + kb > N
    assert lib.dqmc_op_metropolis_block(48, 0, 65, p, 65, p, 0.5, 1, 0, 0, 1,
                                        None, p, p, p, p, None) == 1
    assert lib.dqmc_op_metropolis_block(48, 0, 8, p, 4, p, 0.5, 1, 0, 0, 1,
                                        None, p, p, p, p, None) == 1           # ld_g < kb


def test_batch_create_validation(lib):
    out = (C.c_void_p * 2)()
    assert lib.dqmc_batch_create(0, None, out) == 1
    bad_L = (C.c_double * 12)(4.5, 2.0, 0.1, -4.0, -1.0, 1.0, 4.0, 2.0, 0.1, -4.0, -1.0, 2.0)
    assert lib.dqmc_batch_create(2, bad_L, out) == 1 and out[0] is None and out[1] is None
    bad_seed = (C.c_double * 6)(4.0, 2.0, 0.1, -4.0, -1.0, -1.0)
    assert lib.dqmc_batch_create(1, bad_seed, out) == 1
    assert lib.dqmc_batch_sweep(None, 1, 1, 0) == 1
    dup = (C.c_void_p * 2)(C.c_void_p(16), C.c_void_p(16))
    assert lib.dqmc_batch_sweep(dup, 2, 1, 0) == 1          # the same context twice


def test_autotune_validation(lib):
    """Argument checks of the autotuner, all before any chain is made."""
    ks = (C.c_int * 2)(16, 32)
    ns = (C.c_int * 1)(8)
    kb, nb, sec = C.c_int(0), C.c_int(0), C.c_double(0.0)
    outs = (C.byref(kb), C.byref(nb), C.byref(sec), None)

    def call(ks_=ks, nk=2, ns_=ns, nn=1, prec=1, warmup=1, sweeps=1, bar=1e-6, o=outs):
        return lib.dqmc_autotune(4, 2.0, 0.1, -4.0, -1.0, 1, prec, ks_, nk, ns_, nn, warmup, sweeps, bar, *o)

    assert call(ks_=None) == 1
    assert call(nk=0) == 1
    assert call(nn=0) == 1
    assert call(prec=3) == 1
    assert call(warmup=-1) == 1
    assert call(sweeps=0) == 1
    assert call(bar=0.0) == 1
    assert call(ks_=(C.c_int * 2)(16, 0)) == 1
    assert call(ns_=(C.c_int * 1)(0)) == 1
    assert call(o=(None, C.byref(nb), C.byref(sec), None)) == 1
    assert b"autotune" in lib.dqmc_last_error()


def _checkpoint(M=20, N=48, k=8, n_stab=10, prec=0, chain=0, bin_=10, st=(2, 1920, 900), md=1e-9,
                field=None, ns=0, extra=b""):
    import struct
    f = bytes([1] * (M * N)) if field is None else field
    return (b"DQMCGB31" + struct.pack("<5d", 4, 2.0, 0.1, -4.0, -1.0) + struct.pack("<Q", 1)
            + struct.pack("<7i", k, n_stab, prec, chain, 1, bin_, 0) + struct.pack("<3q", *st)
            + struct.pack("<d", md) + f + struct.pack("<q", ns)
            + b"\0" * (48 * ns if 0 <= ns <= 100 else 0) + extra)


@pytest.mark.parametrize("kw,why", [
    (dict(k=7), "header"), (dict(n_stab=0), "header"), (dict(prec=5), "header"),
    (dict(bin_=0), "header"), (dict(st=(2, 10, 11)), "header"), (dict(md=float("nan")), "header"),
    (dict(ns=-1), "damaged"), (dict(ns=10**15), "damaged"), (dict(ns=1, extra=b"x"), "damaged"),
    (dict(field=bytes([1] * 959 + [0])), "+1 or -1"),
])
def test_load_rejects_damaged_checkpoints_before_any_device_work(lib, tmp_path, kw, why):
    """A damaged checkpoint (bad options, counters, sample count or field
    values) is refused with DQMC_EINVAL before anything is allocated."""
    st, h = _create(lib)
    assert st == 0
    path = tmp_path / "ck.bin"
    path.write_bytes(_checkpoint(**kw))
    assert lib.dqmc_load(h, str(path).encode()) == 1
    assert why in lib.dqmc_last_error().decode()
    lib.dqmc_destroy(h)


@pytest.mark.parametrize("L,n_occ,eps", [(1, 1, 0.0), (2, 4, 0.0), (3, 9, 1e-4), (4, 16, 0.0), (4, 16, 1e-4),
                                         (6, 36, 1e-4), (6, 13, 1e-4), (12, 144, 1e-4)])
def test_trial_state_spans_the_oracle_trial_subspace(lib, L, n_occ, eps):
    """dqmc_op_trial_state (host, momentum blocks) against the oracle's trial
    state (dense eigendecomposition of K + eps diag(1, 0, -1)): orthonormal,
    and the same occupied subspace (equal projectors)."""
    import numpy as np
    from oracle import model as omodel, pqmc
    from paper_2608_03894_gb300 import ops
    P = ops.trial_state(L, n_occ, eps)
    ref = pqmc.trial_state(omodel.Model(L, 1.0, 0.1, -4.0, -1.0), n_occ, eps)
    assert np.max(np.abs(P.T @ P - np.eye(n_occ))) < 1e-12
    assert np.max(np.abs(P @ P.T - ref @ ref.T)) < 1e-9


def test_trial_state_refuses_an_open_shell(lib):
    import numpy as np
    P = np.zeros((27, 9))
    assert lib.dqmc_op_trial_state(3, 9, 0.0, P.ctypes.data_as(C.c_void_p)) == 1
    assert "open shell" in lib.dqmc_last_error().decode()
    assert lib.dqmc_op_trial_state(3, 0, 1e-4, P.ctypes.data_as(C.c_void_p)) == 1
    assert lib.dqmc_op_trial_state(5, 3, 1e-4, P.ctypes.data_as(C.c_void_p)) == 1


def test_trial_state_refuses_exactly_the_open_shells_the_oracle_refuses(lib):
    import numpy as np
    from oracle import model as omodel, pqmc
    m = omodel.Model(6, 1.0, 0.1, -4.0, -1.0)
    P = np.zeros((m.N, m.N))
    for n in range(1, 41):
        try:
            pqmc.trial_state(m, n)
            closed = True
        except ValueError:
            closed = False
        rc = lib.dqmc_op_trial_state(6, n, 1e-4, P.ctypes.data_as(C.c_void_p))
        assert (rc == 0) == closed, n
