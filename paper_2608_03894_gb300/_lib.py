"""ctypes declarations of the C ABI in include/dqmc.h (argument marshalling only)."""

import ctypes as C
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libdqmc_gb300.so")

STATUS = {
    0: "DQMC_OK", 1: "DQMC_EINVAL", 2: "DQMC_ENOMEM", 3: "DQMC_ECUDA",
    4: "DQMC_ENUMERIC", 5: "DQMC_ETIMEOUT", 6: "DQMC_ESTATE",
}


class DQMCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Obs(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("S_pair_G", "S_pair_dk", "phi2_G", "phi2_K", "density", "ekin")] + [
        ("err", C.c_double * 6), ("n_samples", C.c_long), ("n_bins", C.c_long),
        ("R_pair", C.c_double), ("R_pair_err", C.c_double), ("P", C.c_double), ("P_err", C.c_double),
        ("D_G", C.c_double), ("D_K", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("sweeps", C.c_long), ("proposed", C.c_long), ("accepted", C.c_long),
                ("max_drift", C.c_double), ("last_drift", C.c_double),
                ("ms_wrap", C.c_double), ("ms_update", C.c_double), ("ms_stab", C.c_double),
                ("ms_measure", C.c_double), ("ms_kernel", C.c_double * 10), ("n_kernel", C.c_long * 10),
                ("flops_kernel", C.c_double * 10), ("bytes_kernel", C.c_double * 10),
                ("launches", C.c_ulonglong)]

KERNEL_FAMILIES = ("prop", "metropolis", "flush", "gemm", "qr_panel", "measure", "other", "slice",
                   "block_aux", "stab_aux")


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

vp, i32, u32, u64, f64, i8p = C.c_void_p, C.c_int, C.c_uint32, C.c_uint64, C.c_double, C.c_void_p

SIGNATURES = {
    "dqmc_version": (C.c_char_p, []),
    "dqmc_last_error": (C.c_char_p, []),
    "dqmc_create": (i32, [i32, f64, f64, f64, f64, u64, C.POINTER(vp)]),
    "dqmc_set_option": (i32, [vp, C.c_char_p, f64]),
    "dqmc_set_stream": (i32, [vp, vp]),
    "dqmc_set_allocator": (i32, [vp, ALLOC_FN, FREE_FN, vp]),
    "dqmc_sweep": (i32, [vp, i32, i32]),
    "dqmc_green": (i32, [vp, i32, vp]),
    "dqmc_get_running_green": (i32, [vp, vp, C.POINTER(i32)]),
    "dqmc_measure": (i32, [vp, C.POINTER(Obs)]),
    "dqmc_get_stats": (i32, [vp, C.POINTER(Stats)]),
    "dqmc_get_field": (i32, [vp, vp]),
    "dqmc_set_field": (i32, [vp, vp]),
    "dqmc_replay": (i32, [vp, vp, i32, vp]),
    "dqmc_save": (i32, [vp, C.c_char_p]),
    "dqmc_load": (i32, [vp, C.c_char_p]),
    "dqmc_destroy": (None, [vp]),
    "dqmc_batch_create": (i32, [i32, vp, vp]),
    "dqmc_batch_sweep": (i32, [vp, i32, i32, i32]),
    "dqmc_autotune": (i32, [i32, f64, f64, f64, f64, u64, i32, vp, i32, vp, i32, i32, i32, f64,
                            C.POINTER(i32), C.POINTER(i32), C.POINTER(f64), vp]),
    "dqmc_op_propagate_f64": (i32, [i32, f64, i32, vp, vp, i32, i32, vp, vp, vp, vp]),
    "dqmc_op_propagate_f32": (i32, [i32, f64, i32, vp, vp, i32, i32, vp, vp, vp, vp]),
    "dqmc_op_propagate_df": (i32, [i32, f64, i32, vp, vp, i32, i32, vp, vp, vp, vp]),
    "dqmc_op_metropolis_block": (i32, [i32, i32, i32, vp, i32, vp, f64, u64, u32, u32, i32, vp, vp, vp, vp, vp, vp]),
    "dqmc_op_metropolis_block_df": (i32, [i32, i32, i32, vp, i32, vp, f64, u64, u32, u32, i32, vp, vp, vp, vp, vp, vp]),
    "dqmc_op_flush_f64": (i32, [i32, i32, i32, vp, vp, vp, vp, vp, vp, vp]),
    "dqmc_op_flush_df": (i32, [i32, i32, i32, vp, vp, vp, vp, vp, vp, vp]),
    "dqmc_op_flush_f32": (i32, [i32, i32, i32, vp, vp, vp, vp, vp, vp, vp]),
    "dqmc_op_flush_tc": (i32, [i32, i32, i32, vp, vp, vp, vp, vp, vp, vp]),
    "dqmc_op_flush_f64_noalloc": (i32, [i32, i32, i32, vp, vp, vp, vp, vp, vp, vp]),
    "dqmc_op_measure": (i32, [i32, vp, i32, vp, vp]),
    "dqmc_op_measure_fullq": (i32, [i32, vp, i32, vp, vp, vp]),
    "dqmc_op_trial_state": (i32, [i32, i32, C.c_double, vp]),
    "dqmc_op_gemm_f64": (i32, [i32, i32, i32, i32, i32, i32, f64, vp, i32, vp, i32, f64, vp, i32, vp]),
}

_lib = None


def load():
    """Load libdqmc_gb300.so; raises ImportError if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with __graft_entry__.build() or "
            "python -m paper_2608_03894_gb300._build (the CUDA path has no fallback)")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status):
    if status != 0:
        msg = load().dqmc_last_error().decode(errors="replace")
        raise DQMCError(status, msg)
