"""Python binding of the DQMC context API (include/dqmc.h): argument marshalling
only; every step of the sweep runs in the CUDA library."""

import ctypes as C

import numpy as np

from . import _lib
from ._lib import check

OBS_NAMES = ("S_pair_G", "S_pair_dk", "phi2_G", "phi2_K", "density", "ekin")


def _torch():
    import torch
    return torch


class TorchAllocator:
    """Routes the library's device allocations through PyTorch's caching
    allocator (on the current device and stream)."""

    def __init__(self, device=None, stream=None):
        torch = _torch()
        self.device = torch.cuda.current_device() if device is None else device
        self.stream = stream

        def _alloc(nbytes, user):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream))
            except Exception:  # out of memory -> NULL -> DQMC_ENOMEM
                return None

        def _free(ptr, user):
            if ptr:
                torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc_cb = _lib.ALLOC_FN(_alloc)
        self.free_cb = _lib.FREE_FN(_free)


class DQMC:
    """One Markov chain of the kagome attractive-Hubbard DQMC sweep.

    Parameters follow the paper's notation: L (cells per side, N = 3 L^2),
    beta, dtau (M = beta / dtau slices), U <= 0 (attraction), mu, seed.
    Options: k (delay rank), n_stab, precision ("fp64" or "mixed"), chain,
    timing, site_offsets, bin, drift_limit. ``use_torch`` routes device
    memory and the stream through PyTorch."""

    def __init__(self, L, beta, dtau, U, mu, seed=1, k=32, n_stab=10, precision="fp64",
                 chain=0, timing=False, site_offsets=True, bin=10, drift_limit=1e-3,
                 use_torch=True):
        self.lib = _lib.load()
        h = C.c_void_p()
        check(self.lib.dqmc_create(int(L), float(beta), float(dtau), float(U), float(mu),
                                   int(seed) & 0xFFFFFFFFFFFFFFFF, C.byref(h)))
        self.h = h
        self.L = int(L)
        self.N = 3 * self.L * self.L
        self.M = int(round(beta / dtau))
        self._alloc = None
        prec = {"fp64": 0, "mixed": 1, "fp32": 2, 0: 0, 1: 1, 2: 2}[precision]
        opts = dict(k=k, n_stab=n_stab, precision=prec, chain=chain, timing=int(timing),
                    site_offsets=int(bool(site_offsets)), bin=bin, drift_limit=drift_limit)
        for key, v in opts.items():
            self.set_option(key, v)
        if use_torch:
            torch = _torch()
            if torch.cuda.is_available():
                self._alloc = TorchAllocator()
                check(self.lib.dqmc_set_allocator(self.h, self._alloc.alloc_cb, self._alloc.free_cb, None))
                self.set_stream(torch.cuda.current_stream().cuda_stream)

    @classmethod
    def _from_handle(cls, h, L, beta, dtau):
        self = cls.__new__(cls)
        self.lib = _lib.load()
        self.h = h
        self.L = int(L)
        self.N = 3 * self.L * self.L
        self.M = int(round(beta / dtau))
        self._alloc = None
        return self

    # -- options / plumbing
    def set_option(self, key, value):
        check(self.lib.dqmc_set_option(self.h, key.encode(), float(value)))

    def set_stream(self, stream_handle):
        check(self.lib.dqmc_set_stream(self.h, C.c_void_p(int(stream_handle))))

    # -- the hot path
    def sweep(self, n=1, measure=False):
        check(self.lib.dqmc_sweep(self.h, int(n), int(bool(measure))))

    def green(self, slice_index=0):
        G = np.empty((self.N, self.N), dtype=np.float64)
        check(self.lib.dqmc_green(self.h, int(slice_index), G.ctypes.data_as(C.c_void_p)))
        return G

    def running_green(self):
        G = np.empty((self.N, self.N), dtype=np.float64)
        sl = C.c_int(0)
        check(self.lib.dqmc_get_running_green(self.h, G.ctypes.data_as(C.c_void_p), C.byref(sl)))
        return G, sl.value

    def measure(self):
        o = _lib.Obs()
        check(self.lib.dqmc_measure(self.h, C.byref(o)))
        out = {n: getattr(o, n) for n in OBS_NAMES}
        out["err"] = dict(zip(OBS_NAMES, list(o.err)))
        for n in ("n_samples", "n_bins", "R_pair", "R_pair_err", "P", "P_err", "D_G", "D_K"):
            out[n] = getattr(o, n)
        return out

    def stats(self):
        s = _lib.Stats()
        check(self.lib.dqmc_get_stats(self.h, C.byref(s)))
        arrays = ("ms_kernel", "n_kernel", "flops_kernel", "bytes_kernel")
        out = {n: getattr(s, n) for n, _ in _lib.Stats._fields_ if n not in arrays}
        for n in arrays:
            out[n] = dict(zip(_lib.KERNEL_FAMILIES, list(getattr(s, n))))
        return out

    @property
    def field(self):
        f = np.empty((self.M, self.N), dtype=np.int8)
        check(self.lib.dqmc_get_field(self.h, f.ctypes.data_as(C.c_void_p)))
        return f

    @field.setter
    def field(self, value):
        f = np.ascontiguousarray(np.asarray(value, dtype=np.int8).reshape(self.M, self.N))
        check(self.lib.dqmc_set_field(self.h, f.ctypes.data_as(C.c_void_p)))

    def replay(self, target, slice):
        """Forced-flip up pass to `slice` towards the target field; returns the
        fast path's running G(tau_slice) (FP64 N x N)."""
        t = np.ascontiguousarray(np.asarray(target, dtype=np.int8).reshape(self.M, self.N))
        G = np.empty((self.N, self.N), dtype=np.float64)
        check(self.lib.dqmc_replay(self.h, t.ctypes.data_as(C.c_void_p), int(slice),
                                   G.ctypes.data_as(C.c_void_p)))
        return G

    def save(self, path):
        check(self.lib.dqmc_save(self.h, str(path).encode()))

    def load(self, path):
        check(self.lib.dqmc_load(self.h, str(path).encode()))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.dqmc_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Independent chains of possibly different sizes on one GPU
    (dqmc_batch_create / dqmc_batch_sweep): rows of params are
    (L, beta, dtau, U, mu, seed); every chain has its own CUDA stream and
    device memory from cudaMalloc. Options apply to every chain."""

    def __init__(self, params, **options):
        self.lib = _lib.load()
        rows = [tuple(float(x) for x in r) for r in params]
        n = len(rows)
        flat = (C.c_double * (6 * n))(*[x for r in rows for x in r])
        hs = (C.c_void_p * n)()
        check(self.lib.dqmc_batch_create(n, flat, hs))
        self._hs = hs
        self.chains = [DQMC._from_handle(C.c_void_p(hs[i]), r[0], r[1], r[2]) for i, r in enumerate(rows)]
        prec = {"fp64": 0, "mixed": 1, "fp32": 2}
        for key, v in options.items():
            v = prec.get(v, v) if key == "precision" else v
            for c in self.chains:
                c.set_option(key, v)

    def sweep(self, n=1, measure=False):
        check(self.lib.dqmc_batch_sweep(self._hs, len(self.chains), int(n), int(bool(measure))))

    def close(self):
        for c in self.chains:
            c.close()
        self.chains = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def autotune(L, beta, dtau, U, mu, seed=1, precision="mixed", ks=(16, 32, 64), n_stabs=(8,),
             warmup=1, sweeps=1, drift_bar=1e-6):
    """Delay rank and refresh interval by measurement (dqmc_autotune): every
    (k, n_stab) pair timed on a fresh chain; returns the fastest pair whose
    drift stays within drift_bar, its seconds per sweep, and the table of all
    pairs (None for a pair over the bar)."""
    lib = _lib.load()
    prec = {"fp64": 0, "mixed": 1, "fp32": 2, 0: 0, 1: 1, 2: 2}[precision]
    ka = (C.c_int * len(ks))(*[int(k) for k in ks])
    na = (C.c_int * len(n_stabs))(*[int(n) for n in n_stabs])
    times = (C.c_double * (len(ks) * len(n_stabs)))()
    kb, nb, sec = C.c_int(0), C.c_int(0), C.c_double(0.0)
    check(lib.dqmc_autotune(int(L), float(beta), float(dtau), float(U), float(mu),
                            int(seed) & 0xFFFFFFFFFFFFFFFF, prec, ka, len(ks), na, len(n_stabs),
                            int(warmup), int(sweeps), float(drift_bar), C.byref(kb), C.byref(nb),
                            C.byref(sec), times))
    table = {(int(k), int(n)): (times[a * len(n_stabs) + b] if times[a * len(n_stabs) + b] >= 0 else None)
             for a, k in enumerate(ks) for b, n in enumerate(n_stabs)}
    return {"k": kb.value, "n_stab": nb.value, "sec_per_sweep": sec.value, "table": table}
