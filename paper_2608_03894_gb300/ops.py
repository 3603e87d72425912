"""Python binding of the stateless operator API (include/dqmc.h, operator API):
each call validates torch CUDA tensors and passes their device pointers and
the current stream to one hot-path kernel of the library."""

import ctypes as C

from . import _lib
from ._lib import check


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(torch):
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _need(t, dtype, name):
    import torch
    if t is None:
        return
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA tensor of {dtype}")


def propagate(L, scale, side, X, Y=None, pre=None, post=None, vscale=None):
    """Eq. 5-6 kinetic propagator with fused diagonal scalings (see the header).
    side 0: Y = diag(post) e^{scale K} diag(pre) X diag(vscale), X is N x nvec;
    side 1: Y = diag(vscale) X diag(pre) e^{scale K} diag(post), X is nvec x N."""
    import torch
    lib = _lib.load()
    dt = X.dtype
    for t, n in ((X, "X"), (Y, "Y"), (pre, "pre"), (post, "post"), (vscale, "vscale")):
        _need(t, dt, n)
    if Y is None:
        Y = torch.empty_like(X)
    nvec = X.shape[1] if side == 0 else X.shape[0]
    ld = X.shape[1]
    fn = lib.dqmc_op_propagate_f64 if dt == torch.float64 else lib.dqmc_op_propagate_f32
    if dt not in (torch.float64, torch.float32):
        raise ValueError("float32 or float64 only")
    check(fn(int(L), float(scale), int(side), _ptr(X), _ptr(Y), int(nvec), int(ld), _ptr(pre),
             _ptr(post), _ptr(vscale), _stream(torch)))
    return Y


def metropolis_block(N, site0, kb, g, s, lam, seed, chain, sweep_pass, slice1, forced=None):
    """One delayed-update block (FP64): returns (Gamma, accepted, status)."""
    import torch
    lib = _lib.load()
    _need(g, torch.float64, "g")
    _need(s, torch.int8, "s")
    dev = g.device
    Gamma = torch.empty((kb, kb), dtype=torch.float64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    if forced is not None:
        forced = forced.to(device=dev, dtype=torch.uint8).contiguous()
    check(lib.dqmc_op_metropolis_block(int(N), int(site0), int(kb), _ptr(g), int(g.shape[1]), _ptr(s),
                                       float(lam), int(seed), int(chain), int(sweep_pass), int(slice1),
                                       _ptr(forced), _ptr(Gamma), _ptr(cnt), _ptr(st), _stream(torch)))
    return Gamma, int(cnt.item()), int(st.item())


def flush(N, site0, kb, G, Gcol, Grow, Gamma):
    """G <- G - Gcol Gamma (E_S - Grow) in place (FP64 or FP32 G)."""
    import torch
    lib = _lib.load()
    dt = G.dtype
    _need(G, dt, "G")
    _need(Gcol, dt, "Gcol")
    _need(Grow, dt, "Grow")
    _need(Gamma, torch.float64, "Gamma")
    fn = lib.dqmc_op_flush_f64 if dt == torch.float64 else lib.dqmc_op_flush_f32
    check(fn(int(N), int(site0), int(kb), _ptr(G), _ptr(Gcol), _ptr(Grow), _ptr(Gamma), _stream(torch)))
    return G


def measure(L, G, site_offsets=True):
    """The six equal-time estimators of one FP64 G (dict)."""
    import numpy as np
    import torch
    lib = _lib.load()
    _need(G, torch.float64, "G")
    out = np.zeros(6)
    check(lib.dqmc_op_measure(int(L), _ptr(G), int(bool(site_offsets)), out.ctypes.data_as(C.c_void_p),
                              _stream(torch)))
    return dict(zip(("S_pair_G", "S_pair_dk", "phi2_G", "phi2_K", "density", "ekin"), out.tolist()))
