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


def propagate(L, scale, side, X, Y=None, pre=None, post=None, vscale=None, df=False):
    """Eq. 5-6 kinetic propagator with fused diagonal scalings (see the header).
    side 0: Y = diag(post) e^{scale K} diag(pre) X diag(vscale), X is N x nvec;
    side 1: Y = diag(vscale) X diag(pre) e^{scale K} diag(post), X is nvec x N.
    df: float64 data computed in double-float arithmetic."""
    import torch
    lib = _lib.load()
    dt = X.dtype
    for t, n in ((X, "X"), (Y, "Y"), (pre, "pre"), (post, "post"), (vscale, "vscale")):
        _need(t, dt, n)
    if Y is None:
        Y = torch.empty_like(X)
    nvec = X.shape[1] if side == 0 else X.shape[0]
    ld = X.shape[1]
    if dt not in (torch.float64, torch.float32):
        raise ValueError("float32 or float64 only")
    if df and dt != torch.float64:
        raise ValueError("double-float propagation takes float64 data")
    fn = (lib.dqmc_op_propagate_df if df else lib.dqmc_op_propagate_f64) if dt == torch.float64 \
        else lib.dqmc_op_propagate_f32
    check(fn(int(L), float(scale), int(side), _ptr(X), _ptr(Y), int(nvec), int(ld), _ptr(pre),
             _ptr(post), _ptr(vscale), _stream(torch)))
    return Y


def metropolis_block(N, site0, kb, g, s, lam, seed, chain, sweep_pass, slice1, forced=None, df=False):
    """One delayed-update block (FP64, or double-float with df=True): returns
    (alpha, beta, count, status) with count a device int32 tensor (pass it to
    flush) -- alpha/beta rows < count hold the coefficient vectors of the
    accepted flips."""
    import torch
    lib = _lib.load()
    _need(g, torch.float64, "g")
    _need(s, torch.int8, "s")
    dev = g.device
    alpha = torch.empty((kb, kb), dtype=torch.float64, device=dev)
    beta = torch.empty((kb, kb), dtype=torch.float64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    if forced is not None:
        forced = forced.to(device=dev, dtype=torch.uint8).contiguous()
    fn = lib.dqmc_op_metropolis_block_df if df else lib.dqmc_op_metropolis_block
    check(fn(int(N), int(site0), int(kb), _ptr(g), int(g.shape[1]), _ptr(s),
             float(lam), int(seed), int(chain), int(sweep_pass), int(slice1),
             _ptr(forced), _ptr(alpha), _ptr(beta), _ptr(cnt), _ptr(st),
             _stream(torch)))
    return alpha, beta, cnt, int(st.item())


def flush(N, site0, kb, G, Gcol, Grow, alpha, beta, count, mode=None):
    """G <- G - (Gcol alpha^T)(beta (E_S - Grow)) in place. mode: "f64" (default for
    float64 G), "df" (FP64 G, double-float product), "tc" (FP64 G, digit-slice
    product on the tcgen05 tensor cores, kb <= 32) or "f32" (float32 G)."""
    import torch
    lib = _lib.load()
    dt = G.dtype
    for t, n in ((G, "G"), (Gcol, "Gcol"), (Grow, "Grow")):
        _need(t, dt, n)
    _need(alpha, torch.float64, "alpha")
    _need(beta, torch.float64, "beta")
    _need(count, torch.int32, "count")
    mode = mode or ("f64" if dt == torch.float64 else "f32")
    fn = {"f64": lib.dqmc_op_flush_f64, "df": lib.dqmc_op_flush_df, "tc": lib.dqmc_op_flush_tc,
          "f32": lib.dqmc_op_flush_f32}[mode]
    check(fn(int(N), int(site0), int(kb), _ptr(G), _ptr(Gcol), _ptr(Grow), _ptr(alpha), _ptr(beta),
             _ptr(count), _stream(torch)))
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


def measure_fullq(L, G, site_offsets=True):
    """S_Pair(Q) and <phi^+ phi>(Q) at every mesh momentum (two L x L numpy
    arrays indexed [m1, m2]) from one FP64 G."""
    import numpy as np
    import torch
    lib = _lib.load()
    _need(G, torch.float64, "G")
    S = np.zeros((L, L))
    P = np.zeros((L, L))
    check(lib.dqmc_op_measure_fullq(int(L), _ptr(G), int(bool(site_offsets)), S.ctypes.data_as(C.c_void_p),
                                    P.ctypes.data_as(C.c_void_p), _stream(torch)))
    return S, P


def trial_state(L, n_occ, eps=1e-4):
    """Projector-QMC trial orbitals: N x n_occ orthonormal real basis of the
    lowest n_occ eigenstates of K + eps diag(+1, 0, -1) (host numpy array)."""
    import numpy as np
    lib = _lib.load()
    N = 3 * int(L) ** 2
    P = np.zeros((N, int(n_occ)))
    check(lib.dqmc_op_trial_state(int(L), int(n_occ), float(eps), P.ctypes.data_as(C.c_void_p)))
    return P


def gemm(A, B, C=None, alpha=1.0, beta=0.0, ta=False, tb=False, mode="f64"):
    """C = alpha op(A) op(B) + beta C (FP64 tensors). mode: "f64" (FP64 FMA),
    "df" (double-float on the FP32 units), "oz" (exact digit slices on the bf16
    tensor cores, mma.sync), "tc" (the same digit slices on tcgen05)."""
    import torch
    lib = _lib.load()
    for t, n in ((A, "A"), (B, "B")):
        _need(t, torch.float64, n)
    M = A.shape[1] if ta else A.shape[0]
    K = A.shape[0] if ta else A.shape[1]
    N = B.shape[0] if tb else B.shape[1]
    if C is None:
        C = torch.zeros((M, N), dtype=torch.float64, device=A.device)
    _need(C, torch.float64, "C")
    check(lib.dqmc_op_gemm_f64({"f64": 0, "df": 1, "oz": 2, "tc": 3}[mode], int(ta), int(tb), M, N, K, float(alpha),
                               _ptr(A), A.shape[1], _ptr(B), B.shape[1], float(beta), _ptr(C), C.shape[1],
                               _stream(torch)))
    return C
