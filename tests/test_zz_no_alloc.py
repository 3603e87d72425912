"""The fixed-scratch rank-m flush (dqmc_op_flush_f64_noalloc), called
through the C ABI, against the allocating dqmc_op_flush_f64 on the same
inputs, on two calls in a row. Runs last (file name), and alone."""

import ctypes as C

import numpy as np
import pytest

from dqmc_inputs import random_field, random_green_like

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


def _p(t):
    return C.c_void_p(t.data_ptr())


def test_fixed_scratch_flush_matches_allocating_flush(pkg):
    from paper_2608_03894_gb300 import _lib
    lib = _lib.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    N, kb, lam = 432, 32, 0.65
    G0 = torch.tensor(random_green_like(N, seed=11), device="cuda")
    s = torch.tensor(random_field(1, N, seed=12)[0], device="cuda")
    Ga, Gb = G0.clone(), G0.clone()
    for call, site0 in enumerate((0, kb)):   # two calls in a row, consecutive blocks
        g = Ga[site0:site0 + kb, site0:site0 + kb].contiguous()
        al, be, cnt, st = pkg.ops.metropolis_block(N, site0, kb, g, s, lam, 7, 0, 0, 1)
        assert st == 0 and int(cnt.item()) > 0
        # copies (a full-row slice is already contiguous: .contiguous() would alias Ga)
        Gcol = Ga[:, site0:site0 + kb].clone()
        Grow = Ga[site0:site0 + kb, :].clone()
        Gprev = Ga.clone()
        assert lib.dqmc_op_flush_f64(N, site0, kb, _p(Ga), _p(Gcol), _p(Grow), _p(al), _p(be), _p(cnt),
                                     stream) == 0
        assert lib.dqmc_op_flush_f64_noalloc(N, site0, kb, _p(Gb), _p(Gcol), _p(Grow), _p(al), _p(be),
                                             _p(cnt), stream) == 0
        torch.cuda.synchronize()
        m = int(cnt.item())
        E = torch.zeros((kb, N), dtype=torch.float64, device="cuda")
        E[torch.arange(kb), site0 + torch.arange(kb)] = 1.0
        ref = Gprev - (Gcol @ al[:m].T) @ (be[:m] @ (E - Grow))
        err = torch.max(torch.abs(Ga - Gb)).item()
        assert err < 1e-12, (call, err)
        assert torch.max(torch.abs(Gb - ref)).item() < 1e-12
        assert torch.max(torch.abs(Gb - Gprev)).item() > 1e-3   # the flush did change G


def test_fixed_scratch_flush_rejects_sizes_beyond_its_scratch(pkg):
    from paper_2608_03894_gb300 import _lib
    lib = _lib.load()
    p = C.c_void_p(16)
    # N * K = 4000 * 64 > 3888 * 64: rejected on the host before any launch
    assert lib.dqmc_op_flush_f64_noalloc(4000, 0, 64, p, p, p, p, p, p, None) == 1
    assert b"fixed flush scratch" in lib.dqmc_last_error()
