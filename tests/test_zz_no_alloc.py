"""The allocation-free CD++ entry point (cdpp_solve_noalloc) against cdpp_solve.

Some callers cannot call cudaMalloc (their GPU memory belongs to another allocator, or a request
must not block on allocation or fail with out-of-memory half way).  cdpp_solve_noalloc serves them
from a fixed scratch array inside the library.  It runs the general CD++ kernel with cdpp_solve's
launch shape, so the reference here is cdpp_solve with kernel variant 1 (the general kernel): the
iterates must agree within the iterate tolerance of the other parity tests (1e-10 relative) and the
step counts must be equal.  Against the default variant (the dataflow kernels, another summation
order) only the iterate and the residual are compared.  The test calls the entry point twice in a
row (the second call must not see the first call's leftovers) and checks that neither call made a
device allocation.  It lives in its own file, collected last, and passes alone or after the rest of
the suite.
"""
import ctypes

import numpy as np
import pytest

from paper_2501_11673_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_matches_cdpp_solve_twice():
    from paper_2501_11673_gb300 import build as kbuild
    from paper_2501_11673_gb300 import kpp
    kbuild.build()
    kpp.load()
    cases = [(W.spd(512, 8, 1e2, 1e3, 1.0, 10.0, seed_A=70, seed_b=71), 32, 7),
             (W.spd(300, 5, 1e2, 1e3, 1.0, 4.0, seed_A=72, seed_b=73), 24, 8)]  # ragged last block
    for (A, b, _), s, seed in cases:
        n = A.shape[0]
        Ad = torch.as_tensor(A, device="cuda")
        bd = torch.as_tensor(b, device="cuda")
        P = kpp.Partition(n, s)
        F = kpp.Factors(Ad, P, 1e-4, 1)
        prm = kpp.params(lam=1e-4, tol=1e-9, seed=seed)
        x_gen = torch.zeros(n, dtype=torch.float64, device="cuda")
        kpp.set_kernel_variant(1)
        try:
            rep_gen = kpp.cdpp_solve(Ad, bd, x_gen, P, F, prm)
        finally:
            kpp.set_kernel_variant(3)
        x_dflt = torch.zeros(n, dtype=torch.float64, device="cuda")
        rep_dflt = kpp.cdpp_solve(Ad, bd, x_dflt, P, F, prm)
        ev = np.linalg.eigvalsh(A)
        kappa = ev[-1] / ev[0]
        for call in range(2):
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            allocs = kpp.device_alloc_count()
            rep = kpp.cdpp_solve_noalloc(Ad, bd, x, P, F, prm)
            assert kpp.device_alloc_count() == allocs, "cdpp_solve_noalloc allocated device memory"
            assert rep.status == kpp.OK, (call, rep.as_dict())
            assert rep.iters == rep_gen.iters, (call, rep.iters, rep_gen.iters)
            assert rep.rel_res_true <= 1e-9
            err = (torch.linalg.norm(x - x_gen) / torch.linalg.norm(x_gen)).item()
            assert err <= 1e-10, (call, err)
            # the default variant may stop at another checkpoint; both residuals are small, and
            # |x - x'| / |x'| <= kappa (|r| / |b| + |r'| / |b|) bounds how far apart they can be
            err_d = (torch.linalg.norm(x - x_dflt) / torch.linalg.norm(x_dflt)).item()
            assert err_d <= 1.01 * kappa * (rep.rel_res_true + rep_dflt.rel_res_true), (call, err_d)


def test_noalloc_refuses_oversize_without_touching_memory():
    """Sizes beyond the fixed scratch are refused on the host, before any pointer is used; a small
    valid buffer stands behind a matrix descriptor that claims n = 16448."""
    from paper_2501_11673_gb300 import kpp
    kpp.load()
    n_small = 64
    A = torch.eye(n_small, dtype=torch.float64, device="cuda")
    P = kpp.Partition(n_small, 16)
    F = kpp.Factors(A, P, 1e-4, 1)
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    big = 16448
    m = kpp.Matrix(ctypes.c_void_p(buf.data_ptr()), kpp.KPP_F64, 0, big, big, big)
    Pb = kpp.Partition(big, 64)
    prm = kpp.params(lam=1e-4)
    rep = kpp.Report()
    allocs = kpp.device_alloc_count()
    rc = kpp.load().cdpp_solve_noalloc(ctypes.byref(m), ctypes.c_void_p(buf.data_ptr()),
                                       ctypes.c_void_p(buf.data_ptr()), Pb.handle, F.handle, ctypes.byref(prm),
                                       ctypes.byref(rep), None)
    assert rc == kpp.ERR_ARG
    assert "exceed the fixed scratch" in kpp.last_error()
    assert kpp.device_alloc_count() == allocs
