"""The allocation-free CD++ entry point (cdpp_solve_noalloc) against cdpp_solve.

Some callers cannot call cudaMalloc (their GPU memory belongs to another allocator, or a request
must not block on allocation or fail with out-of-memory half way).  cdpp_solve_noalloc serves them
from a fixed scratch array inside the library.  This test calls it through the C ABI twice in a row
(the second call must not see the first call's leftovers) and compares each result with the
allocating entry point, within the iterate tolerance of the other parity tests (1e-10 relative).
It lives in its own file, collected last, and passes alone or after the rest of the suite.
"""
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
        x_ref = torch.zeros(n, dtype=torch.float64, device="cuda")
        rep_ref = kpp.cdpp_solve(Ad, bd, x_ref, P, F, prm)
        for call in range(2):
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            rep = kpp.cdpp_solve_noalloc(Ad, bd, x, P, F, prm)
            assert rep.status == kpp.OK, (call, rep.as_dict())
            assert rep.iters == rep_ref.iters
            assert rep.rel_res_true <= 1e-9
            err = (torch.linalg.norm(x - x_ref) / torch.linalg.norm(x_ref)).item()
            assert err <= 1e-10, (call, err)
    # sizes beyond the fixed scratch are refused, not allocated
    big = torch.zeros((16448, 16448), dtype=torch.float64, device="cuda")
    Pb = kpp.Partition(16448, 64)
    with pytest.raises(kpp.KppError) as e:
        kpp.cdpp_solve_noalloc(big, big[0], big[1], Pb, F, kpp.params(lam=1e-4))
    assert e.value.status == kpp.ERR_ARG and "exceed the fixed scratch" in str(e.value)
    del big
    torch.cuda.empty_cache()
