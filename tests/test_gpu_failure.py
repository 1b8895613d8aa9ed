"""Failure handling on the GPU without a GPU fault: a bounded device wait that runs out.

Every spin-wait of the persistent kernels gives up after a time limit, marks the group's error word,
releases the other waiters and returns.  The test hook kpp_set_wait_test shortens the limit to 1 ms and
makes one CTA of the general kernel leave before its first group barrier without arriving, so the
barrier's count never reaches its target (a flag that nothing sets) and the other CTAs' wait runs out.
The solve must return KPP_ERR_TIMEOUT, and the context must stay usable: the next solve on the same
context matches the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2501_11673_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def K():
    from paper_2501_11673_gb300 import build as kbuild
    from paper_2501_11673_gb300 import kpp
    kbuild.build()
    kpp.load()
    return kpp


def test_wait_that_runs_out_returns_timeout_and_context_stays_usable(K):
    sy = W.kpp_fp64_2000x200()
    m, n = sy.A.shape
    Ad = torch.as_tensor(sy.A, device="cuda")
    bd = torch.as_tensor(sy.b, device="cuda")
    P = K.Partition(m, sy.s)
    F = K.Factors(Ad, P, sy.lam, 0)
    prm = K.params(lam=sy.lam, tol=sy.tol, seed=0, grid=8)
    # the hook is refused by every kernel but the general one, before any launch
    K.set_wait_test(1_000_000, 2)
    try:
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        with pytest.raises(K.KppError) as e:
            K.kpp_solve(Ad, bd, x, P, F, prm)
        assert e.value.status == K.ERR_UNSUPPORTED
        K.set_kernel_variant(1)
        launches = K.launch_count()
        with pytest.raises(K.KppError) as e:
            K.kpp_solve(Ad, bd, x, P, F, prm)
        assert e.value.status == K.ERR_TIMEOUT, str(e.value)
        assert K.launch_count() > launches
    finally:
        K.set_wait_test(0, -1)
        K.set_kernel_variant(3)
    torch.cuda.synchronize()
    # the same context runs the next solve correctly
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    rep = K.kpp_solve(Ad, bd, x, P, F, prm)
    assert rep.status == K.OK and rep.rel_res_true <= 1e-8
    res = oracle.run(sy.A, sy.b, oracle.kpp_factor(sy.A, sy.s, sy.lam), sy.s, lam=sy.lam, tol=sy.tol, seed=0)
    assert rep.iters == res.iters
    err = np.linalg.norm(x.cpu().numpy() - res.x) / np.linalg.norm(res.x)
    assert err <= 1e-10


def test_wait_test_hook_arguments(K):
    with pytest.raises(K.KppError) as e:
        K.set_wait_test(0, -2)
    assert e.value.status == K.ERR_ARG
    K.set_wait_test(0, -1)
