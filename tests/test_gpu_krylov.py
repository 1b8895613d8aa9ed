"""The GPU Krylov reference solvers (kpp_cg, kpp_gmres) against the oracle's CG and GMRES.

In lockstep (tol = 0, a fixed number of steps) the iterates agree to 1e-10 relative: both compute
the same CG recurrence, or the same minimal-residual iterate of the Krylov space (the GPU orthogonalises
by classical Gram-Schmidt with one reorthogonalisation, the oracle by modified Gram-Schmidt: the same
iterate in exact arithmetic).  CG's lockstep runs on a smooth spectrum: with a few isolated outlying
eigenvalues, CG loses orthogonality once they converge and its trajectory amplifies rounding, so
that two correct FP64 CG codes that only sum in another order drift apart by 1e-7 .. 1e-4 within
15 - 25 steps (checked on the CPU against a plain numpy CG).  Run to a tolerance, the solvers stop
within a few percent of each other's step count and both reach it.
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


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _nonsym(n, seed):
    rng = np.random.default_rng(seed)
    A = np.eye(n) * 3.0 + rng.standard_normal((n, n)) * (0.8 / np.sqrt(n))
    return A, rng.standard_normal(n)


@pytest.mark.parametrize("n,T", [(512, 40), (1024, 30), (300, 7)])
def test_cg_lockstep_with_oracle(K, n, T):
    if n == 300:  # outliers, few steps
        A, b, _ = W.spd(n, 6, 1e2, 1e3, 1.0, 10.0, seed_A=90 + n, seed_b=91)
    else:         # smooth spectrum in [1, 12]
        A, b, _ = W.spd(n, 1, 11.0, 12.0, 1.0, 10.0, seed_A=90 + n, seed_b=91)
    x = dev(np.zeros(n))
    rep = K.cg(dev(A), dev(b), x, tol=0.0, max_iters=T, allow_no_conv=True)
    xo, it, _ = oracle.cg(A, b, tol=0.0, max_iters=T)
    assert rep.iters == it == T
    assert rel(x.cpu().numpy(), xo) <= 1e-10


def test_cg_to_tolerance_matches_oracle(K):
    A, b, _ = W.spd(2048, 25, 1e2, 1e4, 1.0, 10.0, seed_A=95, seed_b=96)
    x = dev(np.zeros(2048))
    rep = K.cg(dev(A), dev(b), x, tol=1e-8)
    xo, it, rr = oracle.cg(A, b, tol=1e-8)
    assert rep.status == K.OK and abs(rep.iters - it) <= max(2, 0.05 * it), (rep.iters, it)
    assert rep.rel_res_true <= 1.05e-8 and rr <= 1.05e-8
    kappa = 1e4
    assert rel(x.cpu().numpy(), xo) <= kappa * (rep.rel_res_true + rr)


@pytest.mark.parametrize("k", [1, 5, 20, 45])
def test_gmres_lockstep_with_oracle(K, k):
    n = 300
    A, b = _nonsym(n, 97)
    x0 = np.random.default_rng(98).standard_normal(n) * 0.1
    x = dev(x0)
    rep = K.gmres(dev(A), dev(b), x, restart=64, tol=0.0, max_iters=k, allow_no_conv=True)
    xo, it, _, cyc = oracle.gmres(A, b, restart=64, tol=0.0, max_iters=k, x0=x0)
    assert rep.iters == it == k
    assert rel(x.cpu().numpy(), xo) <= 1e-10, (k, rel(x.cpu().numpy(), xo))


def test_gmres_restarted_to_tolerance(K):
    n = 500
    A, b = _nonsym(n, 99)
    x = dev(np.zeros(n))
    rep = K.gmres(dev(A), dev(b), x, restart=8, tol=1e-10)
    xo, it, rr, cyc = oracle.gmres(A, b, restart=8, tol=1e-10)
    assert rep.status == K.OK and rep.rel_res_true <= 1.05e-10 and rep.outer >= 2
    assert abs(rep.iters - it) <= 2 and abs(rep.outer - cyc) <= 1
    xs = np.linalg.solve(A, b)
    assert rel(x.cpu().numpy(), xs) <= np.linalg.cond(A) * 2.0 * rep.rel_res_true


def test_gmres_on_spd_system(K):
    A, b, _ = W.spd(1024, 12, 1e2, 1e4, 1.0, 10.0, seed_A=100, seed_b=101)
    x = dev(np.zeros(1024))
    rep = K.gmres(dev(A), dev(b), x, restart=512, tol=1e-8)
    assert rep.status == K.OK and rep.rel_res_true <= 1.05e-8
    xc = dev(np.zeros(1024))
    rc = K.cg(dev(A), dev(b), xc, tol=1e-8)
    # full GMRES minimises the residual over the same Krylov spaces CG searches
    assert rep.iters <= rc.iters + 1


def test_krylov_argument_errors(K):
    A = dev(np.eye(16))
    b = dev(np.ones(16))
    x = dev(np.zeros(16))
    for restart in (0, 513):
        with pytest.raises(K.KppError) as e:
            K.gmres(A, b, x, restart=restart)
        assert e.value.status == K.ERR_ARG
    with pytest.raises(K.KppError) as e:
        K.cg(A.float(), b, x)
    assert e.value.status == K.ERR_ARG
    with pytest.raises(K.KppError):
        K.cg(dev(np.ones((16, 8))), b, x)
