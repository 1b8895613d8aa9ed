"""K++ with the inexact projection of Sec. 4.1 on the GPU (kpp_factor_lsqr, kpp_proj_lsqr,
kpp_solve_lsqr) against the oracle (orc_proj_precond, orc_proj_lsqr, orc_run_lsqr).

The oracle's pieces are pinned in test_oracle.py: the sketched Gram against scipy's Hadamard matrix,
LSQR against the normal equations and the rate of the section's lemma, and the run with converged
projections against the exact K++ run.  Here the GPU path is compared element by element:
- the preconditioners L_j to 1e-10 relative;
- a projection after t = 1, 3 and 8 LSQR iterations to 1e-10;
- the K++ iterates in lockstep (the same Philox block draws) to 1e-9 relative;
- the step at which a solve to 1e-8 stops.
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


def _system(m, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n)) @ np.diag(np.geomspace(1, 30, n))
    b = A @ rng.standard_normal(n)
    return A, b


def _sketch(n, s, seed):
    np2 = 1 << (n - 1).bit_length()
    T = np.sort(np.random.default_rng(seed).choice(np2, min(2 * s, np2), replace=False))
    return T, W.rademacher_signs(np2, seed + 1)


@pytest.mark.parametrize("m,n,s", [(240, 40, 12), (512, 300, 64), (2048, 1000, 128)])
def test_preconditioners_match_the_oracle(K, m, n, s):
    A, _ = _system(m, n, 1)
    T, d = _sketch(n, s, 2)
    lam = 0.05
    P = K.Partition(m, s)
    F = K.LsqrFactors(dev(A), P, lam, T, dev(d))
    for j in range(P.nb):
        Lo = oracle.proj_precond(A[j * s:(j + 1) * s], lam, T, d)
        Lg = F.block(j)
        np.testing.assert_allclose(np.tril(Lg), np.tril(Lo), rtol=1e-10, atol=1e-12 * np.abs(Lo).max())


@pytest.mark.parametrize("t", [1, 3, 8])
def test_projection_matches_the_oracle(K, t):
    m, n, s, lam = 512, 300, 64, 0.05
    A, _ = _system(m, n, 3)
    T, d = _sketch(n, s, 4)
    P = K.Partition(m, s)
    F = K.LsqrFactors(dev(A), P, lam, T, dev(d))
    r = np.random.default_rng(5).standard_normal(s)
    for j in (0, 5):
        w = dev(np.zeros(n))
        K.proj_lsqr(dev(A), P, F, j, dev(r), t, w)
        AS = A[j * s:(j + 1) * s]
        wo, _ = oracle.proj_lsqr(AS, r, lam, oracle.proj_precond(AS, lam, T, d), t)
        assert rel(w.cpu().numpy(), wo) <= 1e-10, (j, rel(w.cpu().numpy(), wo))


@pytest.mark.parametrize("steps", [1, 7, 43])
def test_kpp_lsqr_lockstep_with_the_oracle(K, steps):
    m, n, s, lam = 240, 40, 12, 0.05
    A, b = _system(m, n, 6)
    T, d = _sketch(n, s, 7)
    P = K.Partition(m, s)
    F = K.LsqrFactors(dev(A), P, lam, T, dev(d))
    x = dev(np.zeros(n))
    rep = K.solve_lsqr(dev(A), dev(b), x, P, F, 8, K.params(lam=lam, tol=0.0, max_iters=steps, seed=2),
                       allow_no_conv=True)
    res = oracle.run_lsqr(A, b, oracle.lsqr_factors(A, s, lam, T, d), s, 8, lam=lam, tol=0.0, max_iters=steps,
                          seed=2)
    assert rep.iters == res.iters == steps
    assert rel(x.cpu().numpy(), res.x) <= 1e-9


def test_kpp_lsqr_to_tolerance_stops_with_the_oracle(K):
    m, n, s, lam = 1024, 96, 32, 1e-3
    A, b = _system(m, n, 8)
    T, d = _sketch(n, s, 9)
    P = K.Partition(m, s)
    F = K.LsqrFactors(dev(A), P, lam, T, dev(d))
    x = dev(np.zeros(n))
    rep = K.solve_lsqr(dev(A), dev(b), x, P, F, 8, K.params(lam=lam, tol=1e-8, seed=4))
    res = oracle.run_lsqr(A, b, oracle.lsqr_factors(A, s, lam, T, d), s, 8, lam=lam, tol=1e-8, seed=4)
    assert rep.status == K.OK and res.status == oracle.OK
    assert rep.iters == res.iters
    assert rep.rel_res_true <= 1e-8
    assert rel(x.cpu().numpy(), res.x) <= 1e-9


def test_lsqr_argument_errors(K):
    A, b = _system(100, 20, 10)
    T, d = _sketch(20, 10, 11)
    with pytest.raises(K.KppError) as e:  # ragged last block
        K.LsqrFactors(dev(A), K.Partition(100, 12), 0.1, T, dev(d))
    assert e.value.status == K.ERR_ARG
    with pytest.raises(K.KppError) as e:  # a sampled column beyond the padded row
        K.LsqrFactors(dev(A), K.Partition(100, 10), 0.1, np.array([0, 40]), dev(d))
    assert e.value.status == K.ERR_ARG
    P = K.Partition(100, 10)
    F = K.LsqrFactors(dev(A), P, 0.1, T, dev(d))
    with pytest.raises(K.KppError) as e:  # the exact solve does not take these factors
        K.kpp_solve(dev(A), dev(b), dev(np.zeros(20)), P, F, K.params(lam=0.1))
    assert e.value.status == K.ERR_ARG
