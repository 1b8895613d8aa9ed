"""GPU parity of the mixed-precision factor phase against the FP64 oracle.

With BF16 / FP32 storage the block Gram G_j = A_Sj A_Sj^T + lambda I (Eq. 1.3) is built on the tensor
cores with FP32 accumulation, and its Cholesky factor (the memoised factor of Sec. 4) is computed in
FP32.  Only blocks whose Gram is too ill-conditioned for FP32 elimination are factored in FP64: a block
whose FP32 pivots fail, or whose largest-to-smallest pivot ratio (a lower bound on kappa(G_j)) exceeds
2^24 / (s + 1).

Bound for an accepted FP32 factor against the oracle's FP64 factor of the same stored matrix: each Gram
entry carries an FP32 accumulation error of at most n 2^-24 relative to (|A_S| |A_S|^T)_ik (sums over n
columns of products that are exact in FP32 for BF16 and rounded once for FP32), which for these dense
Gaussian blocks is of the size of G's bulk; the FP32 Cholesky adds a backward error of at most (s + 1)
2^-24 relative; and to first order a Cholesky factor moves by at most kappa(G) times the relative change
of G, so
    |L_gpu - L_oracle|_F / |L_oracle|_F <= kappa(G_j) * (n + s + 1) * 2^-24.
"""
import numpy as np
import pytest

import oracle
from paper_2501_11673_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EPS32 = 2.0 ** -24
TDT = {"f32": torch.float32, "bf16": torch.bfloat16}


@pytest.fixture(scope="module")
def K():
    from paper_2501_11673_gb300 import build as kbuild
    from paper_2501_11673_gb300 import kpp
    kbuild.build()
    kpp.load()
    return kpp


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


@pytest.mark.parametrize("dtype,m,n,s", [("bf16", 1000, 1024, 512),   # ragged last block of 488 rows
                                         ("f32", 600, 1024, 128),
                                         ("f32", 230, 300, 33),       # odd block size: ragged panels
                                         ("bf16", 2048, 2048, 1024),  # largest block the partition allows
                                         ("bf16", 256, 512, 64)])
def test_fp32_cholesky_matches_oracle_within_bound(K, record_property, dtype, m, n, s):
    rng = np.random.default_rng(m + n + s)
    A = W.round_to_storage(rng.standard_normal((m, n)), dtype)
    lam = 0.5
    P = K.Partition(m, s)
    F = K.Factors(dev(A, TDT[dtype]), P, lam, 0)
    assert F.fp64_blocks == 0
    Lo = oracle.kpp_factor(A, s, lam)
    worst = 0.0
    for j in range(P.nb):
        Lj = oracle.factor_block(Lo, j, m, s)
        As = A[j * s:(j + 1) * s]
        ev = np.linalg.eigvalsh(As @ As.T + lam * np.eye(As.shape[0]))
        bound = ev[-1] / ev[0] * (n + s + 1) * EPS32
        Lg = F.block(j)
        assert np.all(np.triu(Lg, 1) == 0.0)
        err = np.linalg.norm(Lg - Lj) / np.linalg.norm(Lj)
        worst = max(worst, err / bound)
        assert err <= bound, (j, err, bound)
    record_property("worst_err_over_bound", worst)


def test_fp64_storage_factors_every_block_in_fp64(K):
    A = np.random.default_rng(4).standard_normal((300, 200))
    P = K.Partition(300, 64)
    F = K.Factors(dev(A), P, 1e-3, 0)
    assert F.fp64_blocks == P.nb


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
def test_ill_conditioned_block_is_refactored_in_fp64(K, record_property, dtype):
    """Block 1 holds two rows that differ in one entry by about 0.02, so its Gram has an eigenvalue near
    lambda = 1e-2 beside pivots of order n = 1024: its pivot ratio (about 1e5) is above
    2^24 / (s + 1) = 32704, while the other blocks' ratios stay below 20.  That block alone is factored in
    FP64 (its factor then matches the oracle's up to the Gram's FP32 accumulation), and the refined solve
    still meets 1e-8 and the oracle's solution."""
    m, n, s, lam = 4096, 1024, 512, 1e-2
    rng = np.random.default_rng(77)
    A = rng.standard_normal((m, n))
    A[s + 7] = A[s + 6]
    A[s + 7, 5] += 0.02
    A = W.round_to_storage(A, dtype)
    assert 0.0 < abs(A[s + 7, 5] - A[s + 6, 5]) < 0.05
    x_star = rng.standard_normal(n)
    b = A @ x_star
    Ad = dev(A, TDT[dtype])
    P = K.Partition(m, s)
    F = K.Factors(Ad, P, lam, 0)
    assert F.fp64_blocks == 1
    Lo = oracle.kpp_factor(A, s, lam)
    for j in range(P.nb):
        Lj = oracle.factor_block(Lo, j, m, s)
        As = A[j * s:(j + 1) * s]
        ev = np.linalg.eigvalsh(As @ As.T + lam * np.eye(s))
        # the Gram's FP32 accumulation error, n 2^-24 of its largest entry, moved by kappa(G)
        bound = ev[-1] / ev[0] * (n + s + 1) * EPS32
        err = np.linalg.norm(F.block(j) - Lj) / np.linalg.norm(Lj)
        assert err <= bound, (j, err, bound)
    x = dev(np.zeros(n))
    prm = K.params(lam=lam, tol=1e-8, refine=1, inner_tol=1e-3, seed=2)
    rep = K.kpp_solve(Ad, dev(b), x, P, F, prm)
    assert rep.status == K.OK and rep.rel_res_true <= 1e-8
    res = oracle.run(A, b, Lo, s, lam=lam, tol=1e-12, max_iters=400000, seed=2)
    assert res.status == oracle.OK
    sv = np.linalg.svd(A, compute_uv=False)
    xg = x.cpu().numpy()
    err = np.linalg.norm(xg - res.x) / np.linalg.norm(res.x)
    bound = sv[0] / sv[-1] * (rep.rel_res_true + res.rel_res_true)
    record_property("err_vs_oracle", err)
    assert err <= bound, (err, bound)


def test_not_spd_block_is_reported_under_mixed_storage(K):
    """A zero block row with lambda = 0 fails in FP32, is handed to the FP64 pass, fails there too, and
    the factor phase reports it as not SPD."""
    A = np.random.default_rng(3).standard_normal((512, 256)).astype(np.float32)
    A[300] = 0.0
    F = K.Factors(dev(A, torch.float32), K.Partition(512, 128), 0.0, 0, allow_not_spd=True)
    assert F.status == K.ERR_NOT_SPD and F.bad_block == 2
