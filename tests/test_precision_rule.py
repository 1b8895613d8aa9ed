"""The rule that decides which block Grams the mixed-precision factor phase factors in FP64.

Under BF16 / FP32 storage every block is factored in FP32 and refactored in FP64 only when an FP32 pivot
fails or when the ratio of the largest to the smallest pivot L_cc^2 exceeds 2^24 / (s + 1).  These CPU
tests pin the two facts the rule rests on, with LAPACK factors in FP64:

* the pivots are diagonals of successive Schur complements of G, so every pivot lies in
  [lambda_min(G), lambda_max(G)] and the pivot ratio is a lower bound on kappa(G);
* on the mixed-precision LS workload's recipe (Z D V^T with Z ~ N(0, 1/m), 100 outliers log-spaced
  10..1000 and a bulk in [0.5, 1], lambda = 1e-3, s = 512) the blocks' pivot ratios stay well below the
  threshold (so no block of the bench line goes to FP64), although kappa(G) itself is about 4e5;
* a block with two nearly equal rows has a pivot ratio above the threshold (so it does go to FP64).
"""
import numpy as np
import pytest


def pivots(G):
    return np.diag(np.linalg.cholesky(G)) ** 2


def threshold(s):
    return 2.0 ** 24 / (s + 1)


@pytest.mark.parametrize("n,seed", [(8, 0), (40, 1), (128, 2)])
def test_pivots_lie_in_the_spectrum_and_bound_kappa_from_below(n, seed):
    rng = np.random.default_rng(seed)
    for trial in range(20):
        # spectra from well to badly conditioned, random eigenvectors
        q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        ev = np.logspace(0, rng.uniform(0, 8), n)
        G = (q * ev) @ q.T
        G = 0.5 * (G + G.T)
        p = pivots(G)
        lo, hi = ev.min(), ev.max()
        assert np.all(p >= lo * (1 - 1e-8)) and np.all(p <= hi * (1 + 1e-8))
        assert p.max() / p.min() <= hi / lo * (1 + 1e-8)


def test_lowrank_ls_blocks_stay_below_the_threshold():
    m, n, s = 262144, 4096, 512
    rng = np.random.default_rng(5)
    d = np.concatenate([np.logspace(1, 3, 100), rng.uniform(0.5, 1.0, n - 100)])
    worst, kappa = 0.0, 0.0
    for _ in range(6):
        Z = rng.standard_normal((s, n)) / np.sqrt(m)
        G = (Z * d ** 2) @ Z.T + 1e-3 * np.eye(s)  # A_S A_S^T with A = Z D V^T (V orthogonal drops out)
        p = pivots(G)
        worst = max(worst, p.max() / p.min())
        ev = np.linalg.eigvalsh(G)
        kappa = max(kappa, ev[-1] / ev[0])
    assert kappa > 1e5                      # ill-conditioned by kappa alone
    assert worst < threshold(s) / 2.0       # yet clear of the FP32 elimination floor


def test_nearly_dependent_rows_go_to_fp64():
    rng = np.random.default_rng(77)
    s, n, lam = 512, 1024, 1e-2
    A = rng.standard_normal((s, n))
    A[8] = A[7]
    A[8, 5] += 0.02
    p = pivots(A @ A.T + lam * np.eye(s))
    assert p.max() / p.min() > threshold(s)
    B = rng.standard_normal((s, n))
    p = pivots(B @ B.T + lam * np.eye(s))
    assert p.max() / p.min() < 20.0
