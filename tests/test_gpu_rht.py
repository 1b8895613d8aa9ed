"""GPU parity of the randomized Hadamard preprocessing of CD++ (Sec. 5.1; kpp_rht_forward /
kpp_rht_inverse through the C ABI) against the FP64 oracle's explicit definition Q = H_n diag(d) / sqrt(n).

Both sides scale by d_i d_j / n exactly (d = +-1, n a power of 2) and differ only in the order of the
sums: the oracle adds n terms left to right for each of its two products, the GPU runs log2 n
butterfly levels per side.  For entries of size |A| the difference is a few 1e-15 |A|; the bound used
is 1e-12 max|A| per entry (a wrong sign, index or scale is an O(|A|) error).
"""
import ctypes
import math

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


def _sym(n, seed):
    A = np.random.default_rng(seed).standard_normal((n, n))
    return A + A.T


@pytest.mark.parametrize("n", [1, 2, 8, 16, 32, 64, 512])
@pytest.mark.parametrize("k", [0, 1, 3])
def test_rht_forward_and_inverse_match_oracle(K, n, k):
    """All index-bit splits: n = 2, 8 (one partial radix pass), 16 (one full pass), 32 (full + 1 bit),
    64, 512 (full + 1 / 2 bits); k = 0 (matrix only), a vector and a 3-column panel."""
    A, d = _sym(n, 11 + n), W.rademacher_signs(n, 21 + n)
    B = np.random.default_rng(31 + n).standard_normal((n, max(k, 1)))[:, :k]
    Ao, Bo = oracle.rht_forward(d, A, B if k else None)
    Ad, dd = dev(A), dev(d)
    Abar, bbar = K.rht_forward(dd, Ad, dev(B) if k else None)
    tol = 1e-12 * np.abs(A).max()
    assert np.abs(Abar.cpu().numpy() - Ao).max() <= tol
    if k:
        assert np.abs(bbar.cpu().numpy() - Bo).max() <= 1e-12 * np.abs(B).max() * max(1.0, math.sqrt(n))
        xo = oracle.rht_inverse(d, Bo)
        x = K.rht_inverse(dd, dev(Bo)).cpu().numpy()
        assert np.abs(x - xo).max() <= 1e-12 * np.abs(B).max() * max(1.0, math.sqrt(n))
        assert np.abs(x - B).max() <= 1e-12 * np.abs(B).max() * max(1.0, math.sqrt(n))  # Q^T Q = I
    # the input is left untouched
    assert torch.equal(Ad, dev(A))


def test_rht_in_place_matrix_and_vector(K):
    """Abar may overwrite A, bbar may overwrite b, x may overwrite xbar (raw C-ABI calls)."""
    n = 64
    A, d, b = _sym(n, 5), W.rademacher_signs(n, 6), np.random.default_rng(7).standard_normal(n)
    Ao, bo = oracle.rht_forward(d, A, b)
    Ad, bd, dd = dev(A), dev(b), dev(d)
    m = K.matrix(Ad)
    lib, vp = K.load(), ctypes.c_void_p
    K._check(lib.kpp_rht_forward(n, vp(dd.data_ptr()), ctypes.byref(m), vp(Ad.data_ptr()), vp(bd.data_ptr()),
                                 vp(bd.data_ptr()), 1, None))
    torch.cuda.synchronize()
    assert np.abs(Ad.cpu().numpy() - Ao).max() <= 1e-12 * np.abs(A).max()
    assert np.abs(bd.cpu().numpy() - bo).max() <= 1e-12 * np.abs(b).max() * math.sqrt(n)
    K._check(lib.kpp_rht_inverse(n, vp(dd.data_ptr()), vp(bd.data_ptr()), vp(bd.data_ptr()), 1, None))
    torch.cuda.synchronize()
    assert np.abs(bd.cpu().numpy() - b).max() <= 1e-12 * np.abs(b).max() * math.sqrt(n)


def test_rht_rejects_bad_arguments(K):
    A = dev(np.eye(6))
    with pytest.raises(K.KppError):
        K.rht_forward(dev(np.ones(6)), A)                       # not a power of 2
    with pytest.raises(K.KppError):
        K.rht_forward(dev(np.ones(8)), dev(np.eye(8)).float())  # not FP64


def test_rht_full_size_sampled_entries_and_invariants(K):
    """n = 4096 (the CD++ workload's size): 40 entries of Abar computed one by one by the oracle, bbar
    against the oracle's recursive FHT, and the invariants of an orthogonal similarity (trace,
    Frobenius norm) on the whole matrix."""
    n = 4096
    A, d = _sym(n, 41), W.rademacher_signs(n, 42)
    b = np.random.default_rng(43).standard_normal(n)
    Abar, bbar = K.rht_forward(dev(d), dev(A), dev(b))
    Ab = Abar.cpu().numpy()
    rng = np.random.default_rng(44)
    pts = [(0, 0), (n - 1, n - 1), (0, n - 1), (n - 1, 0), (n // 2, n // 2 - 1)]
    pts += [tuple(int(v) for v in rng.integers(0, n, 2)) for _ in range(35)]
    for i, j in pts:
        assert abs(Ab[i, j] - oracle.rht_entry(d, A, i, j)) <= 1e-12 * np.abs(A).max(), (i, j)
    assert abs(np.trace(Ab) - np.trace(A)) <= 1e-10 * np.abs(A).sum() / n
    assert abs(np.linalg.norm(Ab) - np.linalg.norm(A)) <= 1e-12 * np.linalg.norm(A)
    assert np.abs(Ab - Ab.T).max() <= 1e-12 * np.abs(A).max()
    bo, _ = oracle.fht(d * b / math.sqrt(n))
    assert np.abs(bbar.cpu().numpy() - bo).max() <= 1e-12 * np.abs(b).max() * math.sqrt(n)


def test_cdpp_on_transformed_system_solves_the_original(K):
    """CD++ with the preprocessing (Alg. 3: transform, iterate on Q A Q^T, return Q^T xbar): the FP64
    residual of the original system reaches 1e-8, and x matches numpy's solve within kappa * 1e-8."""
    n, s = 512, 64
    A, b, sig = W.spd(n, 8, 1e2, 1e4, 1.0, 10.0, seed_A=51, seed_b=52)
    d = W.rademacher_signs(n, 53)
    dd = dev(d)
    Abar, bbar = K.rht_forward(dd, dev(A), dev(b))
    P = K.Partition(n, s)
    F = K.Factors(Abar, P, 1e-4, 1)
    xbar = torch.zeros(n, dtype=torch.float64, device="cuda")
    rep = K.cdpp_solve(Abar, bbar, xbar, P, F, K.params(lam=1e-4, tol=1e-8, seed=3))
    assert rep.status == K.OK
    x = K.rht_inverse(dd, xbar).cpu().numpy()
    res = np.linalg.norm(A @ x - b) / np.linalg.norm(b)
    assert res <= 1.0001e-8
    xs = np.linalg.solve(A, b)
    kappa = sig.max() / sig.min()
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= kappa * 1e-8
