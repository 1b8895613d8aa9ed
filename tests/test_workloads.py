"""CPU checks that the seeded input generators build what the input recipe states.

The parity tests and the benchmark both draw their inputs from paper_2501_11673_gb300/workloads.py, so
these checks pin the inputs themselves: Haar factors, planted spectra, row outliers, storage rounding,
the serving stream.  The device generators (torch_*) are device-agnostic and run here on the CPU at
small sizes.
"""
import math

import numpy as np
import pytest

from paper_2501_11673_gb300 import workloads as W

torch = pytest.importorskip("torch")


def test_haar_factor_is_orthogonal_and_uniform():
    """Q^T Q = I, and the sign fix makes Q Haar: its first column is uniform on the sphere, so
    E[q11] = 0 and E[q11^2] = 1/n (without the fix QR's sign convention biases q11)."""
    n, draws = 6, 3000
    rng = np.random.default_rng(1)
    q11 = np.empty(draws)
    for i in range(draws):
        Q = W.haar_orthogonal(n, rng)
        if i < 5:
            np.testing.assert_allclose(Q.T @ Q, np.eye(n), atol=1e-13)
        q11[i] = Q[0, 0]
    assert abs(q11.mean()) <= 0.03                   # sd 0.0075
    assert abs((q11 ** 2).mean() - 1.0 / n) <= 0.015  # sd 0.0034
    gen = torch.Generator(device="cpu")
    gen.manual_seed(3)
    Qt = W.torch_haar(16, gen, device="cpu")
    np.testing.assert_allclose((Qt.T @ Qt).numpy(), np.eye(16), atol=1e-13)


def test_planted_spectrum_layout():
    """k outliers exactly geomspace(hi, lo, k), then the bulk sorted descending inside [bulk_lo, bulk_hi]."""
    sig = W.planted_spectrum(200, 10, 1e2, 1e3, 1.0, 2.0, np.random.default_rng(0))
    assert sig.shape == (200,)
    np.testing.assert_array_equal(sig[:10], np.geomspace(1e3, 1e2, 10))
    bulk = sig[10:]
    assert bulk.min() >= 1.0 and bulk.max() <= 2.0 and np.all(np.diff(bulk) <= 0)
    assert abs(bulk.mean() - 1.5) <= 0.1


def test_spd_has_the_planted_eigenvalues():
    """A = U diag(sigma) U^T is bitwise symmetric and its eigenvalues are sigma (host and device builds)."""
    A, b, sig = W.spd(64, 4, 1e2, 1e4, 1.0, 10.0, seed_A=5, seed_b=6)
    assert np.array_equal(A, A.T) and b.shape == (64,)
    np.testing.assert_allclose(np.linalg.eigvalsh(A), np.sort(sig), rtol=0, atol=1e-10 * sig.max())
    At, sigt = W.torch_spd(64, 4, 1e2, 1e4, 1.0, 10.0, seed=7, dtype="f64", device="cpu")
    At = At.numpy()
    assert np.array_equal(At, At.T)
    np.testing.assert_allclose(np.linalg.eigvalsh(At), np.sort(sigt.numpy()), rtol=0, atol=1e-10 * 1e4)
    np.testing.assert_allclose(sigt.numpy()[:4], np.geomspace(1e4, 1e2, 4), rtol=1e-14)
    Ab, _ = W.torch_spd(64, 4, 1e2, 1e4, 1.0, 10.0, seed=7, dtype="bf16", device="cpu")
    assert Ab.dtype == torch.bfloat16 and torch.equal(Ab, Ab.T)


def test_lowrank_ls_has_the_planted_singular_values_and_a_consistent_rhs():
    """A = Z diag(d) V^T with Z_ij ~ N(0, 1/m): Z^T Z -> I as m / n grows, so the singular values of A
    are d within the Marchenko-Pastur edge factors 1 +- sqrt(n/m); b = A x* exactly, and the noisy
    variant adds noise * N(0, I)."""
    m, n = 8000, 40
    A, b, xs, d = W.lowrank_ls(m, n, 4, 10.0, 1000.0, 0.5, 1.0, seed_A=9, seed_b=10)
    ratio = np.linalg.svd(A, compute_uv=False) / d
    edge = math.sqrt(n / m)
    assert ratio.min() >= 1 - edge - 0.05 and ratio.max() <= (1 + edge) + 0.05
    np.testing.assert_array_equal(b, A @ xs)
    _, bn, xn, _ = W.lowrank_ls(m, n, 4, 10.0, 1000.0, 0.5, 1.0, seed_A=9, seed_b=10, noise=1e-3)
    e = bn - A @ xn
    assert abs(e.std() / 1e-3 - 1.0) <= 0.05 and abs(e.mean()) <= 1e-4
    At, bt, xt, dt = W.torch_lowrank_ls(4096, 32, 3, 10.0, 1000.0, 0.5, 1.0, seed=11, dtype="f32", device="cpu")
    assert At.dtype == torch.float32 and bt.dtype == torch.float64
    torch.testing.assert_close(bt, At.double() @ xt, rtol=1e-15, atol=1e-12)
    rt = np.linalg.svd(At.double().numpy(), compute_uv=False) / dt.numpy()
    assert rt.min() >= 1 - math.sqrt(32 / 4096) - 0.05 and rt.max() <= 1 + math.sqrt(32 / 4096) + 0.05


def test_gaussian_rows_scale_exactly_the_listed_rows():
    """n_big rows chosen by a seeded permutation carry the scale; the rest are i.i.d. N(0, 1)."""
    m, n = 300, 2000
    A, B, rows = W.gaussian_rows(m, n, 5, 100.0, seed_A=12, seed_b=13, k_rhs=3)
    assert B.shape == (m, 3) and len(rows) == 5 and np.all(np.diff(rows) > 0)
    norms = np.linalg.norm(A, axis=1) / math.sqrt(n)
    big = np.zeros(m, dtype=bool)
    big[rows] = True
    assert np.all(np.abs(norms[big] / 100.0 - 1.0) <= 0.1) and np.all(np.abs(norms[~big] - 1.0) <= 0.1)
    lam = W.row_outlier_lambda(A)
    assert abs(lam / (1e-3 * n) - 1.0) <= 0.05  # median squared row norm of N(0,1) rows ~ n
    At, Bt, rt = W.torch_gaussian_rows(m, n, 5, 100.0, seed=14, k_rhs=2, device="cpu")
    nt = (At.double().norm(dim=1) / math.sqrt(n)).numpy()
    bigt = np.zeros(m, dtype=bool)
    bigt[rt.numpy()] = True
    assert bigt.sum() == 5 and np.all(np.abs(nt[bigt] / 100.0 - 1.0) <= 0.1) and np.all(np.abs(nt[~bigt] - 1.0) <= 0.1)


def test_bf16_storage_rounding_matches_torch():
    """Round to nearest even into BF16, including exact ties, against torch's own conversion."""
    rng = np.random.default_rng(15)
    vals = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-30, 30, 5000), [0.0, -0.0, 1.0]])
    hi = rng.integers(0, 0x7F80, 200, dtype=np.uint32) << 16  # finite upper halves, both signs below
    ties = np.concatenate([hi | 0x8000, hi | 0x18000, hi | 0x7FFF, hi | 0x8001]).astype(np.uint32)
    ties = np.concatenate([ties, ties | np.uint32(0x80000000)])
    vals = np.concatenate([vals, ties.view(np.float32).astype(np.float64)])
    vals = vals[np.isfinite(vals.astype(np.float32))]
    ref = torch.tensor(vals.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(W.round_to_storage(vals, "bf16"), ref)
    bits = torch.tensor(vals.astype(np.float32)).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(W.bf16_bits(vals), bits)
    np.testing.assert_array_equal(W.round_to_storage(vals, "f32"), vals.astype(np.float32).astype(np.float64))


def test_serving_catalog_and_request_stream():
    """Matrix sizes are multiples of 64, log-uniform in [512, 8192]; arrivals are Poisson with a 2 ms mean
    gap starting at 0; k in [1, 32]; every request has its own right-hand-side seed."""
    sizes = W.serving_catalog()
    assert len(sizes) == 32 and all(v % 64 == 0 and 512 <= v <= 8192 for v in sizes)
    logs = np.log(sizes)
    assert abs(logs.mean() - 0.5 * (math.log(512) + math.log(8192))) <= 0.5  # sd 0.14
    req = W.serving_requests()
    t = np.array([r[0] for r in req])
    assert len(req) == 1024 and t[0] == 0.0 and np.all(np.diff(t) >= 0)
    gaps = np.diff(t)
    assert abs(gaps.mean() - 2.0) <= 4 * 2.0 / math.sqrt(len(gaps))
    assert abs(gaps.std() / gaps.mean() - 1.0) <= 0.15  # exponential: sd = mean
    ks = np.array([r[2] for r in req])
    assert ks.min() >= 1 and ks.max() <= 32 and set(range(1, 33)) <= set(ks.tolist())
    assert all(0 <= r[1] < 32 for r in req) and len({r[3] for r in req}) == len(req)


def test_rademacher_signs():
    d = W.rademacher_signs(4096, 16)
    assert set(np.unique(d).tolist()) == {-1.0, 1.0} and abs(d.mean()) <= 4 / math.sqrt(4096)
    np.testing.assert_array_equal(d, W.rademacher_signs(4096, 16))
    assert not np.array_equal(d, W.rademacher_signs(4096, 17))


def test_stays_spd_flags_a_rounded_matrix_whose_spectrum_crossed_the_margin():
    """stays_spd(A, margin) is whether A - margin I is positive definite (the check that decides FP32
    storage for a BF16-rounded serving matrix)."""
    A, _ = W.torch_spd(32, 2, 1e2, 1e3, 1.0, 2.0, seed=9, dtype="f64", device="cpu")
    lo = float(torch.linalg.eigvalsh(A).min())
    assert W.stays_spd(A, 0.5 * lo) and not W.stays_spd(A, 1.5 * lo)
    Ab, _ = W.torch_spd(32, 2, 1e2, 1e3, 1.0, 2.0, seed=9, dtype="bf16", device="cpu")
    lob = float(torch.linalg.eigvalsh(Ab.double()).min())
    assert W.stays_spd(Ab, 0.9 * lob) and not W.stays_spd(Ab, 1.1 * lob)
