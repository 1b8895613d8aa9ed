"""Seeded synthetic workloads for Kaczmarz++ / CD++ (inputs only, no solver arithmetic).

The paper evaluates on matrices whose spectrum has a few large outlying singular values over a flat
bulk (Sec. 6 and App. F: scikit-learn low-rank matrices and kernel matrices of public datasets).
Those datasets are not used here; the planted-spectrum matrices below stand in for them:

* ``lowrank_ls``: over-determined ``A = Z diag(d) V^T`` with ``Z`` i.i.d. Gaussian, ``V`` Haar
  orthogonal, ``d`` = k log-spaced outliers plus a uniform bulk; consistent ``b = A x*`` (plus an
  optional Gaussian noise term).
* ``spd``: dense symmetric positive definite ``A = U diag(sigma) U^T`` with ``U`` Haar orthogonal.
* ``gaussian_rows``: under-determined i.i.d. N(0,1) rows, some rows scaled up (row outliers).

Haar matrices come from the QR factorisation of a Gaussian matrix with the signs of ``diag(R)`` moved
into ``Q`` (Mezzadri, "How to generate random matrices from the classical compact groups", 2007).

This module is shared by the tests and the benchmark so that both sides of a parity check see the
same arrays; it never calls the solver, the oracle or the CUDA library.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def haar_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed n x n orthogonal matrix (QR of a Gaussian, sign-fixed)."""
    g = rng.standard_normal((n, n))
    q, r = np.linalg.qr(g)
    q *= np.sign(np.diag(r))[None, :]
    return q


def planted_spectrum(n_total: int, n_out: int, out_lo: float, out_hi: float,
                     bulk_lo: float, bulk_hi: float, rng: np.random.Generator) -> np.ndarray:
    """n_out log-spaced outliers in [out_lo, out_hi] (descending) followed by a uniform bulk."""
    out = np.geomspace(out_hi, out_lo, n_out) if n_out > 0 else np.zeros(0)
    bulk = rng.uniform(bulk_lo, bulk_hi, n_total - n_out)
    return np.concatenate([out, np.sort(bulk)[::-1]])


@dataclasses.dataclass
class System:
    """One linear system A x = b with its metadata (all arrays FP64, row-major, C-contiguous)."""
    A: np.ndarray
    b: np.ndarray
    x_star: np.ndarray | None
    s: int
    lam: float
    tol: float
    name: str
    spectrum: np.ndarray | None = None


def lowrank_ls(m: int, n: int, n_out: int, out_lo: float, out_hi: float, bulk_lo: float,
               bulk_hi: float, seed_A: int, seed_b: int, noise: float = 0.0) -> tuple:
    """Over-determined A = Z diag(d) V^T (Z_ij ~ N(0, 1/m)), x* ~ N(0, I), b = A x* (+ noise)."""
    rng = np.random.default_rng(seed_A)
    z = rng.standard_normal((m, n)) * (1.0 / math.sqrt(m))
    v = haar_orthogonal(n, rng)
    d = planted_spectrum(n, n_out, out_lo, out_hi, bulk_lo, bulk_hi, rng)
    A = np.ascontiguousarray(z @ (d[:, None] * v.T))
    rb = np.random.default_rng(seed_b)
    x_star = rb.standard_normal(n)
    b = A @ x_star
    if noise:
        b = b + noise * rb.standard_normal(m)
    return A, b, x_star, d


def spd(n: int, n_out: int, out_lo: float, out_hi: float, bulk_lo: float, bulk_hi: float,
        seed_A: int, seed_b: int) -> tuple:
    """Exactly symmetric A = U diag(sigma) U^T with U Haar; b ~ N(0, I)."""
    rng = np.random.default_rng(seed_A)
    u = haar_orthogonal(n, rng)
    sig = planted_spectrum(n, n_out, out_lo, out_hi, bulk_lo, bulk_hi, rng)
    A = (u * sig[None, :]) @ u.T
    A = np.ascontiguousarray(0.5 * (A + A.T))  # bitwise symmetric
    b = np.random.default_rng(seed_b).standard_normal(n)
    return A, b, sig


def rademacher_signs(n: int, seed: int) -> np.ndarray:
    """n independent +-1 signs (FP64), the diagonal of the randomized Hadamard transform's D."""
    return np.where(np.random.default_rng(seed).integers(0, 2, n) == 1, 1.0, -1.0)


def gaussian_rows(m: int, n: int, n_big: int, scale: float, seed_A: int, seed_b: int,
                  k_rhs: int = 1) -> tuple:
    """Under-determined A (m < n) with i.i.d. N(0,1) entries; n_big seeded rows scaled by `scale`."""
    rng = np.random.default_rng(seed_A)
    A = rng.standard_normal((m, n))
    rows = rng.permutation(m)[:n_big]
    A[rows] *= scale
    B = np.random.default_rng(seed_b).standard_normal((m, k_rhs))
    return np.ascontiguousarray(A), np.ascontiguousarray(B), np.sort(rows)


# ---------------------------------------------------------------------------------------------
# The five workloads (sizes as stated; `scale` shrinks the big ones for fast test variants).
# ---------------------------------------------------------------------------------------------

def kpp_fp64_2000x200() -> System:
    """K++ FP64: 2000 x 200 consistent LS, 10 outliers 1e2..1e3 over U[1,2]; s=20, lambda=1e-3, seed 0."""
    A, b, xs, d = lowrank_ls(2000, 200, 10, 1e2, 1e3, 1.0, 2.0, seed_A=0, seed_b=0)
    return System(A, b, xs, s=20, lam=1e-3, tol=1e-8, name="kpp_fp64_2000x200", spectrum=d)


def cdpp_fp64_spd(n: int = 4096, s: int = 64) -> System:
    """CD++ FP64: n x n SPD, 50 outliers log-spaced 1e2..1e4 over U[1,10]; s=64, lambda=1e-4."""
    n_out = 50 if n >= 1024 else max(1, n // 80)
    A, b, sig = spd(n, n_out, 1e2, 1e4, 1.0, 10.0, seed_A=1, seed_b=102)
    return System(A, b, None, s=s, lam=1e-4, tol=1e-8, name=f"cdpp_fp64_spd{n}", spectrum=sig)


def kpp_mixed_lowrank(m: int = 262144, n: int = 4096, s: int = 512, n_out: int = 100,
                      noise: float = 0.0) -> System:
    """Mixed-precision K++: m x n LS, n_out outliers log-spaced 10..1000 over U[0.5,1]; s=512."""
    A, b, xs, d = lowrank_ls(m, n, n_out, 10.0, 1000.0, 0.5, 1.0, seed_A=2, seed_b=103, noise=noise)
    return System(A, b, xs, s=s, lam=1e-3, tol=1e-8, name=f"kpp_mixed_{m}x{n}", spectrum=d)


def round_to_storage(A: np.ndarray, dtype: str) -> np.ndarray:
    """Round FP64 entries to the storage type and widen back (the stored matrix is the system)."""
    if dtype == "f64":
        return A
    if dtype == "f32":
        return A.astype(np.float32).astype(np.float64)
    if dtype == "bf16":
        a32 = A.astype(np.float32)
        u = a32.view(np.uint32).astype(np.uint64)
        # round-to-nearest-even on the upper 16 bits (finite inputs only)
        u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
        return u.astype(np.uint32).view(np.float32).astype(np.float64)
    raise ValueError(dtype)


def bf16_bits(A: np.ndarray) -> np.ndarray:
    """The bf16 bit patterns (uint16) of A rounded to nearest-even."""
    a32 = np.ascontiguousarray(A, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return u.astype(np.uint16)


def batched_minnorm(n_sys: int = 64, m: int = 2048, n: int = 65536, k_rhs: int = 8,
                    n_big: int = 20) -> list:
    """Batched under-determined min-norm K++ systems: A_i (m x n, FP32-stored) with row outliers."""
    out = []
    for i in range(n_sys):
        A, B, rows = gaussian_rows(m, n, n_big, 100.0, seed_A=3000 + i, seed_b=4000 + i, k_rhs=k_rhs)
        out.append((A, B, rows))
    return out


def row_outlier_lambda(A: np.ndarray) -> float:
    """lambda = 1e-3 * median squared row norm (the regulariser used for the row-outlier systems)."""
    return 1e-3 * float(np.median(np.einsum("ij,ij->i", A, A)))


def serving_catalog(n_mats: int = 32, n_lo: int = 512, n_hi: int = 8192, seed: int = 5000) -> list:
    """Sizes of the SPD matrices a serving run draws from (log-uniform in [n_lo, n_hi], multiple of 64)."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), n_mats))
    return [int(max(64, round(v / 64) * 64)) for v in sizes]


def serving_requests(n_req: int = 1024, n_mats: int = 32, mean_gap_ms: float = 2.0,
                     k_lo: int = 1, k_hi: int = 32, seed: int = 6000) -> list:
    """Request stream: (arrival_ms, matrix_id, k_rhs, rhs_seed), Poisson arrivals."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(mean_gap_ms, n_req)
    t = np.cumsum(gaps) - gaps[0]
    mats = rng.integers(0, n_mats, n_req)
    ks = rng.integers(k_lo, k_hi + 1, n_req)
    return [(float(t[i]), int(mats[i]), int(ks[i]), 1000 + i) for i in range(n_req)]


# ---------------------------------------------------------------------------------------------
# Device-side generators (torch, seeded) for the workloads too large to build on the host.
# Same recipes as above; the stored (rounded) matrix is the system and b is formed in FP64 from it.
# ---------------------------------------------------------------------------------------------

HOST_QR = False  # factor the Gaussian matrix of torch_haar on the host (see torch_haar)


def torch_haar(n: int, gen, device: str = "cuda"):
    """Haar orthogonal matrix from a seeded device Gaussian.  With HOST_QR the QR factorisation runs on
    the host (the same Gaussian; for profilers under which torch's device linear algebra cannot load)."""
    import torch
    g = torch.randn(n, n, generator=gen, device=device, dtype=torch.float64)
    if HOST_QR:
        q, r = torch.linalg.qr(g.cpu())
        q, r = q.to(device), r.to(device)
    else:
        q, r = torch.linalg.qr(g)
    return q * torch.sign(torch.diagonal(r))[None, :]


def torch_lowrank_ls(m: int, n: int, n_out: int, out_lo: float, out_hi: float, bulk_lo: float, bulk_hi: float,
                     seed: int, dtype: str = "bf16", noise: float = 0.0, device: str = "cuda"):
    """A = Z diag(d) V^T stored in `dtype` (Z_ij ~ N(0, 1/m), V Haar), x* ~ N(0, I), b = A_stored x* (FP64)."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    v = torch_haar(n, gen, device)
    out = torch.logspace(math.log10(out_hi), math.log10(out_lo), n_out, dtype=torch.float64, device=device)
    bulk = torch.rand(n - n_out, generator=gen, device=device, dtype=torch.float64) * (bulk_hi - bulk_lo) + bulk_lo
    d = torch.cat([out, torch.sort(bulk, descending=True).values])
    dvt = (d[:, None] * v.T).to(torch.float32)
    tdt = {"bf16": torch.bfloat16, "f32": torch.float32}[dtype]
    A = torch.empty(m, n, dtype=tdt, device=device)
    chunk = 16384
    old = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for r0 in range(0, m, chunk):
            z = torch.randn(min(chunk, m - r0), n, generator=gen, device=device, dtype=torch.float32)
            A[r0:r0 + z.shape[0]] = (z @ dvt * (1.0 / math.sqrt(m))).to(tdt)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old
    x_star = torch.randn(n, generator=gen, device=device, dtype=torch.float64)
    b = torch.empty(m, dtype=torch.float64, device=device)
    for r0 in range(0, m, chunk):
        b[r0:r0 + chunk] = A[r0:r0 + chunk].double() @ x_star
    if noise:
        b += noise * torch.randn(m, generator=gen, device=device, dtype=torch.float64)
    return A, b, x_star, d


def torch_gaussian_rows(m: int, n: int, n_big: int, scale: float, seed: int, k_rhs: int, dtype: str = "f32",
                        device: str = "cuda"):
    """Under-determined A (m x n, i.i.d. N(0,1), n_big seeded rows scaled), B ~ N(0, I) (m x k_rhs, FP64)."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    tdt = {"bf16": torch.bfloat16, "f32": torch.float32}[dtype]
    A = torch.randn(m, n, generator=gen, device=device, dtype=torch.float32)
    rows = torch.randperm(m, generator=gen, device=device)[:n_big]
    A[rows] *= scale
    B = torch.randn(m, k_rhs, generator=gen, device=device, dtype=torch.float64)
    return A.to(tdt), B, torch.sort(rows).values


def torch_spd(n: int, n_out: int, out_lo: float, out_hi: float, bulk_lo: float, bulk_hi: float, seed: int,
              dtype: str = "f64", device: str = "cuda"):
    """Exactly symmetric A = U diag(sigma) U^T (U Haar) in `dtype`, built in FP64 on the device."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    u = torch_haar(n, gen, device)
    out = torch.logspace(math.log10(out_hi), math.log10(out_lo), n_out, dtype=torch.float64, device=device)
    bulk = torch.rand(n - n_out, generator=gen, device=device, dtype=torch.float64) * (bulk_hi - bulk_lo) + bulk_lo
    sig = torch.cat([out, torch.sort(bulk, descending=True).values])
    A = (u * sig[None, :]) @ u.T
    A = 0.5 * (A + A.T)
    tdt = {"bf16": torch.bfloat16, "f32": torch.float32, "f64": torch.float64}[dtype]
    A = A.to(tdt)
    A = 0.5 * (A + A.T)  # symmetric again after rounding (exact: a + a = 2a, halving is exact)
    return A.contiguous(), sig


def stays_spd(A, margin: float) -> bool:
    """Whether the stored matrix (widened to FP64) minus margin * I is positive definite: rounding a
    matrix with a wide spectrum to BF16 can push its smallest eigenvalues below zero."""
    import torch
    Ad = A.double()
    Ad.diagonal().sub_(margin)
    return int(torch.linalg.cholesky_ex(Ad)[1].item()) == 0
