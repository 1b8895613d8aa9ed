"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances (FP64 path): relative iterate error <= 1e-10 at equal iteration counts, identical block
sequences (bitwise), identical stop iterations; final |Ax-b|/|b| <= 1e-8.  The FP32/BF16 forms are
compared on what is unique: the converged solution, within the bound |x - x_o| <= kappa * (res + res_o)
|x_o| implied by both residuals.
"""
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


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_device_block_draws_match_oracle(K):
    for nb, sys_id, seed in [(100, 0, 0), (64, 3, 123456789), (7, 11, 2**63 + 5), (1, 0, 1)]:
        d = K.sample_blocks(seed, sys_id, 0, 4096, nb).cpu().numpy()
        o = np.array([oracle.sample_block(seed, t, sys_id, nb) for t in range(4096)])
        np.testing.assert_array_equal(d, o)
    d = K.sample_blocks(9, 2, (1 << 33) + 17, 64, 13).cpu().numpy()
    o = np.array([oracle.sample_block(9, (1 << 33) + 17 + t, 2, 13) for t in range(64)])
    np.testing.assert_array_equal(d, o)


# (1003, 24, 5): 201 blocks, more than the GPU's SMs, with a ragged last block: the Cholesky runs as a
# launch of whole rounds of blocks and a launch of the last round, whose inverses follow it
@pytest.mark.parametrize("m,n,s", [(103, 37, 10), (64, 64, 64), (50, 200, 7), (1003, 24, 5)])
def test_kpp_factors_match_oracle(K, m, n, s):
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n))
    lam = 0.05
    P = K.Partition(m, s)
    F = K.Factors(dev(A), P, lam, 0)
    L = oracle.kpp_factor(A, s, lam)
    for j in range(P.nb):
        Lo = oracle.factor_block(L, j, m, s)
        np.testing.assert_allclose(F.block(j), Lo, rtol=1e-11, atol=1e-11 * np.abs(Lo).max())


def test_cdpp_factors_and_not_spd(K):
    A, b, _ = W.spd(96, 4, 10.0, 100.0, 1.0, 2.0, seed_A=5, seed_b=6)
    P = K.Partition(96, 20)
    F = K.Factors(dev(A), P, 1e-4, 1)
    L = oracle.cdpp_factor(A, 20, 1e-4)
    for j in range(P.nb):
        Lo = oracle.factor_block(L, j, 96, 20)
        np.testing.assert_allclose(F.block(j), Lo, rtol=1e-11, atol=1e-12 * np.abs(Lo).max())
    # a block with two equal rows and lambda = 0 is singular: the factor reports it
    Bm = np.random.default_rng(1).standard_normal((40, 30))
    Bm[25] = Bm[21]
    Fb = K.Factors(dev(Bm), K.Partition(40, 10), 0.0, 0, allow_not_spd=True)
    assert Fb.status == K.ERR_NOT_SPD and Fb.bad_block == 2


@pytest.mark.parametrize("zero_rows", [[902], [17, 902]])
def test_not_spd_block_reported_across_the_split_cholesky(K, zero_rows):
    # 200 blocks of 5 rows: blocks 0 .. 151 factor in the first launch, 152 .. 199 in the second.  A zero
    # row with lambda = 0 gives its block an exactly zero pivot; the smallest such block is reported,
    # wherever it is
    Bm = np.random.default_rng(2).standard_normal((1000, 30))
    Bm[zero_rows] = 0.0
    Fb = K.Factors(dev(Bm), K.Partition(1000, 5), 0.0, 0, allow_not_spd=True)
    assert Fb.status == K.ERR_NOT_SPD and Fb.bad_block == min(r // 5 for r in zero_rows)


def _kpp_pair(K, A, b, s, lam, T=None, tol=0.0, seed=3, grid=0, adaptive=True, x0=None, eta=None, cd=False,
              dtype=torch.float64):
    m, n = A.shape
    P = K.Partition(m, s)
    Ad = dev(A, dtype)
    F = K.Factors(Ad, P, lam, 1 if cd else 0)
    x = dev(np.zeros(n) if x0 is None else x0)
    prm = K.params(lam=lam, tol=tol, max_iters=T if T is not None else 10**6, seed=seed, grid=grid,
                   adaptive_rho=int(adaptive), eta=eta)
    solve = K.cdpp_solve if cd else K.kpp_solve
    rep = solve(Ad, dev(b), x, P, F, prm, allow_no_conv=True)
    Lo = oracle.cdpp_factor(A, s, lam) if cd else oracle.kpp_factor(A, s, lam)
    res = oracle.run(A, b, Lo, s, cd=cd, lam=lam, tol=tol, max_iters=T if T is not None else 10**6, seed=seed,
                     adaptive=adaptive, eta=eta, x0=x0)
    return x.cpu().numpy(), rep, res


@pytest.fixture(params=[1, 2, 3], ids=["general", "smallblock", "dataflow"])
def variant(request, K):
    K.set_kernel_variant(request.param)
    yield request.param
    K.set_kernel_variant(3)


@pytest.mark.parametrize("grid", [1, 3, 8, 40])
@pytest.mark.parametrize("shape", [(103, 37, 10), (104, 40, 10)])
def test_kpp_fp64_lockstep_ragged(K, variant, grid, shape):
    rng = np.random.default_rng(7)
    m, n, s = shape  # 11 blocks, the last of 3 (or 4) rows; 40 columns qualify for the small-block kernel
    A = rng.standard_normal((m, n)) @ np.diag(np.geomspace(1, 30, n))
    b = A @ rng.standard_normal(n)
    for T in (1, 5, 2 * 11 * 3, 2 * 11 * 7 + 4):
        x, rep, res = _kpp_pair(K, A, b, s, 1e-2, T=T, grid=grid)
        assert rep.iters == T == res.iters
        assert rel(x, res.x) <= 1e-10, (T, rel(x, res.x))


def test_kpp_fp64_lockstep_fixed_rho_and_no_momentum(K):
    rng = np.random.default_rng(8)
    A = rng.standard_normal((90, 60))
    b = rng.standard_normal(90)
    x, rep, res = _kpp_pair(K, A, b, 9, 0.3, T=150, adaptive=False, eta=0.0)
    assert rel(x, res.x) <= 1e-10
    x, rep, res = _kpp_pair(K, A, b, 9, 0.3, T=150, adaptive=False, eta=0.05)
    assert rel(x, res.x) <= 1e-10


def test_kpp_fp64_single_row_blocks_and_single_block(K):
    rng = np.random.default_rng(9)
    A = rng.standard_normal((30, 20))
    b = A @ rng.standard_normal(20)
    x, rep, res = _kpp_pair(K, A, b, 1, 0.0, T=200, eta=0.0, adaptive=False)
    assert rel(x, res.x) <= 1e-10
    A2 = rng.standard_normal((12, 40))
    b2 = rng.standard_normal(12)
    x, rep, res = _kpp_pair(K, A2, b2, 12, 0.0, T=1, eta=0.0, adaptive=False)
    np.testing.assert_allclose(x, np.linalg.pinv(A2) @ b2, rtol=1e-9, atol=1e-11)


def test_kpp_fp64_2000x200_to_tolerance(K, variant):
    sy = W.kpp_fp64_2000x200()
    x, rep, res = _kpp_pair(K, sy.A, sy.b, sy.s, sy.lam, tol=sy.tol, seed=0)
    assert rep.status == K.OK and res.status == oracle.OK
    assert rep.iters == res.iters
    assert rep.rel_res_true <= 1e-8
    assert rel(x, res.x) <= 1e-10


@pytest.mark.parametrize("grid", [1, 5, 16])
def test_cdpp_fp64_lockstep_ragged(K, variant, grid):
    A, b, _ = W.spd(200, 6, 1e2, 1e3, 1.0, 5.0, seed_A=10, seed_b=11)
    for T in (1, 7, 2 * 13 * 4, 2 * 13 * 9 + 5):
        x, rep, res = _kpp_pair(K, A, b, 16, 1e-4, T=T, grid=grid, cd=True)
        assert rep.iters == T == res.iters
        assert rel(x, res.x) <= 1e-10, (T, rel(x, res.x))


@pytest.mark.parametrize("grid", [0, 20, 24])
def test_cdpp_fp64_single_column_kernel_lockstep(K, grid):
    """The single-column FP64 dataflow kernel (column chunks <= 32, s <= 64): ragged last block, runs
    longer than the mailbox ring and several checkpoints, then a solve to tolerance that stops at the
    oracle's checkpoint (window sums reduced over the group, r republished after the true residual)."""
    A, b, _ = W.spd(640, 10, 1e2, 1e3, 1.0, 5.0, seed_A=14, seed_b=15)
    s = 50  # 13 blocks, the last of 40 rows
    for T in (3, 2 * 13 * 10 + 3, 700):
        x, rep, res = _kpp_pair(K, A, b, s, 1e-4, T=T, grid=grid, cd=True)
        assert rep.iters == T == res.iters
        assert rel(x, res.x) <= 1e-10, (T, rel(x, res.x))
    x, rep, res = _kpp_pair(K, A, b, s, 1e-4, tol=1e-9, grid=grid, cd=True)
    assert rep.status == K.OK and res.status == oracle.OK
    assert rep.iters == res.iters
    assert rep.rel_res_true <= 1e-9
    assert rel(x, res.x) <= 1e-10


def test_cdpp_fp64_nonzero_start(K):
    A, b, _ = W.spd(130, 3, 1e2, 1e3, 1.0, 5.0, seed_A=12, seed_b=13)
    x0 = np.random.default_rng(3).standard_normal(130)
    x, rep, res = _kpp_pair(K, A, b, 13, 1e-4, T=300, cd=True, x0=x0)
    assert rel(x, res.x) <= 1e-10


@pytest.mark.slow
def test_cdpp_fp64_spd4096_to_tolerance(K, variant):
    sy = W.cdpp_fp64_spd()
    x, rep, res = _kpp_pair(K, sy.A, sy.b, sy.s, sy.lam, tol=sy.tol, seed=1, cd=True)
    assert rep.status == K.OK and res.status == oracle.OK
    assert rep.iters == res.iters
    assert rep.rel_res_true <= 1e-8
    assert rel(x, res.x) <= 1e-10


def test_status_no_convergence_keeps_last_iterate(K):
    sy = W.kpp_fp64_2000x200()
    x, rep, res = _kpp_pair(K, sy.A, sy.b, sy.s, sy.lam, T=300, tol=1e-14, seed=0)
    assert rep.status == K.ERR_NO_CONVERGENCE and res.status == oracle.NO_CONVERGENCE
    assert rel(x, res.x) <= 1e-10


def test_argument_errors(K):
    A = dev(np.eye(8))
    P = K.Partition(8, 4)
    F = K.Factors(A, P, 0.1, 0)
    x = dev(np.zeros(8))
    with pytest.raises(K.KppError) as e:
        K.kpp_solve(A, dev(np.ones(8)), x, P, F, K.params(lam=0.2))  # lambda differs from the factors'
    assert e.value.status == K.ERR_ARG
    with pytest.raises(K.KppError):
        K.cdpp_solve(A, dev(np.ones(8)), x, P, F, K.params(lam=0.1))  # K++ factors used for CD++
    with pytest.raises(K.KppError):
        K.Factors(dev(np.ones((8, 5))), P, 0.1, 1)  # CD++ needs a square matrix


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_mixed_precision_refinement_reaches_1e8(K, variant, dtype):
    sy = W.kpp_mixed_lowrank(m=16384, n=512, s=128, n_out=16)
    A = W.round_to_storage(sy.A, dtype)
    b = A @ sy.x_star
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    m, n = A.shape
    P = K.Partition(m, sy.s)
    Ad = dev(A, tdt)
    assert np.array_equal(Ad.double().cpu().numpy(), A)
    F = K.Factors(Ad, P, sy.lam, 0)
    x = dev(np.zeros(n))
    rep = K.kpp_solve(Ad, dev(b), x, P, F, K.params(lam=sy.lam, tol=1e-8, refine=1, inner_tol=1e-3, seed=0))
    assert rep.status == K.OK and rep.rel_res_true <= 1e-8 and rep.outer >= 1
    xo = np.linalg.lstsq(A, b, rcond=None)[0]
    kappa = sy.spectrum.max() / sy.spectrum.min() * 2.0
    assert rel(x.cpu().numpy(), xo) <= kappa * 2e-8


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_single_column_cdpp_kernel_fp32_tracks_general_kernel(K, dtype):
    """CD++ inner FP32 iterations on one column through the single-column kernel (FP32 memo
    W32 = G^-1 A_S) against the general kernel: the same iteration to FP32 rounding after T steps;
    then refinement to 1e-8 reaches the solution of the stored system."""
    A, b, _ = W.spd(512, 8, 1e2, 1e3, 1.0, 10.0, seed_A=30, seed_b=31)
    Ar = W.round_to_storage(A, dtype)
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    P = K.Partition(512, 64)
    Ad = dev(Ar, tdt)
    F = K.Factors(Ad, P, 1e-4, 1)
    out = {}
    for v in (1, 3):
        K.set_kernel_variant(v)
        x = dev(np.zeros(512))
        K.cdpp_solve(Ad, dev(b), x, P, F, K.params(lam=1e-4, tol=0.0, max_iters=2 * 8 * 20 + 3, refine=0, seed=5),
                     allow_no_conv=True)
        out[v] = x.cpu().numpy()
    K.set_kernel_variant(3)
    # W = G^-1 A_S rounded once to FP32 against G^-1 applied to r each step: O(eps32 * kappa) apart
    assert rel(out[3], out[1]) <= 1e-4
    x = dev(np.zeros(512))
    rep = K.cdpp_solve(Ad, dev(b), x, P, F, K.params(lam=1e-4, tol=1e-8, refine=1, inner_tol=1e-3, seed=2))
    assert rep.status == K.OK and rep.rel_res_true <= 1e-8
    xo = np.linalg.solve(Ar, b)
    assert rel(x.cpu().numpy(), xo) <= 1e3 * 2e-8


def test_mixed_cdpp_refinement(K, variant):
    A, b, _ = W.spd(512, 8, 1e2, 1e3, 1.0, 10.0, seed_A=20, seed_b=21)
    A32 = W.round_to_storage(A, "f32")
    P = K.Partition(512, 64)
    Ad = dev(A32, torch.float32)
    F = K.Factors(Ad, P, 1e-4, 1)
    x = dev(np.zeros(512))
    rep = K.cdpp_solve(Ad, dev(b), x, P, F, K.params(lam=1e-4, tol=1e-8, refine=1, inner_tol=1e-3, seed=2))
    assert rep.status == K.OK and rep.rel_res_true <= 1e-8
    xo = np.linalg.solve(A32, b)
    assert rel(x.cpu().numpy(), xo) <= 1e3 * 2e-8


@pytest.mark.parametrize("shape", [(60, 25, 7), (60, 24, 6)])
def test_batched_multi_rhs_matches_single_rhs_oracle(K, variant, shape):
    nsys, k, lam = 3, 3, 0.05
    m, n, s = shape
    As, Bs = [], []
    for i in range(nsys):
        rng = np.random.default_rng(100 + i)
        As.append(rng.standard_normal((m, n)))
        Bs.append(rng.standard_normal((m, k)))
    P = K.Partition(m, s)
    Ad = [dev(a) for a in As]
    Fs = [K.Factors(a, P, lam, 0) for a in Ad]
    Xd = [dev(np.zeros((n, k))) for _ in range(nsys)]
    T = 2 * 9 * 5 + 3
    reps = K.kpp_solve_batched(Ad, [dev(bb) for bb in Bs], Xd, P, Fs,
                               K.params(lam=lam, tol=0.0, max_iters=T, seed=4, sys_id=10), allow_no_conv=True)
    assert len(reps) == nsys * k
    for i in range(nsys):
        L = oracle.kpp_factor(As[i], s, lam)
        for c in range(k):
            res = oracle.run(As[i], Bs[i][:, c], L, s, lam=lam, tol=0.0, max_iters=T, seed=4, sys=10 + i)
            assert rel(Xd[i][:, c].cpu().numpy(), res.x) <= 1e-10


def test_host_entry_point_matches_device_path(K):
    sy = W.kpp_fp64_2000x200()
    x_host = np.zeros(sy.A.shape[1])
    rep = K.solve_host(np.ascontiguousarray(sy.A), sy.b.copy(), x_host, sy.s, 0,
                       K.params(lam=sy.lam, tol=sy.tol, seed=0))
    assert rep.status == K.OK and rep.rel_res_true <= 1e-8
    x, rep2, res = _kpp_pair(K, sy.A, sy.b, sy.s, sy.lam, tol=sy.tol, seed=0)
    np.testing.assert_array_equal(x_host, x)


def _unpack_lower(G, j, rows, s):
    ln = min(s, rows - j * s)
    blk = G[j * s * s: j * s * s + ln * ln].reshape(ln, ln)
    return np.tril(blk)


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
@pytest.mark.parametrize("m,n,s", [(300, 1000, 128), (520, 200, 256), (1100, 776, 512), (64, 104, 64),
                                   (256, 4096, 256)])
def test_tensor_core_gram_matches_fp64_gram(K, dtype, m, n, s):
    """tcgen05 Gram (FP32 accumulation; TF32 products for FP32 storage) against the FP64 CUDA-core Gram
    and the oracle's definition, on the rounded storage values."""
    rng = np.random.default_rng(m + n + s)
    A = W.round_to_storage(rng.standard_normal((m, n)), dtype)
    tdt = torch.bfloat16 if dtype == "bf16" else torch.float32
    Ad = dev(A, tdt)
    lam = 0.25
    Gt, used = K.block_gram(Ad, s, lam, engine=2)
    assert used == 2
    if dtype == "f32":
        Gs, used3 = K.block_gram(Ad, s, lam, engine=3)
        assert used3 == 3
        Gs = Gs.cpu().numpy()
    G64, used64 = K.block_gram(Ad, s, lam, engine=1)
    assert used64 == 1
    Gt, G64 = Gt.cpu().numpy(), G64.cpu().numpy()
    nb = -(-m // s)
    # bf16 products are exact, so only FP32 accumulation errs: the tensor core sums K-slices of 16 exactly
    # enough and rounds once per slice, about (n / 16) * 2^-23 relative on a diagonal entry.  TF32
    # truncates each product to 11 bits (2^-10 relative) on top of that.
    tol = max(1e-6, (n / 16) * 2.0 ** -23) + (0.0 if dtype == "bf16" else 2.0 ** -9)
    for j in range(nb):
        ref = np.tril(A[j * s:(j + 1) * s] @ A[j * s:(j + 1) * s].T) + lam * np.eye(min(s, m - j * s))
        scale = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
        np.testing.assert_allclose(_unpack_lower(G64, j, m, s), ref, rtol=1e-12, atol=1e-12 * scale.max())
        err = np.abs(_unpack_lower(Gt, j, m, s) - ref) / np.tril(scale)
        assert np.nanmax(err) <= tol, (j, float(np.nanmax(err)))
        if dtype == "f32":
            # split TF32: products good to ~2^-21; three MMAs per K-slice round into the FP32 accumulator,
            # so three times the accumulation term above
            err3 = np.abs(_unpack_lower(Gs, j, m, s) - ref) / np.tril(scale)
            assert np.nanmax(err3) <= 3 * max(1e-6, (n / 16) * 2.0 ** -23) + 2.0 ** -19, (j, float(np.nanmax(err3)))


def test_tensor_core_gram_refuses_unaligned_rows_and_auto_falls_back(K):
    A = dev(np.ones((64, 777)), torch.bfloat16)  # 1554-byte rows: not a TMA stride
    with pytest.raises(K.KppError) as e:
        K.block_gram(A, 64, 0.0, engine=2)
    assert e.value.status == K.ERR_UNSUPPORTED
    G, used = K.block_gram(A, 64, 0.0, engine=0)
    assert used == 1
    np.testing.assert_allclose(G.cpu().numpy()[:64 * 64].reshape(64, 64)[5, 3], 777.0)


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
def test_mixed_storage_factors_match_oracle(K, dtype):
    """FP64 Cholesky of the tensor-core / CUDA-core Gram of the stored matrix, against the oracle's factor
    of the same (widened) matrix; tolerance from the FP32 accumulation of the Gram."""
    rng = np.random.default_rng(12)
    m, n, s = 600, 1024, 128
    A = W.round_to_storage(rng.standard_normal((m, n)), dtype)
    P = K.Partition(m, s)
    F = K.Factors(dev(A, torch.bfloat16 if dtype == "bf16" else torch.float32), P, 0.5, 0)
    L = oracle.kpp_factor(A, s, 0.5)
    for j in range(P.nb):
        Lo = oracle.factor_block(L, j, m, s)
        np.testing.assert_allclose(F.block(j), Lo, rtol=1e-4, atol=1e-4 * np.abs(Lo).max())


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
def test_true_residual_is_exact_fp64_of_stored_entries(K, dtype):
    """kpp_rel_residual widens stored entries exactly (integer rebias) and sums in FP64: compare with
    numpy FP64 on the widened matrix, including zeros and subnormal-range bf16 entries."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((300, 520))
    A[0, :10] = 0.0
    A[1, :10] = 1e-39  # subnormal in fp32 / bf16
    A[2, :10] = -3e-42
    Ar = W.round_to_storage(A, dtype) if dtype == "bf16" else A.astype(np.float32).astype(np.float64)
    x = rng.standard_normal(520)
    b = Ar @ x + 1e-3 * rng.standard_normal(300)
    got = K.rel_residual(dev(Ar, torch.bfloat16 if dtype == "bf16" else torch.float32), dev(b), dev(x))
    want = np.linalg.norm(b - Ar @ x) / np.linalg.norm(b)
    assert abs(got - want) <= 1e-12 * want


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_true_residual_widens_subnormal_zero_and_extreme_entries_exactly(K, dtype):
    """Rows made of subnormal, zero and extreme-exponent FP32 / BF16 entries, with x scaled so that each
    row's products are O(1): the FP64 residual is sensitive to every entry's widened value, and matches
    numpy's FP64 on the exactly widened matrix."""
    rng = np.random.default_rng(11)
    m, n = 64, 256
    mag = np.zeros((m, 1))
    mag[0:16] = 1e-40     # subnormal in FP32 and BF16
    mag[16:24] = 1e-44    # deep subnormal (a few mantissa bits)
    mag[24:40] = 1e30     # large normal
    mag[40:56] = 1e-37    # small normal
    mag[56:64] = 1.0
    A = rng.standard_normal((m, n)) * mag
    A[::5, ::7] = 0.0
    A[3, 0] = -0.0
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    Ad = dev(A, tdt)
    Ar = Ad.double().cpu().numpy()  # the stored values, exactly widened by torch on the host side
    assert np.count_nonzero((np.abs(Ar) < 1.1754943508222875e-38) & (Ar != 0)) > 100
    x = rng.standard_normal(n)
    rows_scale = 1.0 / np.maximum(np.abs(Ar).max(axis=1), 1e-300)
    # one x for all rows: scale columns so that each magnitude class contributes O(1) through its rows
    b = np.empty(m)
    res = []
    for lo, hi in [(0, 16), (16, 24), (24, 40), (40, 56), (56, 64)]:
        xs = x * rows_scale[lo]
        bb = Ar[lo:hi] @ xs + 1e-3 * rng.standard_normal(hi - lo)
        got = K.rel_residual(dev(Ar[lo:hi], tdt), dev(bb), dev(xs))
        want = np.linalg.norm(bb - Ar[lo:hi] @ xs) / np.linalg.norm(bb)
        res.append((got, want))
        assert abs(got - want) <= 1e-12 * want, (lo, got, want)


def _wide_batch(nsys, m, n, s, k, dtype, seed=0):
    As, Bs = [], []
    for i in range(nsys):
        A, B, _ = W.gaussian_rows(m, n, 2, 100.0, seed_A=seed + 10 * i, seed_b=seed + 10 * i + 1, k_rhs=k)
        As.append(W.round_to_storage(A, dtype))
        Bs.append(B)
    return As, Bs


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("k", [1, 3])
def test_streaming_batched_refinement_reaches_min_norm(K, dtype, k):
    """Wide under-determined systems (the streaming kernel): FP64 refinement to 1e-8 per column, and the
    result is the minimum-norm solution A^T (A A^T)^{-1} b (K++ from x0 = 0 stays in range(A^T))."""
    nsys, m, n, s = 3, 96, 16384, 32
    As, Bs = _wide_batch(nsys, m, n, s, k, dtype)
    lam = W.row_outlier_lambda(As[0])
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    P = K.Partition(m, s)
    Ad = [dev(a, tdt) for a in As]
    Fs = [K.Factors(a, P, lam, 0) for a in Ad]
    Xd = [dev(np.zeros((n, k))) for _ in range(nsys)]
    reps = K.kpp_solve_batched(Ad, [dev(b) for b in Bs], Xd, P, Fs,
                               K.params(lam=lam, tol=1e-8, refine=1, inner_tol=1e-4, seed=5))
    for i in range(nsys):
        Xmn = As[i].T @ np.linalg.solve(As[i] @ As[i].T, Bs[i])
        for c in range(k):
            r = reps[i * k + c]
            assert r.status == K.OK and r.rel_res_true <= 1e-8, r.as_dict()
            assert rel(Xd[i][:, c].cpu().numpy(), Xmn[:, c]) <= 1e-6


def test_streaming_kernel_tracks_general_kernel_in_fp32(K):
    """Same FP32 iteration through the streaming kernel and the general kernel: iterates agree to FP32
    rounding after T steps (different but fixed summation orders)."""
    nsys, m, n, s, k = 2, 64, 16384, 32, 3
    As, Bs = _wide_batch(nsys, m, n, s, k, "f32", seed=100)
    lam = W.row_outlier_lambda(As[0])
    P = K.Partition(m, s)
    Ad = [dev(a, torch.float32) for a in As]
    Fs = [K.Factors(a, P, lam, 0) for a in Ad]
    out = {}
    for v in (1, 3):
        K.set_kernel_variant(v)
        Xd = [dev(np.zeros((n, k))) for _ in range(nsys)]
        K.kpp_solve_batched(Ad, [dev(b) for b in Bs], Xd, P, Fs,
                            K.params(lam=lam, tol=0.0, max_iters=37, refine=0, seed=9), allow_no_conv=True)
        out[v] = [x.cpu().numpy() for x in Xd]
    K.set_kernel_variant(3)
    for i in range(nsys):
        assert rel(out[3][i], out[1][i]) <= 2e-5


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("k", [3, 8])
def test_streaming_kernel_uneven_short_chunks_track_general_kernel(K, dtype, k):
    """The streaming kernel with 43 column tiles over 5 CTAs (chunks of 8 and 9 tiles, the shortest the
    kernel takes): its prefetch runs close behind the X / M stores of the previous step.  The iterates
    after T steps agree with the general kernel's to FP32 rounding, for the k = 8 panel path and the
    generic one."""
    nsys, m, s = 2, 64, 32
    n = 43 * (32 if dtype == "f32" else 64)  # 43 tiles of 128 bytes per row
    As, Bs = _wide_batch(nsys, m, n, s, k, dtype, seed=300)
    lam = W.row_outlier_lambda(As[0])
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    P = K.Partition(m, s)
    Ad = [dev(a, tdt) for a in As]
    Bd = [dev(b) for b in Bs]
    Fs = [K.Factors(a, P, lam, 0) for a in Ad]
    out = {}
    for v in (1, 3):
        K.set_kernel_variant(v)
        prm = K.params(lam=lam, tol=0.0, max_iters=37, refine=0, seed=9, grid=5)
        Xd = [dev(np.zeros((n, k))) for _ in range(nsys)]
        if v == 3:
            plan = K.Plan(Ad, Bd, Xd, P, Fs, prm)
            info = plan.info()
            plan.close()
            assert info["kernel"] == 4 and info["grid"] == 5, info
        K.kpp_solve_batched(Ad, Bd, Xd, P, Fs, prm, allow_no_conv=True)
        out[v] = [x.cpu().numpy() for x in Xd]
    K.set_kernel_variant(3)
    for i in range(nsys):
        assert np.all(np.isfinite(out[3][i]))
        assert rel(out[3][i], out[1][i]) <= 2e-5


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
def test_large_block_kernel_tracks_general_kernel_in_fp32(K, dtype):
    """The large-block K++ kernel (memoised W = G^-1 A_S, one exchange per step over 4-CTA clusters)
    against the general kernel on the same FP32 iteration: iterates agree to FP32 rounding after T steps,
    and both refine to 1e-8 with the same solution."""
    sy = W.kpp_mixed_lowrank(m=16384, n=512, s=128, n_out=16)
    A = W.round_to_storage(sy.A, dtype)
    b = A @ sy.x_star
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    m, n = A.shape
    P = K.Partition(m, sy.s)
    Ad = dev(A, tdt)
    F = K.Factors(Ad, P, sy.lam, 0)
    out = {}
    for v in (1, 3):
        K.set_kernel_variant(v)
        x = dev(np.zeros(n))
        K.kpp_solve(Ad, dev(b), x, P, F, K.params(lam=sy.lam, tol=0.0, max_iters=2 * 128 * 2 + 7, refine=0, seed=4),
                    allow_no_conv=True)
        out[v] = x.cpu().numpy()
    K.set_kernel_variant(3)
    # the memoised W = G^-1 A_S is rounded once where the general kernel rounds G^-1 r every step; with
    # FP32 arithmetic (eps 6e-8) and block Grams of condition ~1e3 the iterates differ by O(1e-5)
    assert rel(out[3], out[1]) <= 1e-4
    x = dev(np.zeros(n))
    rep = K.kpp_solve(Ad, dev(b), x, P, F, K.params(lam=sy.lam, tol=1e-8, refine=1, inner_tol=1e-3, seed=0))
    assert rep.status == K.OK and rep.rel_res_true <= 1e-8
    kappa = sy.spectrum.max() / sy.spectrum.min() * 2.0
    assert rel(x.cpu().numpy(), sy.x_star) <= kappa * 2e-8


@pytest.mark.parametrize("n,s", [(200, 16), (192, 32)])
def test_batched_cdpp_panels_match_single_rhs_oracle(K, variant, n, s):
    """CD++ with right-hand-side panels (k = 3, two systems): every column against the oracle's
    single-RHS CD++ run with the same Philox stream."""
    nsys, k, lam = 2, 3, 1e-4
    As, Bs = [], []
    for i in range(nsys):
        A, _, _ = W.spd(n, 5, 1e2, 1e3, 1.0, 5.0, seed_A=300 + i, seed_b=301 + i)
        As.append(A)
        Bs.append(np.random.default_rng(310 + i).standard_normal((n, k)))
    P = K.Partition(n, s)
    Ad = [dev(a) for a in As]
    Fs = [K.Factors(a, P, lam, 1) for a in Ad]
    Xd = [dev(np.zeros((n, k))) for _ in range(nsys)]
    T = 2 * (-(-n // s)) * 4 + 5
    K.kpp_solve_batched(Ad, [dev(b) for b in Bs], Xd, P, Fs, K.params(lam=lam, tol=0.0, max_iters=T, seed=6, sys_id=20),
                        allow_no_conv=True, cd=True)
    for i in range(nsys):
        L = oracle.cdpp_factor(As[i], s, lam)
        for c in range(k):
            res = oracle.run(As[i], Bs[i][:, c], L, s, cd=True, lam=lam, tol=0.0, max_iters=T, seed=6, sys=20 + i)
            assert rel(Xd[i][:, c].cpu().numpy(), res.x) <= 1e-10, (variant, i, c)
