"""Pins for the FP64 oracle: each test checks it against something other than itself.

Paper: arXiv 2501.11673.  What pins what:
  * Philox4x32-10       -> published known-answer vectors (tests/golden/philox4x32_10_kat.txt)
  * block draw           -> its counter layout {t_lo, t_hi, system, 0} on the pinned generator; uniformity
  * Cholesky / solve     -> LAPACK through numpy
  * K++ step, lam > 0    -> the argmin definition of Eq. 1.3, solved through the n x n normal equations
  * K++ step, lam = 0    -> the projection invariant A_S x = b_S (Sec. 1.1) and, for s = 1, the classical
                            randomized Kaczmarz update; for one block = all rows, x = pinv(A) b
  * momentum             -> the (x, y, v) recursion of Lemma 2.3 with alpha, beta, gamma of Lemma 2.3
  * CD++ step            -> K++ on Phi with Phi Phi^T = A (Eq. 5.1 / the implicit form in the proof of Thm 5.1)
  * whole solves         -> x*, numpy.linalg.solve / lstsq / the min-norm solution; range invariance (Thm 2.1)
  * CG                   -> numpy.linalg.solve
  * online memo (Sec. 4, 5.2) -> uniform s-subsets (inclusion and pair frequencies), the Bernoulli schedule's
                            expected block count, the argmin / block-residual invariants on arbitrary
                            subsets, convergence to the direct solution, closed-form windows and rho on
                            diagonal systems
  * LSQR projection (Sec. 4.1) -> the regularised argmin (normal equations); one iteration when the sketch is
                            the whole (orthogonal) transform; the preconditioned condition number against tau;
                            the sketched Gram against scipy's Hadamard matrix
  * Hadamard preprocessing (Sec. 5.1) -> scipy.linalg.hadamard (Sylvester construction); the spectrum and
                            the solution are invariant (Q orthogonal); the SymFHT operation count of its
                            theorem, n^2 (2.5 + log2 n), and the recursion's exact count
  * adaptive rho, stop rule (Eq. 5.2, 5.3) -> closed forms on diagonal systems with eta = 0: each residual
                            entry decays by its own factor per draw of its block, so the windows E0 / E1,
                            the ratios, the weighted mean of Eq. 5.3 (written as an explicit weighted sum),
                            rho with its clamps, the confirmations and the stop iteration are all fixed
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2501_11673_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], tuple(v[6:10])))
    return rows


@pytest.mark.parametrize("ctr,key,expected", _kat_rows())
def test_philox_known_answers(ctr, key, expected):
    assert oracle.philox4x32_10(ctr, key) == expected


@pytest.mark.parametrize("seed,t,sys_id,nb", [(0, 0, 0, 100), (1234, 77, 3, 7), (2**40 + 5, 2**33 + 9, 11, 64),
                                             (2**64 - 1, 2**32 - 1, 2**32 - 1, 1), (9, 5, 0, 2**31 - 1)])
def test_block_draw_follows_the_counter_layout(seed, t, sys_id, nb):
    """The block of step t is j = (out0 * nb) >> 32 with out = Philox4x32-10(counter {t_lo, t_hi, system, 0},
    key {seed_lo, seed_hi}) (the sampling reading), built here from the known-answer-pinned generator."""
    m32 = 0xFFFFFFFF
    out = oracle.philox4x32_10([t & m32, t >> 32, sys_id, 0], [seed & m32, seed >> 32])
    assert oracle.sample_block(seed, t, sys_id, nb) == (out[0] * nb) >> 32


def test_block_sampling_uniform_and_in_range():
    nb = 7
    draws = np.array([oracle.sample_block(1234, t, 3, nb) for t in range(14000)])
    assert draws.min() >= 0 and draws.max() < nb
    counts = np.bincount(draws, minlength=nb)
    chi2 = float(((counts - 2000.0) ** 2 / 2000.0).sum())
    assert chi2 < 30.0  # 6 dof; p ~ 4e-5
    # different systems give different streams
    other = np.array([oracle.sample_block(1234, t, 4, nb) for t in range(200)])
    assert (other != draws[:200]).any()


def _rand_spd(n, rng, cond=1e3):
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.geomspace(1.0, cond, n)
    return (q * ev) @ q.T


def test_cholesky_matches_lapack_and_flags_indefinite():
    rng = np.random.default_rng(0)
    for n in (1, 5, 20, 37):
        G = _rand_spd(n, rng)
        G = 0.5 * (G + G.T)
        L = oracle.cholesky(G)
        np.testing.assert_allclose(L, np.linalg.cholesky(G), rtol=1e-10, atol=1e-12)
        r = rng.standard_normal(n)
        np.testing.assert_allclose(oracle.chol_solve(L, r), np.linalg.solve(G, r), rtol=1e-9, atol=1e-12)
    G = np.diag([1.0, 2.0, -1.0, 4.0])
    with pytest.raises(ValueError, match="pivot 2"):
        oracle.cholesky(G)


def _one_step(A, b, s, lam, x0, seed=7, cd=False, mom0=None, eta=0.0, rho=0.0):
    """One block step from x0 through the oracle; returns (x1, m1, j)."""
    rows = A.shape[0]
    L = oracle.cdpp_factor(A, s, lam) if cd else oracle.kpp_factor(A, s, lam)
    nb = -(-rows // s)
    j = oracle.sample_block(seed, 0, 0, nb)
    res = oracle.run(A, b, L, s, cd=cd, lam=lam, tol=0.0, max_iters=1, seed=seed, adaptive=False,
                     eta=eta, rho=rho, x0=x0, mom0=mom0)
    assert res.iters == 1
    return res.x, res.mom, j


@pytest.mark.parametrize("m,n,s", [(50, 30, 8), (47, 60, 10), (23, 5, 4)])
def test_kpp_step_is_regularised_argmin(m, n, s):
    """Eq. 1.3: x1 = argmin |A_S x - b_S|^2 + lam |x - x0|^2 (normal equations, independent of the oracle)."""
    rng = np.random.default_rng(m * n)
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    x0 = rng.standard_normal(n)
    lam = 0.37
    for seed in range(6):  # several blocks, including the ragged last one
        x1, _, j = _one_step(A, b, s, lam, x0, seed=seed)
        S = slice(j * s, min((j + 1) * s, m))
        As, bs = A[S], b[S]
        ref = np.linalg.solve(As.T @ As + lam * np.eye(n), As.T @ bs + lam * x0)
        np.testing.assert_allclose(x1, ref, rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("m,n,s", [(40, 60, 8), (43, 30, 6)])
def test_unregularised_step_is_a_projection(m, n, s):
    """lam = 0, eta = 0: after the step A_S x = b_S exactly (Sec. 1.1), and x1 - x0 lies in range(A_S^T)."""
    rng = np.random.default_rng(1 + m)
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    x0 = rng.standard_normal(n)
    for seed in range(5):
        x1, _, j = _one_step(A, b, s, 0.0, x0, seed=seed)
        S = slice(j * s, min((j + 1) * s, m))
        assert np.linalg.norm(A[S] @ x1 - b[S]) <= 1e-10 * np.linalg.norm(b[S])
        d = x1 - x0
        coef, *_ = np.linalg.lstsq(A[S].T, d, rcond=None)
        assert np.linalg.norm(A[S].T @ coef - d) <= 1e-10 * np.linalg.norm(d)


def test_single_row_blocks_are_classical_randomized_kaczmarz():
    """s = 1, lam = 0, eta = 0: x1 = x0 - (a_i^T x0 - b_i) / |a_i|^2 a_i (Strohmer-Vershynin update)."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((13, 9))
    b = rng.standard_normal(13)
    x0 = rng.standard_normal(9)
    for seed in range(5):
        x1, _, i = _one_step(A, b, 1, 0.0, x0, seed=seed)
        a = A[i]
        ref = x0 - (a @ x0 - b[i]) / (a @ a) * a
        np.testing.assert_allclose(x1, ref, rtol=1e-12, atol=1e-13)


def test_one_block_holding_all_rows_gives_min_norm_solution():
    """s = m, lam = 0, eta = 0, x0 = 0 on an under-determined system: one step gives pinv(A) b."""
    rng = np.random.default_rng(9)
    A = rng.standard_normal((12, 40))
    b = rng.standard_normal(12)
    x1, _, j = _one_step(A, b, 12, 0.0, np.zeros(40))
    assert j == 0
    np.testing.assert_allclose(x1, np.linalg.pinv(A) @ b, rtol=1e-10, atol=1e-12)


def test_momentum_matches_lemma_2_3_recursion():
    """Lemma 2.3: with beta = 1 - rho, gamma = 1 + eta/rho - eta, alpha = rho/(1+rho) and v0 = y0 = x0,
    the (x, y, v) recursion reproduces m <- (1-rho)/(1+rho)(m - w), x <- x - w + eta m (m0 = 0)."""
    rng = np.random.default_rng(11)
    m, n, s, lam = 60, 25, 6, 0.2
    A = rng.standard_normal((m, n))
    b = A @ rng.standard_normal(n)
    x0 = rng.standard_normal(n)
    rho, eta = 0.15, 0.2
    T = 40
    L = oracle.kpp_factor(A, s, lam)
    res = oracle.run(A, b, L, s, lam=lam, tol=0.0, max_iters=T, seed=3, adaptive=False, eta=eta, rho=rho, x0=x0)
    nb = -(-m // s)
    alpha, beta, gamma = rho / (1 + rho), 1 - rho, 1 + eta / rho - eta
    y = x0.copy()
    v = x0.copy()
    for t in range(T):
        x = alpha * v + (1 - alpha) * y
        j = oracle.sample_block(3, t, 0, nb)
        S = slice(j * s, min((j + 1) * s, m))
        As = A[S]
        w = As.T @ np.linalg.solve(As @ As.T + lam * np.eye(As.shape[0]), As @ x - b[S])
        y, v = x - w, beta * v + (1 - beta) * x - gamma * w
    x_T = alpha * v + (1 - alpha) * y
    np.testing.assert_allclose(res.x, x_T, rtol=1e-10, atol=1e-12)
    # the momentum vector itself: m_t = beta (1 - alpha) / (gamma - 1) (v_t - y_t)
    m_T = beta * (1 - alpha) / (gamma - 1) * (v - y)
    np.testing.assert_allclose(res.mom, m_T, rtol=1e-9, atol=1e-11)


def test_fixed_momentum_meets_the_general_convergence_theorem():
    """Sec. 2's general convergence theorem: with its mu and nu computed exactly by enumerating the blocks
    of the partition, rho = rhobar / 2 (c = 1/2) and eta = 1 / (2 nu), the mean of |x_t - x*|^2 over
    300 independent block sequences stays below 8 (1 - rho/2)^t |x_0 - x*|^2; and 1 <= nu <= 1/mu.  A weak,
    statistical pin (the bound is loose), kept because it ties the momentum form to the theorem's rate."""
    rng = np.random.default_rng(41)
    m, n, s, lam = 60, 20, 6, 0.5
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = U @ np.diag(np.concatenate([np.geomspace(30, 10, 3), rng.uniform(1, 2, n - 3)])) @ V.T * math.sqrt(m / n)
    xs = rng.standard_normal(n)
    b = A @ xs
    nb = m // s
    Ps = []
    for j in range(nb):
        As = A[j * s:(j + 1) * s]
        Ps.append(As.T @ np.linalg.solve(As @ As.T + lam * np.eye(s), As))
    Pbar = sum(Ps) / nb
    ev, Q = np.linalg.eigh(Pbar)
    mu = ev.min()
    Ph = Q @ np.diag(ev ** -0.5) @ Q.T
    nu = np.linalg.eigvalsh(sum((Ph @ P @ Ph) @ (Ph @ P @ Ph) for P in Ps) / nb).max()
    assert 1.0 <= nu <= 1.0 / mu
    rho, eta = math.sqrt(mu / nu) / 2, 1.0 / (2.0 * nu)
    L = oracle.kpp_factor(A, s, lam)
    x0 = rng.standard_normal(n)
    e0 = float(np.sum((x0 - xs) ** 2))
    T, ch, S = 300, 10, 300
    mean = np.zeros(T // ch)
    for seed in range(S):
        x, mom, st = x0.copy(), np.zeros(n), None
        for c in range(T // ch):
            r = oracle.run(A, b, L, s, lam=lam, tol=0.0, max_iters=(c + 1) * ch, seed=seed, adaptive=False, eta=eta,
                           rho=rho, x0=x, mom0=mom, state=st)
            x, mom, st = r.x, r.mom, r.state
            mean[c] += float(np.sum((x - xs) ** 2)) / S
    t = np.arange(1, T // ch + 1) * ch
    assert np.all(mean <= 8.0 * (1.0 - rho / 2.0) ** t * e0)


@pytest.mark.parametrize("adaptive", [False, True])
def test_cdpp_is_kpp_on_a_square_root(adaptive):
    """Eq. 5.1 / proof of Thm 5.1: CD++ on A = Phi Phi^T is K++ on Phi z = b with z_t = Phi^T x_t."""
    rng = np.random.default_rng(21)
    n, s, lam = 45, 7, 1e-3
    A = _rand_spd(n, rng, cond=1e2)
    A = 0.5 * (A + A.T)
    b = rng.standard_normal(n)
    Phi = np.linalg.cholesky(A)
    T = 6 * (-(-n // s)) * 2  # six checkpoints
    Lc = oracle.cdpp_factor(A, s, lam)
    Lk = oracle.kpp_factor(Phi, s, lam)
    kw = dict(lam=lam, tol=0.0, max_iters=T, seed=5, adaptive=adaptive, rho=0.0 if adaptive else 0.1,
              eta=s / (2.0 * n))
    rc = oracle.run(A, b, Lc, s, cd=True, **kw)
    rk = oracle.run(Phi, b, Lk, s, cd=False, **kw)
    np.testing.assert_allclose(rk.x, Phi.T @ rc.x, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(rk.trace[:, 1:4], rc.trace[:, 1:4], rtol=1e-9, atol=1e-14)


def test_fixed_point_is_kept():
    """x0 = x*, m0 = 0 on a consistent system: w = 0 up to rounding, so x stays at x*."""
    sy = W.kpp_fp64_2000x200()
    L = oracle.kpp_factor(sy.A, sy.s, sy.lam)
    res = oracle.run(sy.A, sy.b, L, sy.s, lam=sy.lam, tol=0.0, max_iters=400, seed=0, x0=sy.x_star)
    assert np.linalg.norm(res.x - sy.x_star) <= 1e-12 * np.linalg.norm(sy.x_star)


def test_kpp_converges_to_consistent_solution():
    """The 2000 x 200 consistent system: stop at |Ax-b|/|b| <= 1e-8 and x close to x*."""
    sy = W.kpp_fp64_2000x200()
    L = oracle.kpp_factor(sy.A, sy.s, sy.lam)
    res = oracle.run(sy.A, sy.b, L, sy.s, lam=sy.lam, tol=1e-8, max_iters=20000, seed=0)
    assert res.status == oracle.OK
    assert res.rel_res_true <= 1e-8
    x_ls = np.linalg.lstsq(sy.A, sy.b, rcond=None)[0]
    kappa = sy.spectrum.max() / sy.spectrum.min() * 2
    assert np.linalg.norm(res.x - x_ls) <= kappa * 1e-8 * np.linalg.norm(x_ls)
    # stop happens at a checkpoint  t = 2 zeta - 1 (mod 2 zeta)
    zeta = -(-sy.A.shape[0] // sy.s)
    assert res.iters % (2 * zeta) == 0


def test_underdetermined_stays_in_row_space_and_reaches_min_norm():
    """Thm 2.1 (minimum-norm solution): from x0 = 0 every iterate lies in range(A^T)."""
    rng = np.random.default_rng(31)
    m, n, s = 40, 120, 8
    A = rng.standard_normal((m, n))
    A[3] *= 30.0
    b = rng.standard_normal(m)
    L = oracle.kpp_factor(A, s, 1e-2)
    res = oracle.run(A, b, L, s, lam=1e-2, tol=1e-10, max_iters=50000, seed=2)
    assert res.status == oracle.OK
    q, _ = np.linalg.qr(A.T)
    null_part = res.x - q @ (q.T @ res.x)
    assert np.linalg.norm(null_part) <= 1e-12 * np.linalg.norm(res.x)
    x_mn = np.linalg.pinv(A) @ b
    assert np.linalg.norm(res.x - x_mn) <= 1e-7 * np.linalg.norm(x_mn)


def test_cdpp_converges_to_spd_solution():
    rng = np.random.default_rng(41)
    n, s = 256, 16
    A, b, _ = W.spd(n, 6, 1e2, 1e3, 1.0, 4.0, seed_A=41, seed_b=42)
    L = oracle.cdpp_factor(A, s, 1e-4)
    res = oracle.run(A, b, L, s, cd=True, lam=1e-4, tol=1e-9, max_iters=200000, seed=4)
    assert res.status == oracle.OK and res.rel_res_true <= 1e-9
    x = np.linalg.solve(A, b)
    assert np.linalg.norm(res.x - x) <= 1e-9 * 1e3 * np.linalg.norm(x)


def test_adaptive_rho_schedule_structure():
    """Alg. 3's checkpoints: every 2 zeta steps; rho in [0, 1); the first
    rho follows from the first ratio as 1 - (E1/E0)^(1/zeta)."""
    sy = W.kpp_fp64_2000x200()
    L = oracle.kpp_factor(sy.A, sy.s, sy.lam)
    res = oracle.run(sy.A, sy.b, L, sy.s, lam=sy.lam, tol=0.0, max_iters=2000, seed=0)
    zeta = 100
    tr = res.trace
    assert len(tr) == 10
    np.testing.assert_array_equal(tr[:, 0], np.arange(1, 11) * 2 * zeta - 1)
    assert tr[0, 3] == 0.0  # rho_0 = 0 (Alg. 3's initialisation)
    rho1 = 1.0 - (tr[0, 2] / tr[0, 1]) ** (1.0 / zeta)
    assert tr[1, 3] == pytest.approx(max(rho1, 0.0), rel=1e-12)
    assert np.all((res.trace[:, 3] >= 0) & (res.trace[:, 3] < 1))


def _weighted_mean_rhat(q):
    """Eq. 5.3 solved for rhat_i: a_i rhat_i = a_{i-1} rhat_{i-1} + (a_i - a_{i-1}) q_i with rhat_1 = q_1,
    so rhat_i = (a_1 q_1 + sum_{j=2..i} (a_j - a_{j-1}) q_j) / a_i, a_j = (j+1)^{ln(j+1)}."""
    a = [(j + 1.0) ** math.log(j + 1.0) for j in range(len(q) + 1)]
    out, acc = [], 0.0
    for i in range(1, len(q) + 1):
        acc += (a[1] if i == 1 else a[i] - a[i - 1]) * q[i - 1]
        out.append(acc / a[i])
    return out


def _diagonal_windows(cfac, b, s, seed, T):
    """E0/E1 windows of a diagonal system in closed form.  With A = diag(d), one step on block S
    multiplies each residual entry of S by its factor c_i (K++: lambda/(d_i^2 + lambda); CD++:
    lambda/(d_i + lambda)) and leaves the other entries alone, so after k_i draws of i's block the
    entry is -b_i c_i^{k_i}.  Window membership and checkpoint times follow Alg. 3.
    Returns zeta and, per checkpoint, (t, E0, E1, |A x_{t+1} - b|)."""
    n = len(b)
    nb = -(-n // s)
    zeta = nb
    k = np.zeros(n)
    E0 = E1 = 0.0
    ckpt = []
    for t in range(T):
        j = oracle.sample_block(seed, t, 0, nb)
        S = slice(j * s, min((j + 1) * s, n))
        e = float(np.sum((b[S] * cfac[S] ** k[S]) ** 2))
        k[S] += 1
        if t % (2 * zeta) < zeta:
            E0 += e
        else:
            E1 += e
        if t % (2 * zeta) == 2 * zeta - 1:
            ckpt.append((t, E0, E1, float(np.linalg.norm(b * cfac ** k))))
            E0 = E1 = 0.0
    return zeta, ckpt


@pytest.mark.parametrize("cd", [False, True])
@pytest.mark.parametrize("n,s,scales,lam_rel,T,rtol,kind", [
    (9, 9, (1.0,), 4.0, 12, 1e-9, "inside"),             # one block: zeta = 1, every window deterministic
    (12, 4, (1.0, 1.5, 0.7), 0.5, 90, 1e-8, "mixed"),    # zeta = 3 under the Philox draw
    (11, 4, (1.0, 1.5, 0.7), 0.5, 90, 1e-8, "mixed"),    # ragged last block: zeta = ceil(11/4) = 3
    (12, 4, (1.0, 1e2, 1e-2), 4.0, 90, 1e-8, "low"),     # ratios far above 1: rho stays at its lower clamp 0
    (4, 4, (1.0,), 1e-8, 2, 1e-6, "high"),               # ratio below 1e-12: rho hits its upper clamp
])
def test_adaptive_rho_follows_closed_form_windows_on_diagonal_systems(cd, n, s, scales, lam_rel, T, rtol, kind):
    """Eq. 5.2 and Eq. 5.3 with the checkpoints of Alg. 3 on diagonal systems with eta = 0 (momentum off, so
    rho never changes the iterates): the windows E0 and E1, the ratio q_i = E1/E0 at each checkpoint,
    rhat_i as the explicit weighted mean of Eq. 5.3's weights, rho_i = 1 - rhat_i^(1/zeta) clamped to
    [0, 1 - 1e-12] (readings 5 and 6), all from the closed-form residual decay.  The oracle forms each
    residual as A_S x - b_S, which loses digits as the residual shrinks (absolute error ~1e-16 |b| per
    step), so lambda keeps the decay factors >= 0.8 and rtol follows the smallest c_i^{k_i} reached."""
    rng = np.random.default_rng(900 + n + s)
    d = rng.uniform(1.0, 3.0, n)
    b = rng.standard_normal(n) * np.repeat(np.asarray(scales), s)[:n]
    A = np.diag(d)
    lam = lam_rel * (float(np.max(d)) if cd else float(np.max(d)) ** 2)
    cfac = lam / (d + lam) if cd else lam / (d * d + lam)
    L = oracle.cdpp_factor(A, s, lam) if cd else oracle.kpp_factor(A, s, lam)
    res = oracle.run(A, b, L, s, cd=cd, lam=lam, tol=0.0, max_iters=T, seed=7, eta=0.0)
    zeta, ck = _diagonal_windows(cfac, b, s, 7, T)
    tr = res.trace
    assert len(tr) == len(ck) == T // (2 * zeta)
    np.testing.assert_array_equal(tr[:, 0], [c[0] for c in ck])
    np.testing.assert_allclose(tr[:, 1], [c[1] for c in ck], rtol=rtol)
    np.testing.assert_allclose(tr[:, 2], [c[2] for c in ck], rtol=rtol)
    q = [c[2] / c[1] for c in ck]
    rhat = _weighted_mean_rhat(q)
    rho = [min(max(1.0 - r ** (1.0 / zeta), 0.0), 1.0 - 1e-12) for r in rhat]
    # the trace holds the rho in force at each checkpoint: 0 at the first (Alg. 3's initialisation), then rho_{i-1}
    np.testing.assert_allclose(tr[:, 3], [0.0] + rho[:-1], rtol=0, atol=10 * rtol)
    assert res.state.rhat == pytest.approx(rhat[-1], rel=10 * rtol)
    assert res.state.rho == pytest.approx(rho[-1], rel=0, abs=10 * rtol)
    # the reported estimate of Eq. 5.2 at the last checkpoint: sqrt(E1) / |b|
    assert res.rel_res_est == pytest.approx(math.sqrt(ck[-1][2]) / np.linalg.norm(b), rel=rtol)
    np.testing.assert_allclose(res.x, b / d * (1.0 - cfac ** _draw_counts(n, s, 7, T)), rtol=1e-12)
    if kind == "inside":
        assert min(rho) > 0.0 and max(rho) < 1.0 - 1e-12
    elif kind == "mixed":
        assert max(rho) > 0.0 and max(q) > 1.0
    elif kind == "low":
        assert q[0] > 1.0 and max(rho) == 0.0
    else:
        assert q[0] < 1e-12 and res.state.rho == 1.0 - 1e-12


@pytest.mark.parametrize("cd", [False, True])
@pytest.mark.parametrize("n,s,scales,lam_rel", [(9, 9, (1.0,), 4.0), (12, 4, (1.0, 30.0, 0.03), 0.5)])
def test_stop_rule_follows_closed_form_on_diagonal_systems(cd, n, s, scales, lam_rel):
    """Eq. 5.2's stopping test E1 <= eps^2 |b|^2 at each checkpoint (Alg. 3), confirmed by the true
    residual |Ax - b| / |b| <= eps before returning (reading 8): on diagonal systems with eta = 0 both sides
    of both tests are closed forms, so the stop iteration, the checkpoints where the confirmation ran and
    what it found are fixed.  With uneven block scales the window can pass while an undrawn block still
    holds a large residual; the confirmation must then reject and the run continue."""
    rng = np.random.default_rng(700 + n)
    d = rng.uniform(1.0, 3.0, n)
    b = rng.standard_normal(n) * np.repeat(np.asarray(scales), s)[:n]
    if len(scales) > 1:
        d[s:2 * s] *= 0.3  # the large block also converges slowest
    A = np.diag(d)
    lam = lam_rel * (float(np.max(d)) if cd else float(np.max(d)) ** 2)
    cfac = lam / (d + lam) if cd else lam / (d * d + lam)
    L = oracle.cdpp_factor(A, s, lam) if cd else oracle.kpp_factor(A, s, lam)
    eps, T = 1e-3, 3000
    res = oracle.run(A, b, L, s, cd=cd, lam=lam, tol=eps, max_iters=T, seed=7, eta=0.0)
    zeta, ck = _diagonal_windows(cfac, b, s, 7, T)
    bn = float(np.linalg.norm(b))
    stop, tested, rejected = None, [], 0
    for i, (t, _, E1, rn) in enumerate(ck):
        if E1 <= eps * eps * bn * bn:
            tested.append(i)
            if rn <= eps * bn:
                stop = i
                break
            rejected += 1
    assert stop is not None
    assert res.status == oracle.OK and res.iters == ck[stop][0] + 1
    tr = res.trace
    assert len(tr) == stop + 1
    assert np.flatnonzero(~np.isnan(tr[:, 4])).tolist() == tested
    np.testing.assert_allclose(tr[tested, 4], [ck[i][3] / bn for i in tested], rtol=1e-8)
    assert res.rel_res_true == pytest.approx(ck[stop][3] / bn, rel=1e-8)
    if len(scales) > 1:
        assert rejected > 0


def _draw_counts(n, s, seed, T):
    nb = -(-n // s)
    k = np.zeros(n)
    for t in range(T):
        j = oracle.sample_block(seed, t, 0, nb)
        k[j * s:min((j + 1) * s, n)] += 1
    return k


def test_cg_matches_direct_solve():
    rng = np.random.default_rng(51)
    A = _rand_spd(80, rng, cond=1e3)
    A = 0.5 * (A + A.T)
    b = rng.standard_normal(80)
    x, it, rr = oracle.cg(A, b, tol=1e-12)
    assert rr <= 1e-12
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-8)


def _krylov_minres_iterate(A, b, x0, k):
    """The definition of the k-th GMRES iterate: x0 + Q y with Q an orthonormal basis of
    K_k(A, r0) = span(r0, A r0, ..., A^(k-1) r0) (QR of the power basis) and y the least-squares
    minimiser of |b - A (x0 + Q y)|."""
    r0 = b - A @ x0
    Kb = np.empty((A.shape[0], k))
    v = r0 / np.linalg.norm(r0)
    for j in range(k):
        Kb[:, j] = v
        v = A @ v
        v = v / np.linalg.norm(v)
    Q, _ = np.linalg.qr(Kb)
    y = np.linalg.lstsq(A @ Q, r0, rcond=None)[0]
    return x0 + Q @ y


def test_gmres_iterates_are_the_krylov_minimal_residual_ones():
    rng = np.random.default_rng(52)
    n = 40
    A = np.eye(n) * 3.0 + rng.standard_normal((n, n)) * (0.6 / np.sqrt(n))  # nonsymmetric, well conditioned
    b = rng.standard_normal(n)
    x0 = rng.standard_normal(n) * 0.1
    for k in (1, 2, 4, 7):
        x, it, _, cyc = oracle.gmres(A, b, restart=50, tol=0.0, max_iters=k, x0=x0)
        assert it == k and cyc == 1
        xd = _krylov_minres_iterate(A, b, x0, k)
        assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd), k
    # the residual never grows with the steps of one cycle, and n steps solve the system
    res = [np.linalg.norm(b - A @ oracle.gmres(A, b, restart=n, tol=0.0, max_iters=k, x0=x0)[0]) for k in range(1, 12)]
    assert all(r2 <= r1 * (1 + 1e-12) for r1, r2 in zip(res, res[1:]))
    x, it, rr, _ = oracle.gmres(A, b, restart=n, tol=0.0, max_iters=n, x0=x0)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-12)


def test_gmres_restarted_reaches_the_direct_solution():
    rng = np.random.default_rng(53)
    n = 80
    A = np.eye(n) * 2.0 + rng.standard_normal((n, n)) * (0.5 / np.sqrt(n))
    b = rng.standard_normal(n)
    x, it, rr, cyc = oracle.gmres(A, b, restart=6, tol=1e-11)
    assert rr <= 1e-11 * 1.001 and cyc > 1
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-8, atol=1e-12)
    # a cycle that ends on the tolerance: the last cycle's estimate and the true residual agree
    x2, it2, rr2, _ = oracle.gmres(A, b, restart=200, tol=1e-8)
    assert rr2 <= 1e-8 * 1.001 and it2 < it


def test_storage_rounding_is_exact_widening():
    rng = np.random.default_rng(61)
    A = rng.standard_normal((5, 7))
    Ab = W.round_to_storage(A, "bf16")
    # every bf16 value has at most 8 significant bits
    m, e = np.frexp(Ab)
    assert np.all(np.abs(m * 256 - np.round(m * 256)) == 0)
    assert np.all(np.abs(Ab - A) <= 2.0 ** -8 * np.abs(A))
    bits = W.bf16_bits(A).astype(np.uint32) << 16
    np.testing.assert_array_equal(bits.view(np.float32).astype(np.float64), Ab)


# ---------------------------------------------------------------------------------------------
# Randomized Hadamard preprocessing of CD++ (Sec. 5.1, the preprocessing of Alg. 3; App. on FHT / SymFHT)
# ---------------------------------------------------------------------------------------------

def _sym(n, seed):
    A = np.random.default_rng(seed).standard_normal((n, n))
    return A + A.T


def _signs(n, seed):
    return W.rademacher_signs(n, seed)


@pytest.mark.parametrize("n", [1, 2, 4, 16, 64])
def test_rht_matches_scipy_hadamard(n):
    """Q A Q^T, Q b and Q^T x against scipy's Sylvester-Hadamard matrix, Q = H diag(d) / sqrt(n)."""
    import scipy.linalg
    A, d = _sym(n, n), _signs(n, 100 + n)
    B = np.random.default_rng(200 + n).standard_normal((n, 3))
    Q = scipy.linalg.hadamard(n).astype(float) * d[None, :] / math.sqrt(n)
    Abar, Bbar = oracle.rht_forward(d, A, B)
    assert np.abs(Abar - Q @ A @ Q.T).max() <= 1e-13 * n
    assert np.abs(Bbar - Q @ B).max() <= 1e-13 * n
    assert np.abs(oracle.rht_inverse(d, Bbar) - B).max() <= 1e-13 * n
    for i, j in [(0, 0), (n - 1, 0), (n // 2, n - 1)]:
        assert abs(oracle.rht_entry(d, A, i, j) - Abar[i, j]) <= 1e-13 * n


@pytest.mark.parametrize("n", [2, 8, 32])
def test_rht_definition_holds_for_a_general_matrix(n):
    """Q A Q^T and its single entries for a non-symmetric A (the definition does not use symmetry)."""
    import scipy.linalg
    A = np.random.default_rng(300 + n).standard_normal((n, n))
    d = _signs(n, 400 + n)
    Q = scipy.linalg.hadamard(n).astype(float) * d[None, :] / math.sqrt(n)
    ref = Q @ A @ Q.T
    Abar, _ = oracle.rht_forward(d, A, None)
    assert np.abs(Abar - ref).max() <= 1e-13 * n
    for i, j in [(0, n - 1), (n - 1, 0), (1, n // 2)]:
        assert abs(oracle.rht_entry(d, A, i, j) - ref[i, j]) <= 1e-13 * n


def test_symfht_count_at_4096_matches_the_papers_printed_rht_cost():
    """The paper prints the RHT step's cost at n = 4096 as about 2.4e8 FLOPs (tests/golden/rht_flops_n4096.txt).
    The oracle's SymFHT additions on a 4096 x 4096 symmetric matrix, plus the n^2 multiplications of the
    scaling D A D, give that figure to its printed digits; the additions alone stay within the SymFHT
    theorem's n^2 (2.5 + log2 n)."""
    with open(os.path.join(GOLDEN, "rht_flops_n4096.txt")) as f:
        n, printed, digits = next(ln.split() for ln in f if ln.strip() and not ln.startswith("#"))
    n, printed, digits = int(n), float(printed), int(digits)
    A = _sym(n, 5)
    _, ops = oracle.symfht(A)
    assert ops <= n * n * (2.5 + math.log2(n))
    total = ops + n * n
    assert float(f"{total:.{digits - 1}e}") == printed


def test_rht_keeps_spectrum_and_solution():
    """Q is orthogonal: Q A Q^T has the eigenvalues of A, and Q^T (Q A Q^T)^{-1} Q b = A^{-1} b."""
    n = 32
    A, b, _ = W.spd(n, 4, 1e1, 1e3, 1.0, 2.0, seed_A=3, seed_b=6)
    d = W.rademacher_signs(n, 5)
    Abar, bbar = oracle.rht_forward(d, A, b)
    np.testing.assert_allclose(np.linalg.eigvalsh(Abar), np.linalg.eigvalsh(A), rtol=1e-12)
    assert np.abs(Abar - Abar.T).max() <= 1e-12 * np.abs(A).max()
    x = oracle.rht_inverse(d, np.linalg.solve(Abar, bbar))
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-10)


def test_rht_rejects_sizes_that_are_not_powers_of_two():
    with pytest.raises(ValueError):
        oracle.rht_forward(np.ones(6), np.eye(6))


@pytest.mark.parametrize("n", [1, 2, 8, 32, 128])
def test_fht_follows_the_sylvester_definition_with_n_log_n_operations(n):
    """H_2n = [[H_n, H_n], [H_n, -H_n]]: H v = [H(v1 + v2); H(v1 - v2)] for the halves v1, v2 (the
    appendix's listing writes the second half as H(v2 - v1); the definition decides), n log2 n ops."""
    import scipy.linalg
    V = np.random.default_rng(n).standard_normal((n, 2))
    got, ops = oracle.fht(V)
    assert np.abs(got - scipy.linalg.hadamard(n) @ V).max() <= 1e-13 * n
    assert ops == 2 * n * int(round(math.log2(n)))


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 64, 128])
def test_symfht_returns_hah_within_its_operation_bound(n):
    """SymFHT(A) = H A H for symmetric A, using n^2 log2 n + 1.5 n^2 - 1.5 n additions (the recursion
    T(n) = 2 T(n/2) + 2 (n/2)^2 log2(n/2) + 7 (n/2)^2, T(1) = 0), within the theorem's n^2 (2.5 + log2 n)."""
    import scipy.linalg
    A = _sym(n, 7 + n)
    H = scipy.linalg.hadamard(n).astype(float)
    got, ops = oracle.symfht(A)
    assert np.abs(got - H @ A @ H).max() <= 1e-12 * n
    L = int(round(math.log2(n)))
    assert ops == n * n * L + (3 * n * n - 3 * n) // 2
    assert ops <= n * n * (2.5 + L)


# ---------------------------------------------------------------------------------------------
# Online block memoisation with random subsets (Sec. 4 "Block memoization", Sec. 5.2)
# ---------------------------------------------------------------------------------------------

def test_memo_subsets_are_uniform_distinct_and_sorted():
    """Floyd's sampling gives uniform s-subsets: every element is in a subset with probability s/N and
    every pair with probability s(s-1)/(N(N-1))."""
    N, s, T = 20, 5, 20000
    inc = np.zeros(N)
    pair01 = pair_end = 0
    for t in range(T):
        S = oracle.memo_subset(7, t, 3, N, s)
        assert len(set(S.tolist())) == s and np.all(np.diff(S) > 0) and S[0] >= 0 and S[-1] < N
        inc[S] += 1
        ss = set(S.tolist())
        pair01 += (0 in ss and 1 in ss)
        pair_end += (N - 2 in ss and N - 1 in ss)
    assert np.abs(inc / T - s / N).max() <= 0.02           # sd 0.003
    p2 = s * (s - 1) / (N * (N - 1))
    assert abs(pair01 / T - p2) <= 0.01 and abs(pair_end / T - p2) <= 0.01  # sd 0.0016


def test_memo_bernoulli_schedule_and_expected_block_count():
    """p_t = 1 while t <= (n/s) ln n, then (n/s) ln(n) / t (CD++), the K++ form takes the smaller of the
    m and n terms; the number of memoised blocks after T steps is sum_t p_t (the paper's B (1 + ln(T/B)))
    within four standard deviations."""
    n, s = 256, 16
    B = n / s * math.log(n)
    assert oracle.memo_prob(True, n, n, s, 0) == 1.0
    assert oracle.memo_prob(True, n, n, s, int(B)) == 1.0
    assert abs(oracle.memo_prob(True, n, n, s, 1000) - B / 1000) <= 1e-15
    m2 = 1000
    assert abs(oracle.memo_prob(False, m2, 60, 20, 5000) - min(m2, 60) / 20 * math.log(m2) / 5000) <= 1e-15
    T = 4000
    A, b, _ = W.spd(n, 4, 1e1, 1e2, 1.0, 2.0, seed_A=1, seed_b=2)
    res, nb, blocks = oracle.run_memo(A, b, s, cd=True, lam=1e-4, tol=0.0, max_iters=T, seed=11, block_cap=T)
    ps = np.array([oracle.memo_prob(True, n, n, s, t) for t in range(T)])
    mean, sd = ps.sum(), math.sqrt((ps * (1 - ps)).sum())
    assert abs(nb - mean) <= 4 * sd + 1, (nb, mean, sd)
    assert abs(mean - B * (1 + math.log(T / B))) <= 0.05 * mean
    # the first ceil(B) steps all add a block, in order; later steps reuse a memoised one
    k = int(math.ceil(B))
    assert np.array_equal(blocks[:k], np.arange(k))
    assert blocks.max() == nb - 1 and blocks.min() == 0


@pytest.mark.parametrize("seed", [0, 1])
def test_memo_subset_step_is_regularised_argmin(seed):
    """K++ step on an arbitrary row subset (eta = 0, beta = 1): x+ minimises |z - x|^2 + |A_S z - b_S|^2 / lam,
    solved through the n x n normal equations."""
    rng = np.random.default_rng(seed)
    m, n, lam = 40, 12, 0.3
    A, b, x0 = rng.standard_normal((m, n)), rng.standard_normal(m), rng.standard_normal(n)
    S = np.sort(rng.choice(m, 7, replace=False))
    x, _, rn2 = oracle.step_subset(A, b, S, cd=False, lam=lam, x0=x0)
    AS = A[S]
    z = np.linalg.solve(np.eye(n) + AS.T @ AS / lam, x0 + AS.T @ b[S] / lam)
    np.testing.assert_allclose(x, z, rtol=1e-12, atol=1e-12)
    assert abs(rn2 - np.sum((AS @ x0 - b[S]) ** 2)) <= 1e-12 * rn2


def test_memo_subset_cd_step_zeroes_the_block_residual():
    """CD++ step on an arbitrary coordinate subset with lam = 0, eta = 0: (A x+ - b)_S = 0."""
    n = 30
    A, b, _ = W.spd(n, 3, 1e1, 1e2, 1.0, 2.0, seed_A=4, seed_b=5)
    x0 = np.random.default_rng(6).standard_normal(n)
    S = np.array([0, 3, 4, 17, 29])
    x, _, _ = oracle.step_subset(A, b, S, cd=True, lam=0.0, x0=x0)
    assert np.abs((A @ x - b)[S]).max() <= 1e-12 * np.abs(b).max()
    others = np.setdiff1d(np.arange(n), S)
    np.testing.assert_array_equal(x[others], x0[others])


@pytest.mark.parametrize("n", [11, 12])
@pytest.mark.parametrize("cd", [False, True])
def test_memo_windows_follow_closed_form_on_diagonal_systems(cd, n):
    """The online memo's run keeps the windows, ratios and rho of Eq. 5.2 - 5.3 with zeta = ceil(rows / s)
    (here 11 or 12 rows in subsets of 4, zeta = 3): on a diagonal system with eta = 0 each row's residual entry
    decays by its own factor whenever a subset holding it is drawn, so rhat, rho and x after T steps are
    closed forms of the recorded block sequence and subsets."""
    s, T, seed = 4, 96, 5
    rng = np.random.default_rng(31)
    d = rng.uniform(1.0, 3.0, n)
    b = rng.standard_normal(n) * np.where(np.arange(n) < 5, 1.0, 1.8)
    lam = 4.0 * (float(np.max(d)) if cd else float(np.max(d)) ** 2)
    cfac = lam / (d + lam) if cd else lam / (d * d + lam)
    res, nb, blocks = oracle.run_memo(np.diag(d), b, s, cd=cd, lam=lam, tol=0.0, max_iters=T, seed=seed, eta=0.0,
                                      block_cap=T)
    assert res.iters == T and nb == blocks.max() + 1
    first = {}
    for t, j in enumerate(blocks.tolist()):
        first.setdefault(j, t)
    subsets = {j: oracle.memo_subset(seed, t, 0, n, s) for j, t in first.items()}
    zeta = -(-n // s)
    k = np.zeros(n)
    E0 = E1 = 0.0
    q = []
    for t, j in enumerate(blocks.tolist()):
        S = subsets[j]
        e = float(np.sum((b[S] * cfac[S] ** k[S]) ** 2))
        k[S] += 1
        if t % (2 * zeta) < zeta:
            E0 += e
        else:
            E1 += e
        if t % (2 * zeta) == 2 * zeta - 1:
            q.append(E1 / E0)
            E0 = E1 = 0.0
    rhat = _weighted_mean_rhat(q)[-1]
    assert res.state.ci == len(q) == T // (2 * zeta)
    assert res.state.rhat == pytest.approx(rhat, rel=1e-9)
    assert res.state.rho == pytest.approx(min(max(1.0 - rhat ** (1.0 / zeta), 0.0), 1.0 - 1e-12), abs=1e-9)
    np.testing.assert_allclose(res.x, b / d * (1.0 - cfac ** k), rtol=1e-12)


def test_memo_solves_converge_to_the_direct_solution():
    """CD++ (SPD) and K++ (consistent least squares) with the online memo reach 1e-8 and the solution."""
    n, s = 128, 16
    A, b, sig = W.spd(n, 4, 1e1, 1e3, 1.0, 2.0, seed_A=8, seed_b=9)
    res, nb, _ = oracle.run_memo(A, b, s, cd=True, lam=1e-4, tol=1e-8, max_iters=200000, seed=3)
    assert res.status == oracle.OK and res.rel_res_true <= 1e-8
    xs = np.linalg.solve(A, b)
    assert np.linalg.norm(res.x - xs) / np.linalg.norm(xs) <= sig.max() / sig.min() * 1e-8
    rng = np.random.default_rng(10)
    m2, n2 = 400, 40
    A2 = rng.standard_normal((m2, n2)) * np.concatenate([np.full(5, 20.0), np.ones(n2 - 5)])[None, :]
    xstar = rng.standard_normal(n2)
    b2 = A2 @ xstar
    res2, nb2, _ = oracle.run_memo(A2, b2, 20, cd=False, lam=1e-3, tol=1e-8, max_iters=200000, seed=4)
    assert res2.status == oracle.OK and res2.rel_res_true <= 1e-8
    assert np.linalg.norm(res2.x - xstar) / np.linalg.norm(xstar) <= 1e-6
    assert 0 < nb2 < res2.iters


# ---------------------------------------------------------------------------------------------
# Inexact projection by sketch-preconditioned LSQR (Sec. 4.1; the supplement's Proj algorithm)
# ---------------------------------------------------------------------------------------------

def _proj_case(s, n, lam, seed):
    rng = np.random.default_rng(seed)
    AS = rng.standard_normal((s, n)) * np.linspace(10.0, 0.1, s)[:, None]
    r = rng.standard_normal(s)
    w_star = np.linalg.solve(np.eye(n) * lam + AS.T @ AS, AS.T @ r)  # argmin |A_S w - r|^2 + lam |w|^2
    return AS, r, w_star


@pytest.mark.parametrize("s,n,tau", [(8, 100, 16), (12, 64, 40)])
def test_proj_precond_is_the_sketched_gram(s, n, tau):
    """L L^T - lam I = Ahat Ahat^T with Ahat = (A_S D H_n')[:, T] / sqrt(tau) (Sec. 4.1's SRHT sketch), built
    here from scipy's Hadamard matrix on A_S padded with zero columns to n' = the next power of 2."""
    import scipy.linalg
    lam = 0.3
    AS, _, _ = _proj_case(s, n, lam, 20 + s)
    n2 = 1 << (n - 1).bit_length()
    d = W.rademacher_signs(n2, 21)
    T = np.sort(np.random.default_rng(22).choice(n2, tau, replace=False))
    L = oracle.proj_precond(AS, lam, T, d)
    pad = np.hstack([AS, np.zeros((s, n2 - n))])
    Ah = (pad * d[None, :] @ scipy.linalg.hadamard(n2).astype(float))[:, T] / math.sqrt(tau)
    np.testing.assert_allclose(L @ L.T - lam * np.eye(s), Ah @ Ah.T, rtol=1e-12, atol=1e-10)


def test_proj_lsqr_with_the_whole_transform_is_exact_in_one_iteration():
    """tau = n (a power of 2), T = everything: Ahat Ahat^T = A_S A_S^T, the preconditioned operator has
    orthonormal rows, and one LSQR iteration returns the projection."""
    s, n, lam = 16, 128, 0.7
    AS, r, w_star = _proj_case(s, n, lam, 1)
    L = oracle.proj_precond(AS, lam, np.arange(n), W.rademacher_signs(n, 2))
    np.testing.assert_allclose(L @ L.T, AS @ AS.T + lam * np.eye(s), rtol=1e-12, atol=1e-10)
    w, it = oracle.proj_lsqr(AS, r, lam, L, 1)
    assert it == 1
    assert np.linalg.norm(w - w_star) <= 1e-12 * np.linalg.norm(w_star)


def test_proj_lsqr_converges_monotonically_to_the_regularised_projection():
    """tau = 2 s (the supplement's choice), n not a power of 2 (zero padding): the error to the argmin
    falls monotonically and reaches rounding level."""
    s, n, lam = 32, 300, 0.05
    AS, r, w_star = _proj_case(s, n, lam, 3)
    d = W.rademacher_signs(512, 4)
    T = np.sort(np.random.default_rng(5).choice(512, 2 * s, replace=False))
    L = oracle.proj_precond(AS, lam, T, d)
    errs = [np.linalg.norm(oracle.proj_lsqr(AS, r, lam, L, t)[0] - w_star) / np.linalg.norm(w_star)
            for t in range(1, 13)]
    assert all(b <= a * (1 + 1e-9) for a, b in zip(errs, errs[1:]))
    w, _ = oracle.proj_lsqr(AS, r, lam, L, 3 * s)
    assert np.linalg.norm(w - w_star) <= 1e-10 * np.linalg.norm(w_star)


@pytest.mark.parametrize("tau", [64, 128, 256])
def test_proj_lsqr_meets_the_rate_of_its_lemma(tau):
    """Sec. 4.1's inner-solver lemma, with its kappa measured: for r = A_S e the exact projection has
    |[w; v]| <= sqrt(2) |e|, and LSQR from zero on the preconditioned system, of condition number kappa,
    has |z_k - z*| <= kappa |M (z_k - z*)| / sigma_max <= 2 kappa q^k |z*|, q = (kappa - 1)/(kappa + 1).
    So |w_k - w| <= 2 sqrt(2) kappa q^k |e| for every k."""
    s, n, lam = 32, 300, 0.05
    AS, _, _ = _proj_case(s, n, lam, 3)
    e = np.random.default_rng(4).standard_normal(n)
    r = AS @ e
    w_star = np.linalg.solve(np.eye(n) * lam + AS.T @ AS, AS.T @ r)
    T = np.sort(np.random.default_rng(5).choice(512, tau, replace=False))
    L = oracle.proj_precond(AS, lam, T, W.rademacher_signs(512, 4))
    sv = np.linalg.svd(np.linalg.solve(L, np.hstack([AS, math.sqrt(lam) * np.eye(s)])), compute_uv=False)
    kappa = sv[0] / sv[-1]
    q = (kappa - 1.0) / (kappa + 1.0)
    for k in range(1, 9):
        w, _ = oracle.proj_lsqr(AS, r, lam, L, k)
        assert np.linalg.norm(w - w_star) <= 2.0 * math.sqrt(2.0) * kappa * q ** k * np.linalg.norm(e)


def test_proj_preconditioned_condition_number_shrinks_with_the_sketch():
    """kappa(L^{-1} [A_S, sqrt(lam) I]) is 1 for the whole transform and, averaged over draws, smaller for
    a sketch of 8 s columns than for one of s columns; at 2 s it is a small constant."""
    s, n, lam = 24, 256, 0.01
    AS, _, _ = _proj_case(s, n, lam, 6)
    Mfull = np.hstack([AS, math.sqrt(lam) * np.eye(s)])

    def kappa(T, seed):
        L = oracle.proj_precond(AS, lam, T, W.rademacher_signs(n, seed))
        sv = np.linalg.svd(np.linalg.solve(L, Mfull), compute_uv=False)
        return sv[0] / sv[-1]

    assert abs(kappa(np.arange(n), 7) - 1.0) <= 1e-9
    rng = np.random.default_rng(8)
    ks = {tau: np.mean([kappa(np.sort(rng.choice(n, tau, replace=False)), 10 + i) for i in range(5)])
          for tau in (s, 2 * s, 8 * s)}
    assert ks[8 * s] < ks[s]
    assert ks[2 * s] <= 10.0


def test_run_lsqr_with_converged_projections_is_the_exact_kpp_run():
    """K++ with the inexact projection (Sec. 4.1) and enough LSQR iterations for the projection to reach
    rounding level (3 s, see the test above) follows the exact K++ run (Alg. 1 with Cholesky
    projections) step for step: same block draws, same momentum and windows."""
    rng = np.random.default_rng(21)
    m, n, s, lam = 120, 40, 12, 0.05
    A = rng.standard_normal((m, n)) @ np.diag(np.geomspace(1, 20, n))
    b = A @ rng.standard_normal(n)
    T = np.sort(rng.choice(64, 2 * s, replace=False))
    d = W.rademacher_signs(64, 3)
    Lsk = oracle.lsqr_factors(A, s, lam, T, d)
    Lex = oracle.kpp_factor(A, s, lam)
    for steps in (1, 7, 43):
        ri = oracle.run_lsqr(A, b, Lsk, s, 3 * s, lam=lam, tol=0.0, max_iters=steps, seed=2)
        re = oracle.run(A, b, Lex, s, lam=lam, tol=0.0, max_iters=steps, seed=2)
        assert ri.iters == re.iters == steps
        np.testing.assert_allclose(ri.x, re.x, rtol=1e-9, atol=1e-12 * np.abs(re.x).max())


def test_run_lsqr_with_eight_iterations_converges():
    """The supplement's setting (tau = 2 s, t_max = 8): the inexact-projection K++ still reaches 1e-8 on a
    consistent system, confirmed by the true residual, in a number of steps close to the exact run's."""
    rng = np.random.default_rng(22)
    m, n, s, lam = 400, 60, 20, 1e-3
    A = rng.standard_normal((m, n)) @ np.diag(np.geomspace(1, 30, n))
    b = A @ rng.standard_normal(n)
    T = np.sort(rng.choice(64, 2 * s, replace=False))
    Lsk = oracle.lsqr_factors(A, s, lam, T, W.rademacher_signs(64, 5))
    ri = oracle.run_lsqr(A, b, Lsk, s, 8, lam=lam, tol=1e-8, max_iters=200000, seed=4)
    re = oracle.run(A, b, oracle.kpp_factor(A, s, lam), s, lam=lam, tol=1e-8, max_iters=200000, seed=4)
    assert ri.status == oracle.OK and re.status == oracle.OK
    assert ri.rel_res_true <= 1e-8
    assert ri.iters <= 3 * re.iters
