"""GPU parity at the block sizes the mixed-precision and batched workloads ship with, against the FP64
oracle run on the stored (rounded) matrix.

Under BF16 / FP32 storage the stored matrix is the system; the oracle widens the same stored values
to FP64 and runs K++ (Eq. 1.3 - 1.4, Alg. 5) to a residual well below the GPU's.  Two kinds of check:

* refined solutions (FP32 inner iterations, FP64 refinement to 1e-8) against the oracle's solution:
  for a full-column-rank consistent system, or the minimum-norm solution of an under-determined one
  (the iterations start at 0, and every K++ update A_S^T y lies in range(A^T)),
      |x - x_o| / |x_o| <= kappa(A) * (|Ax - b| + |A x_o - b|) / |b|,
  with kappa(A) = sigma_max / sigma_min of the stored matrix computed here.  For an under-determined
  system this holds for the part of x in range(A^T): the FP32 roundings of the inner iterations also
  leave a small component in the null space of A, which no residual sees; it is bounded separately
  by the FP32 drift of the whole run, 4 * T * (2 + sqrt(n)) * 2^-24 relative (T its steps);
* FP32 iterations in lockstep with the FP64 oracle (same Philox block sequence, T steps, no
  refinement) on systems with well-conditioned blocks.  The FP32 Gram, Cholesky factor, inverse and
  residual carry a relative error of about u = (2 + sqrt(n) + sqrt(s)) 2^-24 (a rounding per operation
  plus the random-walk growth of FP32 sums over n columns and over the s terms of the factor); the
  block solve turns it into a perturbation of the step of at most kappa(G_j + lambda I) u relative; a
  projection does not expand the error it inherits and the momentum at most doubles it; so after T steps
      |x_32 - x_64| / |x_64| <= 4 * T * max_j kappa(G_j + lambda I) * (2 + sqrt(n) + sqrt(s)) * 2^-24.
Each test reports its measured error beside the bound (record_property).
The kernel a solve runs is read from a plan of the same solve (kpp_plan_info: 2 small-block,
4 streaming, 6 large-block with the W memo).
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
    kpp.set_kernel_variant(3)
    return kpp


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def kappa(A):
    sv = np.linalg.svd(A, compute_uv=False)
    return float(sv[0] / sv[-1])


def block_kappa(A, s, lam):
    out = 0.0
    for j in range(0, A.shape[0], s):
        As = A[j:j + s]
        ev = np.linalg.eigvalsh(As @ As.T + lam * np.eye(As.shape[0]))
        out = max(out, ev[-1] / ev[0])
    return out


def kernel_of(K, Ads, Bds, n, k, P, Fs, prm):
    Xd = [dev(np.zeros((n, k)) if k > 1 else np.zeros(n)) for _ in Ads]
    plan = K.Plan(Ads, Bds, Xd, P, Fs, prm)
    info = plan.info()
    plan.close()
    return info["kernel"]


@pytest.mark.parametrize("dtype,m,n,s,kern", [("bf16", 8192, 1024, 512, 6),   # large-block kernel, s = 512
                                              ("f32", 4096, 1024, 256, 6),    # large-block kernel, FP32 s = 256
                                              ("f32", 8192, 1024, 512, 2)])   # small-block kernel, distributed y
def test_refined_solution_matches_oracle_at_shipped_block_sizes(K, record_property, dtype, m, n, s, kern):
    sy = W.kpp_mixed_lowrank(m=m, n=n, s=s, n_out=25)
    A = W.round_to_storage(sy.A, dtype)
    b = A @ sy.x_star
    Ad = dev(A, TDT[dtype])
    P = K.Partition(m, s)
    F = K.Factors(Ad, P, sy.lam, 0)
    prm = K.params(lam=sy.lam, tol=1e-8, refine=1, inner_tol=1e-3, seed=0)
    bd = dev(b)
    assert kernel_of(K, [Ad], [bd], n, 1, P, [F], prm) == kern
    x = dev(np.zeros(n))
    rep = K.kpp_solve(Ad, bd, x, P, F, prm)
    assert rep.status == K.OK and rep.rel_res_true <= 1e-8 and rep.outer >= 1
    res = oracle.run(A, b, oracle.kpp_factor(A, s, sy.lam), s, lam=sy.lam, tol=1e-12, max_iters=200000, seed=0)
    assert res.status == oracle.OK
    err = rel(x.cpu().numpy(), res.x)
    bound = kappa(A) * (rep.rel_res_true + res.rel_res_true)
    record_property("err_vs_oracle", err)
    record_property("bound", bound)
    print(f"\n{dtype} {m}x{n} s={s}: |x - x_oracle|/|x_oracle| = {err:.3e} (bound {bound:.3e}), "
          f"residual {rep.rel_res_true:.2e}, {rep.iters} iterations, {rep.outer} refinement steps")
    assert err <= bound


def test_streaming_kernel_s256_k8_two_systems_match_oracle(K, record_property):
    """The batched workload's block size and panel width (s = 256, k = 8) on two 1024 x 16384 FP32
    systems with 20 rows scaled x100: every column against the minimum-norm solution, and columns 0
    and 7 of each system against the oracle's K++ run on the stored matrix."""
    nsys, m, n, s, k = 2, 1024, 16384, 256, 8
    As, Bs = [], []
    for i in range(nsys):
        A, B, _ = W.gaussian_rows(m, n, 20, 100.0, seed_A=500 + 2 * i, seed_b=501 + 2 * i, k_rhs=k)
        As.append(W.round_to_storage(A, "f32"))
        Bs.append(B)
    lam = W.row_outlier_lambda(As[0])
    P = K.Partition(m, s)
    Ad = [dev(a, torch.float32) for a in As]
    Bd = [dev(b) for b in Bs]
    Fs = [K.Factors(a, P, lam, 0) for a in Ad]
    prm = K.params(lam=lam, tol=1e-8, refine=1, inner_tol=1e-4, seed=5)
    assert kernel_of(K, Ad, Bd, n, k, P, Fs, prm) == 4
    Xd = [dev(np.zeros((n, k))) for _ in range(nsys)]
    reps = K.kpp_solve_batched(Ad, Bd, Xd, P, Fs, prm)
    worst, worst_null = 0.0, 0.0
    for i in range(nsys):
        X = Xd[i].cpu().numpy()
        Ai = As[i]
        kap = kappa(Ai)
        G = Ai @ Ai.T
        Xr = Ai.T @ np.linalg.solve(G, Ai @ X)  # the part of X in range(A^T)
        Xmn = Ai.T @ np.linalg.solve(G, Bs[i])
        L = oracle.kpp_factor(Ai, s, lam)
        for c in range(k):
            r = reps[i * k + c]
            assert r.status == K.OK and r.rel_res_true <= 1e-8, r.as_dict()
            assert rel(Xr[:, c], Xmn[:, c]) <= kap * 2.0 * r.rel_res_true + 1e-12
            null = np.linalg.norm(X[:, c] - Xr[:, c]) / np.linalg.norm(Xmn[:, c])
            worst_null = max(worst_null, null)
            assert null <= 4.0 * r.iters * (2.0 + np.sqrt(n)) * EPS32, (i, c, null, r.iters)
        for c in (0, k - 1):
            res = oracle.run(Ai, Bs[i][:, c], L, s, lam=lam, tol=1e-10, max_iters=200000, seed=5, sys=i)
            assert res.status == oracle.OK
            err = rel(Xr[:, c], res.x)
            bound = kap * (reps[i * k + c].rel_res_true + res.rel_res_true)
            worst = max(worst, err / bound)
            print(f"\nsystem {i} column {c}: range(A^T) part |x - x_oracle|/|x_oracle| = {err:.3e} "
                  f"(bound {bound:.3e}); null-space part {np.linalg.norm(X[:, c] - Xr[:, c]) / np.linalg.norm(res.x):.3e}")
            assert err <= bound
    record_property("worst_err_over_bound", worst)
    record_property("worst_null_space_drift", worst_null)


@pytest.mark.parametrize("form", ["large_block", "general", "streaming"])
def test_fp32_iterations_lockstep_with_fp64_oracle(K, record_property, form):
    """T FP32 steps (no refinement) against T FP64 oracle steps on the same stored matrix and block
    sequence, within 4 T kappa_block (2 + sqrt(n) + sqrt(s)) 2^-24 (module docstring)."""
    rng_seed = {"large_block": 610, "general": 620, "streaming": 630}[form]
    if form == "streaming":
        nsys, m, n, s, k = 2, 512, 16384, 256, 3
    else:
        nsys, m, n, s, k = 1, 4096, 1024, 256, 1
    As, Bs = [], []
    for i in range(nsys):
        A, B, _ = W.gaussian_rows(m, n, 0, 1.0, seed_A=rng_seed + 2 * i, seed_b=rng_seed + 1 + 2 * i, k_rhs=k)
        As.append(W.round_to_storage(A, "f32"))
        Bs.append(B)
    lam = W.row_outlier_lambda(As[0])
    nb = m // s
    T = 2 * nb * 3 + 5
    P = K.Partition(m, s)
    Ad = [dev(a, torch.float32) for a in As]
    Bd = [dev(b if k > 1 else b[:, 0]) for b in Bs]
    Fs = [K.Factors(a, P, lam, 0) for a in Ad]
    prm = K.params(lam=lam, tol=0.0, max_iters=T, refine=0, seed=11, sys_id=40)
    K.set_kernel_variant(1 if form == "general" else 3)
    try:
        kern = kernel_of(K, Ad, Bd, n, k, P, Fs, prm)
        assert kern == {"large_block": 6, "general": 1, "streaming": 4}[form]
        Xd = [dev(np.zeros((n, k)) if k > 1 else np.zeros(n)) for _ in range(nsys)]
        K.kpp_solve_batched(Ad, Bd, Xd, P, Fs, prm, allow_no_conv=True)
    finally:
        K.set_kernel_variant(3)
    worst = 0.0
    for i in range(nsys):
        X = Xd[i].cpu().numpy().reshape(n, k)
        L = oracle.kpp_factor(As[i], s, lam)
        bound = 4.0 * T * block_kappa(As[i], s, lam) * (2.0 + np.sqrt(n) + np.sqrt(s)) * EPS32
        for c in range(k):
            res = oracle.run(As[i], Bs[i][:, c], L, s, lam=lam, tol=0.0, max_iters=T, seed=11, sys=40 + i)
            err = rel(X[:, c], res.x)
            worst = max(worst, err)
            assert err <= bound, (i, c, err, bound)
    record_property("err_vs_oracle", worst)
    record_property("bound", bound)
    print(f"\n{form}: T={T} FP32 steps, |x32 - x64|/|x64| = {worst:.3e} (bound {bound:.3e})")
