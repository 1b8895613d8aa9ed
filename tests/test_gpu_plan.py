"""Prepared batched solves (kpp_plan_*): parity with the oracle and with the one-shot batched entry
points, CUDA-graph capture and replay, systems that stop at different refinement steps, and the
launch autotuner with its cache.

A plan runs the same kernels on the same launch shape as kpp_solve_batched / cdpp_solve_batched, and
its device-side refinement check takes the same FP64 decisions in the same order as the host loop, so
the two are compared bitwise; the FP64 forms are also compared with the oracle (1e-10).
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


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _fp64_systems(cd, nsys, n, m, k, seed):
    As, Bs = [], []
    for i in range(nsys):
        if cd:
            A, _, _ = W.spd(n, 5, 1e2, 1e3, 1.0, 5.0, seed_A=seed + 2 * i, seed_b=seed + 2 * i + 1)
        else:
            A = np.random.default_rng(seed + 2 * i).standard_normal((m, n))
        As.append(A)
        Bs.append(np.random.default_rng(seed + 2 * i + 1).standard_normal((A.shape[0], k)))
    return As, Bs


def _graph_replay(plan, Xd, stream):
    """Capture plan.launch on `stream` (after one eager warm-up launch) and replay it once from X = 0."""
    with torch.cuda.stream(stream):
        for x in Xd:
            x.zero_()
        plan.launch(stream)
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        plan.launch(torch.cuda.current_stream())
    for x in Xd:
        x.zero_()
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    return g


@pytest.mark.parametrize("cd", [False, True])
def test_plan_fp64_matches_batched_and_oracle(K, cd):
    nsys, k, lam, s = 2, 3, 1e-4 if cd else 0.05, 16
    n, m = (200, 200) if cd else (25, 60)
    As, Bs = _fp64_systems(cd, nsys, n, m, k, 500)
    P = K.Partition(As[0].shape[0], s)
    Ad = [dev(a) for a in As]
    Bd = [dev(b) for b in Bs]
    Fs = [K.Factors(a, P, lam, 1 if cd else 0) for a in Ad]
    nb = -(-As[0].shape[0] // s)
    T = 2 * nb * 3 + 5
    prm = K.params(lam=lam, tol=0.0, max_iters=T, seed=8, sys_id=30)
    Xp = [dev(np.zeros((n, k))) for _ in range(nsys)]
    plan = K.Plan(Ad, Bd, Xp, P, Fs, prm, cd=cd)
    plan.launch()
    reps = plan.report(allow_no_conv=True)
    Xb = [dev(np.zeros((n, k))) for _ in range(nsys)]
    repb = K.kpp_solve_batched(Ad, Bd, Xb, P, Fs, prm, allow_no_conv=True, cd=cd)
    for i in range(nsys):
        assert torch.equal(Xp[i], Xb[i])
        fac = oracle.cdpp_factor(As[i], s, lam) if cd else oracle.kpp_factor(As[i], s, lam)
        for c in range(k):
            assert reps[i * k + c].iters == repb[i * k + c].iters == T
            res = oracle.run(As[i], Bs[i][:, c], fac, s, cd=cd, lam=lam, tol=0.0, max_iters=T, seed=8, sys=30 + i)
            assert rel(Xp[i][:, c].cpu().numpy(), res.x) <= 1e-10, (i, c)
    plan.close()


def test_plan_fp64_cdpp_graph_replay_to_tolerance(K):
    """CD++ FP64 (the dataflow kernel) solved to 1e-8 inside a replayed CUDA graph; new right-hand sides
    written into the bound buffers between replays are picked up."""
    n, s, nsys = 1024, 64, 2
    As, Bs = [], []
    for i in range(nsys):
        A, b, _ = W.spd(n, 8, 1e2, 1e3, 1.0, 10.0, seed_A=40 + i, seed_b=50 + i)
        As.append(A)
        Bs.append(b)
    lam = 1e-4
    P = K.Partition(n, s)
    Ad = [dev(a) for a in As]
    Bd = [dev(b) for b in Bs]
    Fs = [K.Factors(a, P, lam, 1) for a in Ad]
    prm = K.params(lam=lam, tol=1e-8, seed=1)
    Xp = [dev(np.zeros(n)) for _ in range(nsys)]
    plan = K.Plan(Ad, Bd, Xp, P, Fs, prm, cd=True)
    st = torch.cuda.Stream()
    g = _graph_replay(plan, Xp, st)
    reps = plan.report(stream=st)
    Xb = [dev(np.zeros(n)) for _ in range(nsys)]
    repb = K.kpp_solve_batched(Ad, Bd, Xb, P, Fs, prm, cd=True)
    for i in range(nsys):
        assert torch.equal(Xp[i], Xb[i])
        assert reps[i].status == K.OK and reps[i].rel_res_true <= 1e-8
        assert reps[i].iters == repb[i].iters
    # new right-hand sides in place, replay again
    for i in range(nsys):
        Bd[i].copy_(dev(np.random.default_rng(70 + i).standard_normal(n)))
        Xp[i].zero_()
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    reps2 = plan.report()
    Xb2 = [dev(np.zeros(n)) for _ in range(nsys)]
    K.kpp_solve_batched(Ad, Bd, Xb2, P, Fs, prm, cd=True)
    for i in range(nsys):
        assert torch.equal(Xp[i], Xb2[i])
        assert reps2[i].status == K.OK and reps2[i].rel_res_true <= 1e-8
    del g
    plan.close()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_plan_mixed_refinement_in_graph_matches_host_loop(K, dtype):
    """FP32 / BF16 storage with FP64 refinement: the device-side refinement loop inside a replayed graph
    equals the host loop of kpp_solve_batched bitwise (x, steps, refinement count).  System 1 has a zero
    right-hand side and stops at the first check (its inner solves run zero steps)."""
    sy = W.kpp_mixed_lowrank(m=16384, n=512, s=128, n_out=16)
    A = W.round_to_storage(sy.A, dtype)
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    m, n = A.shape
    rng = np.random.default_rng(9)
    Bs = [A @ sy.x_star, np.zeros(m), A @ rng.standard_normal(n)]
    nsys = len(Bs)
    P = K.Partition(m, sy.s)
    Ad = [dev(A, tdt) for _ in range(nsys)]
    Bd = [dev(b) for b in Bs]
    Fs = [K.Factors(a, P, sy.lam, 0) for a in Ad]
    prm = K.params(lam=sy.lam, tol=1e-8, refine=1, inner_tol=1e-3, seed=0)
    Xp = [dev(np.zeros(n)) for _ in range(nsys)]
    plan = K.Plan(Ad, Bd, Xp, P, Fs, prm)
    st = torch.cuda.Stream()
    g = _graph_replay(plan, Xp, st)
    reps = plan.report()
    Xb = [dev(np.zeros(n)) for _ in range(nsys)]
    repb = K.kpp_solve_batched(Ad, Bd, Xb, P, Fs, prm)
    for i in range(nsys):
        assert torch.equal(Xp[i], Xb[i]), i
        assert (reps[i].iters, reps[i].outer) == (repb[i].iters, repb[i].outer), (reps[i].as_dict(), repb[i].as_dict())
        assert reps[i].status == K.OK and reps[i].rel_res_true <= 1e-8
    assert reps[1].iters == 0 and reps[1].outer == 0 and float(Xp[1].abs().max()) == 0.0
    assert reps[0].outer >= 1 and reps[2].outer >= 1
    del g
    plan.close()


def test_plan_streaming_kernel_refinement_in_graph(K):
    """Wide FP32 systems (the streaming kernel, k = 3 panels): graph replay equals the host loop and
    reaches the minimum-norm solution."""
    nsys, m, n, s, k = 3, 96, 16384, 32, 3
    As, Bs = [], []
    for i in range(nsys):
        A, B, _ = W.gaussian_rows(m, n, 2, 100.0, seed_A=600 + 10 * i, seed_b=601 + 10 * i, k_rhs=k)
        As.append(W.round_to_storage(A, "f32"))
        Bs.append(B)
    lam = W.row_outlier_lambda(As[0])
    P = K.Partition(m, s)
    Ad = [dev(a, torch.float32) for a in As]
    Bd = [dev(b) for b in Bs]
    Fs = [K.Factors(a, P, lam, 0) for a in Ad]
    prm = K.params(lam=lam, tol=1e-8, refine=1, inner_tol=1e-4, seed=5)
    Xp = [dev(np.zeros((n, k))) for _ in range(nsys)]
    plan = K.Plan(Ad, Bd, Xp, P, Fs, prm)
    assert plan.info()["kernel"] == 4
    st = torch.cuda.Stream()
    g = _graph_replay(plan, Xp, st)
    reps = plan.report()
    Xb = [dev(np.zeros((n, k))) for _ in range(nsys)]
    K.kpp_solve_batched(Ad, Bd, Xb, P, Fs, prm)
    for i in range(nsys):
        assert torch.equal(Xp[i], Xb[i])
        Xmn = As[i].T @ np.linalg.solve(As[i] @ As[i].T, Bs[i])
        for c in range(k):
            assert reps[i * k + c].status == K.OK and reps[i * k + c].rel_res_true <= 1e-8
            assert rel(Xp[i][:, c].cpu().numpy(), Xmn[:, c]) <= 1e-6
    del g
    plan.close()


def test_plan_mixed_cdpp_refinement(K):
    A, b, _ = W.spd(512, 8, 1e2, 1e3, 1.0, 10.0, seed_A=20, seed_b=21)
    A32 = W.round_to_storage(A, "f32")
    P = K.Partition(512, 64)
    Ad = dev(A32, torch.float32)
    Bd = dev(b)
    F = K.Factors(Ad, P, 1e-4, 1)
    prm = K.params(lam=1e-4, tol=1e-8, refine=1, inner_tol=1e-3, seed=2)
    xp = dev(np.zeros(512))
    plan = K.Plan([Ad], [Bd], [xp], P, [F], prm, cd=True)
    plan.launch()
    rep = plan.report()[0]
    xb = dev(np.zeros(512))
    repb = K.cdpp_solve(Ad, Bd, xb, P, F, prm)
    assert torch.equal(xp, xb)
    assert rep.status == K.OK and rep.rel_res_true <= 1e-8 and (rep.iters, rep.outer) == (repb.iters, repb.outer)


def test_plan_argument_errors(K):
    A = dev(np.ones((8, 5)))
    P = K.Partition(8, 4)
    F = K.Factors(A, P, 0.1, 0)
    b, x = dev(np.ones(8)), dev(np.zeros(5))
    with pytest.raises(K.KppError):
        K.Plan([A], [b], [x], P, [F], K.params(lam=0.1), cd=True)  # K++ factors for a CD++ plan
    with pytest.raises(K.KppError):
        K.Plan([A], [b], [x], P, [F], K.params(lam=0.2))  # lambda differs from the factors'


def test_autotuner_choice_is_cached_saved_and_reproducible(K, tmp_path):
    """grid = GRID_TUNE: the tuned plan equals the one-shot solve run with the chosen (generation, grid)
    bitwise; the choice is cached once per shape and survives a save / clear / load round trip."""
    n, s, lam = 1024, 64, 1e-4
    A, b, _ = W.spd(n, 8, 1e2, 1e3, 1.0, 10.0, seed_A=80, seed_b=81)
    P = K.Partition(n, s)
    Ad, Bd = dev(A), dev(b)
    F = K.Factors(Ad, P, lam, 1)
    K.tune_cache_clear()
    prm = K.params(lam=lam, tol=1e-8, seed=3, grid=K.GRID_TUNE)
    xp = dev(np.zeros(n))
    plan = K.Plan([Ad], [Bd], [xp], P, [F], prm, cd=True)
    info = plan.info()
    assert K.tune_cache_size() == 1 and info["grid"] >= 1 and info["variant"] in (2, 3)
    plan.launch()
    rep = plan.report()[0]
    assert rep.status == K.OK and rep.rel_res_true <= 1e-8
    # the one-shot path with the tuned choice
    K.set_kernel_variant(info["variant"])
    try:
        xb = dev(np.zeros(n))
        K.cdpp_solve(Ad, Bd, xb, P, F, K.params(lam=lam, tol=1e-8, seed=3, grid=info["grid"]))
    finally:
        K.set_kernel_variant(3)
    assert torch.equal(xp, xb)
    # a second tuned plan of the same shape uses the cache
    plan2 = K.Plan([Ad], [Bd], [dev(np.zeros(n))], P, [F], prm, cd=True)
    assert plan2.info() == info and K.tune_cache_size() == 1
    path = tmp_path / "tune.txt"
    K.tune_cache_save(path)
    K.tune_cache_clear()
    assert K.tune_cache_size() == 0
    K.tune_cache_load(path)
    assert K.tune_cache_size() == 1
    xt = dev(np.zeros(n))
    K.cdpp_solve(Ad, Bd, xt, P, F, prm)  # one-shot solve, tuned shape from the loaded cache
    assert torch.equal(xt, xp)
    plan.close()
    plan2.close()
