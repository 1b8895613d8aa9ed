"""The block-size autotuner (kpp_tune_block_size) on a batched FP32 system set and a CD++ system.

It must return one of the candidates with finite estimates, the smallest estimate must belong to the
returned size, and a solve with the returned size must reach the tolerance.  Its estimate of the time
to tolerance must also be of the right size: within a factor 4 of the measured time of that solve
(the estimate extrapolates a contraction rate measured over six sweeps).
"""
import numpy as np
import pytest

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


def test_block_size_tuner_on_wide_fp32_batch(K, record_property):
    nsys, m, n, k = 2, 1024, 16384, 8
    As, Bs = [], []
    for i in range(nsys):
        A, B, _ = W.gaussian_rows(m, n, 20, 100.0, seed_A=800 + 2 * i, seed_b=801 + 2 * i, k_rhs=k)
        As.append(torch.as_tensor(W.round_to_storage(A, "f32"), dtype=torch.float32, device="cuda"))
        Bs.append(torch.as_tensor(B, device="cuda"))
    lam = W.row_outlier_lambda(As[0].double().cpu().numpy())
    prm = K.params(lam=lam, tol=1e-8, refine=1, inner_tol=1e-3, seed=3)
    cands = [64, 128, 256]
    s, est = K.tune_block_size(As, Bs, cands, prm)
    record_property("estimates_ms", est)
    print(f"\nblock-size estimates (ms to 1e-8): {est}; chosen s = {s}")
    assert s in cands and all(np.isfinite(v) for v in est.values())
    assert est[s] == min(est.values())
    P = K.Partition(m, s)
    Xd = [torch.zeros((n, k), dtype=torch.float64, device="cuda") for _ in range(nsys)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    Fs = [K.Factors(a, P, lam, 0) for a in As]
    reps = K.kpp_solve_batched(As, Bs, Xd, P, Fs, prm)
    e1.record()
    e1.synchronize()
    assert all(r.status == K.OK and r.rel_res_true <= 1e-8 for r in reps)
    measured = e0.elapsed_time(e1)
    record_property("measured_ms", measured)
    assert est[s] / 4 <= measured <= est[s] * 4, (est[s], measured)


def test_block_size_tuner_on_cdpp(K):
    A, b, _ = W.spd(1024, 12, 1e2, 1e4, 1.0, 10.0, seed_A=810, seed_b=811)
    Ad = torch.as_tensor(A, device="cuda")
    bd = torch.as_tensor(b, device="cuda")
    prm = K.params(lam=1e-4, tol=1e-8, seed=4)
    s, est = K.tune_block_size([Ad], [bd], [16, 32, 64], prm, cd=True)
    assert s in (16, 32, 64) and est[s] == min(est.values())
    x = torch.zeros(1024, dtype=torch.float64, device="cuda")
    P = K.Partition(1024, s)
    rep = K.cdpp_solve(Ad, bd, x, P, K.Factors(Ad, P, 1e-4, 1), prm)
    assert rep.status == K.OK and rep.rel_res_true <= 1e-8
    with pytest.raises(K.KppError) as e:
        K.tune_block_size([Ad], [bd], [0], prm, cd=True)
    assert e.value.status == K.ERR_ARG
