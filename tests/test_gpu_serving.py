"""Serving runtime (kpp_server_*): continuous batching under a memory budget, run by the device-resident
request loop (a persistent kernel whose slots claim queued jobs).

Each result must be bitwise the same whether the request ran alone or in a mix of concurrent requests
(a job runs on one slot's CTAs with fixed reduction orders and no floating-point atomics), every column
must reach its tolerance, and the peak device memory charged to admitted work must stay within the budget.
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


def _catalog():
    mats = []
    for i, (n, dt) in enumerate([(256, "f64"), (384, "f32"), (512, "bf16")]):
        A, _, _ = W.spd(n, 6, 1e2, 1e3, 1.0, 10.0, seed_A=900 + i, seed_b=901 + i)
        Ar = W.round_to_storage(A, dt)
        tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dt]
        mats.append((n, dt, torch.as_tensor(Ar, dtype=tdt, device="cuda"), Ar))
    return mats


def _requests():
    rng = np.random.default_rng(77)
    out = []
    for r in range(12):
        mid = r % 3
        k = [1, 3, 8][r % 4 % 3]
        out.append((mid, k, 1000 + r))
    return out


def _run(K, mats, reqs, max_concurrent, budget=8 << 30):
    sv = K.Server(budget, max_concurrent=max_concurrent, grid_per_solve=8)
    ids = [sv.add_matrix(A, 32, 1e-4, 1) for (_, _, A, _) in mats]
    rids = []
    for (mid, k, seed) in reqs:
        n = mats[mid][0]
        B = np.random.default_rng(seed).standard_normal((n, k))
        prm = K.params(tol=1e-8, refine=1 if mats[mid][1] != "f64" else 0, inner_tol=1e-3, seed=seed, sys_id=seed)
        rids.append(sv.submit(ids[mid], B, prm))
    sv.wait_all(300.0)
    results = []
    for rid, (mid, k, seed) in zip(rids, reqs):
        done, rc, X, reps = sv.poll(rid, mats[mid][0], k)
        assert done
        results.append((rc, X, reps))
    st = sv.stats()
    sv.close()
    return results, st


def test_results_are_the_same_alone_and_in_the_mix(K):
    mats = _catalog()
    reqs = _requests()
    mixed, st = _run(K, mats, reqs, max_concurrent=6)
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["peak_bytes"] <= st["budget_bytes"]
    assert st["p99_ms"] >= st["p50_ms"] > 0
    for i, req in enumerate(reqs):
        alone, _ = _run(K, mats, [req], max_concurrent=1)
        rc_a, X_a, _ = alone[0]
        rc_m, X_m, reps = mixed[i]
        assert rc_a == rc_m == K.OK
        np.testing.assert_array_equal(X_m, X_a)
        mid, k, seed = req
        n, dt, _, Ar = mats[mid]
        B = np.random.default_rng(seed).standard_normal((n, k))
        for c in range(k):
            assert reps[c].status == K.OK
            assert np.linalg.norm(Ar @ X_m[:, c] - B[:, c]) <= 1e-8 * np.linalg.norm(B[:, c]) * 1.0001
        if dt == "f64":
            # FP64 requests against the oracle's CD++ run on the same column and Philox stream: the
            # solve freezes a column at its own stop checkpoint, so each column's iterate equals the
            # oracle's single-column run to 1e-10 relative (the report's step count is the panel's)
            L = oracle.cdpp_factor(Ar, 32, 1e-4)
            for c in range(k):
                res = oracle.run(Ar, B[:, c], L, 32, cd=True, lam=1e-4, tol=1e-8, seed=seed, sys=seed)
                assert res.status == oracle.OK and reps[c].iters >= res.iters, (i, c, reps[c].iters, res.iters)
                err = np.linalg.norm(X_m[:, c] - res.x) / np.linalg.norm(res.x)
                assert err <= 1e-10, (i, c, err)


def test_budget_admission_and_refusal(K):
    mats = _catalog()
    # a budget that holds about one request at a time: all still complete, never above the budget
    small = 24 << 20
    res, st = _run(K, mats[:1], [(0, 1, 1), (0, 3, 2), (0, 1, 3)], max_concurrent=3, budget=small)
    assert st["completed"] == 3 and st["failed"] == 0 and st["peak_bytes"] <= small
    # a budget no request fits (the matrix's factors alone take about 0.7 MB): refused at submission
    sv = K.Server(1 << 18, max_concurrent=1)
    mid = sv.add_matrix(mats[0][2], 32, 1e-4, 1)
    rid = sv.submit(mid, np.ones(256), K.params(tol=1e-8))
    done, rc, _, _ = sv.poll(rid, 256, 1)
    assert done and rc == K.ERR_BUDGET
    sv.close()


def test_loop_goes_idle_and_relaunches_and_splits_wide_requests(K):
    """A request of 20 columns runs as jobs of 8, 8 and 4 columns; after the loop has gone idle (its
    slots leave after 50 ms without work), a second batch relaunches it; every column meets 1e-8 in the
    FP64 residual of the stored matrix."""
    import time
    mats = _catalog()
    sv = K.Server(8 << 30, max_concurrent=4, grid_per_solve=8)
    ids = [sv.add_matrix(A, 32, 1e-4, 1) for (_, _, A, _) in mats]
    def batch(seeds):
        rids = []
        for mid, k, seed in seeds:
            n = mats[mid][0]
            B = np.random.default_rng(seed).standard_normal((n, k))
            prm = K.params(tol=1e-8, refine=1 if mats[mid][1] != "f64" else 0, inner_tol=1e-3, seed=seed,
                           sys_id=seed)
            rids.append((sv.submit(ids[mid], B, prm), mid, k, B))
        sv.wait_all(300.0)
        for rid, mid, k, B in rids:
            done, rc, X, reps = sv.poll(rid, mats[mid][0], k)
            assert done and rc == K.OK, (rid, rc)
            Ar = mats[mid][3]
            for c in range(k):
                assert reps[c].status == K.OK
                assert np.linalg.norm(Ar @ X[:, c] - B[:, c]) <= 1e-8 * np.linalg.norm(B[:, c]) * 1.0001
    batch([(2, 20, 11), (1, 1, 12)])
    first = sv.stats()["loop_launches"]
    time.sleep(0.5)
    batch([(0, 2, 13), (2, 9, 14)])
    st = sv.stats()
    assert first >= 1 and st["loop_launches"] > first and st["loop_slots"] >= 1
    sv.close()
