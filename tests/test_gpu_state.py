"""Checkpoint and resume (kpp_state_*, kpp_solve_resume, cdpp_solve_resume) on the GPU.

A solve split into calls, with the state and x written to a host checkpoint and loaded into a new
state between them, must follow the uninterrupted solve bitwise: same iterate, same step count,
same rho.  Splits are taken at a window boundary (t = 2 zeta q, where the window sums are zero) and
in the middle of a window (the sums E0 / E1 travel in the checkpoint).  The uninterrupted
trajectory itself matches the FP64 oracle to 1e-10 relative (Alg. 5 for K++, Alg. 3 for CD++).
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


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _run(K, Ad, bd, P, F, prm_of, splits, total, cd, k):
    """Run `total` steps as calls of the given split lengths; between calls the state and x go
    through a host checkpoint into a fresh state."""
    n = Ad.shape[1]
    x = dev(np.zeros((n, k)) if k > 1 else np.zeros(n))
    st = K.State(Ad.shape[0], n, k, cd)
    done, reps = 0, None
    for length in splits + [total - sum(splits)]:
        reps = K.solve_resume(Ad, bd, x, P, F, prm_of(length), st, cd=cd)
        done += length
        blob = st.save(x)
        st = K.State(Ad.shape[0], n, k, cd)
        x.zero_()
        st.load(blob, x)
        assert st.step == reps[0].iters
        if all(r.status == K.OK for r in reps):
            break
    return x.cpu().numpy(), reps


def test_kpp_split_solve_is_bitwise_the_uninterrupted_one(K):
    sy = W.kpp_fp64_2000x200()
    m, n = sy.A.shape
    P = K.Partition(m, sy.s)
    Ad, bd = dev(sy.A), dev(sy.b)
    F = K.Factors(Ad, P, sy.lam, 0)
    T, zeta = 1000, -(-m // sy.s)

    def prm(length):
        return K.params(lam=sy.lam, tol=0.0, max_iters=length, seed=0, grid=8)

    x_one, r_one = _run(K, Ad, bd, P, F, prm, [], T, False, 1)
    assert r_one[0].iters == T
    for splits in ([2 * zeta * 2], [437], [2 * zeta, 2 * zeta + 37, 100]):
        x_sp, r_sp = _run(K, Ad, bd, P, F, prm, splits, T, False, 1)
        np.testing.assert_array_equal(x_sp, x_one)
        assert r_sp[0].iters == T and r_sp[0].rho_final == r_one[0].rho_final
    res = oracle.run(sy.A, sy.b, oracle.kpp_factor(sy.A, sy.s, sy.lam), sy.s, lam=sy.lam, tol=0.0, max_iters=T, seed=0)
    assert rel(x_one, res.x) <= 1e-10


def test_cdpp_split_solve_to_tolerance_is_bitwise_the_uninterrupted_one(K):
    n, s, k, lam = 512, 32, 3, 1e-4
    A, _, _ = W.spd(n, 8, 1e2, 1e3, 1.0, 10.0, seed_A=81, seed_b=82)
    B = np.random.default_rng(83).standard_normal((n, k))
    P = K.Partition(n, s)
    Ad, Bd = dev(A), dev(B)
    F = K.Factors(Ad, P, lam, 1)
    zeta = n // s

    def prm(length):
        return K.params(lam=lam, tol=1e-9, max_iters=length, seed=9, sys_id=4)

    big = 10 ** 6
    x_one, r_one = _run(K, Ad, Bd, P, F, prm, [], big, True, k)
    assert all(r.status == K.OK and r.rel_res_true <= 1e-9 for r in r_one)
    t_stop = r_one[0].iters
    for splits in ([2 * zeta * 3], [2 * zeta * 3 + 11, 2 * zeta * 5]):
        assert sum(splits) < t_stop
        x_sp, r_sp = _run(K, Ad, Bd, P, F, prm, splits, big, True, k)
        np.testing.assert_array_equal(x_sp, x_one)
        assert [r.iters for r in r_sp] == [r.iters for r in r_one]
        assert [r.status for r in r_sp] == [K.OK] * k
    L = oracle.cdpp_factor(A, s, lam)
    for c in range(k):
        res = oracle.run(A, B[:, c], L, s, cd=True, lam=lam, tol=1e-9, seed=9, sys=4)
        assert res.status == oracle.OK
        assert rel(x_one[:, c], res.x) <= 1e-10


def test_state_argument_errors(K):
    A = dev(np.eye(64))
    P = K.Partition(64, 16)
    F = K.Factors(A, P, 0.1, 0)
    x = dev(np.zeros(64))
    st = K.State(64, 64, 1, False)
    with pytest.raises(K.KppError) as e:  # a state of another shape
        K.solve_resume(A, dev(np.ones(64)), x, P, F, K.params(lam=0.1, max_iters=4), K.State(64, 32, 1, False))
    assert e.value.status == K.ERR_ARG
    with pytest.raises(K.KppError) as e:  # FP32 storage is not resumable
        A32 = A.float()
        K.solve_resume(A32, dev(np.ones(64)), x, P, K.Factors(A32, P, 0.1, 0), K.params(lam=0.1, max_iters=4), st)
    assert e.value.status == K.ERR_UNSUPPORTED
    blob = st.save(x)
    with pytest.raises(K.KppError) as e:  # a checkpoint of another shape
        K.State(64, 64, 2, False).load(blob, dev(np.zeros((64, 2))))
    assert e.value.status == K.ERR_ARG
    with pytest.raises(K.KppError) as e:  # not a checkpoint
        st.load(b"\0" * len(blob), x)
    assert e.value.status == K.ERR_ARG
    with pytest.raises(K.KppError):
        K.State(64, 32, 1, True)  # CD++ needs a square system
