"""The online block memoisation on the GPU (kpp_solve_memo) against the oracle's memo run
(oracle.run_memo: Sec. 4 "Block memoization", Sec. 5.2, the sampling steps of Alg. 3 and Alg. 5).

Both draw from the same Philox stream, so they take the same new subsets and picks.  In lockstep (tol = 0,
T steps) the FP64 iterates agree to 1e-10 relative and the numbers of memoised blocks are equal; to a
tolerance both stop at the same step.  The solve runs in windows of steps (the block sequence is
drawn ahead); T is chosen so that several windows and a growth of the memo store are crossed, and the
windows must not change the trajectory.
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


@pytest.mark.parametrize("T", [1, 37, 700])
def test_kpp_memo_lockstep_with_oracle(K, T):
    sy = W.kpp_fp64_2000x200()
    x = dev(np.zeros(200))
    rep, nb = K.solve_memo(dev(sy.A), dev(sy.b), x, sy.s, K.params(lam=sy.lam, tol=0.0, max_iters=T, seed=3),
                           allow_no_conv=True)
    res, nbo, _ = oracle.run_memo(sy.A, sy.b, sy.s, lam=sy.lam, tol=0.0, max_iters=T, seed=3)
    assert rep.iters == res.iters == T and nb == nbo
    assert rel(x.cpu().numpy(), res.x) <= 1e-10


@pytest.mark.parametrize("n,s,T", [(300, 24, 1), (300, 24, 45), (256, 16, 600)])
def test_cdpp_memo_lockstep_with_oracle(K, n, s, T):
    # (256, 16, 600): about 260 memoised blocks, so the store grows from 64 to 512 blocks across windows
    A, b, _ = W.spd(n, 5, 1e2, 1e3, 1.0, 10.0, seed_A=120 + n, seed_b=121)
    x = dev(np.zeros(n))
    rep, nb = K.solve_memo(dev(A), dev(b), x, s, K.params(lam=1e-4, tol=0.0, max_iters=T, seed=5, sys_id=2),
                           cd=True, allow_no_conv=True)
    res, nbo, _ = oracle.run_memo(A, b, s, cd=True, lam=1e-4, tol=0.0, max_iters=T, seed=5, sys=2)
    assert rep.iters == res.iters == T and nb == nbo
    assert rel(x.cpu().numpy(), res.x) <= 1e-10


@pytest.mark.parametrize("cd", [False, True])
def test_memo_to_tolerance_stops_with_the_oracle(K, cd):
    if cd:
        A, b, _ = W.spd(256, 5, 1e2, 1e3, 1.0, 10.0, seed_A=130, seed_b=131)
        s, lam = 16, 1e-4
    else:
        sy = W.kpp_fp64_2000x200()
        A, b, s, lam = sy.A, sy.b, sy.s, sy.lam
    x = dev(np.zeros(A.shape[1]))
    rep, nb = K.solve_memo(dev(A), dev(b), x, s, K.params(lam=lam, tol=1e-8, seed=7), cd=cd)
    res, nbo, _ = oracle.run_memo(A, b, s, cd=cd, lam=lam, tol=1e-8, seed=7)
    assert rep.status == K.OK and res.status == oracle.OK
    assert rep.iters == res.iters and nb == nbo
    assert rep.rel_res_true <= 1e-8
    assert rel(x.cpu().numpy(), res.x) <= 1e-10


def test_memo_singular_block_is_reported(K):
    # one nonzero row: every drawn subset of 4 of the 40 rows holds a zero row, so with lambda = 0 the
    # first memoised block (memo index 0) has a zero pivot
    A = np.zeros((40, 12))
    A[7] = np.arange(1, 13)
    x = dev(np.zeros(12))
    with pytest.raises(K.KppError) as e:
        K.solve_memo(dev(A), dev(np.ones(40)), x, 4, K.params(lam=0.0, tol=0.0, max_iters=10, seed=1))
    assert e.value.status == K.ERR_NOT_SPD


def test_memo_argument_errors(K):
    A = dev(np.eye(16))
    b = dev(np.ones(16))
    x = dev(np.zeros(16))
    with pytest.raises(K.KppError) as e:
        K.solve_memo(A, b, x, 0, K.params(lam=0.1))
    assert e.value.status == K.ERR_ARG
    with pytest.raises(K.KppError) as e:
        K.solve_memo(A.float(), b, x, 4, K.params(lam=0.1))
    assert e.value.status == K.ERR_ARG
    with pytest.raises(K.KppError) as e:
        K.solve_memo(dev(np.ones((16, 8))), b, dev(np.zeros(8)), 4, K.params(lam=0.1), cd=True)
    assert e.value.status == K.ERR_ARG
