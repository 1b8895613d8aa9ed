"""FP64 CPU oracle for Kaczmarz++ / CD++ -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg import this package.
The product library (``paper_2501_11673_gb300``) never imports, links or runs anything here, and this
package never imports the product library.  The C source (``kpp_oracle.c``) is the oracle proper;
this module compiles it with gcc and marshals numpy arrays through ctypes.

Paper: Derezinski, Needell, Rebrova, Yang, "Randomized Kaczmarz Methods with Beyond-Krylov
Convergence" (arXiv 2501.11673).  Functions cite the passage they follow:

* ``kpp_factor`` / ``cdpp_factor``: memoised Cholesky factor per block (Sec. 4, Sec. 5.2).
* ``run``: the K++ iteration (Alg. 1's loop with exact Cholesky projection, i.e. the
  ``K++(Cholesky)`` variant of App. F; Alg. 5's adaptive rho and stopping rule) and the CD++
  iteration (Eq. 5.1, Alg. 3's loop), both without the randomized Hadamard preprocessing.
* ``cg``: plain conjugate gradients (context, Sec. 6).
* ``run_memo`` (with ``memo_prob``, ``memo_subset``, ``memo_draw``, ``step_subset``): K++ / CD++ with the
  online block memoisation over random s-subsets (Sec. 4 "Block memoization", Sec. 5.2, the sampling
  steps of Alg. 3 and Alg. 5), the readings for its random draws stated in kpp_oracle.c.
* ``proj_precond`` / ``proj_lsqr``: the inexact projection by sketch-preconditioned LSQR (Sec. 4.1 and the
  supplement's Proj algorithm) with the SRHT sketch; the signs and the column subset are inputs.
* ``rht_forward`` / ``rht_inverse`` / ``rht_entry``: the randomized Hadamard preprocessing of CD++
  (Sec. 5.1, the preprocessing of Alg. 3 and its return D FHT(x)) from the definition Q = H_n D, written out
  with the explicit Sylvester-Hadamard entries.  ``fht`` / ``symfht``: the paper's recursive FHT and
  SymFHT (App. on the symmetric fast Hadamard transform), with their operation counts.
* ``philox4x32_10`` / ``sample_block``: Philox4x32-10 of Salmon et al. (SC'11).

The adaptive-rho schedule and the stopping rule have no worked values in the paper.  They are pinned
instead by closed forms: on diagonal systems with the momentum off, every windowed residual sum, every
ratio, the weighted mean of Eq. 5.3, each rho and the stop iteration follow from the per-entry decay
factors alone (tests/test_oracle.py).
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kpp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libkpp_oracle.so")
_lock = threading.Lock()
_lib = None

OK, NO_CONVERGENCE, NOT_SPD, BAD_ARG = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction so x86 and Arm give the same bits)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("s", ctypes.c_int32), ("cd", ctypes.c_int32), ("lam", ctypes.c_double),
                ("tol", ctypes.c_double), ("max_iters", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("sys", ctypes.c_uint32), ("adaptive", ctypes.c_int32), ("eta", ctypes.c_double),
                ("confirm", ctypes.c_int32)]


class _State(ctypes.Structure):
    _fields_ = [("t", ctypes.c_int64), ("ci", ctypes.c_int64), ("E0", ctypes.c_double),
                ("E1", ctypes.c_double), ("rhat", ctypes.c_double), ("rho", ctypes.c_double)]


class _Report(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("rel_res_true", ctypes.c_double),
                ("rel_res_est", ctypes.c_double), ("status", ctypes.c_int32), ("pad", ctypes.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.orc_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                              ctypes.POINTER(ctypes.c_uint32)]
            lib.orc_sample_block.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int32]
            lib.orc_sample_block.restype = ctypes.c_int32
            lib.orc_cholesky.argtypes = [ctypes.c_int, dp]
            lib.orc_cholesky.restype = ctypes.c_int
            lib.orc_chol_solve.argtypes = [ctypes.c_int, dp, dp]
            lib.orc_rel_residual.argtypes = [ctypes.c_int64, ctypes.c_int64, dp, dp, dp]
            lib.orc_rel_residual.restype = ctypes.c_double
            lib.orc_kpp_factor.argtypes = [ctypes.c_int64, ctypes.c_int64, dp, ctypes.c_int, ctypes.c_double, dp]
            lib.orc_kpp_factor.restype = ctypes.c_int
            lib.orc_cdpp_factor.argtypes = [ctypes.c_int64, dp, ctypes.c_int, ctypes.c_double, dp]
            lib.orc_cdpp_factor.restype = ctypes.c_int
            lib.orc_run.argtypes = [ctypes.c_int64, ctypes.c_int64, dp, dp, dp, ctypes.POINTER(_Params),
                                    ctypes.POINTER(_State), dp, dp, ctypes.POINTER(_Report), dp, ctypes.c_int64]
            lib.orc_run.restype = ctypes.c_int
            lib.orc_cg.argtypes = [ctypes.c_int64, dp, dp, dp, ctypes.c_double, ctypes.c_int64, dp]
            lib.orc_cg.restype = ctypes.c_int64
            lib.orc_gmres.argtypes = [ctypes.c_int64, dp, dp, dp, ctypes.c_int64, ctypes.c_double, ctypes.c_int64, dp,
                                      ctypes.POINTER(ctypes.c_int64)]
            lib.orc_gmres.restype = ctypes.c_int64
            lib.orc_rht_forward.argtypes = [ctypes.c_int64, dp, dp, ctypes.c_int64, dp, dp, dp]
            lib.orc_rht_inverse.argtypes = [ctypes.c_int64, dp, ctypes.c_int64, dp, dp]
            lib.orc_rht_entry.argtypes = [ctypes.c_int64, dp, dp, ctypes.c_int64, ctypes.c_int64]
            lib.orc_rht_entry.restype = ctypes.c_double
            lib.orc_fht.argtypes = [ctypes.c_int64, ctypes.c_int64, dp]
            lib.orc_fht.restype = ctypes.c_int64
            lib.orc_symfht.argtypes = [ctypes.c_int64, dp]
            lib.orc_symfht.restype = ctypes.c_int64
            i64p = ctypes.POINTER(ctypes.c_int64)
            lib.orc_memo_prob.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int64]
            lib.orc_memo_prob.restype = ctypes.c_double
            lib.orc_memo_subset.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int64,
                                            ctypes.c_int, i64p]
            lib.orc_memo_draw.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int,
                                          ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int64]
            lib.orc_memo_draw.restype = ctypes.c_int64
            lib.orc_step_subset.argtypes = [ctypes.c_int64, ctypes.c_int64, dp, dp, i64p, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp, dp]
            lib.orc_step_subset.restype = ctypes.c_int
            lib.orc_run_memo.argtypes = [ctypes.c_int64, ctypes.c_int64, dp, dp, ctypes.POINTER(_Params),
                                         ctypes.POINTER(_State), dp, dp, ctypes.POINTER(_Report), i64p, i64p,
                                         ctypes.c_int64]
            lib.orc_run_memo.restype = ctypes.c_int
            lib.orc_proj_precond.argtypes = [ctypes.c_int64, dp, ctypes.c_int, ctypes.c_double, ctypes.c_int64,
                                             i64p, dp, dp]
            lib.orc_proj_precond.restype = ctypes.c_int
            lib.orc_proj_lsqr.argtypes = [ctypes.c_int64, dp, ctypes.c_int, dp, ctypes.c_double, dp, ctypes.c_int, dp]
            lib.orc_proj_lsqr.restype = ctypes.c_int
            lib.orc_run_lsqr.argtypes = [ctypes.c_int64, ctypes.c_int64, dp, dp, dp, ctypes.c_int,
                                         ctypes.POINTER(_Params), ctypes.POINTER(_State), dp, dp,
                                         ctypes.POINTER(_Report)]
            lib.orc_run_lsqr.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11)
# ----------------------------------------------------------------------------------------------

def philox4x32_10(ctr, key) -> tuple:
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib.orc_philox4x32_10(c, k, o)
    return tuple(int(v) for v in o)


def sample_block(seed: int, t: int, sys: int, nb: int) -> int:
    """Block index drawn at step t of system `sys` (uniform over the nb partition blocks)."""
    return int(_load().orc_sample_block(seed, t, sys, nb))


# ----------------------------------------------------------------------------------------------
# Dense pieces
# ----------------------------------------------------------------------------------------------

def cholesky(G: np.ndarray) -> np.ndarray:
    """Lower Cholesky factor; raises ValueError on a non-positive pivot."""
    L = _f64(G).copy()
    rc = _load().orc_cholesky(L.shape[0], _dp(L))
    if rc:
        raise ValueError(f"not SPD at pivot {rc - 1}")
    return L


def chol_solve(L: np.ndarray, r: np.ndarray) -> np.ndarray:
    y = _f64(r).copy()
    _load().orc_chol_solve(L.shape[0], _dp(_f64(L)), _dp(y))
    return y


def rel_residual(A: np.ndarray, b: np.ndarray, x: np.ndarray) -> float:
    A = _f64(A)
    return float(_load().orc_rel_residual(A.shape[0], A.shape[1], _dp(A), _dp(_f64(b)), _dp(_f64(x))))


def kpp_factor(A: np.ndarray, s: int, lam: float) -> np.ndarray:
    """Per-block factors chol(A_S A_S^T + lam I) (Sec. 4); array of shape (nb, s, s)."""
    A = _f64(A)
    m, n = A.shape
    nb = -(-m // s)
    L = np.zeros((nb, s, s))
    rc = _load().orc_kpp_factor(m, n, _dp(A), s, lam, _dp(L))
    if rc:
        raise ValueError(f"block {rc - 1} not SPD")
    return L


def cdpp_factor(A: np.ndarray, s: int, lam: float) -> np.ndarray:
    """Per-block factors chol(A_SS + lam I) (Sec. 5.2); array of shape (nb, s, s)."""
    A = _f64(A)
    n = A.shape[0]
    nb = -(-n // s)
    L = np.zeros((nb, s, s))
    rc = _load().orc_cdpp_factor(n, _dp(A), s, lam, _dp(L))
    if rc:
        raise ValueError(f"block {rc - 1} not SPD")
    return L


def factor_block(L: np.ndarray, j: int, rows: int, s: int) -> np.ndarray:
    """The (len x len) factor of block j out of the packed (nb, s, s) array."""
    ln = min(s, rows - j * s)
    return L[j].reshape(-1)[: ln * ln].reshape(ln, ln)


# ----------------------------------------------------------------------------------------------
# The iteration
# ----------------------------------------------------------------------------------------------

@dataclasses.dataclass
class State:
    t: int = 0
    ci: int = 0
    E0: float = 0.0
    E1: float = 0.0
    rhat: float = 0.0
    rho: float = 0.0


@dataclasses.dataclass
class Result:
    x: np.ndarray
    mom: np.ndarray
    state: State
    iters: int
    rel_res_true: float
    rel_res_est: float
    status: int
    trace: np.ndarray  # (n_checkpoints, 5): t, E0, E1, rho, true residual (NaN if not computed)


def default_eta(rows: int, cols: int, s: int) -> float:
    """eta = s / (2 min(rows, cols)) (Sec. 5.4; Alg. 3 and Alg. 5 print s/(2n))."""
    return s / (2.0 * min(rows, cols))


def run(A: np.ndarray, b: np.ndarray, L: np.ndarray, s: int, *, cd: bool = False, lam: float = 0.0,
        tol: float = 1e-8, max_iters: int = 100000, seed: int = 0, sys: int = 0, adaptive: bool = True,
        eta: float | None = None, rho: float = 0.0, confirm: bool = True, x0=None, mom0=None,
        state: State | None = None, trace_cap: int = 4096) -> Result:
    """Run K++ (cd=False) or CD++ (cd=True) iterations from a state until the stop rule or max_iters.

    K++ step: Eq. 1.3 with the memoised factor L (Alg. 1); CD++ step: Eq. 5.1.
    Adaptive rho, residual estimate and stop: Eq. 5.2, Eq. 5.3, the checkpoints of Alg. 3 / Alg. 5.
    """
    lib = _load()
    A = _f64(A)
    b = _f64(b)
    rows, n = A.shape
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    mom = np.zeros(n) if mom0 is None else _f64(mom0).copy()
    st = state or State(rho=rho)
    p = _Params(s=s, cd=int(cd), lam=lam, tol=tol, max_iters=max_iters, seed=seed, sys=sys,
                adaptive=int(adaptive), eta=default_eta(rows, n, s) if eta is None else eta,
                confirm=int(confirm))
    cst = _State(st.t, st.ci, st.E0, st.E1, st.rhat, st.rho)
    rep = _Report()
    tr = np.full((trace_cap, 5), np.nan)
    Lc = _f64(L)
    lib.orc_run(rows, n, _dp(A), _dp(b), _dp(Lc), ctypes.byref(p), ctypes.byref(cst), _dp(x), _dp(mom),
                ctypes.byref(rep), _dp(tr), trace_cap)
    nst = State(cst.t, cst.ci, cst.E0, cst.E1, cst.rhat, cst.rho)
    ntr = min(nst.ci - (st.ci if state else 0), trace_cap)
    return Result(x, mom, nst, rep.iters, rep.rel_res_true, rep.rel_res_est, rep.status, tr[:max(ntr, 0)])


def cg(A: np.ndarray, b: np.ndarray, tol: float = 1e-8, max_iters: int = 100000, x0=None):
    """Plain FP64 conjugate gradients (context only).  Returns (x, iterations, |Ax-b|/|b|)."""
    A = _f64(A)
    x = np.zeros(A.shape[0]) if x0 is None else _f64(x0).copy()
    rr = ctypes.c_double()
    it = _load().orc_cg(A.shape[0], _dp(A), _dp(_f64(b)), _dp(x), tol, max_iters, ctypes.byref(rr))
    return x, int(it), rr.value


def gmres(A: np.ndarray, b: np.ndarray, restart: int = 256, tol: float = 1e-8, max_iters: int = 100000, x0=None):
    """Restarted FP64 GMRES (context only; textbook Arnoldi with modified Gram-Schmidt and Givens
    rotations).  Returns (x, steps, |Ax-b|/|b|, cycles)."""
    A = _f64(A)
    x = np.zeros(A.shape[0]) if x0 is None else _f64(x0).copy()
    rr = ctypes.c_double()
    cyc = ctypes.c_int64()
    it = _load().orc_gmres(A.shape[0], _dp(A), _dp(_f64(b)), _dp(x), int(restart), tol, max_iters, ctypes.byref(rr),
                           ctypes.byref(cyc))
    return x, int(it), rr.value, int(cyc.value)


# ----------------------------------------------------------------------------------------------
# Randomized Hadamard preprocessing of CD++ (Sec. 5.1; App. on FHT / SymFHT)
# ----------------------------------------------------------------------------------------------

def _pow2(n: int) -> None:
    if n < 1 or n & (n - 1):
        raise ValueError("n must be a power of 2")


def rht_forward(d: np.ndarray, A: np.ndarray, b: np.ndarray | None = None):
    """(Q A Q^T, Q b) with Q = H_n diag(d) / sqrt(n), H_n Sylvester-Hadamard, d = +-1 signs.  b is a
    vector or an n x k panel (or None).  Explicit O(n^3) definition."""
    A = _f64(A)
    n = A.shape[0]
    _pow2(n)
    B = np.zeros((n, 0)) if b is None else _f64(np.asarray(b).reshape(n, -1))
    k = B.shape[1]
    Abar = np.empty((n, n))
    Bbar = np.empty((n, max(k, 1)))
    _load().orc_rht_forward(n, _dp(_f64(d)), _dp(A), k, _dp(B if k else np.zeros((n, 1))), _dp(Abar), _dp(Bbar))
    if b is None:
        return Abar, None
    return Abar, Bbar[:, :k].reshape(np.shape(b))


def rht_inverse(d: np.ndarray, xbar: np.ndarray) -> np.ndarray:
    """x = Q^T xbar = diag(d) H_n xbar / sqrt(n) (vector or n x k panel)."""
    Xb = _f64(np.asarray(xbar).reshape(len(d), -1))
    n, k = Xb.shape
    _pow2(n)
    X = np.empty_like(Xb)
    _load().orc_rht_inverse(n, _dp(_f64(d)), k, _dp(Xb), _dp(X))
    return X.reshape(np.shape(xbar))


def rht_entry(d: np.ndarray, A: np.ndarray, i: int, j: int) -> float:
    """One entry of Q A Q^T in O(n^2) (for sampled checks at large n)."""
    A = _f64(A)
    _pow2(A.shape[0])
    return float(_load().orc_rht_entry(A.shape[0], _dp(_f64(d)), _dp(A), int(i), int(j)))


def fht(V: np.ndarray):
    """(H_n V, additions used) for a vector or n x k panel, by the halving recursion."""
    W = _f64(np.asarray(V).reshape(np.shape(V)[0], -1)).copy()
    n, k = W.shape
    _pow2(n)
    ops = _load().orc_fht(n, k, _dp(W))
    return W.reshape(np.shape(V)), int(ops)


def symfht(A: np.ndarray):
    """(H_n A H_n, additions used) for a symmetric A, by the paper's SymFHT recursion."""
    W = _f64(A).copy()
    _pow2(W.shape[0])
    ops = _load().orc_symfht(W.shape[0], _dp(W))
    return W, int(ops)


# ----------------------------------------------------------------------------------------------
# Online block memoisation with random subsets (Sec. 4, Sec. 5.2; the sampling steps of Alg. 3 / Alg. 5)
# ----------------------------------------------------------------------------------------------

def memo_prob(cd: bool, rows: int, n: int, s: int, t: int) -> float:
    """Probability that step t draws a new block (CD++: min(1, (n/s) ln n / t); K++: the minimum with
    (m/s) ln m / t and (n/s) ln m / t; 1 at t = 0)."""
    return float(_load().orc_memo_prob(int(cd), rows, n, s, t))


def memo_subset(seed: int, t: int, sys: int, N: int, s: int) -> np.ndarray:
    """The uniform s-subset of range(N) drawn at step t (Floyd's sampling), sorted."""
    S = np.empty(s, dtype=np.int64)
    _load().orc_memo_subset(seed, t, sys, N, s, S.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return S


def memo_draw(seed: int, t: int, sys: int, cd: bool, rows: int, n: int, s: int, nb: int) -> int:
    """-1 when step t draws a new subset, else the index in [0, nb) of the memoised block it reuses."""
    return int(_load().orc_memo_draw(seed, t, sys, int(cd), rows, n, s, nb))


def step_subset(A: np.ndarray, b: np.ndarray, S, *, cd: bool, lam: float, beta: float = 1.0, eta: float = 0.0,
                x0=None, mom0=None):
    """One step on the rows S (factor computed here): (x, mom, |r|^2)."""
    A, b = _f64(A), _f64(b)
    rows, n = A.shape
    Sv = np.ascontiguousarray(S, dtype=np.int64)
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    mom = np.zeros(n) if mom0 is None else _f64(mom0).copy()
    rn2 = ctypes.c_double()
    rc = _load().orc_step_subset(rows, n, _dp(A), _dp(b), Sv.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(Sv),
                                 int(cd), lam, beta, eta, _dp(x), _dp(mom), ctypes.byref(rn2))
    if rc:
        raise ValueError("subset block not SPD")
    return x, mom, rn2.value


def run_memo(A: np.ndarray, b: np.ndarray, s: int, *, cd: bool = False, lam: float = 0.0, tol: float = 1e-8,
             max_iters: int = 100000, seed: int = 0, sys: int = 0, adaptive: bool = True, eta: float | None = None,
             confirm: bool = True, block_cap: int = 0):
    """K++ / CD++ with the online memo from x0 = 0.  Returns (Result, number of memoised blocks,
    memo index of each of the first block_cap steps)."""
    lib = _load()
    A, b = _f64(A), _f64(b)
    rows, n = A.shape
    x, mom = np.zeros(n), np.zeros(n)
    cst = _State(0, 0, 0.0, 0.0, 0.0, 0.0)
    p = _Params(s=s, cd=int(cd), lam=lam, tol=tol, max_iters=max_iters, seed=seed, sys=sys,
                adaptive=int(adaptive), eta=default_eta(rows, n, s) if eta is None else eta, confirm=int(confirm))
    rep = _Report()
    nb = ctypes.c_int64()
    blocks = np.full(max(block_cap, 1), -2, dtype=np.int64)
    lib.orc_run_memo(rows, n, _dp(A), _dp(b), ctypes.byref(p), ctypes.byref(cst), _dp(x), _dp(mom), ctypes.byref(rep),
                     ctypes.byref(nb), blocks.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), block_cap)
    st = State(cst.t, cst.ci, cst.E0, cst.E1, cst.rhat, cst.rho)
    res = Result(x, mom, st, rep.iters, rep.rel_res_true, rep.rel_res_est, rep.status, np.zeros((0, 5)))
    return res, int(nb.value), blocks[:block_cap]


# ----------------------------------------------------------------------------------------------
# Inexact projection: sketch-preconditioned LSQR (Sec. 4.1; the supplement's Proj algorithm)
# ----------------------------------------------------------------------------------------------

def proj_precond(AS: np.ndarray, lam: float, T, d) -> np.ndarray:
    """Lower L with L L^T = Ahat Ahat^T + lam I, Ahat = (A_S D H)[:, T] / sqrt(tau) (SRHT sketch; A_S padded
    with zero columns to the next power of 2; d: that many signs)."""
    AS = _f64(AS)
    s, n = AS.shape
    Tv = np.ascontiguousarray(T, dtype=np.int64)
    L = np.empty((s, s))
    rc = _load().orc_proj_precond(n, _dp(AS), s, lam, len(Tv), Tv.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  _dp(_f64(d)), _dp(L))
    if rc:
        raise ValueError("sketched Gram not SPD")
    return L


def proj_lsqr(AS: np.ndarray, r: np.ndarray, lam: float, L: np.ndarray, t_max: int):
    """(w, iterations): LSQR on L^{-1} [A_S, sqrt(lam) I] [w; v] = L^{-1} r from zero, the first n entries."""
    AS = _f64(AS)
    s, n = AS.shape
    w = np.empty(n)
    it = _load().orc_proj_lsqr(n, _dp(AS), s, _dp(_f64(r)), lam, _dp(_f64(L)), int(t_max), _dp(w))
    return w, int(it)



def lsqr_factors(A: np.ndarray, s: int, lam: float, T, d) -> np.ndarray:
    """The sketch preconditioner of every block of the contiguous partition (proj_precond per block),
    stacked as nb x s x s (block j: len x len, leading dimension len, as the exact factors)."""
    A = _f64(A)
    rows = A.shape[0]
    nb = -(-rows // s)
    L = np.zeros((nb, s, s))
    for j in range(nb):
        ln = min(s, rows - j * s)
        Lj = proj_precond(A[j * s:j * s + ln], lam, T, d)
        L[j].reshape(-1)[:ln * ln] = Lj.reshape(-1)
    return L


def run_lsqr(A: np.ndarray, b: np.ndarray, Lsk: np.ndarray, s: int, t_max: int, *, lam: float = 0.0,
             tol: float = 1e-8, max_iters: int = 100000, seed: int = 0, sys: int = 0, adaptive: bool = True,
             eta: float | None = None, confirm: bool = True) -> Result:
    """K++ from x0 = 0 with the block step's projection computed by t_max iterations of
    sketch-preconditioned LSQR (Sec. 4.1; orc_run_lsqr); Lsk from lsqr_factors."""
    lib = _load()
    A, b = _f64(A), _f64(b)
    rows, n = A.shape
    x, mom = np.zeros(n), np.zeros(n)
    cst = _State(0, 0, 0.0, 0.0, 0.0, 0.0)
    p = _Params(s=s, cd=0, lam=lam, tol=tol, max_iters=max_iters, seed=seed, sys=sys, adaptive=int(adaptive),
                eta=default_eta(rows, n, s) if eta is None else eta, confirm=int(confirm))
    rep = _Report()
    rc = lib.orc_run_lsqr(rows, n, _dp(A), _dp(b), _dp(_f64(Lsk)), int(t_max), ctypes.byref(p), ctypes.byref(cst),
                          _dp(x), _dp(mom), ctypes.byref(rep))
    if rc == 3:  # ORC_BAD_ARG
        raise ValueError("orc_run_lsqr: bad argument")
    st = State(cst.t, cst.ci, cst.E0, cst.E1, cst.rhat, cst.rho)
    return Result(x, mom, st, rep.iters, rep.rel_res_true, rep.rel_res_est, rep.status, np.zeros((0, 5)))