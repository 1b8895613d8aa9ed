"""The Krylov reference points of the SPD bench line (the library's FP64 CG and GMRES), on the CPU
with a stand-in for the library: the fields come out whole and the flop counts follow the paper's
models (CG 2n^2 + 11n per iteration; GMRES 2n^2 T + 4n T (T + 1))."""
import os
import sys
import types

import numpy as np
import pytest

from paper_2501_11673_gb300 import workloads as W

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


class _FakeKpp:
    """Stands in for the library: fixed step counts and times."""

    def __init__(self):
        self.calls = []

    def cg(self, A, b, x, tol):
        self.calls.append(("cg", tol))
        return types.SimpleNamespace(iters=40, kernel_ms=2.0 + len(self.calls), rel_res_true=0.9 * tol)

    def gmres(self, A, b, x, restart, tol):
        self.calls.append(("gmres", restart, tol))
        return types.SimpleNamespace(iters=37, kernel_ms=3.0 - 0.1 * len(self.calls), rel_res_true=0.8 * tol)


@pytest.mark.parametrize("method", ["cg", "gmres"])
def test_krylov_reference_fields_and_flop_models(method, monkeypatch):
    bench = _bench()
    n = 64
    monkeypatch.setattr(torch, "zeros", lambda *a, **k: None)  # no device vectors on the CPU
    fk = _FakeKpp()
    out = bench.krylov_reference(fk, np.eye(n), np.ones(n), 1e-8, method)
    T = 40 if method == "cg" else 37
    assert out["iters"] == T and out["rel_res_true"] <= 1e-8
    model = (2 * n * n + 11 * n) * T if method == "cg" else 2 * n * n * T + 4 * n * T * (T + 1)
    assert out["flops_paper_model"] == model
    assert len(fk.calls) == 3 and out["time_to_tol_ms"] == min(
        (3.0, 4.0, 5.0) if method == "cg" else (2.9, 2.8, 2.7))


def test_cdpp_flop_fields_of_the_spd_line():
    bench = _bench()
    A, b, _ = W.spd(128, 4, 1e2, 1e4, 1.0, 10.0, seed_A=3, seed_b=4)
    wl = object.__new__(bench.SingleFP64)
    wl.cd, wl.name = True, "cdpp4096"
    wl.run_cg_reference = False
    wl.sy = W.System(A, b, None, s=16, lam=1e-4, tol=1e-8, name="spd128")
    out = wl.extra([{"iters": 1000}])
    assert out["cdpp_flops"]["iterations"] == wl.per_iter()[0] * 1000
    assert out["cdpp_flops"]["factor_phase"] == 8 * (16 ** 3 / 3 + 2 * 16 * 16 * 128)
