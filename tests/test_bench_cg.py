"""The Krylov reference point of the SPD bench line (plain FP64 CG in torch), on the CPU: it takes the
oracle's iterations and reaches the same solution, and the bench's extra fields come out whole."""
import os
import sys

import numpy as np
import pytest

import oracle
from paper_2501_11673_gb300 import workloads as W

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


@pytest.mark.parametrize("n,seed", [(256, 1), (512, 2)])
def test_torch_cg_matches_the_oracle_cg(n, seed):
    bench = _bench()
    A, b, sig = W.spd(n, 8, 1e2, 1e4, 1.0, 10.0, seed_A=seed, seed_b=seed + 100)
    xo, ito, ro = oracle.cg(A, b, tol=1e-8, max_iters=20000)
    xt, itt, rt = bench.cg_torch(torch.as_tensor(A), torch.as_tensor(b), 1e-8, 20000)
    # same recurrences; the sums round differently (torch blocks its dot products), and CG's loss of
    # orthogonality on the outliers turns that into a few iterations either way
    assert abs(itt - ito) <= max(2, 0.06 * ito) and rt <= 1e-8 and ro <= 1e-8
    xs = np.linalg.solve(A, b)
    err = np.linalg.norm(xt.numpy() - xs) / np.linalg.norm(xs)
    assert err <= sig.max() / sig.min() * 1e-8


def test_cg_reference_and_flop_fields_of_the_spd_line():
    bench = _bench()
    A, b, _ = W.spd(128, 4, 1e2, 1e4, 1.0, 10.0, seed_A=3, seed_b=4)
    wl = object.__new__(bench.SingleFP64)
    wl.cd, wl.name = True, "cdpp4096"
    wl.sy = W.System(A, b, None, s=16, lam=1e-4, tol=1e-8, name="spd128")
    wl.Ad, wl.bd = torch.as_tensor(A), torch.as_tensor(b)
    out = wl.extra([{"iters": 1000}])
    cg = out["cg_reference"]
    assert "error" not in cg and cg["rel_res_true"] <= 1e-8 and cg["iters"] > 0 and cg["time_to_tol_ms"] > 0
    assert cg["flops_paper_model"] == (2 * 128 * 128 + 11 * 128) * cg["iters"]
    assert out["cdpp_flops"]["iterations"] == wl.per_iter()[0] * 1000
    assert out["cdpp_flops"]["factor_phase"] == 8 * (16 ** 3 / 3 + 2 * 16 * 16 * 128)
