"""The FP32 memo W_j = G_j^{-1} A_{S_j} (Sec. 4's memoised projection folded into one operator per
block) built on the tcgen05 tensor cores for BF16 storage, against the library GEMM (cuBLAS with the
BF16x9 FP32 emulation, KPP_WMEMO_TC=0) on the same G^{-1}, and against the FP64 product.

Both builds compute sum_k g_ak A_kc with g the FP32 inverse and A exact in BF16: the tensor-core path
splits g into three BF16 pieces (g - hi - mid - lo at most 2^-24 |g|), forms exact products and sums
3 s of them in FP32, so each entry is within (3 + 3 s) 2^-24 (|G^-1| |A_S|)_ac of the exact sum with
the FP32 g; the two builds are therefore within twice that of each other.  Against the FP64 product
with the FP64 inverse from the factor the FP32 rounding of the inverse itself enters as well; that
relative error is reported.
"""
import os

import numpy as np
import pytest

from paper_2501_11673_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def K():
    from paper_2501_11673_gb300 import build as kbuild
    from paper_2501_11673_gb300 import kpp
    kbuild.build()
    kpp.load()
    return kpp


def _factors_both(K, Ad, P, lam, mode):
    F_tc = K.Factors(Ad, P, lam, mode)
    os.environ["KPP_WMEMO_TC"] = "0"
    try:
        F_bl = K.Factors(Ad, P, lam, mode)
    finally:
        del os.environ["KPP_WMEMO_TC"]
    return F_tc, F_bl


@pytest.mark.parametrize("m,n,s,mode", [(2048, 1024, 512, 0),   # K++ large blocks, s = 512
                                        (4096, 512, 256, 0),    # K++, s = 256
                                        (6400, 256, 32, 0),     # K++, 200 blocks: the memo of the first
                                                                # 152 overlaps the last blocks' Cholesky
                                        (576, 576, 64, 1)])     # CD++ single-column memo, N tail (576 = 2.25 x 256)
def test_tensor_core_memo_matches_library_gemm(K, record_property, m, n, s, mode):
    if mode == 0:
        A, _, _ = W.gaussian_rows(m, n, 0, 1.0, seed_A=700 + s, seed_b=701, k_rhs=1)
        lam = W.row_outlier_lambda(A)
    else:
        A, _, _ = W.spd(n, 6, 1e2, 1e3, 1.0, 10.0, seed_A=702, seed_b=703)
        lam = 1e-4
    A = W.round_to_storage(A, "bf16")
    Ad = torch.as_tensor(A, dtype=torch.bfloat16, device="cuda")
    P = K.Partition(m, s)
    F_tc, F_bl = _factors_both(K, Ad, P, lam, mode)
    W_tc = F_tc.memo(0, m, n).astype(np.float64)
    W_bl = F_bl.memo(0, m, n).astype(np.float64)
    assert np.all(np.isfinite(W_tc))
    worst_pair, worst_fp64 = 0.0, 0.0
    for j in range(m // s):
        As = A[j * s:(j + 1) * s]
        L = F_tc.block(j)
        Ginv = np.linalg.inv(L @ L.T)
        M = np.abs(Ginv) @ np.abs(As)
        d = np.abs(W_tc[j * s:(j + 1) * s] - W_bl[j * s:(j + 1) * s])
        bound = 2.0 * (3.0 + 3.0 * s) * EPS32 * M
        assert np.all(d <= bound + 1e-30), (j, float(np.max(d / (M + 1e-300))))
        worst_pair = max(worst_pair, float(np.max(d / (M + 1e-300))))
        Wref = Ginv @ As
        worst_fp64 = max(worst_fp64, float(np.linalg.norm(W_tc[j * s:(j + 1) * s] - Wref) / np.linalg.norm(Wref)))
    record_property("max_diff_over_abs_product", worst_pair)
    record_property("rel_err_vs_fp64", worst_fp64)
    print(f"\nm={m} n={n} s={s}: tensor-core vs library memo {worst_pair:.2e} of |G^-1||A_S|; "
          f"vs FP64 product {worst_fp64:.2e} relative")
