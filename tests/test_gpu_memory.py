"""The library's device memory caches (kpp_device_cache_bytes / kpp_device_cache_trim): a released
factor set's buffers are kept and handed out again for the same shape, the results do not depend on
whether a buffer came from the cache, and a trim returns everything to the driver."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def K():
    from paper_2501_11673_gb300 import build as kbuild
    from paper_2501_11673_gb300 import kpp
    kbuild.build()
    kpp.load()
    return kpp


def test_factor_buffers_are_cached_reused_and_trimmed(K):
    rng = np.random.default_rng(11)
    m, n, s = 1024, 256, 64
    A_h = rng.standard_normal((m, n))
    A = torch.as_tensor(A_h, device="cuda")
    b = torch.as_tensor(A_h @ rng.standard_normal(n), device="cuda")  # consistent: the residual reaches 0
    P = K.Partition(m, s)
    prm = K.params(lam=0.1, tol=1e-10, seed=4)
    K.device_cache_trim()
    assert K.device_cache_bytes() == 0

    outs = []
    for _ in range(3):
        F = K.Factors(A, P, 0.1, 0)
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        rep = K.kpp_solve(A, b, x, P, F, prm)
        outs.append((F.block(5), x.cpu().numpy(), rep.iters))
        del F
        # the factors (L and G^-1: 16 blocks of 64 x 64 doubles each) wait for the next request
        assert K.device_cache_bytes() >= 2 * (m // s) * s * s * 8
    for Lb, xb, it in outs[1:]:
        assert np.array_equal(Lb, outs[0][0])
        assert np.array_equal(xb, outs[0][1]) and it == outs[0][2]

    K.device_cache_trim()
    assert K.device_cache_bytes() == 0
    # the library still works after a trim
    F = K.Factors(A, P, 0.1, 0)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    K.kpp_solve(A, b, x, P, F, prm)
    assert np.array_equal(x.cpu().numpy(), outs[0][1])
