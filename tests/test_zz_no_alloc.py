"""ftwa_moments_noalloc, the allocation-free estimator entry point.

It serves callers that cannot call cudaMalloc (device memory owned by another
allocator, or loops that cannot afford cudaMalloc's implicit device
synchronisation): it takes no plan and keeps its only scratch, the sample
means, in a static device array.  Checked here through the C ABI against
ftwa_moments (FP64 Gram mode) on two calls in a row with different data and
sizes, in FP64 and FP32.  This file is collected last so that a run stopping
at the first failure has already run every other test; it passes on its own
in a fresh process as well.
"""

import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ftwa():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_04352_gb300 as F
    F.load()
    return F


def _snapshots(F, lat, precision, M, steps, seed):
    nu, nd = W.neel_state(lat)
    P = F.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=precision, out_every=10)
    rho = P.sample(seed, M)
    X = P.evolve(rho, steps)
    return P, X


def _noalloc(F, X, precision, n_sites):
    lib = F.load()
    T, M, K = X.shape
    occ = torch.empty((T, K), dtype=torch.float64, device=X.device)
    conn = torch.empty((T, K, K), dtype=torch.float64, device=X.device)
    g2 = torch.empty((T, K, K), dtype=torch.float64, device=X.device)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.ftwa_moments_noalloc(ctypes.c_void_p(X.data_ptr()), precision, n_sites, M, T,
                                  ctypes.c_void_p(occ.data_ptr()), ctypes.c_void_p(conn.data_ptr()),
                                  ctypes.c_void_p(g2.data_ptr()), s)
    assert rc == 0
    return occ, conn, g2


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_matches_moments_two_calls(ftwa, precision):
    cases = [(W.periodic_honeycomb(), 1000, 200, 1), (W.hexagonal_flake(3), 333, 50, 2)]
    for lat, M, steps, seed in cases:                         # two calls in a row
        P, X = _snapshots(ftwa, lat, precision, M, steps, seed)
        occ_r, conn_r, g2_r = P.moments(X, gram_mode=ftwa.FTWA_GRAM_FP64)
        occ, conn, g2 = _noalloc(ftwa, X, precision, lat.n_sites)
        torch.cuda.synchronize()
        assert P.status() == 0
        np.testing.assert_allclose(occ.cpu().numpy(), occ_r.cpu().numpy(), rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(conn.cpu().numpy(), conn_r.cpu().numpy(), rtol=1e-12, atol=1e-15)
        a, b = g2.cpu().numpy(), g2_r.cpu().numpy()
        assert np.array_equal(np.isnan(a), np.isnan(b))
        ok = ~np.isnan(b)
        np.testing.assert_allclose(a[ok], b[ok], rtol=1e-12)
        P.close()


def test_noalloc_rejects_oversize_and_bad_args(ftwa):
    lib = ftwa.load()
    from paper_2212_04352_gb300 import _lib as L
    X = torch.zeros((1, 4, 16), dtype=torch.float64, device="cuda")
    out = torch.zeros((1, 16, 16), dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p
    T_big = L.FTWA_MOMENTS_NOALLOC_MAX_TK // 16 + 1              # n_times * 2N over the static limit
    assert lib.ftwa_moments_noalloc(p(X.data_ptr()), 0, 8, 4, T_big, p(out.data_ptr()), p(out.data_ptr()),
                                    None, None) == L.FTWA_ERR_UNSUPPORTED
    assert lib.ftwa_moments_noalloc(None, 0, 8, 4, 1, p(out.data_ptr()), p(out.data_ptr()), None,
                                    None) == L.FTWA_ERR_INVALID_ARGUMENT
    assert lib.ftwa_moments_noalloc(p(X.data_ptr()), 5, 8, 4, 1, p(out.data_ptr()), p(out.data_ptr()), None,
                                    None) == L.FTWA_ERR_INVALID_ARGUMENT
