"""ftwa_moments_noalloc, the allocation-free estimator entry point.

It serves callers that cannot call cudaMalloc (device memory owned by another
allocator, or loops that cannot afford cudaMalloc's implicit device
synchronisation): it takes no plan and keeps its only scratch, the sample
means, in a static device array.  Checked here through the C ABI against
ftwa_moments (FP64 Gram mode) on two calls in a row with different data and
sizes, in FP64 and FP32.  This file is collected last so that a run stopping
at the first failure has already run every other test; it passes on its own
in a fresh process as well.  A device reset between two calls (in a child
process, which owns its context) must not leave a stale scratch address.
"""

import ctypes
import os
import subprocess
import sys

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
    # n_times beyond the grid limit of the two kernels, inside the size limit
    assert lib.ftwa_moments_noalloc(p(X.data_ptr()), 0, 1, 4, 65536, p(out.data_ptr()), p(out.data_ptr()), None,
                                    None) == L.FTWA_ERR_UNSUPPORTED


def test_noalloc_python_wrapper(ftwa):
    """The binding's moments_noalloc: the same results as ftwa_moments, and
    mismatched shapes or types rejected before the library is called."""
    lat = W.periodic_honeycomb()
    P, X = _snapshots(ftwa, lat, 0, 200, 50, 4)
    occ_r, conn_r, g2_r = P.moments(X, gram_mode=ftwa.FTWA_GRAM_FP64)
    occ, conn, g2 = ftwa.moments_noalloc(X, 0, lat.n_sites)
    torch.cuda.synchronize()
    np.testing.assert_allclose(occ.cpu().numpy(), occ_r.cpu().numpy(), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(conn.cpu().numpy(), conn_r.cpu().numpy(), rtol=1e-12, atol=1e-15)
    with pytest.raises(ValueError):
        ftwa.moments_noalloc(X, 0, lat.n_sites + 1)                  # 2N does not match X
    with pytest.raises(ValueError):
        ftwa.moments_noalloc(X, 1, lat.n_sites)                      # FP32 precision, FP64 data
    bad = (occ, conn[:, :8], g2)
    with pytest.raises(ValueError):
        ftwa.moments_noalloc(X, 0, lat.n_sites, out=bad)             # wrong output shape
    P.close()


_RESET_CHILD = r"""
import ctypes, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2212_04352_gb300 import _lib
lib = _lib.load()
rt = ctypes.CDLL("libcudart.so.13")
P = ctypes.c_void_p
rt.cudaMalloc.argtypes = [ctypes.POINTER(P), ctypes.c_size_t]
rt.cudaFree.argtypes = [P]
rt.cudaMemcpy.argtypes = [P, P, ctypes.c_size_t, ctypes.c_int]
T, M, N = 3, 500, 8
K = 2 * N
X = np.random.default_rng(3).random((T, M, K)) - 0.5

def call():
    dx, do, dc = P(), P(), P()
    for d, n in ((dx, X.nbytes), (do, T * K * 8), (dc, T * K * K * 8)):
        assert rt.cudaMalloc(ctypes.byref(d), n) == 0
    assert rt.cudaMemcpy(dx, X.ctypes.data, X.nbytes, 1) == 0
    assert lib.ftwa_moments_noalloc(dx, 0, N, M, T, do, dc, None, None) == 0
    occ, conn = np.zeros((T, K)), np.zeros((T, K, K))
    assert rt.cudaMemcpy(occ.ctypes.data, do, occ.nbytes, 2) == 0
    assert rt.cudaMemcpy(conn.ctypes.data, dc, conn.nbytes, 2) == 0
    for d in (dx, do, dc):
        rt.cudaFree(d)
    return occ, conn

a = call()
assert rt.cudaDeviceReset() == 0
b = call()
assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
assert np.allclose(a[0], X.mean(1) + 0.5, rtol=1e-13, atol=1e-15)
assert np.allclose(a[1][1], np.cov(X[1].T, bias=True), rtol=1e-12, atol=1e-15)
print("reset ok")
"""


def test_noalloc_after_device_reset(ftwa):
    """Call, reset the device, call again (in a child process with its own
    context): the second call looks up the scratch array's new address and
    gives the same results as the first."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _RESET_CHILD, root], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "reset ok" in r.stdout
