"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every symbol include/ftwa.h declares, and rejects bad arguments before any
device work."""

import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W
from tests.conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    from paper_2212_04352_gb300 import build as b
    b.build()
    from paper_2212_04352_gb300 import _lib
    return _lib.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "ftwa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ftwa_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    from paper_2212_04352_gb300 import _lib
    names = _declared()
    assert set(names) == set(_lib.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_strings(lib):
    assert lib.ftwa_version() == 10000
    for code in range(0, -7, -1):
        assert lib.ftwa_error_string(code)
    assert lib.ftwa_error_string(-99) == b"unknown status"


def _plan(lib, bonds, n, nu=None, nd=None, U=1.0, filling=0.0, precision=0, dt=0.0, out_every=0, t_bond=None):
    from paper_2212_04352_gb300 import _lib
    b = np.ascontiguousarray(bonds, dtype=np.int32).reshape(-1, 2)
    tb = None if t_bond is None else np.ascontiguousarray(t_bond, dtype=np.float64)
    lat = _lib.Lattice(n, b.shape[0], b.ctypes.data if b.size else None, None if tb is None else tb.ctypes.data)
    init = None
    if nu is not None:
        nu = np.ascontiguousarray(nu, dtype=np.float64)
        nd = np.ascontiguousarray(nd, dtype=np.float64)
        init = _lib.InitState(nu.ctypes.data, nd.ctypes.data)
    opts = _lib.Options(precision, dt, out_every, 0, 0, 0, 0, 0)
    h = ctypes.c_void_p()
    rc = lib.ftwa_plan(ctypes.byref(lat), U, 1.0, filling, None if init is None else ctypes.byref(init),
                       ctypes.byref(opts), ctypes.byref(h))
    if rc == 0:
        lib.ftwa_destroy(h)
    return rc


def test_plan_rejects_bad_input(lib):
    from paper_2212_04352_gb300 import _lib as L
    star = [(0, 1), (0, 2), (0, 3), (0, 4)]                         # degree 4
    assert _plan(lib, star, 5, np.ones(5) * 0.5, np.ones(5) * 0.5) == L.FTWA_ERR_UNSUPPORTED
    assert _plan(lib, [(1, 0)], 2, [1, 0], [0, 1]) == L.FTWA_ERR_INVALID_ARGUMENT       # i > j
    assert _plan(lib, [(0, 1), (0, 1)], 2, [1, 0], [0, 1]) == L.FTWA_ERR_INVALID_ARGUMENT  # duplicate
    assert _plan(lib, [(0, 2)], 2, [1, 0], [0, 1]) == L.FTWA_ERR_INVALID_ARGUMENT       # out of range
    assert _plan(lib, [(0, 1)], 2, [1.5, 0], [0, 1]) == L.FTWA_ERR_INVALID_ARGUMENT     # n > 1
    assert _plan(lib, [(0, 1)], 2, [1, 0], [0, 1], filling=0.7) == L.FTWA_ERR_INVALID_ARGUMENT
    assert _plan(lib, [(0, 1)], 2, [1, 0], [0, 1], dt=-0.1) == L.FTWA_ERR_INVALID_ARGUMENT
    assert _plan(lib, [(0, 1)], 2, [1, 0], [0, 1], precision=7) == L.FTWA_ERR_INVALID_ARGUMENT
    assert _plan(lib, [(0, 1)], 2, [1, 0], [0, 1], out_every=-1) == L.FTWA_ERR_INVALID_ARGUMENT
    assert _plan(lib, [(0, 1)], 2, [1, 0], [0, 1], t_bond=[np.nan]) == L.FTWA_ERR_INVALID_ARGUMENT
    assert _plan(lib, [], 1) == L.FTWA_ERR_UNSUPPORTED                                # too small
    assert _plan(lib, [], 300) == L.FTWA_ERR_UNSUPPORTED                              # too large
    tri = [(0, 1), (1, 2), (0, 2)]                                                      # odd ring, no init
    assert _plan(lib, tri, 3, filling=0.5) == L.FTWA_ERR_INVALID_ARGUMENT
    assert lib.ftwa_plan(None, 1.0, 1.0, 0.0, None, None, None) == L.FTWA_ERR_INVALID_ARGUMENT


def test_null_plan_calls_rejected(lib):
    from paper_2212_04352_gb300 import _lib as L
    assert lib.ftwa_sample(None, 1, 0, 4, None, None) == L.FTWA_ERR_INVALID_ARGUMENT
    assert lib.ftwa_evolve(None, None, 4, 10, None, None) == L.FTWA_ERR_INVALID_ARGUMENT
    assert lib.ftwa_moments(None, None, 4, 1, None, None, None, 0, None) == L.FTWA_ERR_INVALID_ARGUMENT
    assert lib.ftwa_adjoint(None, 1, 4, 10, 10, None, None, None, None, None) == L.FTWA_ERR_INVALID_ARGUMENT
    assert lib.ftwa_status(None, None) == L.FTWA_ERR_INVALID_ARGUMENT
    assert lib.ftwa_philox(1, 0, 0, 0, -1, None, None) == L.FTWA_ERR_INVALID_ARGUMENT
    lib.ftwa_destroy(None)


def test_workload_inputs():
    """Input generators: sizes and bond counts of the synthetic geometries."""
    assert W.brick_wall_flake().n_sites == 198 and W.brick_wall_flake().n_bonds == 277
    for k, n in [(2, 24), (3, 54), (4, 96), (5, 150)]:
        lat = W.hexagonal_flake(k)
        assert lat.n_sites == n and lat.n_bonds == 9 * k * k - 3 * k
        assert lat.degrees().max() <= 3
    lat = W.brick_wall_flake()
    nu, nd = W.charge_imbalanced_state(lat)
    assert nu.sum() == 99 and nd.sum() == 99
    assert ((nu + nd) == 2).sum() == 6 and ((nu + nd) == 0).sum() == 6


def test_adjoint_checkpoint_default():
    """The autograd wrapper's default checkpoint spacing divides n_steps, is a
    multiple of out_every and lies near sqrt(n_steps)."""
    import paper_2212_04352_gb300 as F
    for n_steps, every, want in [(40, 10, 10), (1000, 10, 40), (30, 10, 10), (400, 20, 20), (3600, 10, 60)]:
        c = F._default_ckpt(n_steps, every)
        assert c == want and n_steps % c == 0 and c % every == 0


def test_autograd_function_is_exposed():
    """FTWAFunction is a torch.autograd.Function (created without touching the
    CUDA library); occupations() is the entry point that applies it."""
    torch = pytest.importorskip("torch")
    import paper_2212_04352_gb300 as F
    assert issubclass(F.FTWAFunction, torch.autograd.Function)
    assert F.FTWAFunction is F.FTWAFunction and callable(F.occupations)
