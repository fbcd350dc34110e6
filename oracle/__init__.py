"""CPU oracle for the fTWA hot path (TEST INFRASTRUCTURE ONLY).

A plain FP64 implementation of what the GPU path computes, written from the
paper (arXiv:2212.04352) and kept independent of the CUDA library: it shares
no code, header or helper with it and never imports it.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
it.  Its C part (``ftwa_oracle.c``) is compiled on first use with the host
gcc; ``ed.py`` and ``closed_forms.py`` hold the independent checks the oracle
itself is pinned to; ``adjoint.py`` is the discrete RK4 adjoint (numpy),
pinned to finite differences of this integration.

Parity status: every function here is pinned by a test in ``tests/``
(closed forms, worked values of the paper, invariants, exact
diagonalisation); the site-resolved curves of the paper's figures are parity
unpinned because the figures' data are not available.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ftwa_oracle.c")
_LIB = os.path.join(_HERE, "libftwa_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle in place (gcc, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i32, i64, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            lib.orc_philox4x32_10.argtypes = [P, P, P]
            lib.orc_philox_block.argtypes = [u64, i64, i32, i64, i64, P]
            lib.orc_normals.argtypes = [i32, u64, i64, P]
            lib.orc_sample.argtypes = [i32, P, P, u64, i64, P]
            lib.orc_rhs.argtypes = [i32, i32, P, P, f64, P, P]
            lib.orc_evolve.argtypes = [i32, i32, P, P, f64, f64, i64, i64, P, P]
            lib.orc_evolve_longrange.argtypes = [i32, i32, P, P, P, f64, i64, i64, P, P]
            lib.orc_evolve_drive.argtypes = [i32, i32, P, P, f64, f64, i64, i64, P, P, P, f64, f64, f64, f64, f64,
                                             f64, f64, f64, f64, f64]
            lib.orc_run.argtypes = [i32, i32, P, P, f64, P, P, u64, i64, i64, f64, i64, i64, P, P, i32]
            lib.orc_run.restype = ctypes.c_int
            lib.orc_energy.argtypes = [i32, i32, P, P, f64, P, P]
            lib.orc_moments.argtypes = [i64, i64, i64, P, P, P, P]
            lib.orc_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _lat_arrays(lat, t_bond=None):
    bonds = np.ascontiguousarray(lat.bonds, dtype=np.int32)
    t = np.ascontiguousarray(lat.t_bond if t_bond is None else t_bond, dtype=np.float64)
    return bonds, t


def philox4x32_10(ctr, key):
    """Philox4x32-10 of one 128-bit counter under a 64-bit key (4 + 2 words)."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def philox_block(seed, m, spin, p0, count):
    lib = _load()
    out = np.zeros((count, 4), dtype=np.uint32)
    lib.orc_philox_block(seed, m, spin, p0, count, _p(out))
    return out


def normals(N, seed, m):
    """xi_ij,s for i < j (upper triangle; zero elsewhere), shape [2, N, N]."""
    lib = _load()
    out = np.zeros((2, N, N), dtype=np.complex128)
    lib.orc_normals(N, seed, m, _p(out))
    return out


def sample(N, n_up, n_dn, seed, m):
    """One initial sample rho(0) of Eq. 7, shape [2, N, N] complex."""
    lib = _load()
    nu = np.ascontiguousarray(n_up, dtype=np.float64)
    nd = np.ascontiguousarray(n_dn, dtype=np.float64)
    out = np.zeros((2, N, N), dtype=np.complex128)
    lib.orc_sample(N, _p(nu), _p(nd), seed, m, _p(out))
    return out


def sample_general(N, lam, V, seed, m):
    """One initial sample of a general state n_s = V_s diag(lam_s) V_s^dagger
    (App. A covariance, Eq. 7 in the diagonalising basis): rho~ drawn by Eq. 7
    with the eigen-occupations lam (same counters as :func:`sample`), then
    rho_s = V_s rho~_s V_s^dagger.  lam [2, N], V [2, N, N]; shape [2, N, N]."""
    rt = sample(N, lam[0], lam[1], seed, m)
    V = np.asarray(V, dtype=np.complex128)
    return np.stack([V[s] @ rt[s] @ V[s].conj().T for s in range(2)])


def rhs(lat, U, rho, t_bond=None):
    """Right-hand side of Eq. 6 for a state [2, N, N]."""
    lib = _load()
    b, t = _lat_arrays(lat, t_bond)
    r = np.ascontiguousarray(rho, dtype=np.complex128)
    out = np.zeros_like(r)
    lib.orc_rhs(lat.n_sites, lat.n_bonds, _p(b), _p(t), U, _p(r), _p(out))
    return out


def evolve(lat, U, rho0, dt, n_steps, out_every=0, t_bond=None, drive=None, t_start=0.0, u=None):
    """RK4-integrate one state; returns (rho(T), snapshots [n_out, 2N] or None).

    drive: optional time-dependent on-site potential v_i,s(t) = amp[s][i] f(t),
    f(t) = exp(-(t - t0)^2 / (2 sigma^2)) cos(omega (t - t0) + phase), given as
    dict(amp=[2, N], t0=, sigma=, omega=, phase=) (amp may be None), optionally
    with hop=dict(eps=, t0=, sigma=, omega=, phase=): every hopping scaled by
    m(t) = 1 + eps g(t), g the same pulse shape; t_start is the time of rho0.
    u: optional symmetric interaction matrix [N, N] of Eq. 1 (replaces U)."""
    lib = _load()
    b, t = _lat_arrays(lat, t_bond)
    r = np.array(rho0, dtype=np.complex128, order="C", copy=True)
    snap = None
    if out_every > 0:
        snap = np.zeros((n_steps // out_every + 1, 2 * lat.n_sites))
    if u is not None:
        if drive is not None:
            raise ValueError("the oracle integrates a drive or a long-range u, not both")
        um = np.ascontiguousarray(u, dtype=np.float64).reshape(lat.n_sites, lat.n_sites)
        lib.orc_evolve_longrange(lat.n_sites, lat.n_bonds, _p(b), _p(t), _p(um), dt, n_steps, out_every, _p(r),
                                 _p(snap))
    elif drive is None:
        lib.orc_evolve(lat.n_sites, lat.n_bonds, _p(b), _p(t), U, dt, n_steps, out_every, _p(r), _p(snap))
    else:
        amp = drive.get("amp")
        amp = None if amp is None else np.ascontiguousarray(amp, dtype=np.float64).reshape(2, lat.n_sites)
        hop = drive.get("hop") or {}
        lib.orc_evolve_drive(lat.n_sites, lat.n_bonds, _p(b), _p(t), U, dt, n_steps, out_every, _p(r), _p(snap),
                             _p(amp), float(t_start), float(drive.get("t0", 0.0)), float(drive.get("sigma", 0.0)),
                             float(drive.get("omega", 0.0)), float(drive.get("phase", 0.0)),
                             float(hop.get("eps", 0.0)), float(hop.get("t0", 0.0)), float(hop.get("sigma", 0.0)),
                             float(hop.get("omega", 0.0)), float(hop.get("phase", 0.0)))
    return r, snap


def run(lat, U, n_up, n_dn, seed, m0, M, dt, n_steps, out_every, t_bond=None,
        want_final=False, threads=0):
    """Sample + integrate trajectories m0..m0+M-1.

    Returns (snap [n_out, M, 2N], rho_final [M, 2, N, N] or None)."""
    lib = _load()
    b, t = _lat_arrays(lat, t_bond)
    N = lat.n_sites
    nu = np.ascontiguousarray(n_up, dtype=np.float64)
    nd = np.ascontiguousarray(n_dn, dtype=np.float64)
    n_out = n_steps // out_every + 1
    snap = np.zeros((n_out, M, 2 * N))
    fin = np.zeros((M, 2, N, N), dtype=np.complex128) if want_final else None
    lib.orc_run(N, lat.n_bonds, _p(b), _p(t), U, _p(nu), _p(nd), seed, m0, M, dt, n_steps,
                out_every, _p(snap), _p(fin), threads)
    return snap, fin


def energy(lat, U, rho, t_bond=None):
    """Classical energy H_W of Eq. A10 (complex; the imaginary part is 0)."""
    lib = _load()
    b, t = _lat_arrays(lat, t_bond)
    r = np.ascontiguousarray(rho, dtype=np.complex128)
    out = np.zeros(2)
    lib.orc_energy(lat.n_sites, lat.n_bonds, _p(b), _p(t), U, _p(r), _p(out))
    return complex(out[0], out[1])


def moments(X, want_g2=True):
    """Estimators from diagonal snapshots X [T, M, K]: (occ, conn, g2)."""
    lib = _load()
    X = np.ascontiguousarray(X, dtype=np.float64)
    T, M, K = X.shape
    occ = np.zeros((T, K))
    conn = np.zeros((T, K, K))
    g2 = np.zeros((T, K, K)) if want_g2 else None
    lib.orc_moments(T, M, K, _p(X), _p(occ), _p(conn), _p(g2))
    return occ, conn, g2


def max_threads():
    return int(_load().orc_max_threads())


def occupation_loss(lat, U, n_up, n_dn, seed, M, dt, n_steps, out_every, target, t_bond=None):
    """L = sum_t sum_{i,s} (<n_is>(t) - target[t, s*N+i])^2 over output rows 1..T
    (row 0, the initial state, is excluded)."""
    snap, _ = run(lat, U, n_up, n_dn, seed, 0, M, dt, n_steps, out_every, t_bond=t_bond)
    occ = snap.mean(axis=1) + 0.5
    return float(((occ[1:] - target) ** 2).sum())


def correlation_loss(lat, U, n_up, n_dn, seed, M, dt, n_steps, out_every, weight, t_bond=None):
    """L = sum_t sum_kl weight[t, k, l] C_kl(t) over all output rows (the
    connected correlator of Eq. 5 from this oracle's moments)."""
    snap, _ = run(lat, U, n_up, n_dn, seed, 0, M, dt, n_steps, out_every, t_bond=t_bond)
    _, conn, _ = moments(snap, want_g2=False)
    return float((weight * conn).sum())


def fd_gradient_corr(lat, U, n_up, n_dn, seed, M, dt, n_steps, out_every, weight, which, h=1e-5):
    """Central finite differences of :func:`correlation_loss` (common random
    numbers); ``which`` as in :func:`fd_gradient`."""
    out = []
    for w in which:
        def L(delta):
            tb = np.array(lat.t_bond, dtype=np.float64)
            u, nu, nd = U, np.array(n_up, dtype=np.float64), np.array(n_dn, dtype=np.float64)
            if w[0] == "U":
                u = U + delta
            elif w[0] == "t":
                tb[w[1]] += delta
            else:
                (nu if w[1] == 0 else nd)[w[2]] += delta
            return correlation_loss(lat, u, nu, nd, seed, M, dt, n_steps, out_every, weight, t_bond=tb)
        out.append((L(h) - L(-h)) / (2 * h))
    return np.array(out)


def fd_gradient(lat, U, n_up, n_dn, seed, M, dt, n_steps, out_every, target, which, h=1e-5):
    """Central finite differences of :func:`occupation_loss` with common random
    numbers (same seed).  ``which`` is a list of ("U",), ("t", b) or ("n", s, i)."""
    out = []
    for w in which:
        def L(delta):
            tb = np.array(lat.t_bond, dtype=np.float64)
            u, nu, nd = U, np.array(n_up, dtype=np.float64), np.array(n_dn, dtype=np.float64)
            if w[0] == "U":
                u = U + delta
            elif w[0] == "t":
                tb[w[1]] += delta
            else:
                (nu if w[1] == 0 else nd)[w[2]] += delta
            return occupation_loss(lat, u, nu, nd, seed, M, dt, n_steps, out_every, target, t_bond=tb)
        out.append((L(h) - L(-h)) / (2 * h))
    return np.array(out)
