"""GB300 (sm_103a) fTWA hot path: Python binding of the libftwa C ABI.

fermionic truncated Wigner approximation for the Fermi-Hubbard model of
arXiv:2212.04352: Gaussian Wigner samples of a diagonal state (Eq. 7),
RK4 integration of the fTWA equation of motion (Eq. 6) and sample-mean
estimators (Eqs. 5 and 10), each a hand-written CUDA kernel behind
include/ftwa.h.  This module only marshals arguments: device buffers are
torch CUDA tensors, passed to the library as raw pointers on torch's current
stream.  There is no CPU fallback; a missing libftwa.so raises.
"""

from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (  # noqa: F401
    FTWA_FP32, FTWA_FP64, FTWA_GRAM_BF16X3, FTWA_GRAM_FP64, FtwaError, check, load,
)

__all__ = ["Plan", "Batch", "ED", "plan", "philox", "measure_peak", "moments_noalloc", "occupations",
           "correlations",
           "FTWAFunction", "FTWACorrFunction", "FTWA_FP32",
           "FTWA_FP64", "FTWA_GRAM_FP64", "FTWA_GRAM_BF16X3", "FtwaError", "load"]


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Plan:
    """Owner of one ftwa_plan_t (lattice tables, launch shape, status word)."""

    def __init__(self, lattice, U, t=1.0, filling=0.0, n_up=None, n_dn=None, precision=FTWA_FP64,
                 dt=0.01, out_every=10, cluster=0, timeout_us=0, variant=0, threads=0):
        lib = load()
        self.N = int(lattice.n_sites)
        self.n_bonds = int(lattice.n_bonds)
        self._bonds = np.ascontiguousarray(lattice.bonds, dtype=np.int32)
        tb = getattr(lattice, "t_bond", None)
        self._t = None if tb is None else np.ascontiguousarray(tb, dtype=np.float64)
        lat = _lib.Lattice(self.N, self.n_bonds, self._bonds.ctypes.data,
                           None if self._t is None else self._t.ctypes.data)
        init = None
        if n_up is not None:
            self._nu = np.ascontiguousarray(n_up, dtype=np.float64)
            self._nd = np.ascontiguousarray(n_dn, dtype=np.float64)
            init = _lib.InitState(self._nu.ctypes.data, self._nd.ctypes.data)
        opts = _lib.Options(int(precision), float(dt), int(out_every), int(cluster), int(threads), 0, int(timeout_us),
                            int(variant))
        h = ctypes.c_void_p()
        check(lib.ftwa_plan(ctypes.byref(lat), float(U), float(t), float(filling),
                            None if init is None else ctypes.byref(init), ctypes.byref(opts), ctypes.byref(h)),
              "ftwa_plan")
        self._h = h
        self.U = float(U)
        self.precision = int(precision)
        self.dt = float(dt)
        self.out_every = int(out_every)

    # -- lifetime --------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            load().ftwa_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- helpers ---------------------------------------------------------------
    @property
    def real_dtype(self):
        import torch
        return torch.float64 if self.precision == FTWA_FP64 else torch.float32

    @property
    def complex_dtype(self):
        import torch
        return torch.complex128 if self.precision == FTWA_FP64 else torch.complex64

    def info(self):
        inf = _lib.PlanInfo()
        check(load().ftwa_get_info(self._h, ctypes.byref(inf)), "ftwa_get_info")
        return {n: getattr(inf, n) for n, _ in _lib.PlanInfo._fields_}

    def new_state(self, M, device="cuda"):
        import torch
        return torch.empty((M, 2, self.N, self.N), dtype=self.complex_dtype, device=device)

    def n_out(self, n_steps):
        return n_steps // self.out_every + 1

    # -- entry points ----------------------------------------------------------
    def sample(self, seed, M, first_sample=0, out=None, stream=None):
        rho = self.new_state(M) if out is None else out
        check(load().ftwa_sample(self._h, int(seed), int(first_sample), int(M), _ptr(rho), _stream(stream)),
              "ftwa_sample")
        return rho

    def set_initial_basis(self, lam, V):
        """General initial state n_s = V_s diag(lam_s) V_s^dagger (lam [2, N] in
        [0, 1], V [2, N, N] unitary, columns = eigenvectors); None, None returns
        to the diagonal state of the plan's occupations."""
        import numpy as np
        if lam is None:
            check(load().ftwa_set_initial_basis(self._h, None, None, None), "ftwa_set_initial_basis")
            return
        lam = np.ascontiguousarray(lam, dtype=np.float64).reshape(2, self.N)
        V = np.asarray(V).reshape(2, self.N, self.N)
        vr = np.ascontiguousarray(V.real, dtype=np.float64)
        vi = np.ascontiguousarray(V.imag, dtype=np.float64) if np.iscomplexobj(V) else None
        check(load().ftwa_set_initial_basis(self._h, ctypes.c_void_p(lam.ctypes.data), ctypes.c_void_p(vr.ctypes.data),
                                            None if vi is None else ctypes.c_void_p(vi.ctypes.data)),
              "ftwa_set_initial_basis")

    def set_drive(self, amp, t0=0.0, sigma=0.0, omega=0.0, phase=0.0):
        """Time-dependent on-site drive v_i,s(t) = amp[s][i] f(t) with
        f(t) = exp(-(t - t0)^2 / (2 sigma^2)) cos(omega (t - t0) + phase);
        amp None removes it."""
        import numpy as np
        if amp is None:
            check(load().ftwa_set_drive(self._h, None, 0.0, 0.0, 0.0, 0.0), "ftwa_set_drive")
            return
        a = np.ascontiguousarray(amp, dtype=np.float64).reshape(2, self.N)
        check(load().ftwa_set_drive(self._h, ctypes.c_void_p(a.ctypes.data), float(t0), float(sigma), float(omega),
                                    float(phase)), "ftwa_set_drive")

    def set_hopping_drive(self, eps, t0=0.0, sigma=0.0, omega=0.0, phase=0.0):
        """Scale every hopping by m(t) = 1 + eps g(t), g the pulse shape of
        set_drive; eps = 0 removes it."""
        check(load().ftwa_set_hopping_drive(self._h, float(eps), float(t0), float(sigma), float(omega), float(phase)),
              "ftwa_set_hopping_drive")

    def set_interaction(self, u):
        """Long-range interaction u [N, N] (symmetric, u_ii = on-site term) of
        Eq. 1 in place of U; None returns to the on-site U."""
        import numpy as np
        if u is None:
            check(load().ftwa_set_interaction(self._h, None), "ftwa_set_interaction")
            return
        a = np.ascontiguousarray(u, dtype=np.float64).reshape(self.N, self.N)
        check(load().ftwa_set_interaction(self._h, ctypes.c_void_p(a.ctypes.data)), "ftwa_set_interaction")

    def evolve(self, rho, n_steps, snap=True, stream=None, t_start=None):
        """Advance rho in place (from time t_start, default 0); returns
        snapshots [n_out, M, 2N] (or None)."""
        import torch
        M = rho.shape[0]
        X = None
        if snap is True:
            X = torch.empty((self.n_out(n_steps), M, 2 * self.N), dtype=self.real_dtype, device=rho.device)
        elif snap is not None and snap is not False:
            X = snap
        if t_start is None:
            check(load().ftwa_evolve(self._h, _ptr(rho), int(M), int(n_steps), _ptr(X), _stream(stream)),
                  "ftwa_evolve")
        else:
            check(load().ftwa_evolve_at(self._h, _ptr(rho), int(M), int(n_steps), float(t_start), _ptr(X),
                                        _stream(stream)), "ftwa_evolve_at")
        return X

    def moments(self, X, gram_mode=FTWA_GRAM_FP64, g2=True, stream=None):
        """(occ [T, 2N], conn [T, 2N, 2N], g2 [T, 2N, 2N] or None), float64."""
        import torch
        T, M, K = X.shape
        occ = torch.empty((T, K), dtype=torch.float64, device=X.device)
        conn = torch.empty((T, K, K), dtype=torch.float64, device=X.device)
        g = torch.empty((T, K, K), dtype=torch.float64, device=X.device) if g2 else None
        check(load().ftwa_moments(self._h, _ptr(X), int(M), int(T), _ptr(occ), _ptr(conn), _ptr(g),
                                  int(gram_mode), _stream(stream)), "ftwa_moments")
        return occ, conn, g

    def adjoint(self, seed, M, n_steps, ckpt_every, dL_docc, dL_dconn=None, occ=None, stream=None):
        """(dL/dU [1], dL/dt_b [n_bonds], dL/dn0 [2, N]), float64 device tensors.

        dL_docc [T+1, 2N] (or None with dL_dconn) is dL/d<n>; dL_dconn
        [T+1, 2N, 2N] is dL/dC of the connected correlator and needs the
        forward occupations ``occ`` [T+1, 2N] of the same samples."""
        import torch
        T1, K = int(n_steps) // self.out_every + 1, 2 * self.N
        ref = dL_docc if dL_docc is not None else dL_dconn
        if ref is None:
            raise ValueError("give dL_docc, dL_dconn or both")
        for name, t, shape in (("dL_docc", dL_docc, (T1, K)), ("dL_dconn", dL_dconn, (T1, K, K)),
                               ("occ", occ, (T1, K))):
            if t is None:
                continue
            if tuple(t.shape) != shape:
                raise ValueError(f"{name} must be {shape} (n_steps/out_every + 1 rows), got {tuple(t.shape)}")
            if not t.is_cuda:
                raise ValueError(f"{name} must be a CUDA tensor")
        if dL_dconn is not None and occ is None:
            raise ValueError("dL_dconn needs the forward occupations occ")
        dev = ref.device
        gU = torch.zeros(1, dtype=torch.float64, device=dev)
        gt = torch.zeros(self.n_bonds, dtype=torch.float64, device=dev)
        gn = torch.zeros((2, self.N), dtype=torch.float64, device=dev)
        dl = None if dL_docc is None else dL_docc.contiguous().to(torch.float64)
        if dL_dconn is None:
            check(load().ftwa_adjoint(self._h, int(seed), int(M), int(n_steps), int(ckpt_every), _ptr(dl), _ptr(gU),
                                      _ptr(gt), _ptr(gn), _stream(stream)), "ftwa_adjoint")
        else:
            dc = dL_dconn.contiguous().to(torch.float64)
            oc = occ.contiguous().to(torch.float64)
            check(load().ftwa_adjoint_corr(self._h, int(seed), int(M), int(n_steps), int(ckpt_every), _ptr(dl),
                                           _ptr(dc), _ptr(oc), _ptr(gU), _ptr(gt), _ptr(gn), _stream(stream)),
                  "ftwa_adjoint_corr")
        return gU, gt, gn

    def autotune(self, M, probe_steps=20, stream=None):
        """Time every feasible stepper shape and pin the fastest (synchronous)."""
        check(load().ftwa_autotune(self._h, int(M), int(probe_steps), _stream(stream)), "ftwa_autotune")
        return self.info()

    def status(self, stream=None):
        """Synchronise the stream and return (and clear) the device status word."""
        return int(load().ftwa_status(self._h, _stream(stream)))

    def debug_force_timeout(self, armed=True):
        check(load().ftwa_debug_force_timeout(self._h, 1 if armed else 0), "ftwa_debug_force_timeout")


def plan(lattice, U, **kw) -> Plan:
    return Plan(lattice, U, **kw)


class _Bonds:
    """Lattice view (sites, bonds, per-bond hopping) handed to ftwa_plan."""

    def __init__(self, n_sites, bonds, t_bond):
        self.n_sites = int(n_sites)
        self.bonds = np.ascontiguousarray(bonds, dtype=np.int32)
        self.t_bond = np.ascontiguousarray(t_bond, dtype=np.float64)
        self.n_bonds = int(self.bonds.shape[0])


def _default_ckpt(n_steps, out_every):
    """Checkpoint spacing for the adjoint: the multiple of out_every dividing
    n_steps that is closest to sqrt(n_steps) (memory ~ n_steps/c + c)."""
    cands = [c for c in range(out_every, n_steps + 1, out_every) if n_steps % c == 0]
    if not cands:
        return out_every
    return min(cands, key=lambda c: abs(c - n_steps ** 0.5))


_OCC_FN = None


def _occupation_function():
    global _OCC_FN
    if _OCC_FN is not None:
        return _OCC_FN
    import torch

    class FTWAFunction(torch.autograd.Function):
        """Forward: Eq. 7 samples -> RK4 of Eq. 6 -> FP64 sample means (Eq. 5)
        of the occupations, all in libftwa.  Backward: the discrete RK4
        adjoint (ftwa_adjoint) of the same samples (same seed, regenerated
        on the device), given dL/d<n> from autograd."""

        @staticmethod
        def forward(ctx, U, t_bond, n0, bonds, seed, M, n_steps, precision, dt, out_every, ckpt_every):
            n0h = n0.detach().to("cpu", torch.float64).numpy()
            lat = _Bonds(n0h.shape[1], bonds, t_bond.detach().to("cpu", torch.float64).numpy())
            P = Plan(lat, float(U.detach()), n_up=n0h[0], n_dn=n0h[1], precision=precision, dt=dt,
                     out_every=out_every)
            try:
                rho = P.sample(seed, M)
                X = P.evolve(rho, n_steps)
                del rho
                occ = P.moments(X, g2=False)[0]
                st = P.status()
                if st != 0:
                    raise FtwaError(st, "ftwa_evolve", "device status word set (timeout)")
            except BaseException:
                P.close()
                raise
            ctx.plan = P
            ctx.args = (seed, M, n_steps, ckpt_every)
            ctx.like = [(x.shape, x.device, x.dtype) for x in (U, t_bond, n0)]
            return occ

        @staticmethod
        def backward(ctx, g):
            P = ctx.plan
            seed, M, n_steps, ckpt_every = ctx.args
            gU, gt, gn = P.adjoint(seed, M, n_steps, ckpt_every, g.contiguous())
            st = P.status()
            if st != 0:
                raise FtwaError(st, "ftwa_adjoint", "device status word set (timeout)")
            grads = [x.reshape(shape).to(dev, dt) for x, (shape, dev, dt) in zip((gU, gt, gn), ctx.like)]
            return (*grads, None, None, None, None, None, None, None, None)

    _OCC_FN = FTWAFunction
    return _OCC_FN


_CORR_FN = None


def _correlation_function():
    global _CORR_FN
    if _CORR_FN is not None:
        return _CORR_FN
    import torch

    class FTWACorrFunction(torch.autograd.Function):
        """Forward: Eq. 7 samples -> RK4 of Eq. 6 -> FP64 estimators of Eq. 5
        (occupations and the connected correlator), all in libftwa.
        Backward: the discrete RK4 adjoint (ftwa_adjoint_corr) of the same
        samples, given dL/d<n> and dL/dC from autograd."""

        @staticmethod
        def forward(ctx, U, t_bond, n0, bonds, seed, M, n_steps, precision, dt, out_every, ckpt_every):
            n0h = n0.detach().to("cpu", torch.float64).numpy()
            lat = _Bonds(n0h.shape[1], bonds, t_bond.detach().to("cpu", torch.float64).numpy())
            P = Plan(lat, float(U.detach()), n_up=n0h[0], n_dn=n0h[1], precision=precision, dt=dt,
                     out_every=out_every)
            try:
                rho = P.sample(seed, M)
                X = P.evolve(rho, n_steps)
                del rho
                occ, conn, _ = P.moments(X, g2=False)
                st = P.status()
                if st != 0:
                    raise FtwaError(st, "ftwa_evolve", "device status word set (timeout)")
            except BaseException:
                P.close()
                raise
            ctx.plan = P
            ctx.args = (seed, M, n_steps, ckpt_every)
            ctx.occ = occ
            ctx.like = [(x.shape, x.device, x.dtype) for x in (U, t_bond, n0)]
            return occ, conn

        @staticmethod
        def backward(ctx, g_occ, g_conn):
            P = ctx.plan
            seed, M, n_steps, ckpt_every = ctx.args
            g_occ = torch.zeros_like(ctx.occ) if g_occ is None else g_occ.contiguous()
            if g_conn is None:
                gU, gt, gn = P.adjoint(seed, M, n_steps, ckpt_every, g_occ)
            else:
                gU, gt, gn = P.adjoint(seed, M, n_steps, ckpt_every, g_occ, dL_dconn=g_conn.contiguous(),
                                       occ=ctx.occ)
            st = P.status()
            if st != 0:
                raise FtwaError(st, "ftwa_adjoint_corr", "device status word set (timeout)")
            grads = [x.reshape(shape).to(dev, dt) for x, (shape, dev, dt) in zip((gU, gt, gn), ctx.like)]
            return (*grads, None, None, None, None, None, None, None, None)

    _CORR_FN = FTWACorrFunction
    return _CORR_FN


def __getattr__(name):
    # FTWAFunction / FTWACorrFunction: the autograd.Functions behind
    # occupations() and correlations(), created on first use so that
    # importing the package does not import torch.
    if name == "FTWAFunction":
        return _occupation_function()
    if name == "FTWACorrFunction":
        return _correlation_function()
    raise AttributeError(name)


def occupations(lattice, U, t_bond, n0, seed, M, n_steps, precision=FTWA_FP64, dt=0.01, out_every=10,
                ckpt_every=None):
    """Differentiable fTWA occupations <n_k>(t) (Eq. 5 estimator of Re rho_kk
    + 1/2 over samples m = 0 .. M-1 of ``seed``), [n_steps/out_every + 1, 2N]
    float64 on the device, k = s*N + i.

    U (0-dim), t_bond ([n_bonds], the lattice's bond order) and n0 ([2, N]
    initial occupations) are torch tensors; those with requires_grad receive
    dL/dU, dL/dt_b, dL/dn0 from the RK4 adjoint on backward (exact for the
    integrated samples, common random numbers).  The lattice supplies only
    the sites and bonds.  ckpt_every must divide n_steps and be a multiple of
    out_every (default: near sqrt(n_steps)).  Each call builds a plan for the
    given values; the plan is released with the autograd graph (backward may
    run more than once with retain_graph)."""
    import torch
    if ckpt_every is None:
        ckpt_every = _default_ckpt(int(n_steps), int(out_every))
    U = torch.as_tensor(U, dtype=torch.float64)
    t_bond = torch.as_tensor(t_bond, dtype=torch.float64)
    n0 = torch.as_tensor(n0, dtype=torch.float64)
    return _occupation_function().apply(U, t_bond, n0, np.asarray(lattice.bonds), int(seed), int(M), int(n_steps),
                                        int(precision), float(dt), int(out_every), int(ckpt_every))


def correlations(lattice, U, t_bond, n0, seed, M, n_steps, precision=FTWA_FP64, dt=0.01, out_every=10,
                 ckpt_every=None):
    """Differentiable fTWA estimators of Eq. 5: (occ, conn), the occupations
    <n_k>(t) [n_steps/out_every + 1, 2N] and the connected correlator
    C_kl(t) = <n_k n_l> - <n_k><n_l> [.., 2N, 2N] over samples m = 0 .. M-1
    of ``seed`` (float64, on the device).  Losses of <n_k n_l> = C + <n_k><n_l>
    or of g2 (Eq. 10) are differentiable through these two outputs.
    Arguments and gradients as for :func:`occupations`."""
    import torch
    if ckpt_every is None:
        ckpt_every = _default_ckpt(int(n_steps), int(out_every))
    U = torch.as_tensor(U, dtype=torch.float64)
    t_bond = torch.as_tensor(t_bond, dtype=torch.float64)
    n0 = torch.as_tensor(n0, dtype=torch.float64)
    return _correlation_function().apply(U, t_bond, n0, np.asarray(lattice.bonds), int(seed), int(M), int(n_steps),
                                         int(precision), float(dt), int(out_every), int(ckpt_every))


class ED:
    """Exact diagonalisation on the GPU (ftwa_ed_*): the Hubbard model of a
    small lattice with fixed N_up, N_dn, propagated from a Fock state."""

    def __init__(self, lattice, U, n_up, n_dn):
        import numpy as np
        self.N = lattice.n_sites
        bonds = np.ascontiguousarray(lattice.bonds, dtype=np.int32)
        tb = np.ascontiguousarray(lattice.t_bond, dtype=np.float64)
        self._keep = (bonds, tb)
        lat = _lib.Lattice(self.N, int(bonds.shape[0]), ctypes.c_void_p(bonds.ctypes.data),
                           ctypes.c_void_p(tb.ctypes.data))
        h = ctypes.c_void_p()
        check(load().ftwa_ed_plan(ctypes.byref(lat), float(U), int(n_up), int(n_dn), ctypes.byref(h)), "ftwa_ed_plan")
        self._h = h

    def info(self):
        """(basis size, a, b) with H~ = (H - b) / a the Chebyshev map."""
        d, a, b = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        check(load().ftwa_ed_info(self._h, ctypes.byref(d), ctypes.cast(ctypes.byref(a), ctypes.c_void_p),
                                  ctypes.cast(ctypes.byref(b), ctypes.c_void_p)), "ftwa_ed_info")
        return d.value, a.value, b.value

    def evolve(self, n_up, n_dn, dt_out, n_out, nn=True, stream=None):
        """(occ [n_out+1, 2N], nn [n_out+1, 2N, 2N] or None), float64 device tensors."""
        import numpy as np
        import torch
        nu = np.ascontiguousarray(n_up, dtype=np.float64)
        nd = np.ascontiguousarray(n_dn, dtype=np.float64)
        K = 2 * self.N
        occ = torch.empty((n_out + 1, K), dtype=torch.float64, device="cuda")
        mm = torch.empty((n_out + 1, K, K), dtype=torch.float64, device="cuda") if nn else None
        check(load().ftwa_ed_evolve(self._h, ctypes.c_void_p(nu.ctypes.data), ctypes.c_void_p(nd.ctypes.data),
                                    float(dt_out), int(n_out), _ptr(occ), _ptr(mm), _stream(stream)), "ftwa_ed_evolve")
        return occ, mm

    def close(self):
        if self._h:
            load().ftwa_ed_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """One CUDA graph advancing several plans' samples (ftwa_batch_*).

    persistent=False: the graph's branches are the plans' own persistent
    steppers (ftwa_batch_create).  persistent=True: one persistent kernel
    drawing (problem, sample batch) items from a cost-ordered queue
    (ftwa_batch_create_persistent; FP32 plans); tune=True times the cluster
    and CTA sizes on a probe first."""

    def __init__(self, plans, rhos, n_steps, snaps=None, persistent=False, tune=False):
        n = len(plans)
        self._plans = list(plans)          # keep the plans and buffers alive
        self._rhos = list(rhos)
        self._snaps = list(snaps) if snaps is not None else None
        P = ctypes.c_void_p
        hp = (P * n)(*[pl._h for pl in plans])
        hr = (P * n)(*[r.data_ptr() for r in rhos])
        hm = (ctypes.c_int64 * n)(*[r.shape[0] for r in rhos])
        hs = None
        if snaps is not None:
            hs = (P * n)(*[0 if x is None else x.data_ptr() for x in snaps])
        h = P()
        if persistent:
            check(load().ftwa_batch_create_persistent(hp, n, hr, hm, int(n_steps), hs, 1 if tune else 0,
                                                      ctypes.byref(h)), "ftwa_batch_create_persistent")
        else:
            check(load().ftwa_batch_create(hp, n, hr, hm, int(n_steps), hs, ctypes.byref(h)), "ftwa_batch_create")
        self._h = h

    def launch(self, stream=None):
        check(load().ftwa_batch_launch(self._h, _stream(stream)), "ftwa_batch_launch")

    def close(self):
        if getattr(self, "_h", None):
            load().ftwa_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def moments_noalloc(X, precision, n_sites, g2=True, stream=None, out=None):
    """ftwa_moments_noalloc: FP64 estimators without any allocation inside the
    library (for callers that cannot call cudaMalloc).  X is [T, M, 2N] of the
    given precision; ``out`` = (occ, conn, g2-or-None) preallocated float64
    tensors, or None to have them allocated here by torch."""
    import torch
    if X.dim() != 3:
        raise ValueError(f"X must be [T, M, 2N], got shape {tuple(X.shape)}")
    T, M, K = X.shape
    want = torch.float64 if int(precision) == FTWA_FP64 else torch.float32
    if int(precision) not in (FTWA_FP64, FTWA_FP32):
        raise ValueError(f"precision must be FTWA_FP64 or FTWA_FP32, got {precision}")
    if K != 2 * int(n_sites):
        raise ValueError(f"X has {K} columns, expected 2 * n_sites = {2 * int(n_sites)}")
    if X.dtype != want:
        raise ValueError(f"X is {X.dtype}, precision {precision} needs {want}")
    if not X.is_cuda or not X.is_contiguous():
        raise ValueError("X must be a contiguous CUDA tensor")
    if out is None:
        occ = torch.empty((T, K), dtype=torch.float64, device=X.device)
        conn = torch.empty((T, K, K), dtype=torch.float64, device=X.device)
        g = torch.empty((T, K, K), dtype=torch.float64, device=X.device) if g2 else None
    else:
        occ, conn, g = out
        for name, t, shape in (("occ", occ, (T, K)), ("conn", conn, (T, K, K)), ("g2", g, (T, K, K))):
            if t is None and name != "g2":
                raise ValueError(f"{name} output is required")
            if t is None:
                continue
            if tuple(t.shape) != shape or t.dtype != torch.float64 or not t.is_contiguous() \
                    or t.device != X.device:
                raise ValueError(f"{name} output must be a contiguous float64 tensor {shape} on {X.device}")
    check(load().ftwa_moments_noalloc(_ptr(X), int(precision), int(n_sites), int(M), int(T), _ptr(occ), _ptr(conn),
                                      _ptr(g), _stream(stream)), "ftwa_moments_noalloc")
    return occ, conn, g


def measure_peak(kind, stream=None):
    """On-chip peak of the current device (ftwa_measure_peak): "fp32" / "fp32x2"
    (FMA flop/s, scalar / packed pairs), "fp64" (FMA flop/s) or "smem"
    (shared-memory load bytes/s)."""
    k = {"fp32": 0, "fp64": 1, "smem": 2, "fp32x2": 3}[kind]
    v = ctypes.c_double()
    check(load().ftwa_measure_peak(k, ctypes.byref(v), _stream(stream)), "ftwa_measure_peak")
    return v.value


def philox(seed, m, spin, p0, count, stream=None):
    """Raw Philox4x32-10 words [count, 4] (uint32 as int64 tensor on the device)."""
    import torch
    out = torch.empty((count, 4), dtype=torch.int32, device="cuda")
    check(load().ftwa_philox(int(seed), int(m), int(spin), int(p0), int(count), _ptr(out), _stream(stream)),
          "ftwa_philox")
    return out.to(torch.int64) & 0xFFFFFFFF
