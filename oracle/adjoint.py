"""Discrete adjoint of the RK4 integration of Eq. 6 (TEST INFRASTRUCTURE ONLY).

Plain FP64 numpy on full N x N matrices, written from Eq. 6, Eq. 7 and the
RK4 recursion; it shares nothing with the CUDA library and does not use its
reductions (every derivative below is taken from its definition).  The loss
is given through its gradient with respect to the occupations,
g[t, s*N + i] = dL/d<n_is>(t) at the output rows t = 0 .. n_steps/out_every,
with <n_is>(t) = (1/M) sum_m Re rho^m_ii,s(t) + 1/2 (Eq. 5); the result is
dL/dU, dL/dt_b (the lattice's bond order) and dL/dn_is for the samples
m = 0 .. M-1 of ``seed`` drawn by Eq. 7.

Inner product <A, B> = Re tr(A^dagger B), summed over the two spins.
  f_s(rho) = i [h_s, rho_s],  h_s = -J + U diag(Re rho_kk,sbar + 1/2)   (Eq. 6)
  VJP of f at Y for a cotangent v:
    w_s = -i [h_s, v_s]                               (h frozen at Y)
        + diag_k U Re( i ((Y_sbar v_sbar^dagger)_kk - (v_sbar^dagger Y_sbar)_kk) )
          (the dependence of h_sbar on Re rho_kk,s)
  dL/dU   gets <v_s, i [diag(Re Y_kk,sbar + 1/2), Y_s]>
  dL/dt_b gets <v_s, -i [E_b, Y_s]>,  E_b = e_x e_y^T + e_y e_x^T, b = (x, y)
RK4 with stages Y1 = y, Y2 = y + h/2 k1, Y3 = y + h/2 k2, Y4 = y + h k3 and
y' = y + h/6 (k1 + 2 k2 + 2 k3 + k4), reversed for the cotangent l of y':
  kbar4 = h/6 l;             Ybar4 = VJP(Y4)[kbar4]
  kbar3 = h/3 l + h Ybar4;   Ybar3 = VJP(Y3)[kbar3]
  kbar2 = h/3 l + h/2 Ybar3; Ybar2 = VJP(Y2)[kbar2]
  kbar1 = h/6 l + h/2 Ybar2; Ybar1 = VJP(Y1)[kbar1]
  l_n = l + Ybar1 + Ybar2 + Ybar3 + Ybar4
and every stage adds <kbar_s, df/dtheta (Y_s)> to the parameter gradients.
Eq. 7: rho_ii(0) = n_i - 1/2, rho_ij(0) = xi_ij s_ij for i < j and
rho_ji = conj(rho_ij), s_ij = sqrt((n_i + n_j - 2 n_i n_j)/2), so
ds_ij/dn_i = (1 - 2 n_j) / (4 s_ij); pairs with s_ij = 0 are skipped (n -> s
is not differentiable there).

Correlation losses: with gC[t, k, l] = dL/dC_kl(t) for the connected
correlator of Eq. 5, C_kl = (1/M) sum_m x_mk x_ml - mu_k mu_l (x_mk =
Re rho^m_kk, mu = mean over samples), the derivative of C_kl with respect
to one sample's diagonal is (1/M)[delta_jk (x_ml - mu_l) + delta_jl
(x_mk - mu_k)], so sample m's cotangent gets
  (1/M) sum_l (gC_jl + gC_lj)(x_ml - mu_l)
on its diagonal entry j at every output step, mu being the mean over the M
samples at that step (given as ``mu``).

Parity: pinned by central finite differences of the C oracle's integration
(``tests/test_oracle_pins.py``).
"""

from __future__ import annotations

import numpy as np

from . import normals, sample


def hopping_matrix(lat, t_bond=None):
    """J with J_xy = J_yx = t_b for every bond b = (x, y) (Eq. 1)."""
    N = lat.n_sites
    t = np.asarray(lat.t_bond if t_bond is None else t_bond, dtype=np.float64)
    J = np.zeros((N, N))
    for b, (x, y) in enumerate(np.asarray(lat.bonds)):
        J[x, y] = J[y, x] = t[b]
    return J


def _h(J, U, Y, s):
    return -J + U * np.diag(Y[1 - s].diagonal().real + 0.5)


def f(J, U, Y):
    """Right-hand side of Eq. 6 for a state [2, N, N] (full matrices)."""
    out = np.empty_like(Y)
    for s in range(2):
        h = _h(J, U, Y, s)
        out[s] = 1j * (h @ Y[s] - Y[s] @ h)
    return out


def _inner(A, B):
    return float((np.conj(A) * B).real.sum())


def vjp(J, U, bonds, Y, v):
    """(w, dL/dU, dL/dt [n_bonds]) of one evaluation of f at Y for the cotangent v."""
    N = Y.shape[1]
    w = np.empty_like(Y)
    gU = 0.0
    gt = np.zeros(len(bonds))
    for s in range(2):
        h = _h(J, U, Y, s)
        w[s] = -1j * (h @ v[s] - v[s] @ h)
    for s in range(2):
        sb = 1 - s
        # h_sbar depends on Re rho_kk,s through U diag(...)
        c = U * (1j * (np.diag(Y[sb] @ v[sb].conj().T) - np.diag(v[sb].conj().T @ Y[sb]))).real
        w[s] += np.diag(c)
        D = np.diag(Y[sb].diagonal().real + 0.5)
        gU += _inner(v[s], 1j * (D @ Y[s] - Y[s] @ D))
        for b, (x, y) in enumerate(bonds):
            E = np.zeros((N, N))
            E[x, y] = E[y, x] = 1.0
            gt[b] += _inner(v[s], -1j * (E @ Y[s] - Y[s] @ E))
    return w, gU, gt


def adjoint(lat, U, n_up, n_dn, seed, M, dt, n_steps, out_every, g, t_bond=None, gC=None, mu=None):
    """(dL/dU, dL/dt [n_bonds], dL/dn [2, N]) for the linearised loss
    L = sum_t sum_k g[t, k] <n_k>(t) (+ sum_t sum_kl gC[t, k, l] C_kl(t) when
    gC is given, with mu[t, k] the sample means of Re rho_kk) over the
    samples 0 .. M-1 of ``seed``."""
    N = lat.n_sites
    J = hopping_matrix(lat, t_bond)
    bonds = [tuple(int(v) for v in b) for b in np.asarray(lat.bonds)]
    nocc = np.stack([np.asarray(n_up, dtype=np.float64), np.asarray(n_dn, dtype=np.float64)])
    g = np.asarray(g, dtype=np.float64)
    h = dt
    gU, gt, gn = 0.0, np.zeros(len(bonds)), np.zeros((2, N))
    for m in range(M):
        ys = [sample(N, nocc[0], nocc[1], seed, m)]
        for _ in range(n_steps):
            y = ys[-1]
            k1 = f(J, U, y)
            k2 = f(J, U, y + h / 2 * k1)
            k3 = f(J, U, y + h / 2 * k2)
            k4 = f(J, U, y + h * k3)
            ys.append(y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4))

        def inject(lam, step):
            if step % out_every == 0:
                row = g[step // out_every]
                if gC is not None:
                    t = step // out_every
                    x = np.concatenate([ys[step][0].diagonal().real, ys[step][1].diagonal().real])
                    row = row + (gC[t] + gC[t].T) @ (x - mu[t])
                for s in range(2):
                    lam[s] += np.diag(row[s * N:(s + 1) * N] / M)

        lam = np.zeros((2, N, N), dtype=np.complex128)
        inject(lam, n_steps)
        for n in range(n_steps - 1, -1, -1):
            y = ys[n]
            Y1 = y
            Y2 = y + h / 2 * f(J, U, Y1)
            Y3 = y + h / 2 * f(J, U, Y2)
            Y4 = y + h * f(J, U, Y3)
            kb = h / 6 * lam
            Yb4, a, b = vjp(J, U, bonds, Y4, kb)
            gU, gt = gU + a, gt + b
            kb = h / 3 * lam + h * Yb4
            Yb3, a, b = vjp(J, U, bonds, Y3, kb)
            gU, gt = gU + a, gt + b
            kb = h / 3 * lam + h / 2 * Yb3
            Yb2, a, b = vjp(J, U, bonds, Y2, kb)
            gU, gt = gU + a, gt + b
            kb = h / 6 * lam + h / 2 * Yb2
            Yb1, a, b = vjp(J, U, bonds, Y1, kb)
            gU, gt = gU + a, gt + b
            lam = lam + Yb1 + Yb2 + Yb3 + Yb4
            inject(lam, n)
        # Eq. 7: rho(0) as a function of the occupations
        xi = normals(N, seed, m)
        for s in range(2):
            n_s = nocc[s]
            gn[s] += lam[s].diagonal().real
            for a_ in range(N):
                for b_ in range(a_ + 1, N):
                    sab = np.sqrt(max(0.5 * (n_s[a_] + n_s[b_] - 2.0 * n_s[a_] * n_s[b_]), 0.0))
                    if sab == 0.0:
                        continue
                    # d rho_ab / d s = xi_ab, d rho_ba / d s = conj(xi_ab)
                    dL_ds = (np.conj(lam[s, a_, b_]) * xi[s, a_, b_]).real + \
                            (np.conj(lam[s, b_, a_]) * np.conj(xi[s, a_, b_])).real
                    gn[s, a_] += dL_ds * (1.0 - 2.0 * n_s[b_]) / (4.0 * sab)
                    gn[s, b_] += dL_ds * (1.0 - 2.0 * n_s[a_]) / (4.0 * sab)
    return gU, gt, gn
