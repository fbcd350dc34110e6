"""Closed forms that pin the oracle (TEST INFRASTRUCTURE ONLY).

Each function states a result fixed by the paper or by the mathematics of the
method, computed without the oracle's integrator.
"""

from __future__ import annotations

import math

import numpy as np


def hopping_matrix(lat, t_bond=None):
    """Dense real symmetric j_ij of Eq. 1 (both orders of every bond)."""
    tb = lat.t_bond if t_bond is None else t_bond
    J = np.zeros((lat.n_sites, lat.n_sites))
    for (i, j), t in zip(lat.bonds, tb):
        J[i, j] = J[j, i] = t
    return J


def rk4_free(lat, rho0, dt, n_steps):
    """U = 0: RK4 applied to the linear flow d rho/dt = i(rho J - J rho) in
    J's eigenbasis J = V diag(lam) V^T.  Each rotated entry rho~_ab evolves as
    d/dt rho~_ab = i(lam_b - lam_a) rho~_ab, and one RK4 step multiplies it by
    the Taylor polynomial T4(z) = 1 + z + z^2/2 + z^3/6 + z^4/24 of z =
    i(lam_b - lam_a) dt."""
    J = hopping_matrix(lat)
    lam, V = np.linalg.eigh(J)
    z = 1j * (lam[None, :] - lam[:, None]) * dt
    amp = (1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24) ** n_steps
    out = np.empty_like(rho0)
    for s in range(rho0.shape[0]):
        rt = V.T @ rho0[s] @ V
        out[s] = V @ (amp * rt) @ V.T
    return out


def exact_free(lat, rho0, t):
    """U = 0 exact flow: rho(t) = W rho0 W^dagger with W = exp(-iJt) = exp(iht),
    h = -J the one-body Hamiltonian."""
    J = hopping_matrix(lat)
    lam, V = np.linalg.eigh(J)
    W = (V * np.exp(-1j * lam * t)) @ V.T
    return np.stack([W @ rho0[s] @ W.conj().T for s in range(rho0.shape[0])])


def free_fermion_one_body(lat, n0, t):
    """Exact <c+_i c_j>(t) of a diagonal (Fock or thermal) state at U = 0,
    in the index convention of Eq. 5: W diag(n0) W^dagger, W = exp(-iJt)."""
    J = hopping_matrix(lat)
    lam, V = np.linalg.eigh(J)
    W = (V * np.exp(-1j * lam * t)) @ V.T
    return W @ np.diag(n0) @ W.conj().T


def wick_same_spin(nmat):
    """Same-spin <n_i n_j> (i != j) of a Slater determinant, Eq. A4 (wickthm):
    <c+_i c+_j c_j c_i> = n_ii n_jj - |n_ij|^2."""
    d = np.real(np.diag(nmat))
    out = d[:, None] * d[None, :] - np.abs(nmat) ** 2
    np.fill_diagonal(out, np.nan)
    return out


def dimer_eigenvalues(U, t=1.0):
    """Hubbard dimer, one up and one down electron: 0, U, (U +- sqrt(U^2 + 16 t^2))/2."""
    r = math.sqrt(U * U + 16 * t * t)
    return np.sort(np.array([0.0, U, (U + r) / 2, (U - r) / 2]))


def g2_long_time(n):
    """Table 1 (Eq. C11): g2(inf) = 2 C(n-2, n/2-2) / C(n-1, n/2-1), half filling."""
    return 2 * math.comb(n - 2, n // 2 - 2) / math.comb(n - 1, n // 2 - 1)


def g2_short_time(j12, j2):
    """Eq. C8 (form_g_st_2): g2_12(0+) = (sum_i j_2i^2 - j_12^2) / sum_i j_2i^2."""
    s = float(np.sum(np.asarray(j2) ** 2))
    return (s - j12 ** 2) / s


def rho11_taylor(eps, j1, xi1, U):
    """Eq. C3 (ro11u), filled site 1 whose neighbours are empty (Neel start):
    rho_11(eps) = 1/2 - sum_i j_1i eta2_1i eps - sum_i j_1i^2 eps^2
                  + U/2 sum_i j_1i eta1_1i eps^2 + O(eps^3),
    with eta1 = sqrt(2) Re xi and eta2 = sqrt(2) Im xi (App. C: xi/sqrt(2) =
    (eta1 + i eta2)/2)."""
    j1 = np.asarray(j1, dtype=np.float64)
    eta1 = math.sqrt(2) * np.real(xi1)
    eta2 = math.sqrt(2) * np.imag(xi1)
    return 0.5 - np.sum(j1 * eta2) * eps - np.sum(j1 ** 2) * eps ** 2 + U / 2 * np.sum(j1 * eta1) * eps ** 2


def general_state_covariance(lam, V, idx):
    """cov(rho*_ab, rho_mn) of the Gaussian Wigner density of a one-body state
    n = V diag(lam) V^dagger (one spin), App. A:
        1/2 (nt_ma n_bn + nt_bn n_ma),   nt = 1 - n,
    minus the part carried by the eigen-diagonal, sum_k conj(V_ak) V_bk V_mk
    conj(V_nk) lam_k (1 - lam_k), which Eq. 7 (applied in the diagonalising
    basis) leaves without noise.  idx: list of (a, b, m, n)."""
    lam = np.asarray(lam, dtype=np.float64)
    V = np.asarray(V, dtype=np.complex128)
    n = (V * lam[None, :]) @ V.conj().T
    nt = np.eye(len(lam)) - n
    out = []
    for a, b, m, k in idx:
        full = 0.5 * (nt[m, a] * n[b, k] + nt[b, k] * n[m, a])
        diag = np.sum(V[a].conj() * V[b] * V[m] * V[k].conj() * lam * (1 - lam))
        out.append(full - diag)
    return np.array(out)


def energy_longrange(lat, u, rho):
    """Classical energy of Eq. A10 with the full interaction sum of Eq. 1,
    H_W = -sum_ij,s j_ij rho_ij,s + sum_ij u_ij (rho_ii,up + 1/2)(rho_jj,dn + 1/2),
    for a symmetric u; conserved by the flow of Eq. 6 with that u."""
    J = hopping_matrix(lat)
    e = -sum(np.sum(J * rho[s]) for s in range(2))
    du = np.real(np.diag(rho[0])) + 0.5
    dd = np.real(np.diag(rho[1])) + 0.5
    return float(np.real(e) + du @ np.asarray(u) @ dd)
