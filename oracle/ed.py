"""Exact diagonalisation of the Hubbard model of Eq. 1 (TEST INFRASTRUCTURE ONLY).

The comparison method of Sec. III.A / App. B: the many-body state is written
in the basis of Slater determinants with fixed N_up, N_dn, and propagated
exactly.  The paper's Eq. 8 (shro) prints the propagator as exp(+iHt); the
Schroedinger form |Psi(t)> = exp(-iHt)|Psi_0> is used here (hbar = 1).  The
paper propagates with Krylov subspaces (expokit); scipy's expm_multiply is
used here, exact to its tolerance.

Fermionic signs: spin-up orbitals are ordered before spin-down ones, so a
same-spin hop c+_i c_j (i != j) picks up (-1)^(number of occupied same-spin
orbitals strictly between i and j); the other species contributes an even
count and no sign.
"""

from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _configs(n_sites, n_part):
    out = []
    for occ in itertools.combinations(range(n_sites), n_part):
        m = 0
        for i in occ:
            m |= 1 << i
        out.append(m)
    return out


def _hop_matrix(n_sites, configs, hop):
    """Single-species -sum_ij j_ij c+_i c_j in a fixed particle-number sector."""
    index = {c: k for k, c in enumerate(configs)}
    rows, cols, vals = [], [], []
    for k, c in enumerate(configs):
        for (i, j), t in hop.items():
            # term -t c+_i c_j
            if not (c >> j) & 1 or ((c >> i) & 1):
                continue
            lo, hi = min(i, j), max(i, j)
            between = bin(c & (((1 << hi) - 1) ^ ((1 << (lo + 1)) - 1))).count("1")
            sign = -1.0 if between % 2 else 1.0
            c2 = (c & ~(1 << j)) | (1 << i)
            rows.append(index[c2])
            cols.append(k)
            vals.append(-t * sign)
    d = len(configs)
    return sp.csr_matrix((vals, (rows, cols)), shape=(d, d))


class HubbardED:
    """Sparse H = -sum j_ij c+_is c_js + U sum_i n_i,up n_i,dn in the sector (N_up, N_dn)."""

    def __init__(self, lat, U, n_up, n_dn, t_bond=None):
        self.N = lat.n_sites
        tb = lat.t_bond if t_bond is None else t_bond
        hop = {}
        for (i, j), t in zip(lat.bonds, tb):
            hop[(int(i), int(j))] = float(t)
            hop[(int(j), int(i))] = float(t)
        self.up = _configs(self.N, n_up)
        self.dn = _configs(self.N, n_dn)
        hu = _hop_matrix(self.N, self.up, hop)
        hd = _hop_matrix(self.N, self.dn, hop)
        iu, idn = sp.identity(len(self.up), format="csr"), sp.identity(len(self.dn), format="csr")
        self.occ_up = np.array([[(c >> i) & 1 for i in range(self.N)] for c in self.up], dtype=np.float64)
        self.occ_dn = np.array([[(c >> i) & 1 for i in range(self.N)] for c in self.dn], dtype=np.float64)
        double = (self.occ_up @ self.occ_dn.T).reshape(-1)       # sum_i n_i,up n_i,dn
        self.H = (sp.kron(hu, idn) + sp.kron(iu, hd) + U * sp.diags(double)).tocsr()
        self.dim = self.H.shape[0]

    def fock_index(self, n_up, n_dn):
        mu = sum(1 << i for i in range(self.N) if n_up[i] > 0.5)
        md = sum(1 << i for i in range(self.N) if n_dn[i] > 0.5)
        return self.up.index(mu) * len(self.dn) + self.dn.index(md)

    def evolve(self, psi0, times):
        """|Psi(t)> = exp(-iHt)|Psi0> at the given, evenly spaced times."""
        times = np.asarray(times, dtype=np.float64)
        if len(times) == 1:
            return spla.expm_multiply(-1j * self.H * times[0], psi0)[None, :]
        return spla.expm_multiply(-1j * self.H, psi0, start=times[0], stop=times[-1],
                                  num=len(times), endpoint=True)

    def observables(self, psis):
        """<n_is> as [T, 2N] (s-major) and <n_a n_b> as [T, 2N, 2N] for a != b."""
        nu, nd = len(self.up), len(self.dn)
        occ, nn = [], []
        for psi in psis:
            p = (np.abs(psi) ** 2).reshape(nu, nd)
            pu, pd = p.sum(axis=1), p.sum(axis=0)
            n_up = pu @ self.occ_up
            n_dn = pd @ self.occ_dn
            occ.append(np.concatenate([n_up, n_dn]))
            uu = self.occ_up.T @ (pu[:, None] * self.occ_up)
            dd = self.occ_dn.T @ (pd[:, None] * self.occ_dn)
            ud = self.occ_up.T @ p @ self.occ_dn
            nn.append(np.block([[uu, ud], [ud.T, dd]]))
        return np.array(occ), np.array(nn)

    def eigenvalues(self):
        return np.linalg.eigvalsh(self.H.toarray())
