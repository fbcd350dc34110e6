"""Diagonal initial occupations n_{i sigma} (input data only).

The fTWA initial distribution of Eq. 7 is built from a diagonal state with
site occupations n_{ii sigma}; these helpers only choose those occupations.
"""

from __future__ import annotations

import numpy as np

from .lattices import Lattice


def neel_state(lat: Lattice):
    """Spin up on sublattice A, spin down on sublattice B (one electron per site)."""
    a = (lat.sublattice == 0).astype(np.float64)
    return a.copy(), 1.0 - a


def _central_hexagon(lat: Lattice):
    """The 6-cycle of the brick-wall embedding whose centre is closest to the
    centroid of the sites (ties: smallest (row, col) of its lower-left site)."""
    xy = lat.coords
    cols = int(round(xy[:, 0].max())) + 1
    rows = int(round(xy[:, 1].max())) + 1
    if rows * cols != lat.n_sites:
        raise ValueError("central hexagon rule is defined for brick-wall flakes only")
    cen = xy.mean(axis=0)
    best = None
    for r in range(rows - 1):
        for c in range(cols - 2):
            if (r + c) % 2:
                continue
            fx, fy = c + 1.0, r + 0.5
            d = (fx - cen[0]) ** 2 + (fy - cen[1]) ** 2
            cand = (round(d, 9), r, c)
            if best is None or cand < best:
                best = cand
    _, r, c = best
    return [r * cols + c + k for k in range(3)] + [(r + 1) * cols + c + k for k in range(3)]


def charge_imbalanced_state(lat: Lattice):
    """Neel start with a doubly occupied central hexagon and six emptied edge sites.

    The six sites of the central hexagon get n_up = n_dn = 1.  The six emptied
    sites are the first three of each sublattice in the order (lowest degree,
    largest distance from the centroid, lowest index).  This keeps
    N_up = N_dn = N / 2, i.e. half filling.
    """
    n_up, n_dn = neel_state(lat)
    hexa = _central_hexagon(lat)
    n_up[hexa] = 1.0
    n_dn[hexa] = 1.0
    deg = lat.degrees()
    dist = np.linalg.norm(lat.coords - lat.coords.mean(axis=0), axis=1)
    order = sorted(range(lat.n_sites), key=lambda i: (deg[i], -round(dist[i], 9), i))
    picked = {0: [], 1: []}
    for i in order:
        s = int(lat.sublattice[i])
        if i in hexa or len(picked[s]) >= 3:
            continue
        picked[s].append(i)
    for i in picked[0] + picked[1]:
        n_up[i] = 0.0
        n_dn[i] = 0.0
    return n_up, n_dn


def softened(n, eps: float = 0.05):
    """Map Fock occupations {0, 1} to {eps, 1 - eps} (smooth sampler map)."""
    n = np.asarray(n, dtype=np.float64)
    return eps + (1.0 - 2.0 * eps) * n


# ---- general (non-diagonal) initial states, given in a diagonalising basis ----
# A one-body state n_s = V_s diag(lam_s) V_s^dagger per spin is described by
# (lam [2, N], V [2, N, N], columns of V_s = eigenvectors).  These helpers only
# build such inputs (eigen-decompositions with numpy's LAPACK routines).

def thermal_basis(lat: Lattice, beta: float, mu: float = 0.0):
    """Grand-canonical thermal state of the hopping Hamiltonian h = -J of
    Eq. 1 (U = 0) at inverse temperature beta and chemical potential mu,
    both spins: lam_k = 1 / (exp(beta (eps_k - mu)) + 1), V = eigenvectors."""
    J = np.zeros((lat.n_sites, lat.n_sites))
    for (i, j), t in zip(lat.bonds, lat.t_bond):
        J[i, j] = J[j, i] = t
    eps, V = np.linalg.eigh(-J)
    lam = 1.0 / (np.exp(np.clip(beta * (eps - mu), -700, 700)) + 1.0)
    return np.stack([lam, lam]), np.stack([V, V]).astype(np.complex128)


def random_basis(n_sites: int, seed: int, lam_up, lam_dn):
    """Seeded Haar-like random unitary bases (QR of a complex Gaussian matrix,
    phases fixed by the diagonal of R) with the given eigen-occupations."""
    rng = np.random.default_rng(seed)
    Vs = []
    for _ in range(2):
        z = rng.standard_normal((n_sites, n_sites)) + 1j * rng.standard_normal((n_sites, n_sites))
        q, r = np.linalg.qr(z)
        d = np.diag(r)
        Vs.append(q * (d / np.abs(d))[None, :])
    return np.stack([np.asarray(lam_up, dtype=np.float64), np.asarray(lam_dn, dtype=np.float64)]), np.stack(Vs)
