"""Honeycomb lattice generators (input data only).

Every generator returns a :class:`Lattice`: ``n_sites`` sites, a list of
unique bonds ``(i, j)`` with ``i < j`` and one hopping amplitude per bond, a
bipartition (0 = sublattice A, 1 = sublattice B) and planar coordinates used
only to pick sites for initial states.  The Hamiltonian of Eq. 1 only needs
nearest-neighbour hoppings ``j_ij = t`` on these bonds and an on-site ``U``.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Lattice:
    name: str
    n_sites: int
    bonds: np.ndarray        # int32 [B, 2], i < j, unique, sorted
    t_bond: np.ndarray       # float64 [B]
    sublattice: np.ndarray   # int8 [N], 0 = A, 1 = B
    coords: np.ndarray       # float64 [N, 2]

    @property
    def n_bonds(self) -> int:
        return int(self.bonds.shape[0])

    def degrees(self) -> np.ndarray:
        deg = np.zeros(self.n_sites, dtype=np.int64)
        np.add.at(deg, self.bonds[:, 0], 1)
        np.add.at(deg, self.bonds[:, 1], 1)
        return deg

    def with_t(self, t) -> "Lattice":
        """Same geometry with hoppings replaced (scalar or one per bond)."""
        t_arr = np.broadcast_to(np.asarray(t, dtype=np.float64), (self.n_bonds,)).copy()
        return dataclasses.replace(self, t_bond=t_arr)


def _finish(name, n, bonds, coords, sub=None, t=1.0) -> Lattice:
    b = np.array(sorted({(min(i, j), max(i, j)) for i, j in bonds if i != j}), dtype=np.int32)
    if b.size == 0:
        b = np.zeros((0, 2), dtype=np.int32)
    if sub is None:
        sub = _two_colour(n, b)
    return Lattice(name=name, n_sites=n, bonds=b,
                   t_bond=np.full(b.shape[0], float(t)),
                   sublattice=np.asarray(sub, dtype=np.int8),
                   coords=np.asarray(coords, dtype=np.float64).reshape(n, 2))


def _two_colour(n, bonds) -> np.ndarray:
    """Bipartition by breadth-first search; raises if the graph is not bipartite."""
    adj = [[] for _ in range(n)]
    for i, j in bonds:
        adj[i].append(j)
        adj[j].append(i)
    col = -np.ones(n, dtype=np.int64)
    for s in range(n):
        if col[s] >= 0:
            continue
        col[s] = 0
        queue = [s]
        while queue:
            u = queue.pop(0)
            for v in adj[u]:
                if col[v] < 0:
                    col[v] = 1 - col[u]
                    queue.append(v)
                elif col[v] == col[u]:
                    raise ValueError("lattice is not bipartite")
    return col.astype(np.int8)


def periodic_honeycomb(lx: int = 2, ly: int = 2, t: float = 1.0) -> Lattice:
    """Periodic honeycomb of ``lx * ly`` unit cells (2 sites each).

    Site ``2*(x + lx*y)`` is A(x, y), site ``2*(x + lx*y) + 1`` is B(x, y).
    A(x, y) is bonded to B(x, y), B(x-1, y) and B(x, y-1) (indices mod lx, ly).
    With lx = ly = 2 this is the 8-site torus with three distinct neighbours per
    site.
    """
    def a(x, y):
        return 2 * ((x % lx) + lx * (y % ly))

    bonds = []
    coords = []
    for y in range(ly):
        for x in range(lx):
            cx, cy = x + 0.5 * y, y * math.sqrt(3) / 2
            coords += [(cx, cy), (cx + 0.5, cy + 0.29)]
            bonds += [(a(x, y), a(x, y) + 1), (a(x, y), a(x - 1, y) + 1), (a(x, y), a(x, y - 1) + 1)]
    return _finish(f"periodic_honeycomb_{lx}x{ly}", 2 * lx * ly, bonds, coords,
                   sub=[k % 2 for k in range(2 * lx * ly)], t=t)


def brick_wall_flake(rows: int = 11, cols: int = 18, t: float = 1.0) -> Lattice:
    """Open honeycomb flake in its brick-wall embedding (rows x cols sites).

    Site (r, c) has index ``r*cols + c``.  Row bonds join (r, c)-(r, c+1);
    vertical bonds join (r, c)-(r+1, c) when r + c is even.  Sublattice is
    (r + c) mod 2.  Corner sites with a single bond are kept.  11 x 18 gives
    198 sites and 277 bonds.
    """
    bonds = []
    coords = []
    for r in range(rows):
        for c in range(cols):
            coords.append((float(c), float(r)))
            if c + 1 < cols:
                bonds.append((r * cols + c, r * cols + c + 1))
            if r + 1 < rows and (r + c) % 2 == 0:
                bonds.append((r * cols + c, (r + 1) * cols + c))
    sub = [(r + c) % 2 for r in range(rows) for c in range(cols)]
    return _finish(f"brick_wall_{rows}x{cols}", rows * cols, bonds, coords, sub=sub, t=t)


def _hexagon_union(centres_axial, name, t=1.0) -> Lattice:
    """Sites and bonds of the union of the given hexagons (axial coordinates).

    Hexagon (q, r) has its centre at x = sqrt(3) (q + r/2), y = 1.5 r and
    corners at unit distance, angles 30 + 60 k degrees.  Sites are ordered by
    (y, x) so that the site ordering runs row by row across the flake.
    """
    key_to_xy = {}
    bonds = set()
    for q, r in centres_axial:
        cx, cy = math.sqrt(3) * (q + r / 2.0), 1.5 * r
        keys = []
        for k in range(6):
            ang = math.radians(30 + 60 * k)
            x, y = cx + math.cos(ang), cy + math.sin(ang)
            key = (round(y, 6), round(x, 6))
            key_to_xy[key] = (x, y)
            keys.append(key)
        for k in range(6):
            bonds.add((keys[k], keys[(k + 1) % 6]))
    order = sorted(key_to_xy)
    index = {k: i for i, k in enumerate(order)}
    coords = [key_to_xy[k] for k in order]
    bond_idx = [(index[a], index[b]) for a, b in bonds]
    return _finish(name, len(order), bond_idx, coords, t=t)


def hexagonal_flake(k: int, t: float = 1.0) -> Lattice:
    """Zigzag-edged hexagonal flake with k rings: 6 k^2 sites, 9 k^2 - 3 k bonds.

    k = 1 is a single hexagon, k = 2 coronene (24 sites); k = 3, 4, 5 give 54,
    96 and 150 sites.
    """
    cent = [(q, r) for q in range(-k + 1, k) for r in range(-k + 1, k) if abs(q + r) <= k - 1]
    return _hexagon_union(cent, f"hex_flake_k{k}", t=t)


def hexagon_chain(n_hex: int = 2, t: float = 1.0) -> Lattice:
    """Chain of edge-sharing hexagons; two hexagons give the 10-site system."""
    return _hexagon_union([(q, 0) for q in range(n_hex)], f"hexagon_chain_{n_hex}", t=t)


def ring(n: int, t: float = 1.0) -> Lattice:
    """Closed ring of n sites (n even keeps it bipartite)."""
    coords = [(math.cos(2 * math.pi * i / n), math.sin(2 * math.pi * i / n)) for i in range(n)]
    return _finish(f"ring_{n}", n, [(i, (i + 1) % n) for i in range(n)], coords, t=t)


def dimer(t: float = 1.0) -> Lattice:
    """Two sites, one bond (the Hubbard dimer)."""
    return _finish("dimer", 2, [(0, 1)], [(0.0, 0.0), (1.0, 0.0)], sub=[0, 1], t=t)


def chain(n: int, t: float = 1.0) -> Lattice:
    """Open chain of n sites (bipartite for every n, so odd sizes are possible)."""
    return _finish(f"chain_{n}", n, [(i, i + 1) for i in range(n - 1)], [(float(i), 0.0) for i in range(n)], t=t)


def coulomb_interaction(lat: Lattice, U: float, V: float) -> np.ndarray:
    """Symmetric interaction matrix u_ij of Eq. 1 with a long-range tail:
    u_ii = U and u_ij = V / |r_i - r_j| (distances in the lattice's coordinate
    units) for i != j."""
    d = np.linalg.norm(lat.coords[:, None, :] - lat.coords[None, :, :], axis=-1)
    u = np.where(d > 0, V / np.where(d > 0, d, 1.0), 0.0)
    np.fill_diagonal(u, U)
    return u
