"""Seeded, synthetic inputs for the fTWA hot path.

This package holds only input generation: honeycomb lattice geometries (bond
lists with hopping amplitudes) and diagonal initial occupations.  It contains
none of the method's arithmetic (no sampling of phase-space variables, no
equations of motion, no estimators), so both the CUDA path and the CPU oracle
may use it without sharing any of the method's code.

The paper's own geometries (the two-hexagon 10-site system of Fig. 1 and the
198-site flake of Fig. 7) exist only in figures that are not available; the
generators below are deterministic stand-ins with the same site counts and
coordination (honeycomb, nearest-neighbour bonds, degree <= 3).
"""

from .lattices import (  # noqa: F401
    Lattice,
    periodic_honeycomb,
    brick_wall_flake,
    hexagonal_flake,
    hexagon_chain,
    ring,
    dimer,
    chain,
    coulomb_interaction,
)
from .states import (  # noqa: F401
    neel_state,
    charge_imbalanced_state,
    softened,
    thermal_basis,
    random_basis,
)
