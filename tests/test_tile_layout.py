"""The tiled stepper's work decomposition, checked on the host (no device).

ftwa_debug_tile_check builds the decomposition the kernel uses (ranks of a
cluster, block-major shared-memory regions, tiles per warp, per-row and
per-lane offset tables) and simulates every shared-memory address the
kernel forms for one sample: each read of an active lane must hit the
element Eq. 6 asks for, no read may leave the buffer of the CTA it
addresses, each computed element of the upper triangle must be written once
per stage and each mirror-band entry once.  This runs before the kernel ever
does, for every lattice family and cluster size in use.
"""

import ctypes

import numpy as np
import pytest

import workloads as W

LATTICES = {
    "brick198": lambda: W.brick_wall_flake(11, 18),
    "brick35": lambda: W.brick_wall_flake(5, 7),
    "brick16": lambda: W.brick_wall_flake(4, 4),
    "flake24": lambda: W.hexagonal_flake(2),
    "flake54": lambda: W.hexagonal_flake(3),
    "flake96": lambda: W.hexagonal_flake(4),
    "flake150": lambda: W.hexagonal_flake(5),
    "periodic8": W.periodic_honeycomb,
    "chain10": lambda: W.hexagon_chain(2),
    "chain7": lambda: W.chain(7),
    "ring40": lambda: W.ring(40),
    "dimer": W.dimer,
}


@pytest.fixture(scope="module")
def lib():
    from paper_2212_04352_gb300 import _lib
    try:
        return _lib.load()
    except ImportError as e:
        pytest.skip(str(e))


def _check(lib, lat, cluster, slots, t_bond=None):
    from paper_2212_04352_gb300 import _lib as L
    bonds = np.ascontiguousarray(lat.bonds, dtype=np.int32)
    tb = None if t_bond is None else np.ascontiguousarray(t_bond, dtype=np.float64)
    v = ctypes.c_int64(-1)
    msg = ctypes.create_string_buffer(256)
    rc = lib.ftwa_debug_tile_check(lat.n_sites, len(bonds), bonds.ctypes.data,
                                   None if tb is None else tb.ctypes.data, cluster, slots, ctypes.byref(v), msg, 256)
    return rc, v.value, msg.value.decode()


@pytest.mark.parametrize("name", sorted(LATTICES))
def test_tile_layout_every_cluster_size(lib, name):
    from paper_2212_04352_gb300 import _lib as L
    lat = LATTICES[name]()
    fitted = 0
    for cluster in (1, 2, 4, 8):
        for slots in (1, 3):
            rc, bad, msg = _check(lib, lat, cluster, slots)
            if rc == L.FTWA_ERR_UNSUPPORTED:
                continue
            assert rc == 0
            assert bad == 0, f"{name} cluster {cluster} slots {slots}: {bad} violations, first: {msg}"
            fitted += 1
    assert fitted >= 1


def test_tile_layout_per_bond_hoppings(lib):
    lat = W.brick_wall_flake(11, 18)
    t = np.random.default_rng(3).uniform(0.5, 1.5, lat.n_bonds)
    rc, bad, msg = _check(lib, lat, 4, 1, t)
    assert rc == 0 and bad == 0, msg


def test_tile_layout_198_fits_four_ctas(lib):
    """The 198-site flake fits a cluster of four CTAs (one sample)."""
    rc, bad, _ = _check(lib, W.brick_wall_flake(11, 18), 4, 1)
    assert rc == 0 and bad == 0


def test_tile_layout_rejects_bad_arguments(lib):
    from paper_2212_04352_gb300 import _lib as L
    v = ctypes.c_int64()
    assert lib.ftwa_debug_tile_check(1, 0, None, None, 1, 1, ctypes.byref(v), None, 0) == L.FTWA_ERR_INVALID_ARGUMENT
    b = np.array([[1, 0]], dtype=np.int32)
    assert lib.ftwa_debug_tile_check(2, 1, b.ctypes.data, None, 1, 1, ctypes.byref(v), None, 0) == \
        L.FTWA_ERR_INVALID_ARGUMENT
