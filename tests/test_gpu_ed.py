"""GPU exact diagonalisation (ftwa_ed_*) against the oracle's sparse ED
(scipy expm_multiply on the same Fock basis).

Tolerance: 1e-10 absolute on <n> and <n n> (the Chebyshev series is cut
where its Bessel coefficients fall below 1e-17; expm_multiply works to its
own ~1e-13 tolerance).
"""

import numpy as np
import pytest

import workloads as W
from oracle.ed import HubbardED

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ftwa():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_04352_gb300 as F
    F.load()
    return F


@pytest.mark.parametrize("lat_name,U,state", [("chain10", 1.6, "neel"), ("periodic8", 2.5, "neel"),
                                              ("brick12", 1.0, "imbalanced"), ("dimer", 0.7, "neel")])
def test_ed_matches_oracle(ftwa, lat_name, U, state):
    lat = {"chain10": W.hexagon_chain(2), "periodic8": W.periodic_honeycomb(), "brick12": W.brick_wall_flake(3, 4),
           "dimer": W.dimer()}[lat_name]
    nu, nd = W.neel_state(lat)
    if state == "imbalanced":        # one up electron moved onto a down site: N_up != N_dn
        nd = nd.copy()
        nu = nu.copy()
        a = np.flatnonzero(nu)[:1]
        nu[a] = 0.0
        nd[a] = 1.0
    n_up, n_dn = int(nu.sum()), int(nd.sum())
    dt, n_out = 0.25, (4 if lat.n_sites >= 12 else 8)
    ed = HubbardED(lat, U, n_up, n_dn)
    psi0 = np.zeros(ed.dim, dtype=np.complex128)
    psi0[ed.fock_index(nu, nd)] = 1.0
    occ_o, nn_o = ed.observables(ed.evolve(psi0, np.arange(n_out + 1) * dt))
    with ftwa.ED(lat, U, n_up, n_dn) as G:
        assert G.info()[0] == ed.dim
        occ, nn = G.evolve(nu, nd, dt, n_out)
        occ, nn = occ.cpu().numpy(), nn.cpu().numpy()
    assert np.abs(occ - occ_o).max() <= 1e-10
    K = 2 * lat.n_sites
    off = ~np.eye(K, dtype=bool)
    assert np.abs(nn[:, off] - nn_o[:, off]).max() <= 1e-10
    assert np.abs(np.diagonal(nn, axis1=1, axis2=2) - occ).max() <= 1e-12
    # particle number per spin is conserved
    N = lat.n_sites
    assert np.abs(occ[:, :N].sum(axis=1) - n_up).max() <= 1e-10
    assert np.abs(occ[:, N:].sum(axis=1) - n_dn).max() <= 1e-10


def test_ed_argument_errors(ftwa):
    lat = W.dimer()
    with ftwa.ED(lat, 1.0, 1, 1) as G:
        with pytest.raises(ftwa.FtwaError):
            G.evolve([1, 1], [0, 1], 0.1, 2)         # wrong N_up
        with pytest.raises(ftwa.FtwaError):
            G.evolve([0.5, 0.5], [0, 1], 0.1, 2)     # not a Fock state
        with pytest.raises(ftwa.FtwaError):
            G.evolve([1, 0], [0, 1], 0.0, 2)         # dt_out must be positive
    with pytest.raises(ftwa.FtwaError):
        ftwa.ED(W.chain(25), 1.0, 12, 12)            # above 24 sites
