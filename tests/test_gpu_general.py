"""GPU parity of general (non-diagonal) initial states: ftwa_set_initial_basis
+ ftwa_sample against the oracle's sample_general (Eq. 7 in the
diagonalising basis, rotated by V), and the trajectories started from them.

Tolerances: FP64 samples 1e-12 absolute (two complex N x N products in a
different summation order); FP32 samples 2e-5 absolute (values O(1), float
rounding of 2 x N products); FP64 trajectories 1e-10 relative at T = 5.
"""

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import closed_forms as cf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ftwa():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_04352_gb300 as F
    F.load()
    return F


def _basis(kind, lat):
    N = lat.n_sites
    if kind == "thermal":
        return W.thermal_basis(lat, beta=2.0, mu=0.3)
    rng = np.random.default_rng(N)
    return W.random_basis(N, 5, rng.uniform(0, 1, N), rng.uniform(0, 1, N))


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 2e-5)])
@pytest.mark.parametrize("lat_name,kind", [("chain7", "random"), ("flake54", "random"), ("brick198", "thermal"),
                                           ("brick35", "random")])
def test_general_sample_parity(ftwa, lat_name, kind, precision, tol):
    lat = {"chain7": W.chain(7), "flake54": W.hexagonal_flake(3), "brick198": W.brick_wall_flake(),
           "brick35": W.brick_wall_flake(5, 7)}[lat_name]
    nu, nd = W.neel_state(lat)
    lam, V = _basis(kind, lat)
    M, seed = 3, 21
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=precision) as P:
        P.set_initial_basis(lam, V)
        rho = P.sample(seed, M, first_sample=4).cpu().numpy().astype(np.complex128)
        assert P.status() == 0
    for m in range(M):
        want = oracle.sample_general(lat.n_sites, lam, V, seed, 4 + m)
        assert np.abs(rho[m] - want).max() <= tol


def test_general_trajectories_fp64(ftwa):
    """GPU sample + evolve of a general state against the oracle's
    trajectory from its own sample (54 sites, random complex basis)."""
    lat = W.hexagonal_flake(3)
    nu, nd = W.neel_state(lat)
    lam, V = _basis("random", lat)
    M, steps, seed = 3, 500, 9
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=0, out_every=100) as P:
        P.set_initial_basis(lam, V)
        rho = P.sample(seed, M)
        X = P.evolve(rho, steps)
        assert P.status() == 0
        fin = rho.cpu().numpy()
        X = X.cpu().numpy()
    for m in range(M):
        r0 = oracle.sample_general(lat.n_sites, lam, V, seed, m)
        fo, so = oracle.evolve(lat, 1.6, r0, 0.01, steps, out_every=100)
        assert np.linalg.norm(fin[m] - fo) / np.linalg.norm(fo) <= 1e-10
        assert np.abs(X[:, m, :] - so).max() <= 1e-10


def test_general_state_free_fermion_occupations(ftwa):
    """U = 0: fTWA is exact, so the mean occupations of a general state follow
    diag(W n W^dagger), W = exp(-iJt) (FP32 state, 20000 samples, |z| < 5)."""
    lat = W.hexagonal_flake(2)
    nu, nd = W.neel_state(lat)
    lam, V = _basis("random", lat)
    M, steps, every = 20000, 100, 50
    with ftwa.Plan(lat, 0.0, n_up=nu, n_dn=nd, precision=1, out_every=every) as P:
        P.set_initial_basis(lam, V)
        rho = P.sample(3, M)
        X = P.evolve(rho, steps)
        occ, conn, _ = P.moments(X, g2=False)
        assert P.status() == 0
    occ, conn = occ.cpu().numpy(), conn.cpu().numpy()
    N = lat.n_sites
    for k, t in enumerate([0.0, 0.5, 1.0]):
        for s in range(2):
            n = (V[s] * lam[s][None, :]) @ V[s].conj().T
            want = np.real(np.diag(cf.exact_free(lat, n[None], t)[0]))
            se = np.sqrt(np.diagonal(conn[k])[s * N:(s + 1) * N] / M) + 1e-9
            assert np.all(np.abs(occ[k, s * N:(s + 1) * N] - want) < 5 * se)


def test_general_basis_validation_and_reset(ftwa):
    lat = W.hexagon_chain(2)
    nu, nd = W.neel_state(lat)
    lam, V = _basis("random", lat)
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=0, out_every=10) as P:
        ref = P.sample(2, 2).cpu().numpy()
        bad = V.copy()
        bad[0, 0, 0] += 1e-6
        with pytest.raises(ftwa.FtwaError):
            P.set_initial_basis(lam, bad)                  # not unitary
        bad_lam = lam.copy()
        bad_lam[1, 3] = 1.5
        with pytest.raises(ftwa.FtwaError):
            P.set_initial_basis(bad_lam, V)                # occupation outside [0, 1]
        P.set_initial_basis(lam, V)
        g = torch.zeros((5, 2 * lat.n_sites), dtype=torch.float64, device="cuda")
        with pytest.raises(ftwa.FtwaError):
            P.adjoint(1, 2, 40, 20, g)                     # no adjoint through the basis
        P.set_initial_basis(None, None)
        again = P.sample(2, 2).cpu().numpy()
        assert np.array_equal(ref, again)
        assert P.status() == 0
