"""GPU parity of the long-range interaction u_ij of Eq. 1
(ftwa_set_interaction) against the oracle's Eq. 6 with the literal sum over k.

Tolerances as for the on-site stepper: FP64 1e-10 relative per trajectory,
FP32 1e-4 relative after 100 steps.
"""

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ftwa():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_04352_gb300 as F
    F.load()
    return F


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("cluster", [1, 2, 4, 8])
def test_longrange_fp64_parity(ftwa, cluster):
    lat = W.hexagonal_flake(3)
    nu, nd = W.neel_state(lat)
    u = W.coulomb_interaction(lat, 1.6, 0.5)
    M, steps = 3, 300
    rho0 = np.stack([oracle.sample(lat.n_sites, nu, nd, 8, m) for m in range(M)])
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=0, out_every=50, cluster=cluster) as P:
        P.set_interaction(u)
        rho = torch.from_numpy(rho0).cuda()
        X = P.evolve(rho, steps)
        assert P.status() == 0
        fin, X = rho.cpu().numpy(), X.cpu().numpy()
    for m in range(M):
        fo, so = oracle.evolve(lat, 0.0, rho0[m], 0.01, steps, out_every=50, u=u)
        assert _rel(fin[m], fo) <= 1e-10
        assert np.abs(X[:, m, :] - so).max() <= 1e-10


def test_longrange_fp32_parity_198(ftwa):
    lat = W.brick_wall_flake()
    nu, nd = W.charge_imbalanced_state(lat)
    u = W.coulomb_interaction(lat, 1.6, 0.4)
    M, steps = 3, 100
    rho0 = np.stack([oracle.sample(lat.n_sites, nu, nd, 9, m) for m in range(M)])
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=1) as P:
        P.set_interaction(u)
        rho = torch.from_numpy(rho0.astype(np.complex64)).cuda()
        P.evolve(rho, steps, snap=None)
        assert P.status() == 0
        fin = rho.cpu().numpy().astype(np.complex128)
    for m in range(M):
        fo, _ = oracle.evolve(lat, 0.0, rho0[m], 0.01, steps, u=u)
        assert _rel(fin[m], fo) <= 1e-4


def test_longrange_onsite_limit_and_errors(ftwa):
    """u = U 1 follows the on-site stepper (to rounding: the field is
    tabulated); a non-symmetric u is rejected; the adjoint refuses the plan;
    removing u restores the on-site stepper bit for bit."""
    lat = W.hexagon_chain(2)
    nu, nd = W.neel_state(lat)
    N = lat.n_sites
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=0, out_every=10, variant=1) as P:
        ref = P.sample(5, 4)
        P.evolve(ref, 200, snap=None)
        P.set_interaction(1.6 * np.eye(N))
        r1 = P.sample(5, 4)
        P.evolve(r1, 200, snap=None)
        assert _rel(r1.cpu().numpy(), ref.cpu().numpy()) <= 1e-12
        bad = W.coulomb_interaction(lat, 1.6, 0.5)
        bad[0, 1] += 1e-3
        with pytest.raises(ftwa.FtwaError):
            P.set_interaction(bad)
        g = torch.zeros((21, 2 * N), dtype=torch.float64, device="cuda")
        with pytest.raises(ftwa.FtwaError):
            P.adjoint(1, 2, 200, 100, g)
        P.set_interaction(None)
        r2 = P.sample(5, 4)
        P.evolve(r2, 200, snap=None)
        assert torch.equal(r2, ref)
        assert P.status() == 0
