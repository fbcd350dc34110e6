"""GPU parity of the time-dependent on-site drive (ftwa_set_drive +
ftwa_evolve_at) against the oracle's driven RK4 of Eq. 6.

Tolerances as for the undriven stepper: FP64 1e-10 relative per trajectory,
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


def _drive(N, seed=2):
    rng = np.random.default_rng(seed)
    return dict(amp=rng.uniform(-1.5, 1.5, (2, N)), t0=1.0, sigma=0.4, omega=4.0, phase=0.3)


@pytest.mark.parametrize("cluster", [1, 2, 4, 8])
def test_drive_fp64_parity(ftwa, cluster):
    """54 sites, every cluster split, start time 0.25, 300 steps (through the
    pulse), trajectories and snapshots against the oracle."""
    lat = W.hexagonal_flake(3)
    nu, nd = W.neel_state(lat)
    d = _drive(lat.n_sites)
    M, steps, t_start = 3, 300, 0.25
    rho0 = np.stack([oracle.sample(lat.n_sites, nu, nd, 4, m) for m in range(M)])
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=0, out_every=50, cluster=cluster) as P:
        P.set_drive(d["amp"], d["t0"], d["sigma"], d["omega"], d["phase"])
        rho = torch.from_numpy(rho0).cuda()
        X = P.evolve(rho, steps, t_start=t_start)
        assert P.status() == 0
        fin, X = rho.cpu().numpy(), X.cpu().numpy()
    for m in range(M):
        fo, so = oracle.evolve(lat, 1.6, rho0[m], 0.01, steps, out_every=50, drive=d, t_start=t_start)
        assert _rel(fin[m], fo) <= 1e-10
        assert np.abs(X[:, m, :] - so).max() <= 1e-10


def test_drive_fp32_parity_198(ftwa):
    lat = W.brick_wall_flake()
    nu, nd = W.charge_imbalanced_state(lat)
    d = _drive(lat.n_sites, seed=3)
    M, steps = 3, 100
    rho0 = np.stack([oracle.sample(lat.n_sites, nu, nd, 6, m) for m in range(M)])
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=1) as P:
        P.set_drive(d["amp"], d["t0"], d["sigma"], d["omega"], d["phase"])
        rho = torch.from_numpy(rho0.astype(np.complex64)).cuda()
        P.evolve(rho, steps, snap=None, t_start=0.6)
        assert P.status() == 0
        fin = rho.cpu().numpy().astype(np.complex128)
    for m in range(M):
        fo, _ = oracle.evolve(lat, 1.6, rho0[m], 0.01, steps, drive=d, t_start=0.6)
        assert _rel(fin[m], fo) <= 1e-4


def test_drive_neutral_and_unsupported(ftwa):
    """A zero-amplitude drive reproduces the undriven stepper (to rounding:
    the driven stepper tabulates the diagonal field); removing the drive
    restores it bit for bit; evolve_at without a drive ignores the start time;
    the adjoint and CUDA-graph batches refuse a driven plan."""
    lat = W.hexagon_chain(2)
    nu, nd = W.neel_state(lat)
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=0, out_every=10, variant=1) as P:
        ref = P.sample(3, 4)
        P.evolve(ref, 120, snap=None)
        r1 = P.sample(3, 4)
        P.evolve(r1, 120, snap=None, t_start=7.0)
        assert torch.equal(r1, ref)
        P.set_drive(np.zeros((2, lat.n_sites)), 1.0, 0.4, 4.0, 0.3)
        r2 = P.sample(3, 4)
        P.evolve(r2, 120, snap=None, t_start=0.5)
        assert _rel(r2.cpu().numpy(), ref.cpu().numpy()) <= 1e-12
        P.set_drive(_drive(lat.n_sites)["amp"], 1.0, 0.4, 4.0, 0.3)
        r3 = P.sample(3, 4)
        P.evolve(r3, 120, snap=None)
        assert not torch.equal(r3, ref)
        g = torch.zeros((13, 2 * lat.n_sites), dtype=torch.float64, device="cuda")
        with pytest.raises(ftwa.FtwaError):
            P.adjoint(1, 2, 120, 60, g)
        with pytest.raises(ftwa.FtwaError):
            ftwa.Batch([P], [r3], 10)
        P.set_drive(None)
        r4 = P.sample(3, 4)
        P.evolve(r4, 120, snap=None)
        assert torch.equal(r4, ref)
        assert P.status() == 0


@pytest.mark.parametrize("precision,cluster,tol", [(0, 1, 1e-10), (0, 4, 1e-10), (1, 0, 1e-4)])
def test_hopping_drive_parity(ftwa, precision, cluster, tol):
    """Every hopping scaled by m(t) = 1 + eps g(t), together with the site
    pulse, against the oracle (54 sites, start time 0.3, 200 steps)."""
    lat = W.hexagonal_flake(3)
    nu, nd = W.neel_state(lat)
    d = _drive(lat.n_sites, seed=5)
    hop = dict(eps=0.5, t0=1.2, sigma=0.6, omega=3.0, phase=0.1)
    M, steps, t_start = 3, 200, 0.3
    rho0 = np.stack([oracle.sample(lat.n_sites, nu, nd, 12, m) for m in range(M)])
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=precision, cluster=cluster) as P:
        P.set_drive(d["amp"], d["t0"], d["sigma"], d["omega"], d["phase"])
        P.set_hopping_drive(hop["eps"], hop["t0"], hop["sigma"], hop["omega"], hop["phase"])
        dtype = np.complex128 if precision == 0 else np.complex64
        rho = torch.from_numpy(rho0.astype(dtype)).cuda()
        P.evolve(rho, steps, snap=None, t_start=t_start)
        assert P.status() == 0
        fin = rho.cpu().numpy().astype(np.complex128)
        P.set_hopping_drive(0.0)
    for m in range(M):
        fo, _ = oracle.evolve(lat, 1.6, rho0[m], 0.01, steps, drive=dict(d, hop=hop), t_start=t_start)
        assert _rel(fin[m], fo) <= tol
