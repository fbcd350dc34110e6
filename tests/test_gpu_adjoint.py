"""GPU discrete adjoint against central finite differences of the CPU oracle.

Loss L = sum_{t=0..T} sum_k (<n_k>(t) - target_tk)^2 over the output rows;
its gradient with respect to U, every bond hopping t_b and every initial
occupation n_i,s is computed by the adjoint from dL/d<n> = 2(<n> - target)
and compared with central differences (h = 1e-5, common random numbers:
same seed) of the oracle.  Occupations are softened (0.05 / 0.95) so that
every noise scale s_ij of Eq. 7 is positive.  Gate (FP64): relative error
<= 1e-6.
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


def _loss(lat, U, nu, nd, seed, M, steps, every, target, t_bond):
    snap, _ = oracle.run(lat, U, nu, nd, seed, 0, M, 0.01, steps, every, t_bond=t_bond)
    occ = snap.mean(axis=1) + 0.5
    return float(((occ - target) ** 2).sum()), occ


@pytest.mark.parametrize("precision,tol", [(0, 1e-6), (1, 2e-3)])
def test_adjoint_matches_finite_differences(ftwa, precision, tol):
    lat = W.hexagon_chain(2)
    n0u, n0d = W.neel_state(lat)
    nu, nd = W.softened(n0u), W.softened(n0d)
    U, seed, M, steps, every, ckpt = 1.6, 5, 6, 40, 10, 20
    rng = np.random.default_rng(0)
    target = 0.5 + 0.1 * rng.standard_normal((steps // every + 1, 2 * lat.n_sites))
    tb = np.array(lat.t_bond, dtype=np.float64)
    L0, occ = _loss(lat, U, nu, nd, seed, M, steps, every, target, tb)
    g = torch.from_numpy(2.0 * (occ - target)).cuda()
    with ftwa.Plan(lat, U, n_up=nu, n_dn=nd, precision=precision, out_every=every) as P:
        gU, gt, gn = P.adjoint(seed, M, steps, ckpt, g)
        assert P.status() == 0
    gU, gt, gn = gU.item(), gt.cpu().numpy(), gn.cpu().numpy()

    h = 1e-5
    def fd(fn):
        return (fn(h) - fn(-h)) / (2 * h)
    fdU = fd(lambda d: _loss(lat, U + d, nu, nd, seed, M, steps, every, target, tb)[0])
    fdt = np.array([fd(lambda d, b=b: _loss(lat, U, nu, nd, seed, M, steps, every, target,
                                            tb + d * (np.arange(lat.n_bonds) == b))[0])
                    for b in range(lat.n_bonds)])
    fdn = np.zeros((2, lat.n_sites))
    for s in range(2):
        for i in range(lat.n_sites):
            def Ln(d):
                a, b = nu.copy(), nd.copy()
                (a if s == 0 else b)[i] += d
                return _loss(lat, U, a, b, seed, M, steps, every, target, tb)[0]
            fdn[s, i] = fd(Ln)
    scale = max(abs(fdU), np.abs(fdt).max(), np.abs(fdn).max())
    assert abs(gU - fdU) <= tol * scale
    assert np.max(np.abs(gt - fdt)) <= tol * scale
    assert np.max(np.abs(gn - fdn)) <= tol * scale


def test_adjoint_checkpoint_invariance(ftwa):
    """The gradient does not depend on the checkpoint spacing (FP64)."""
    lat = W.periodic_honeycomb()
    nu, nd = W.softened(W.neel_state(lat)[0]), W.softened(W.neel_state(lat)[1])
    g = torch.full((5, 16), 0.3, dtype=torch.float64, device="cuda")
    out = []
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=0, out_every=10) as P:
        for ck in (10, 20, 40):
            out.append([x.cpu().numpy() for x in P.adjoint(3, 4, 40, ck, g)])
        assert P.status() == 0
    for o in out[1:]:
        for a, b in zip(o, out[0]):
            np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-14)


def test_adjoint_96_sites_fp64_spot_check(ftwa):
    """96-site flake (the adjoint workload's lattice) in FP64: dL/dU, three
    bond gradients and two occupation gradients against central differences
    of the oracle."""
    lat = W.hexagonal_flake(4)
    n0u, n0d = W.neel_state(lat)
    nu, nd = W.softened(n0u), W.softened(n0d)
    U, seed, M, steps, every, ckpt = 1.6, 7, 2, 20, 10, 10
    rng = np.random.default_rng(1)
    target = 0.5 + 0.1 * rng.standard_normal((steps // every + 1, 2 * lat.n_sites))
    tb = np.array(lat.t_bond, dtype=np.float64)
    L0, occ = _loss(lat, U, nu, nd, seed, M, steps, every, target, tb)
    g = torch.from_numpy(2.0 * (occ - target)).cuda()
    with ftwa.Plan(lat, U, n_up=nu, n_dn=nd, precision=0, out_every=every) as P:
        gU, gt, gn = P.adjoint(seed, M, steps, ckpt, g)
        assert P.status() == 0
    gU, gt, gn = gU.item(), gt.cpu().numpy(), gn.cpu().numpy()
    h = 1e-5
    def fd(fn):
        return (fn(h) - fn(-h)) / (2 * h)
    checks = [(gU, fd(lambda d: _loss(lat, U + d, nu, nd, seed, M, steps, every, target, tb)[0]))]
    for b in (0, 57, lat.n_bonds - 1):
        checks.append((gt[b], fd(lambda d, b=b: _loss(lat, U, nu, nd, seed, M, steps, every, target,
                                                      tb + d * (np.arange(lat.n_bonds) == b))[0])))
    for s, i in ((0, 3), (1, 90)):
        def Ln(d, s=s, i=i):
            a, b = nu.copy(), nd.copy()
            (a if s == 0 else b)[i] += d
            return _loss(lat, U, a, b, seed, M, steps, every, target, tb)[0]
        checks.append((gn[s, i], fd(Ln)))
    scale = max(abs(f) for _, f in checks)
    for got, want in checks:
        assert abs(got - want) <= 1e-6 * scale, (got, want)


def test_adjoint_fd_gate_at_adjoint_workload_size(ftwa):
    """The adjoint workload's lattice, horizon and checkpointing (96-site
    flake, U/t = 1.6, T = 5: 500 RK4 steps, checkpoints every 50, outputs
    every 10) in FP64 on 8 samples: dL/dU, two bond gradients and two
    initial-occupation gradients against central differences (h = 1e-5,
    same seed) of the oracle, relative error <= 1e-6."""
    lat = W.hexagonal_flake(4)
    n0u, n0d = W.neel_state(lat)
    nu, nd = W.softened(n0u), W.softened(n0d)
    U, seed, M, steps, every, ckpt = 1.6, 11, 8, 500, 10, 50
    rng = np.random.default_rng(4)
    target = 0.5 + 0.05 * rng.standard_normal((steps // every + 1, 2 * lat.n_sites))
    tb = np.array(lat.t_bond, dtype=np.float64)
    _, occ = _loss(lat, U, nu, nd, seed, M, steps, every, target, tb)
    g = torch.from_numpy(2.0 * (occ - target)).cuda()
    with ftwa.Plan(lat, U, n_up=nu, n_dn=nd, precision=0, out_every=every) as P:
        gU, gt, gn = P.adjoint(seed, M, steps, ckpt, g)
        assert P.status() == 0
    gU, gt, gn = gU.item(), gt.cpu().numpy(), gn.cpu().numpy()
    h = 1e-5

    def fd(fn):
        return (fn(h) - fn(-h)) / (2 * h)
    checks = [(gU, fd(lambda d: _loss(lat, U + d, nu, nd, seed, M, steps, every, target, tb)[0]))]
    for b in (0, lat.n_bonds // 2):
        checks.append((gt[b], fd(lambda d, b=b: _loss(lat, U, nu, nd, seed, M, steps, every, target,
                                                      tb + d * (np.arange(lat.n_bonds) == b))[0])))
    for s_, i in ((0, 5), (1, 70)):
        def Ln(d, s_=s_, i=i):
            a, b = nu.copy(), nd.copy()
            (a if s_ == 0 else b)[i] += d
            return _loss(lat, U, a, b, seed, M, steps, every, target, tb)[0]
        checks.append((gn[s_, i], fd(Ln)))
    scale = max(abs(w) for _, w in checks)
    for got, want in checks:
        assert abs(got - want) <= 1e-6 * max(abs(want), 1e-3 * scale), (got, want)


@pytest.mark.parametrize("lat_name", ["flake96", "flake150", "brick198"])
def test_adjoint_fp32_follows_fp64_large(ftwa, lat_name):
    """The FP32 adjoint (row-pass VJP, one 1024-thread CTA per SM) against the
    FP64 adjoint (dot-product VJP) on the larger lattices (8 samples, 20
    steps).  Gate: 2e-3 of the largest gradient entry (the FP32 gate of the
    finite-difference test)."""
    lat = {"flake96": W.hexagonal_flake(4), "flake150": W.hexagonal_flake(5),
           "brick198": W.brick_wall_flake()}[lat_name]
    n0u, n0d = W.neel_state(lat)
    nu, nd = W.softened(n0u), W.softened(n0d)
    seed, M, steps, every, ckpt = 11, 8, 20, 10, 10
    rng = np.random.default_rng(2)
    g = torch.from_numpy(rng.standard_normal((steps // every + 1, 2 * lat.n_sites))).cuda()
    res = []
    for precision in (0, 1):
        with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=precision, out_every=every) as P:
            res.append([x.cpu().numpy() for x in P.adjoint(seed, M, steps, ckpt, g)])
            assert P.status() == 0
    scale = max(np.abs(x).max() for x in res[0])
    for a, b in zip(res[1], res[0]):
        assert np.abs(a - b).max() <= 2e-3 * scale


@pytest.mark.parametrize("lat_name,U,ckpt", [("chain10", 1.6, 10), ("periodic8", 2.5, 30), ("flake24", 1.0, 15)])
def test_adjoint_matches_oracle_adjoint(ftwa, lat_name, U, ckpt):
    """The GPU adjoint against the oracle's discrete RK4 adjoint (numpy, full
    matrices, pinned to finite differences at 1e-8) for a random linear loss:
    FP64 to 1e-10 of the largest gradient entry (the two differ only by
    rounding), FP32 to 2e-3."""
    from oracle import adjoint as OA
    lat = {"chain10": W.hexagon_chain(2), "periodic8": W.periodic_honeycomb(),
           "flake24": W.hexagonal_flake(2)}[lat_name]
    n0u, n0d = W.neel_state(lat)
    nu, nd = W.softened(n0u), W.softened(n0d)
    N, seed, M, steps, every = lat.n_sites, 9, 5, 30, 5
    g = np.random.default_rng(3).standard_normal((steps // every + 1, 2 * N))
    want = OA.adjoint(lat, U, nu, nd, seed, M, 0.01, steps, every, g)
    scale = max(abs(want[0]), np.abs(want[1]).max(), np.abs(want[2]).max())
    for precision, tol in ((0, 1e-10), (1, 2e-3)):
        with ftwa.Plan(lat, U, n_up=nu, n_dn=nd, precision=precision, out_every=every) as P:
            got = [x.cpu().numpy() for x in P.adjoint(seed, M, steps, ckpt, torch.from_numpy(g).cuda())]
            assert P.status() == 0
        assert abs(got[0][0] - want[0]) <= tol * scale
        assert np.abs(got[1] - want[1]).max() <= tol * scale
        assert np.abs(got[2] - want[2]).max() <= tol * scale


@pytest.mark.parametrize("lat_name,U,ckpt", [("chain10", 1.6, 10), ("periodic8", 2.5, 30), ("flake24", 1.0, 15)])
def test_adjoint_corr_matches_oracle_adjoint(ftwa, lat_name, U, ckpt):
    """Correlation losses (ftwa_adjoint_corr): the GPU adjoint for a random
    linear loss sum g <n> + sum G C (G not symmetric, C the connected
    correlator of Eq. 5) against the oracle's discrete RK4 adjoint (pinned to
    finite differences at 1e-8): FP64 to 1e-10 of the largest gradient entry,
    FP32 to 2e-3.  The forward means come from the GPU's own moments."""
    from oracle import adjoint as OA
    lat = {"chain10": W.hexagon_chain(2), "periodic8": W.periodic_honeycomb(),
           "flake24": W.hexagonal_flake(2)}[lat_name]
    n0u, n0d = W.neel_state(lat)
    nu, nd = W.softened(n0u), W.softened(n0d)
    N, seed, M, steps, every = lat.n_sites, 10, 5, 30, 5
    rng = np.random.default_rng(4)
    T = steps // every + 1
    g = rng.standard_normal((T, 2 * N))
    G = rng.standard_normal((T, 2 * N, 2 * N))
    snap, _ = oracle.run(lat, U, nu, nd, seed, 0, M, 0.01, steps, every)
    want = OA.adjoint(lat, U, nu, nd, seed, M, 0.01, steps, every, g, gC=G, mu=snap.mean(axis=1))
    scale = max(abs(want[0]), np.abs(want[1]).max(), np.abs(want[2]).max())
    for precision, tol in ((0, 1e-10), (1, 2e-3)):
        with ftwa.Plan(lat, U, n_up=nu, n_dn=nd, precision=precision, out_every=every) as P:
            X = P.evolve(P.sample(seed, M), steps)
            occ, _, _ = P.moments(X, g2=False)
            got = [x.cpu().numpy() for x in P.adjoint(seed, M, steps, ckpt, torch.from_numpy(g).cuda(),
                                                      dL_dconn=torch.from_numpy(G).cuda(), occ=occ)]
            # the correlation term alone (no occupation cotangent) is accepted too
            P.adjoint(seed, M, steps, ckpt, None, dL_dconn=torch.from_numpy(G).cuda(), occ=occ)
            assert P.status() == 0
        assert abs(got[0][0] - want[0]) <= tol * scale
        assert np.abs(got[1] - want[1]).max() <= tol * scale
        assert np.abs(got[2] - want[2]).max() <= tol * scale


def test_adjoint_corr_rejects_missing_means(ftwa):
    from paper_2212_04352_gb300 import _lib as L
    import ctypes
    lat = W.periodic_honeycomb()
    nu, nd = W.softened(W.neel_state(lat)[0]), W.softened(W.neel_state(lat)[1])
    G = torch.zeros((5, 16, 16), dtype=torch.float64, device="cuda")
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=0, out_every=10) as P:
        p = ctypes.c_void_p
        rc = ftwa.load().ftwa_adjoint_corr(P._h, 1, 2, 40, 20, None, p(G.data_ptr()), None, None, None, None, None)
        assert rc == L.FTWA_ERR_INVALID_ARGUMENT
        rc = ftwa.load().ftwa_adjoint_corr(P._h, 1, 2, 40, 20, None, None, None, None, None, None, None)
        assert rc == L.FTWA_ERR_INVALID_ARGUMENT
        with pytest.raises(ValueError):
            P.adjoint(1, 2, 40, 20, None, dL_dconn=G)
