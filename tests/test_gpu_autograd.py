"""torch.autograd wrapper (occupations) of the fTWA forward (ftwa_sample ->
ftwa_evolve -> ftwa_moments) with the discrete RK4 adjoint (ftwa_adjoint) as
its backward.

Gates (FP64): the forward equals the oracle's sample mean to 1e-10; the
gradients equal a direct ftwa_adjoint call with the same dL/d<n> to 1e-12
of their scale, and central differences of the wrapped forward (h = 1e-5,
same seed) to 1e-6; torch.autograd.gradcheck passes.  FP32: within 2e-3 of
the FP64 gradients.  Occupations are softened (0.05 / 0.95) so that every
noise scale s_ij of Eq. 7 is positive and n0 -> loss is differentiable.
"""

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SEED, M, STEPS, EVERY, CKPT = 5, 6, 40, 10, 20


@pytest.fixture(scope="module")
def ftwa():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_04352_gb300 as F
    F.load()
    return F


def _setup():
    lat = W.hexagon_chain(2)
    nu, nd = W.neel_state(lat)
    return lat, np.stack([W.softened(nu), W.softened(nd)])


def _leaves(lat, n0, U=1.6):
    return (torch.tensor(U, dtype=torch.float64, requires_grad=True),
            torch.tensor(lat.t_bond, dtype=torch.float64, requires_grad=True),
            torch.tensor(n0, dtype=torch.float64, requires_grad=True))


def _target(shape):
    rng = np.random.default_rng(0)
    return torch.from_numpy(0.5 + 0.1 * rng.standard_normal(shape)).cuda()


def test_forward_and_backward_fp64(ftwa):
    lat, n0 = _setup()
    U, tb, n = _leaves(lat, n0)
    occ = ftwa.occupations(lat, U, tb, n, SEED, M, STEPS, out_every=EVERY, ckpt_every=CKPT)
    assert occ.shape == (STEPS // EVERY + 1, 2 * lat.n_sites) and occ.dtype == torch.float64
    snap, _ = oracle.run(lat, 1.6, n0[0], n0[1], SEED, 0, M, 0.01, STEPS, EVERY, t_bond=lat.t_bond)
    assert np.abs(occ.detach().cpu().numpy() - (snap.mean(axis=1) + 0.5)).max() <= 1e-10

    target = _target(tuple(occ.shape))
    ((occ - target) ** 2).sum().backward()
    g = 2.0 * (occ.detach() - target)
    with ftwa.Plan(lat, 1.6, n_up=n0[0], n_dn=n0[1], precision=0, out_every=EVERY) as P:
        gU, gt, gn = (x.cpu().numpy() for x in P.adjoint(SEED, M, STEPS, CKPT, g))
    scale = max(abs(gU).max(), abs(gt).max(), abs(gn).max())
    assert abs(U.grad.item() - gU[0]) <= 1e-12 * scale
    assert np.abs(tb.grad.numpy() - gt).max() <= 1e-12 * scale
    assert np.abs(n.grad.numpy() - gn).max() <= 1e-12 * scale

    def loss(Uv, tv, nv):
        with torch.no_grad():
            o = ftwa.occupations(lat, Uv, tv, nv, SEED, M, STEPS, out_every=EVERY, ckpt_every=CKPT)
            return float(((o - target) ** 2).sum())

    h, t0 = 1e-5, np.array(lat.t_bond, dtype=np.float64)
    fdU = (loss(1.6 + h, t0, n0) - loss(1.6 - h, t0, n0)) / (2 * h)
    fdt = np.array([(loss(1.6, t0 + h * e, n0) - loss(1.6, t0 - h * e, n0)) / (2 * h)
                    for e in np.eye(lat.n_bonds)])
    fdn = np.array([(loss(1.6, t0, n0 + h * e) - loss(1.6, t0, n0 - h * e)) / (2 * h)
                    for e in np.eye(2 * lat.n_sites).reshape(-1, 2, lat.n_sites)]).reshape(2, lat.n_sites)
    scale = max(abs(fdU), np.abs(fdt).max(), np.abs(fdn).max())
    assert abs(U.grad.item() - fdU) <= 1e-6 * scale
    assert np.abs(tb.grad.numpy() - fdt).max() <= 1e-6 * scale
    assert np.abs(n.grad.numpy() - fdn).max() <= 1e-6 * scale


def test_gradcheck(ftwa):
    """torch.autograd.gradcheck (numerical Jacobian-vector products against
    the adjoint; fast mode) on a 16-site periodic lattice."""
    lat = W.periodic_honeycomb()
    nu, nd = W.neel_state(lat)
    n0 = np.stack([W.softened(nu), W.softened(nd)])
    U, tb, n = _leaves(lat, n0, U=2.0)

    def f(Uv, tv, nv):
        return ftwa.occupations(lat, Uv, tv, nv, 3, 4, 30, out_every=10, ckpt_every=10)

    assert ftwa.FTWAFunction.__name__ == "FTWAFunction"
    assert torch.autograd.gradcheck(f, (U, tb, n), eps=1e-6, atol=1e-7, rtol=1e-5, nondet_tol=1e-10,
                                    fast_mode=True)


def test_fp32_and_partial_requires_grad(ftwa):
    """FP32 plan gradients within 2e-3 of FP64; inputs without requires_grad
    receive none; a second backward through a retained graph repeats the
    first (to rounding: the adjoint sums with atomics)."""
    lat, n0 = _setup()
    res = []
    for precision in (0, 1):
        U, tb, n = _leaves(lat, n0)
        n.requires_grad_(False)
        occ = ftwa.occupations(lat, U, tb, n, SEED, M, STEPS, precision=precision, out_every=EVERY,
                               ckpt_every=CKPT)
        L = ((occ - _target(tuple(occ.shape))) ** 2).sum()
        L.backward(retain_graph=True)
        first = (U.grad.clone(), tb.grad.clone())
        U.grad, tb.grad = None, None
        L.backward()
        # sums are reduced with atomics (in FP32 plans partly in FP32): equal
        # to rounding of the plan's precision
        sc, rt = float(first[1].abs().max()), (1e-12 if precision == 0 else 1e-6)
        assert abs(float(U.grad - first[0])) <= rt * sc
        assert float((tb.grad - first[1]).abs().max()) <= rt * sc
        assert n.grad is None
        res.append(np.concatenate([U.grad.reshape(1).numpy(), tb.grad.numpy()]))
    assert np.abs(res[1] - res[0]).max() <= 2e-3 * np.abs(res[0]).max()


def test_errors(ftwa):
    lat, n0 = _setup()
    with pytest.raises(ftwa.FtwaError):          # ckpt_every does not divide n_steps
        occ = ftwa.occupations(lat, torch.tensor(1.6, requires_grad=True), lat.t_bond, n0, SEED, M, STEPS,
                               out_every=EVERY, ckpt_every=30)
        occ.sum().backward()
    with pytest.raises(ftwa.FtwaError):          # occupation outside [0, 1]
        ftwa.occupations(lat, 1.6, lat.t_bond, n0 + 1.0, SEED, M, STEPS)


def test_correlations_autograd_matches_finite_differences(ftwa):
    """correlations(): a nonlinear loss of the occupations, the connected
    correlator and g2 (Eq. 10, formed in torch from occ and conn) differentiated
    by the RK4 adjoint (ftwa_adjoint_corr) against central differences of the
    wrapped forward (FP64, h = 1e-5, same seed): dL/dU, every dL/dt_b and
    every dL/dn0 to 1e-6 of the largest entry.  Occupations 0.2 / 0.8: g2
    divides by <n_k><n_l>, and near-empty sites make the loss so curved that
    central differences at h = 1e-5 are off by 1e-3."""
    lat, _ = _setup()
    nu, nd = W.neel_state(lat)
    n0 = np.stack([W.softened(nu, 0.2), W.softened(nd, 0.2)])
    tb0 = np.array(lat.t_bond, dtype=np.float64)
    rng = np.random.default_rng(8)
    T, K = STEPS // EVERY + 1, 2 * lat.n_sites
    w_c = torch.from_numpy(rng.standard_normal((T, K, K))).cuda()
    w_g = torch.from_numpy(rng.standard_normal((T, K, K)) * 0.01).cuda()

    def loss(U, tb, n):
        occ, conn = ftwa.correlations(lat, U, tb, n, SEED, M, STEPS, out_every=EVERY, ckpt_every=CKPT)
        nn = occ[:, :, None] * occ[:, None, :]
        g2 = (conn + nn) / nn
        return (occ ** 2).sum() + (w_c * conn).sum() + (w_c * conn ** 2).sum() + (w_g * g2).sum()

    U = torch.tensor(1.6, dtype=torch.float64, requires_grad=True)
    tb = torch.tensor(tb0, requires_grad=True)
    n = torch.tensor(n0, requires_grad=True)
    L = loss(U, tb, n)
    L.backward()
    h = 1e-5
    with torch.no_grad():
        def f(du=0.0, dt=None, dn=None):
            return float(loss(torch.tensor(1.6 + du, dtype=torch.float64),
                              torch.tensor(tb0 + (0 if dt is None else dt)),
                              torch.tensor(n0 + (0 if dn is None else dn))))
        fdU = (f(du=h) - f(du=-h)) / (2 * h)
        fdt = np.array([(f(dt=h * e) - f(dt=-h * e)) / (2 * h) for e in np.eye(lat.n_bonds)])
        fdn = np.zeros_like(n0)
        for s in range(2):
            for i in range(lat.n_sites):
                e = np.zeros_like(n0)
                e[s, i] = h
                fdn[s, i] = (f(dn=e) - f(dn=-e)) / (2 * h)
    scale = max(abs(fdU), np.abs(fdt).max(), np.abs(fdn).max())
    assert abs(U.grad.item() - fdU) <= 1e-6 * scale
    assert np.abs(tb.grad.numpy() - fdt).max() <= 1e-6 * scale
    assert np.abs(n.grad.numpy() - fdn).max() <= 1e-6 * scale
