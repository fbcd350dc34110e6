"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each check uses a closed form,
a value printed in the paper, an invariant of the flow, an independent
implementation of a different equation (Hartree-Fock), or exact
diagonalisation.
"""

import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import closed_forms as cf
from oracle.ed import HubbardED
from tests.conftest import read_golden


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------- sampler
def test_philox_known_answers():
    for row in read_golden("philox4x32_10_kat.txt"):
        words = [int(x, 16) for x in row]
        out = oracle.philox4x32_10(words[0:4], words[4:6])
        assert out.tolist() == words[6:10]


def test_philox_counter_layout():
    """Block output equals single calls at counter (m_lo, m_hi, spin, p)."""
    seed, m = 0x1234_5678_9ABC_DEF0, (3 << 32) + 17
    blk = oracle.philox_block(seed, m, 1, 5, 3)
    for q in range(3):
        ref = oracle.philox4x32_10([m & 0xFFFFFFFF, m >> 32, 1, 5 + q], [seed & 0xFFFFFFFF, seed >> 32])
        assert blk[q].tolist() == ref.tolist()


def test_complex_normal_moments():
    """xi is standard complex normal: E xi = 0, E|xi|^2 = 1, E xi^2 = 0
    (Re, Im i.i.d. N(0, 1/2)), as fixed by the covariance of App. A.3."""
    N = 12
    iu = (slice(None),) + np.triu_indices(N, 1)
    xs = np.concatenate([oracle.normals(N, 7, m)[iu].ravel() for m in range(3000)])
    n = xs.size
    assert abs(xs.mean()) < 5 / math.sqrt(n)
    assert abs(np.mean(np.abs(xs) ** 2) - 1.0) < 5 * math.sqrt(1.0 / n)
    assert abs(np.mean(xs ** 2)) < 5 * math.sqrt(1.0 / n)
    # Box-Muller output is Gaussian: 4th moment E|xi|^4 = 2 for a standard complex normal
    assert abs(np.mean(np.abs(xs) ** 4) - 2.0) < 6 * math.sqrt(20.0 / n)
    from scipy import stats
    assert stats.kstest(np.sqrt(2) * xs.real, "norm").pvalue > 1e-4


def test_sample_structure_eq12():
    """Eq. 7: rho_ii = n_i - 1/2; rho Hermitian; rho_ij = xi_ij s_ij with
    s_ij = sqrt((n_i + n_j - 2 n_i n_j)/2)."""
    lat = W.hexagon_chain(2)
    rng = np.random.default_rng(0)
    nu, nd = rng.uniform(size=10), rng.uniform(size=10)
    rho = oracle.sample(10, nu, nd, 99, 5)
    xi = oracle.normals(10, 99, 5)
    for s, n in enumerate([nu, nd]):
        assert np.allclose(np.diag(rho[s]).real, n - 0.5, atol=0, rtol=0)
        assert np.array_equal(rho[s], rho[s].conj().T)
        iu = np.triu_indices(10, 1)
        sd = np.sqrt((n[:, None] + n[None, :] - 2 * n[:, None] * n[None, :]) / 2)
        assert np.allclose(rho[s][iu], xi[s][iu] * sd[iu], rtol=1e-15, atol=0)


def test_sample_covariance_fock():
    """E|rho_ij|^2 = (n_i + n_j - 2 n_i n_j)/2: 1/2 for a filled/empty pair, 0 otherwise."""
    lat = W.periodic_honeycomb()
    nu, nd = W.neel_state(lat)
    acc = np.zeros((2, 8, 8))
    M = 4000
    for m in range(M):
        acc += np.abs(oracle.sample(8, nu, nd, 3, m)) ** 2
    acc /= M
    for s, n in enumerate([nu, nd]):
        expect = (n[:, None] + n[None, :] - 2 * n[:, None] * n[None, :]) / 2
        np.fill_diagonal(expect, (n - 0.5) ** 2)
        assert np.max(np.abs(acc[s] - expect)) < 5 * math.sqrt(1.0 / M)
        zero = expect == 0
        assert np.all(acc[s][zero] == 0)


# ---------------------------------------------------------------- equations of motion
def test_rk4_closed_form_U0():
    """U = 0: the oracle's RK4 equals the eigenbasis closed form to 1e-12 per trajectory."""
    for lat in [W.periodic_honeycomb(), W.hexagonal_flake(2), W.brick_wall_flake(3, 6)]:
        nu, nd = W.neel_state(lat)
        rho0 = oracle.sample(lat.n_sites, nu, nd, 11, 2)
        rho, _ = oracle.evolve(lat, 0.0, rho0, 0.01, 1000)
        assert _rel(rho, cf.rk4_free(lat, rho0, 0.01, 1000)) < 1e-12


def test_exact_propagator_U0():
    """U = 0: fTWA is exact; with a step small enough that RK4's error is below
    1e-13 the oracle matches rho(t) = W rho0 W^dagger, W = exp(-iJt), to 1e-12."""
    lat = W.periodic_honeycomb()
    nu, nd = W.neel_state(lat)
    rho0 = oracle.sample(8, nu, nd, 5, 0)
    rho, _ = oracle.evolve(lat, 0.0, rho0, 2.5e-4, 4000)
    assert _rel(rho, cf.exact_free(lat, rho0, 1.0)) < 1e-12


def test_initial_derivative_paper_value():
    """App. C: for a filled site 1 and an empty neighbour 2 (Neel start),
    d rho_12,up/dt (0) = -i U xi_12 / sqrt(2) + i j_12, exactly."""
    lat = W.hexagon_chain(2)
    nu, nd = W.neel_state(lat)
    U = 1.3
    rho0 = oracle.sample(10, nu, nd, 21, 4)
    xi = oracle.normals(10, 21, 4)
    f = oracle.rhs(lat, U, rho0)
    checked = 0
    for (i, j), t in zip(lat.bonds, lat.t_bond):
        a, b = (i, j) if nu[i] > 0.5 else (j, i)      # a filled (up), b empty (up)
        x = xi[0][a, b] if a < b else np.conj(xi[0][b, a])
        expect = -1j * U * x / math.sqrt(2) + 1j * t
        assert abs(f[0][a, b] - expect) < 1e-14
        checked += 1
    assert checked == lat.n_bonds


def test_short_time_taylor_paper():
    """Eq. C3 (ro11u): rho_11(eps) to second order; the residual is O(eps^3)."""
    lat = W.brick_wall_flake(4, 6)
    nu, nd = W.neel_state(lat)
    U = 1.6
    rho0 = oracle.sample(lat.n_sites, nu, nd, 8, 1)
    xi = oracle.normals(lat.n_sites, 8, 1)
    site = 7                          # interior site, filled with spin up
    assert nu[site] == 1
    nb = [(j if i == site else i, t) for (i, j), t in zip(lat.bonds, lat.t_bond) if site in (i, j)]
    j1 = [t for _, t in nb]
    x1 = [xi[0][site, k] if site < k else np.conj(xi[0][k, site]) for k, _ in nb]
    res = []
    for eps in [0.02, 0.01]:
        rho, _ = oracle.evolve(lat, U, rho0, eps / 200, 200)
        res.append(abs(rho[0][site, site].real - cf.rho11_taylor(eps, j1, x1, U)))
    assert res[0] < 1e-4
    assert 5.5 < res[0] / res[1] < 11.0      # third-order residual: ratio ~ 8


def test_hartree_fock_identity():
    """Sec. III.A: with zero noise the fTWA flow is Hartree-Fock.  Eq. A6
    (Heis_HF2) is integrated here independently on n = rho + 1/2 and compared."""
    lat = W.hexagon_chain(2)
    nu, nd = W.neel_state(lat)
    U, dt, steps = 1.6, 0.01, 300
    J = cf.hopping_matrix(lat)
    rho0 = np.stack([np.diag(nu - 0.5), np.diag(nd - 0.5)]).astype(np.complex128)
    rho0[0][2, 5] = rho0[0][5, 2] = 0.1          # a non-trivial (not stationary) HF state
    rho, _ = oracle.evolve(lat, U, rho0, dt, steps)

    def hf_rhs(n):
        # d/dt n_ij,s = i sum_l (j_jl n_il,s - j_li n_lj,s + (u_il - u_lj) n_ll,sbar n_ij,s)
        out = np.empty_like(n)
        for s in range(2):
            d = np.real(np.diag(n[1 - s]))
            out[s] = 1j * (n[s] @ J - J @ n[s] + U * (d[:, None] - d[None, :]) * n[s])
        return out

    n = rho0 + 0.5 * np.eye(10)[None]
    for _ in range(steps):
        k1 = hf_rhs(n)
        k2 = hf_rhs(n + dt / 2 * k1)
        k3 = hf_rhs(n + dt / 2 * k2)
        k4 = hf_rhs(n + dt * k3)
        n = n + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    assert _rel(rho + 0.5 * np.eye(10)[None], n) < 1e-13


def test_invariants_per_trajectory():
    """Per trajectory: trace per spin is conserved, rho stays Hermitian, and the
    classical energy H_W (Eq. A10) and the spectrum of each rho_s drift only by
    the RK4 error (halving dt cuts the drift by ~16)."""
    lat = W.hexagonal_flake(2)
    nu, nd = W.neel_state(lat)
    U = 1.6
    rho0 = oracle.sample(lat.n_sites, nu, nd, 4, 9)
    e0 = oracle.energy(lat, U, rho0)
    ev0 = [np.linalg.eigvalsh(rho0[s]) for s in range(2)]
    drift_e, drift_ev = [], []
    for dt, steps in [(0.04, 250), (0.02, 500)]:
        rho, _ = oracle.evolve(lat, U, rho0, dt, steps)
        for s, n in enumerate([nu, nd]):
            assert abs(np.trace(rho[s]) - (n.sum() - lat.n_sites / 2)) < 1e-11
            # the two neighbour sums of Eq. 6 associate differently for
            # (i, j) and (j, i), so Hermiticity holds to rounding
            assert np.max(np.abs(rho[s] - rho[s].conj().T)) < 1e-13
        e = oracle.energy(lat, U, rho)
        assert abs(e.imag) < 1e-12
        drift_e.append(abs(e.real - e0.real))
        drift_ev.append(max(np.max(np.abs(np.linalg.eigvalsh(rho[s]) - ev0[s])) for s in range(2)))
    assert drift_e[0] < 1e-3 and drift_ev[0] < 1e-3
    assert 10 < drift_e[0] / drift_e[1] < 24
    assert 10 < drift_ev[0] / drift_ev[1] < 24


# ---------------------------------------------------------------- exact diagonalisation
def test_ed_dimer_closed_form():
    for U in [0.0, 1.6, 4.0]:
        lat = W.dimer()
        ed = HubbardED(lat, U, 1, 1)
        assert np.allclose(ed.eigenvalues(), cf.dimer_eigenvalues(U), atol=1e-12)


def test_ed_free_fermions():
    """ED at U = 0 against the one-body propagator and Wick's theorem (Eq. A4)."""
    lat = W.periodic_honeycomb()
    nu, nd = W.neel_state(lat)
    ed = HubbardED(lat, 0.0, 4, 4)
    psi0 = np.zeros(ed.dim, dtype=np.complex128)
    psi0[ed.fock_index(nu, nd)] = 1
    times = np.linspace(0, 2, 5)
    occ, nn = ed.observables(ed.evolve(psi0, times))
    for k, t in enumerate(times):
        n1 = cf.free_fermion_one_body(lat, nu, t)
        assert np.allclose(occ[k][:8], np.real(np.diag(n1)), atol=1e-9)
        w = cf.wick_same_spin(n1)
        off = ~np.eye(8, dtype=bool)
        assert np.allclose(nn[k][:8, :8][off], w[off], atol=1e-9)


def test_ftwa_statistics_equal_exact_at_U0():
    """U = 0: fTWA sample means equal the exact free-fermion <n_i>(t) and the
    same-spin <n_i n_j>(t) of Wick's theorem (Eq. 5 estimators), within the
    sampling error (|z| < 5)."""
    lat = W.periodic_honeycomb()
    nu, nd = W.neel_state(lat)
    M = 4000
    snap, _ = oracle.run(lat, 0.0, nu, nd, 17, 0, M, 0.01, 200, 50)
    occ, conn, _ = oracle.moments(snap, want_g2=False)
    for k in range(snap.shape[0]):
        t = k * 0.5
        n1 = cf.free_fermion_one_body(lat, nu, t)
        se = np.sqrt(conn[k].diagonal()[:8] / M) + 1e-12
        z = (occ[k][:8] - np.real(np.diag(n1))) / se
        assert np.max(np.abs(z)) < 5
        if t > 0:
            x = snap[k][:, :8] + 0.5
            nn = (x[:, :, None] * x[:, None, :]).mean(axis=0)
            nn_se = (x[:, :, None] * x[:, None, :]).std(axis=0) / math.sqrt(M)
            w = cf.wick_same_spin(n1)
            off = ~np.eye(8, dtype=bool)
            z = (nn[off] - w[off]) / (nn_se[off] + 1e-12)
            assert np.max(np.abs(z)) < 5


# ---------------------------------------------------------------- estimators
def test_moments_definitions():
    rng = np.random.default_rng(1)
    X = rng.normal(size=(3, 500, 6)) * 0.3
    occ, conn, g2 = oracle.moments(X)
    for t in range(3):
        assert np.allclose(occ[t], X[t].mean(axis=0) + 0.5, rtol=1e-14)
        assert np.allclose(conn[t], np.cov(X[t].T, bias=True), rtol=1e-12, atol=1e-15)
        x = X[t] + 0.5
        g = (x.T @ x / 500) / np.outer(x.mean(0), x.mean(0))
        assert np.allclose(g2[t], g, rtol=1e-12)


def _g2_delta_se(x, k, l):
    """Standard error of the ratio estimator mean(x_k x_l) / (mean(x_k) mean(x_l))
    by the delta method (per-sample influence function), from the samples."""
    a, b = x[:, k], x[:, l]
    A, B, C = np.mean(a * b), a.mean(), b.mean()
    psi = (a * b - A) / (B * C) - A * (a - B) / (B * B * C) - A * (b - C) / (B * C * C)
    return psi.std() / math.sqrt(x.shape[0])


def test_g2_estimator_equals_wick_at_U0():
    """Eq. 10 (g2_fTWA) pinned without the estimator's own formula: at U = 0 the
    method is exact for the quadratic Hamiltonian, so the oracle's g2 output
    must equal the free-fermion value.  Same spin, Wick (Eq. A4):
    g2_ij = 1 - |n_ij|^2 / (n_ii n_jj) with n(t) = W diag(n0) W^dagger;
    opposite spin: the up and down Slater determinants are independent, so
    g2 = 1 exactly.  |z| < 5 with the delta-method standard error of the ratio
    (pairs with an occupation below 0.05 are skipped: the ratio is ill
    conditioned there)."""
    lat = W.periodic_honeycomb()
    nu, nd = W.neel_state(lat)
    N, M = 8, 20000
    snap, _ = oracle.run(lat, 0.0, nu, nd, 23, 0, M, 0.01, 300, 50)
    _, _, g2 = oracle.moments(snap)
    checked = 0
    for k in range(1, snap.shape[0]):
        t = 0.5 * k
        x = snap[k] + 0.5
        n_up = cf.free_fermion_one_body(lat, nu, t)
        n_dn = cf.free_fermion_one_body(lat, nd, t)
        for s, nm in ((0, n_up), (1, n_dn)):
            d = np.real(np.diag(nm))
            for i in range(N):
                for j in range(N):
                    if i == j or d[i] < 0.05 or d[j] < 0.05:
                        continue
                    exact = 1.0 - abs(nm[i, j]) ** 2 / (d[i] * d[j])
                    kk, ll = s * N + i, s * N + j
                    z = (g2[k][kk, ll] - exact) / _g2_delta_se(x, kk, ll)
                    assert abs(z) < 5, (t, s, i, j, g2[k][kk, ll], exact)
                    checked += 1
        du, dd = np.real(np.diag(n_up)), np.real(np.diag(n_dn))
        for i in range(N):
            for j in range(N):
                if du[i] < 0.05 or dd[j] < 0.05:
                    continue
                z = (g2[k][i, N + j] - 1.0) / _g2_delta_se(x, i, N + j)
                assert abs(z) < 5, (t, i, j, g2[k][i, N + j])
                checked += 1
    assert checked > 500


def test_g2_short_time_limit_app_c():
    """App. C, Eq. C8 (form_g_st_2): for a filled site next to an empty site
    whose three bonds all have hopping j, the same-spin g2 tends to
    (3 j^2 - j^2) / (3 j^2) = 2/3 as t -> 0+ (independent of U).  Statistical
    check of the oracle's g2 at t = 0.05 on the 8-site periodic lattice
    (Neel start, U = 1.6): the mean over the 12 bonds, spin up, is within 0.02
    of 2/3 (sampling error about 0.004 at M = 200000; the O(t) correction is
    smaller)."""
    vals = {r[0]: float(r[1]) for r in read_golden("paper_values.txt")}
    lat = W.periodic_honeycomb()
    nu, nd = W.neel_state(lat)
    snap, _ = oracle.run(lat, 1.6, nu, nd, 29, 0, 200000, 0.01, 5, 5)
    _, _, g2 = oracle.moments(snap)
    bond_vals = [g2[1][i, j] for (i, j) in lat.bonds]
    assert abs(np.mean(bond_vals) - vals["g2_short_time_three_neighbours"]) < 0.02


def test_paper_asymptotes():
    vals = {r[0]: float(r[1]) for r in read_golden("paper_values.txt")}
    for n in [4, 6, 10]:
        assert abs(cf.g2_long_time(n) - vals[f"g2_long_time_n{n}"]) < 1e-12
    assert round(cf.g2_long_time(198), 3) == vals["g2_long_time_n198"]
    assert abs(cf.g2_short_time(1.0, [1.0, 1.0]) - vals["g2_short_time_two_neighbours"]) < 1e-15
    assert abs(cf.g2_short_time(1.0, [1.0, 1.0, 1.0]) - vals["g2_short_time_three_neighbours"]) < 1e-15


def test_fd_gradient_converges():
    """Central differences with common random numbers: halving h changes the
    U-derivative only at O(h^2)."""
    lat = W.periodic_honeycomb()
    nu, nd = W.neel_state(lat)
    tgt = np.full((2, 16), 0.5)
    g1 = oracle.fd_gradient(lat, 1.6, nu, nd, 3, 8, 0.01, 40, 20, tgt, [("U",), ("t", 0)], h=1e-3)
    g2 = oracle.fd_gradient(lat, 1.6, nu, nd, 3, 8, 0.01, 40, 20, tgt, [("U",), ("t", 0)], h=5e-4)
    assert np.all(np.abs(g1 - g2) <= 1e-5 * np.maximum(1, np.abs(g2)))


# ---- general (non-diagonal) initial states ---------------------------------------
def test_general_sampler_identity_basis_is_eq7():
    """With V = 1 the general sampler is the diagonal sampler of Eq. 7."""
    lat = W.hexagon_chain(2)
    nu, nd = W.softened(W.neel_state(lat)[0]), W.softened(W.neel_state(lat)[1])
    V = np.stack([np.eye(lat.n_sites), np.eye(lat.n_sites)]).astype(np.complex128)
    for m in range(3):
        a = oracle.sample_general(lat.n_sites, np.stack([nu, nd]), V, 11, m)
        b = oracle.sample(lat.n_sites, nu, nd, 11, m)
        assert np.array_equal(a, b)


def test_general_sampler_moments_match_app_a_covariance():
    """Statistics of the general sampler (random complex basis, fractional
    eigen-occupations, 40000 samples): the mean is n - 1/2 and
    cov(rho*_ab, rho_mn) is the covariance of App. A minus the eigen-diagonal
    part that Eq. 7 leaves noiseless (|z| < 5); the trace and Hermiticity
    hold per sample."""
    N, K = 4, 40000
    lam, V = W.random_basis(N, 3, [0.1, 0.6, 0.9, 0.3], [0.2, 0.5, 0.7, 1.0])
    X = np.stack([oracle.sample_general(N, lam, V, 7, m) for m in range(K)])
    for s in range(2):
        assert np.abs(np.trace(X[:, s], axis1=1, axis2=2) - (lam[s].sum() - N / 2)).max() < 1e-12
        assert np.abs(X[:, s] - np.conj(np.transpose(X[:, s], (0, 2, 1)))).max() < 1e-14
        n = (V[s] * lam[s][None, :]) @ V[s].conj().T
        mean = X[:, s].mean(axis=0)
        se = np.maximum(X[:, s].std(axis=0) / np.sqrt(K), 1e-12)
        assert (np.abs(mean - (n - 0.5 * np.eye(N))) / se).max() < 5
        idx = [(0, 1, 0, 1), (0, 1, 2, 3), (1, 1, 2, 2), (0, 2, 0, 2), (3, 0, 1, 2), (2, 2, 2, 2), (0, 0, 1, 1)]
        want = cf.general_state_covariance(lam[s], V[s], idx)
        D = X[:, s] - mean
        for (a, b, m, k), w in zip(idx, want):
            prod = np.conj(D[:, a, b]) * D[:, m, k]
            sd = np.sqrt(np.var(prod.real) + np.var(prod.imag)) / np.sqrt(K)
            assert abs(prod.mean() - w) < 5 * sd + 1e-12


# ---- time-dependent on-site drive ----------------------------------------------
def _drive_case():
    lat = W.hexagon_chain(2)
    N = lat.n_sites
    rng = np.random.default_rng(4)
    amp = rng.uniform(-1.0, 1.0, (2, N))
    drive = dict(amp=amp, t0=1.2, sigma=0.5, omega=3.0, phase=0.4)
    nu, nd = W.softened(W.neel_state(lat)[0]), W.softened(W.neel_state(lat)[1])
    return lat, drive, oracle.sample(N, nu, nd, 5, 0)


def test_drive_phases_closed_form():
    """J = 0, U = 0: d rho_ij/dt = i (v_i - v_j) rho_ij, so
    rho_ij(t) = rho_ij(0) exp(i (a_i - a_j) F(t)), F the integral of the pulse
    (by quadrature); RK4 converges to it at fourth order in dt."""
    from scipy.integrate import quad
    lat, drive, r0 = _drive_case()
    tb = np.zeros(lat.n_bonds)
    T = 2.4
    F = quad(lambda t: np.exp(-(t - drive["t0"]) ** 2 / (2 * drive["sigma"] ** 2))
             * np.cos(drive["omega"] * (t - drive["t0"]) + drive["phase"]), 0.3, 0.3 + T, epsabs=1e-14)[0]
    amp = drive["amp"]
    want = np.stack([r0[s] * np.exp(1j * (amp[s][:, None] - amp[s][None, :]) * F) for s in range(2)])
    errs = []
    for dt in (0.02, 0.01):
        got, _ = oracle.evolve(lat, 0.0, r0, dt, int(round(T / dt)), t_bond=tb, drive=drive, t_start=0.3)
        errs.append(np.abs(got - want).max())
    assert errs[1] < 1e-8
    assert 10 < errs[0] / errs[1] < 24          # fourth order: ratio 16


def test_drive_neutral_cases():
    """Zero amplitudes, or equal amplitudes on every site, leave the
    trajectory unchanged (the drive enters only through v_i - v_j); a later
    start time equals an earlier pulse centre."""
    lat, drive, r0 = _drive_case()
    base, _ = oracle.evolve(lat, 1.6, r0, 0.01, 150)
    z = dict(drive, amp=np.zeros_like(drive["amp"]))
    assert np.array_equal(oracle.evolve(lat, 1.6, r0, 0.01, 150, drive=z)[0], base)
    u = dict(drive, amp=np.full_like(drive["amp"], 0.7))
    assert np.array_equal(oracle.evolve(lat, 1.6, r0, 0.01, 150, drive=u)[0], base)
    a, _ = oracle.evolve(lat, 1.6, r0, 0.01, 150, drive=drive, t_start=0.5)
    b, _ = oracle.evolve(lat, 1.6, r0, 0.01, 150, drive=dict(drive, t0=drive["t0"] - 0.5), t_start=0.0)
    assert np.abs(a - b).max() < 1e-12
    assert np.abs(a - base).max() > 1e-3          # and the drive does act


# ---- long-range interaction u_ij -------------------------------------------------
def test_longrange_reduces_to_onsite():
    """u = U 1 gives the on-site oracle (same trajectory to rounding)."""
    lat = W.hexagon_chain(2)
    nu, nd = W.neel_state(lat)
    r0 = oracle.sample(lat.n_sites, nu, nd, 2, 0)
    a, sa = oracle.evolve(lat, 1.6, r0, 0.01, 200, out_every=50)
    b, sb = oracle.evolve(lat, 0.0, r0, 0.01, 200, out_every=50, u=1.6 * np.eye(lat.n_sites))
    assert np.abs(a - b).max() < 1e-13 and np.abs(sa - sb).max() < 1e-13


def test_longrange_energy_conservation():
    """With a Coulomb-like u the energy of Eq. A10 with the full sum of Eq. 1
    is conserved by the flow: the RK4 drift falls at least at fourth order in
    dt (measured: fifth); and the tail changes the trajectory."""
    lat = W.hexagon_chain(2)
    nu, nd = W.softened(W.neel_state(lat)[0]), W.softened(W.neel_state(lat)[1])
    u = W.coulomb_interaction(lat, 1.6, 0.8)
    r0 = oracle.sample(lat.n_sites, nu, nd, 4, 0)
    e0 = cf.energy_longrange(lat, u, r0)
    drift = []
    for dt in (0.04, 0.02):
        r, _ = oracle.evolve(lat, 0.0, r0, dt, int(round(2.0 / dt)), u=u)
        drift.append(abs(cf.energy_longrange(lat, u, r) - e0))
    assert drift[1] < 1e-6
    assert drift[0] / drift[1] > 12
    onsite, _ = oracle.evolve(lat, 1.6, r0, 0.02, 100)
    assert np.abs(r - onsite).max() > 1e-3


def test_hopping_modulation_closed_form():
    """U = 0 with every hopping scaled by m(t) = 1 + eps g(t): h(t) = -m(t) J
    commutes with itself, so rho(t) = W rho0 W^dagger with W = exp(-i J M),
    M = int m(t) dt (quadrature); RK4 converges to it at fourth order."""
    from scipy.integrate import quad
    lat = W.hexagon_chain(2)
    nu, nd = W.softened(W.neel_state(lat)[0]), W.softened(W.neel_state(lat)[1])
    r0 = oracle.sample(lat.n_sites, nu, nd, 3, 0)
    hop = dict(eps=0.6, t0=1.0, sigma=0.5, omega=2.5, phase=0.2)
    drive = dict(amp=None, hop=hop)
    T, ts = 2.0, 0.4
    g = lambda t: np.exp(-(t - hop["t0"]) ** 2 / (2 * hop["sigma"] ** 2)) * np.cos(hop["omega"] * (t - hop["t0"]) + hop["phase"])
    Mt = T + hop["eps"] * quad(g, ts, ts + T, epsabs=1e-14)[0]
    want = cf.exact_free(lat, r0, Mt)
    errs = []
    for dt in (0.01, 0.005):
        got, _ = oracle.evolve(lat, 0.0, r0, dt, int(round(T / dt)), drive=drive, t_start=ts)
        errs.append(np.abs(got - want).max())
    assert errs[1] < 5e-8                       # the RK4 error of the undriven flow is of this size too
    assert errs[0] / errs[1] > 12
    z, _ = oracle.evolve(lat, 1.6, r0, 0.01, 100, drive=dict(amp=None, hop=dict(hop, eps=0.0)))
    assert np.array_equal(z, oracle.evolve(lat, 1.6, r0, 0.01, 100)[0])


def test_adjoint_oracle_forward_is_eq6():
    """The adjoint oracle's f (full matrices, numpy) is the C oracle's
    right-hand side of Eq. 6."""
    from oracle import adjoint as OA
    lat = W.hexagon_chain(2)
    nu, nd = W.softened(W.neel_state(lat)[0]), W.softened(W.neel_state(lat)[1])
    rho = oracle.sample(lat.n_sites, nu, nd, 5, 1)
    J = OA.hopping_matrix(lat)
    assert np.abs(OA.f(J, 1.6, rho) - oracle.rhs(lat, 1.6, rho)).max() <= 1e-14


@pytest.mark.parametrize("lat_name,U", [("chain10", 1.6), ("periodic8", 2.5)])
def test_adjoint_oracle_matches_finite_differences(lat_name, U):
    """The discrete RK4 adjoint of the oracle against central differences
    (h = 1e-5, same seed) of the C oracle's integration, for the linear loss
    L = sum_t sum_k g_tk <n_k>(t): dL/dU, every dL/dt_b and every dL/dn_is
    (softened occupations) to 1e-8 of the largest entry."""
    from oracle import adjoint as OA
    lat = {"chain10": W.hexagon_chain(2), "periodic8": W.periodic_honeycomb()}[lat_name]
    n0u, n0d = W.neel_state(lat)
    nu, nd = W.softened(n0u), W.softened(n0d)
    N, seed, M, steps, every = lat.n_sites, 5, 3, 30, 10
    g = np.random.default_rng(0).standard_normal((steps // every + 1, 2 * N))
    gU, gt, gn = OA.adjoint(lat, U, nu, nd, seed, M, 0.01, steps, every, g)
    tb0 = np.array(lat.t_bond, dtype=np.float64)

    def L(u, tb, a, b):
        snap, _ = oracle.run(lat, u, a, b, seed, 0, M, 0.01, steps, every, t_bond=tb)
        return float((g * (snap.mean(axis=1) + 0.5)).sum())

    h = 1e-5
    fdU = (L(U + h, tb0, nu, nd) - L(U - h, tb0, nu, nd)) / (2 * h)
    fdt = np.array([(L(U, tb0 + h * e, nu, nd) - L(U, tb0 - h * e, nu, nd)) / (2 * h)
                    for e in np.eye(lat.n_bonds)])
    fdn = np.zeros((2, N))
    for s in range(2):
        for i in range(N):
            e = np.zeros(N)
            e[i] = h
            if s == 0:
                fdn[s, i] = (L(U, tb0, nu + e, nd) - L(U, tb0, nu - e, nd)) / (2 * h)
            else:
                fdn[s, i] = (L(U, tb0, nu, nd + e) - L(U, tb0, nu, nd - e)) / (2 * h)
    scale = max(abs(fdU), np.abs(fdt).max(), np.abs(fdn).max())
    assert abs(gU - fdU) <= 1e-8 * scale
    assert np.abs(gt - fdt).max() <= 1e-8 * scale
    assert np.abs(gn - fdn).max() <= 1e-8 * scale


@pytest.mark.parametrize("lat_name,U", [("chain10", 1.6), ("periodic8", 2.5)])
def test_adjoint_oracle_correlation_loss_matches_finite_differences(lat_name, U):
    """Correlation losses (Eq. 5's connected correlator): the oracle's RK4
    adjoint with the per-sample cotangent (1/M) sum_l (gC_jl + gC_lj)(x_ml -
    mu_l) against central differences (h = 1e-5, same seed) of
    L = sum_t sum_kl gC_tkl C_kl(t) + sum_t sum_k g_tk <n_k>(t), C taken from
    the C oracle's moments (a non-symmetric random weight gC): dL/dU, every
    dL/dt_b and every dL/dn_is to 1e-8 of the largest entry."""
    from oracle import adjoint as OA
    lat = {"chain10": W.hexagon_chain(2), "periodic8": W.periodic_honeycomb()}[lat_name]
    n0u, n0d = W.neel_state(lat)
    nu, nd = W.softened(n0u), W.softened(n0d)
    N, seed, M, steps, every = lat.n_sites, 6, 4, 30, 10
    rng = np.random.default_rng(2)
    T = steps // every + 1
    g = rng.standard_normal((T, 2 * N))
    gC = rng.standard_normal((T, 2 * N, 2 * N))
    snap, _ = oracle.run(lat, U, nu, nd, seed, 0, M, 0.01, steps, every)
    mu = snap.mean(axis=1)
    gU, gt, gn = OA.adjoint(lat, U, nu, nd, seed, M, 0.01, steps, every, g, gC=gC, mu=mu)
    tb0 = np.array(lat.t_bond, dtype=np.float64)

    def L(u, tb, a, b):
        s, _ = oracle.run(lat, u, a, b, seed, 0, M, 0.01, steps, every, t_bond=tb)
        occ, conn, _ = oracle.moments(s, want_g2=False)
        return float((g * occ).sum() + (gC * conn).sum())

    h = 1e-5
    fdU = (L(U + h, tb0, nu, nd) - L(U - h, tb0, nu, nd)) / (2 * h)
    fdt = np.array([(L(U, tb0 + h * e, nu, nd) - L(U, tb0 - h * e, nu, nd)) / (2 * h)
                    for e in np.eye(lat.n_bonds)])
    fdn = np.zeros((2, N))
    for s in range(2):
        for i in range(N):
            e = np.zeros(N)
            e[i] = h
            if s == 0:
                fdn[s, i] = (L(U, tb0, nu + e, nd) - L(U, tb0, nu - e, nd)) / (2 * h)
            else:
                fdn[s, i] = (L(U, tb0, nu, nd + e) - L(U, tb0, nu, nd - e)) / (2 * h)
    scale = max(abs(fdU), np.abs(fdt).max(), np.abs(fdn).max())
    assert abs(gU - fdU) <= 1e-8 * scale
    assert np.abs(gt - fdt).max() <= 1e-8 * scale
    assert np.abs(gn - fdn).max() <= 1e-8 * scale
