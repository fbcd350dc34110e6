"""GPU parity: the CUDA path, called through the C ABI, against the CPU oracle
on the same seeded inputs.

Tolerances:
 - integer stage (Philox words): bit-exact;
 - FP64 sampler: |rho_gpu - rho_oracle| <= 1e-14 (both evaluate log, sqrt,
   cos/sin in double; a few ulp of the O(1) normals);
 - FP64 trajectories: ||rho_gpu - rho_oracle||_F / ||rho_oracle||_F <= 1e-10
   per sample at T = 10 (1000 RK4 steps, dt = 0.01);
 - FP32 trajectories: <= 1e-4 relative after 100 steps (float rounding,
   ~1e-7 per step, amplified by the flow);
 - FP64 moments: 1e-12 relative (same data, different summation order).
"""

import math

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


def _oracle_states(lat, nu, nd, seed, M):
    return np.stack([oracle.sample(lat.n_sites, nu, nd, seed, m) for m in range(M)])


# ------------------------------------------------------------------ sampler
def test_philox_bit_exact(ftwa):
    for seed, m, spin, p0, count in [(0, 0, 0, 0, 64), (2**64 - 1, 2**40 + 3, 1, 12345, 100),
                                     (0x243F6A8885A308D3, 7, 0, 2**31 - 5, 10)]:
        g = ftwa.philox(seed, m, spin, p0, count).cpu().numpy().astype(np.uint32)
        o = oracle.philox_block(seed, m, spin, p0, count)
        assert np.array_equal(g, o)


@pytest.mark.parametrize("precision", [0, 1])
def test_sample_parity(ftwa, precision):
    lat = W.hexagonal_flake(2)
    rng = np.random.default_rng(3)
    nu, nd = rng.uniform(size=24), rng.uniform(size=24)
    nu[:4] = [0, 1, 0, 1]                       # Fock entries give s_ij = 0 pairs
    nd[:4] = [1, 1, 0, 0]
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=precision) as P:
        rho = P.sample(seed=77, M=5, first_sample=3).cpu().numpy()
    ref = np.stack([oracle.sample(24, nu, nd, 77, 3 + m) for m in range(5)])
    if precision == 0:
        assert np.max(np.abs(rho - ref)) <= 1e-14
    else:
        assert np.max(np.abs(rho - ref)) <= 2e-6


def test_sample_independent_of_split(ftwa):
    """Sample m depends only on (seed, m): drawing [0, 10) at once or as
    [0, 4) + [4, 10) gives the same states (what lets ranks shard samples)."""
    lat = W.hexagonal_flake(2)
    nu, nd = W.neel_state(lat)
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=0) as P:
        full = P.sample(5, 10)
        a = P.sample(5, 4, first_sample=0)
        b = P.sample(5, 6, first_sample=4)
    assert torch.equal(full, torch.cat([a, b]))


# ------------------------------------------------------------------ stepper
CASES = [
    ("periodic8", lambda: W.periodic_honeycomb(), 1.6, "neel", 7),
    ("hexflake24", lambda: W.hexagonal_flake(2), 1.6, "neel", 5),
    ("hexchain10_thermal", lambda: W.hexagon_chain(2), 2.5, "thermal", 3),
]


def _state(lat, kind):
    if kind == "neel":
        return W.neel_state(lat)
    rng = np.random.default_rng(11)
    return rng.uniform(size=lat.n_sites), rng.uniform(size=lat.n_sites)


@pytest.mark.parametrize("name,make,U,kind,M", CASES)
def test_evolve_fp64_matches_oracle(ftwa, name, make, U, kind, M):
    """Per trajectory, FP64, T = 10 (1000 steps), snapshots every 10 steps."""
    lat = make()
    nu, nd = _state(lat, kind)
    seed, steps, every = 1, 1000, 10
    snap_o, fin_o = oracle.run(lat, U, nu, nd, seed, 0, M, 0.01, steps, every, want_final=True)
    with ftwa.Plan(lat, U, n_up=nu, n_dn=nd, precision=0, out_every=every) as P:
        rho = P.sample(seed, M)
        X = P.evolve(rho, steps)
        assert P.status() == 0
        fin = rho.cpu().numpy()
        X = X.cpu().numpy()
    for m in range(M):
        assert _rel(fin[m], fin_o[m]) <= 1e-10, (name, m, _rel(fin[m], fin_o[m]))
    assert np.max(np.abs(X - snap_o)) <= 1e-10


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("cluster", [1, 2, 4, 8])
def test_evolve_cluster_shapes(ftwa, cluster, variant):
    """Both steppers (1: banded, 2: packed triangle), every cluster split of
    the spin-rows: the oracle's trajectory (oracle-drawn rho(0) fed to the
    GPU; ragged M)."""
    lat = W.hexagonal_flake(3)          # 54 sites
    nu, nd = W.neel_state(lat)
    M, steps = 3, 200
    rho0 = _oracle_states(lat, nu, nd, 9, M)
    fin_o = np.stack([oracle.evolve(lat, 1.6, rho0[m], 0.01, steps)[0] for m in range(M)])
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=0, cluster=cluster, variant=variant) as P:
        assert P.info()["cluster"] == cluster and P.info()["variant"] == variant
        rho = torch.from_numpy(rho0).cuda()
        P.evolve(rho, steps, snap=None)
        assert P.status() == 0
        fin = rho.cpu().numpy()
    for m in range(M):
        assert _rel(fin[m], fin_o[m]) <= 1e-11


@pytest.mark.parametrize("variant", [1, 2])
def test_evolve_198_sites_fp64(ftwa, variant):
    """The 198-site brick-wall flake, charge-imbalanced start: a few sampled
    trajectories, full T = 10."""
    lat = W.brick_wall_flake()
    nu, nd = W.charge_imbalanced_state(lat)
    M, steps = 2, 1000
    snap_o, fin_o = oracle.run(lat, 1.6, nu, nd, 2, 0, M, 0.01, steps, 100, want_final=True)
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=0, out_every=100, variant=variant) as P:
        rho = P.sample(2, M)
        X = P.evolve(rho, steps)
        assert P.status() == 0
        fin = rho.cpu().numpy()
    for m in range(M):
        assert _rel(fin[m], fin_o[m]) <= 1e-10
    assert np.max(np.abs(X.cpu().numpy() - snap_o)) <= 1e-10


def _tile_fits(lat, cluster):
    """Whether the tiled stepper (variant 3) has a decomposition for this
    lattice and cluster size (host-side check, no launch)."""
    import ctypes
    from paper_2212_04352_gb300 import _lib as L
    b = np.ascontiguousarray(lat.bonds, dtype=np.int32)
    v = ctypes.c_int64()
    return L.load().ftwa_debug_tile_check(lat.n_sites, len(b), b.ctypes.data, None, cluster, 1, ctypes.byref(v),
                                          None, 0) == 0


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("lat_name", ["periodic8", "brick198"])
def test_evolve_fp32_short(ftwa, lat_name, variant):
    lat = W.periodic_honeycomb() if lat_name == "periodic8" else W.brick_wall_flake()
    nu, nd = W.neel_state(lat)
    M, steps = 3, 100
    rho0 = _oracle_states(lat, nu, nd, 4, M)
    fin_o = np.stack([oracle.evolve(lat, 1.6, rho0[m], 0.01, steps)[0] for m in range(M)])
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=1, variant=variant) as P:
        assert P.info()["variant"] == variant
        rho = torch.from_numpy(rho0.astype(np.complex64)).cuda()
        P.evolve(rho, steps, snap=None)
        assert P.status() == 0
        fin = rho.cpu().numpy().astype(np.complex128)
    for m in range(M):
        assert _rel(fin[m], fin_o[m]) <= 1e-4


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("cluster", [1, 2, 4, 8])
@pytest.mark.parametrize("lat_name", ["chain7", "brick35", "flake54", "flake96", "brick198"])
def test_evolve_fp32_shapes(ftwa, lat_name, cluster, variant):
    """FP32 steppers (1: banded, 2: packed triangle, 3: tiled) on odd and
    even lattice sizes (ragged first column block), lattices with and without
    the p -+ 1 neighbour order, and every cluster split that fits; ragged M."""
    lat = {"chain7": W.chain(7), "brick35": W.brick_wall_flake(5, 7), "flake54": W.hexagonal_flake(3),
           "flake96": W.hexagonal_flake(4), "brick198": W.brick_wall_flake()}[lat_name]
    if lat.n_sites > 60 and variant != 3:
        pytest.skip("large lattices: tiled stepper only (the others are covered above)")
    if variant == 3 and not _tile_fits(lat, cluster):
        pytest.skip("no tiled decomposition for this cluster size")
    nu, nd = W.neel_state(lat)
    M, steps = 5, 100
    rho0 = _oracle_states(lat, nu, nd, 21, M)
    fin_o = np.stack([oracle.evolve(lat, 1.6, rho0[m], 0.01, steps)[0] for m in range(M)])
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=1, cluster=cluster, variant=variant) as P:
        assert P.info()["cluster"] == cluster and P.info()["variant"] == variant
        rho = torch.from_numpy(rho0.astype(np.complex64)).cuda()
        P.evolve(rho, steps, snap=None)
        assert P.status() == 0
        fin = rho.cpu().numpy().astype(np.complex128)
    for m in range(M):
        assert _rel(fin[m], fin_o[m]) <= 1e-4, (m, _rel(fin[m], fin_o[m]))
        for sp in range(2):
            assert np.array_equal(fin[m, sp], fin[m, sp].conj().T)


def test_hermitian_output_and_trace(ftwa):
    lat = W.hexagonal_flake(2)
    nu, nd = W.neel_state(lat)
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=0) as P:
        rho = P.sample(5, 4)
        P.evolve(rho, 300, snap=None)
        r = rho.cpu().numpy()
    for m in range(4):
        for s, n in enumerate([nu, nd]):
            assert np.array_equal(r[m, s], r[m, s].conj().T)
            assert abs(np.trace(r[m, s]) - (n.sum() - 12)) < 1e-11


def test_edge_cases(ftwa):
    lat = W.dimer()
    with ftwa.Plan(lat, 1.0, n_up=[1, 0], n_dn=[0, 1], precision=0) as P:
        rho = P.sample(1, 1)
        r0 = rho.clone()
        P.evolve(rho, 0, snap=None)                 # zero steps: state unchanged
        assert torch.equal(rho, r0)
        P.evolve(rho[:0], 10, snap=None)             # empty batch
        with pytest.raises(ftwa.FtwaError):
            ftwa.load()
            from paper_2212_04352_gb300 import check, load
            check(load().ftwa_evolve(P._h, None, 4, 10, None, None), "evolve")
        assert P.status() == 0
    # dimer: fTWA at U = 0 is exact -> <n_1,up>(t) = cos^2(t)
    with ftwa.Plan(lat, 0.0, n_up=[1, 0], n_dn=[0, 1], precision=0, out_every=50) as P:
        rho = P.sample(3, 20000)
        X = P.evolve(rho, 100)
        occ, conn, _ = P.moments(X, g2=False)
        occ = occ.cpu().numpy()
        se = np.sqrt(np.diagonal(conn.cpu().numpy(), axis1=1, axis2=2) / 20000) + 1e-12
        for k, t in enumerate([0.0, 0.5, 1.0]):
            assert abs(occ[k, 0] - math.cos(t) ** 2) < 5 * se[k, 0] + 1e-12


def test_timeout_hook_returns_status(ftwa):
    """A bounded wait that runs out (a barrier nothing arrives at) reports
    FTWA_ERR_DEVICE_TIMEOUT; the context stays usable afterwards."""
    lat = W.hexagonal_flake(3)
    nu, nd = W.neel_state(lat)
    for cluster, variant, prec in [(1, 1, 0), (2, 1, 0), (1, 2, 0), (2, 2, 0), (1, 3, 1), (4, 3, 1)]:
        with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=prec, cluster=cluster, timeout_us=2000,
                       variant=variant) as P:
            rho = P.sample(1, 2)
            r0 = rho.clone()
            P.debug_force_timeout(True)
            P.evolve(rho, 50, snap=None)
            assert P.status() == -5
            assert torch.equal(rho, r0)
            P.debug_force_timeout(False)
            P.evolve(rho, 10, snap=None)
            assert P.status() == 0


# ------------------------------------------------------------------ moments
@pytest.mark.parametrize("precision", [0, 1])
def test_moments_fp64_parity(ftwa, precision):
    lat = W.periodic_honeycomb()
    nu, nd = W.neel_state(lat)
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=precision) as P:
        rho = P.sample(1, 1000)
        X = P.evolve(rho, 200)
        occ, conn, g2 = P.moments(X)
        Xh = X.cpu().numpy().astype(np.float64)
    occ_o, conn_o, g2_o = oracle.moments(Xh)
    assert np.max(np.abs(occ.cpu().numpy() - occ_o)) <= 1e-13
    assert np.max(np.abs(conn.cpu().numpy() - conn_o)) <= 1e-13
    g = g2.cpu().numpy()
    # at t = 0 an empty site has <n> = 0 and g2 is 0/0 on both sides
    assert np.array_equal(np.isnan(g), np.isnan(g2_o))
    ok = ~np.isnan(g2_o)
    assert np.max(np.abs(g[ok] - g2_o[ok]) / np.abs(g2_o[ok])) <= 1e-11


def test_full_path_config1_against_oracle(ftwa):
    """8-site periodic honeycomb, U/t = 1.6, Neel, M = 1000, T = 10, 100 output
    times: GPU FP64 path (sample -> evolve -> moments) equals the oracle's."""
    lat = W.periodic_honeycomb()
    nu, nd = W.neel_state(lat)
    M = 1000
    snap_o, _ = oracle.run(lat, 1.6, nu, nd, 1, 0, M, 0.01, 1000, 10)
    occ_o, conn_o, _ = oracle.moments(snap_o, want_g2=False)
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=0, out_every=10) as P:
        rho = P.sample(1, M)
        X = P.evolve(rho, 1000)
        occ, conn, _ = P.moments(X, g2=False)
        assert P.status() == 0
    assert X.shape == (101, M, 16)
    assert np.max(np.abs(occ.cpu().numpy() - occ_o)) <= 1e-10
    assert np.max(np.abs(conn.cpu().numpy() - conn_o)) <= 1e-10


# ------------------------------------------------------------------ tensor-core Gram
@pytest.mark.parametrize("lat_name,M,steps", [("periodic8", 1000, 50), ("hexflake54", 777, 30),
                                              ("hexflake96", 2000, 20), ("brick198", 1500, 20),
                                              ("brick198", 300, 250), ("brick35", 900, 30)])
def test_gram_bf16x3_matches_fp64(ftwa, lat_name, M, steps):
    """BF16x3 tensor-core Gram against the FP64 Gram of the same FP32
    snapshots.  Each product y_k y_l loses at most the lo*lo term (2^-16
    relative), so |C_bf16 - C_fp64| <= 3e-5 sqrt(C_kk C_ll) (+ FP32
    accumulation); ragged M, 1 to 10 output tiles, several batches of
    output times (26 times of the 198-site case), odd K (35 sites)."""
    lat = {"periodic8": W.periodic_honeycomb, "hexflake54": lambda: W.hexagonal_flake(3),
           "hexflake96": lambda: W.hexagonal_flake(4), "brick198": W.brick_wall_flake,
           "brick35": lambda: W.brick_wall_flake(5, 7)}[lat_name]()
    nu, nd = W.neel_state(lat)
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=1, out_every=10) as P:
        rho = P.sample(3, M)
        X = P.evolve(rho, steps)
        occ64, c64, g64 = P.moments(X, gram_mode=ftwa.FTWA_GRAM_FP64)
        occ16, c16, g16 = P.moments(X, gram_mode=ftwa.FTWA_GRAM_BF16X3)
        assert P.status() == 0
    c64, c16 = c64.cpu().numpy(), c16.cpu().numpy()
    assert torch.equal(occ64, occ16)
    d = np.sqrt(np.abs(np.einsum("tkk->tk", c64)))
    bound = 3e-5 * d[:, :, None] * d[:, None, :] + 1e-7
    assert np.all(np.abs(c16 - c64) <= bound)
    assert np.array_equal(c16, np.transpose(c16, (0, 2, 1)))


def test_gram_bf16x3_error_below_tenth_of_sampling_error(ftwa):
    """At M = 65536 samples (the correlator workload's size) the BF16x3 Gram
    differs from the FP64 Gram by less than 10% of the sampling error
    sigma_k sigma_l / sqrt(M) of each entry."""
    M, K, T = 65536, 396, 3
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    X = torch.rand((T, M, K), generator=g, device="cuda", dtype=torch.float32) - 0.5
    X += 0.1 * torch.rand((1, 1, K), generator=g, device="cuda")
    lat = W.brick_wall_flake()
    nu, nd = W.neel_state(lat)
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=1) as P:
        _, c64, _ = P.moments(X, gram_mode=ftwa.FTWA_GRAM_FP64, g2=False)
        _, c16, _ = P.moments(X, gram_mode=ftwa.FTWA_GRAM_BF16X3, g2=False)
        assert P.status() == 0
    d = torch.sqrt(torch.diagonal(c64, dim1=1, dim2=2))
    stat = d[:, :, None] * d[:, None, :] / M ** 0.5
    assert ((c16 - c64).abs() / stat).max().item() < 0.1


@pytest.mark.parametrize("threads", [512, 768])
@pytest.mark.parametrize("cluster", [1, 2, 4])
@pytest.mark.parametrize("lat_name", ["brick35", "flake54", "brick198"])
def test_evolve_fp32_tiled_threads(ftwa, lat_name, cluster, threads):
    """The tiled stepper with 16 or 24 warps per CTA (different tile
    assignments and tensor-memory splits): the oracle's trajectory to 1e-4
    after 100 FP32 steps; output Hermitian."""
    lat = {"brick35": W.brick_wall_flake(5, 7), "flake54": W.hexagonal_flake(3), "brick198": W.brick_wall_flake()}[lat_name]
    if not _tile_fits(lat, cluster):
        pytest.skip("no tiled decomposition for this cluster size")
    nu, nd = W.neel_state(lat)
    M, steps = 3, 100
    rho0 = _oracle_states(lat, nu, nd, 23, M)
    fin_o = np.stack([oracle.evolve(lat, 1.6, rho0[m], 0.01, steps)[0] for m in range(M)])
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=1, cluster=cluster, variant=3, threads=threads) as P:
        inf = P.info()
        assert inf["variant"] == 3 and inf["threads"] == threads and inf["cluster"] == cluster
        rho = torch.from_numpy(rho0.astype(np.complex64)).cuda()
        P.evolve(rho, steps, snap=None)
        assert P.status() == 0
        fin = rho.cpu().numpy().astype(np.complex128)
    for m in range(M):
        assert _rel(fin[m], fin_o[m]) <= 1e-4
        for sp in range(2):
            assert np.array_equal(fin[m, sp], fin[m, sp].conj().T)
