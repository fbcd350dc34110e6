"""Batched launch of heterogeneous problems (one CUDA graph) and the
launch-shape autotuner."""

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


def test_batch_equals_individual_evolves(ftwa):
    """Uneven lattices and U values in one graph: every problem's state and
    snapshots equal those of its own ftwa_evolve, bit for bit."""
    specs = [(W.periodic_honeycomb(), 1.6, 0, 300), (W.hexagonal_flake(2), 0.5, 0, 77),
             (W.hexagonal_flake(3), 2.5, 1, 130), (W.hexagon_chain(2), 1.0, 0, 5),
             (W.brick_wall_flake(), 1.6, 1, 40)]
    plans, rhos, refs, snaps, snap_refs = [], [], [], [], []
    steps = 60
    for k, (lat, U, prec, M) in enumerate(specs):
        nu, nd = W.neel_state(lat)
        P = ftwa.Plan(lat, U, n_up=nu, n_dn=nd, precision=prec, out_every=10)
        rho = P.sample(10 + k, M)
        ref = rho.clone()
        snap_refs.append(P.evolve(ref, steps))
        refs.append(ref)
        plans.append(P)
        rhos.append(rho)
        snaps.append(torch.empty_like(snap_refs[-1]))
    B = ftwa.Batch(plans, rhos, steps, snaps)
    B.launch()
    torch.cuda.synchronize()
    for P, rho, ref, X, Xr in zip(plans, rhos, refs, snaps, snap_refs):
        assert P.status() == 0
        assert torch.equal(rho, ref)
        assert torch.equal(X, Xr)
    # the graph can be replayed: a second launch continues from the new state
    for P, ref in zip(plans, refs):
        P.evolve(ref, steps, snap=None)
    B.launch()
    torch.cuda.synchronize()
    for rho, ref in zip(rhos, refs):
        assert torch.equal(rho, ref)
    B.close()
    for P in plans:
        P.close()


def test_autotune_keeps_parity(ftwa):
    lat = W.hexagonal_flake(3)
    nu, nd = W.neel_state(lat)
    M, steps = 3, 100
    rho0 = np.stack([oracle.sample(lat.n_sites, nu, nd, 9, m) for m in range(M)])
    fin_o = np.stack([oracle.evolve(lat, 1.6, rho0[m], 0.01, steps)[0] for m in range(M)])
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=0) as P:
        info = P.autotune(M=512, probe_steps=10)
        assert info["variant"] in (1, 2) and info["cluster"] in (1, 2, 4, 8)
        rho = torch.from_numpy(rho0).cuda()
        P.evolve(rho, steps, snap=None)
        assert P.status() == 0
        fin = rho.cpu().numpy()
    for m in range(M):
        assert np.linalg.norm(fin[m] - fin_o[m]) / np.linalg.norm(fin_o[m]) <= 1e-11


def _oracle_run(lat, U, rho0, steps, every):
    outs = [oracle.evolve(lat, U, rho0[m], 0.01, steps, out_every=every) for m in range(rho0.shape[0])]
    return np.stack([o[0] for o in outs]), np.stack([o[1] for o in outs], axis=1)


@pytest.mark.parametrize("tune", [False, True])
def test_persistent_batch_against_oracle(ftwa, tune):
    """One persistent kernel over a cost-ordered queue of (problem, sample
    batch) items of lattices of uneven size and several U (FP32): every
    problem's trajectories and snapshots against the oracle directly
    (oracle-drawn rho(0) fed to the GPU), 1e-4 relative per trajectory;
    output Hermitian."""
    specs = [(W.hexagonal_flake(2), 0.5), (W.hexagonal_flake(2), 2.5), (W.brick_wall_flake(5, 7), 1.6),
             (W.hexagonal_flake(3), 1.0), (W.brick_wall_flake(11, 18), 1.6)]
    M, steps, every = 3, 60, 20
    plans, rhos, snaps, refs = [], [], [], []
    for k, (lat, U) in enumerate(specs):
        nu, nd = W.neel_state(lat)
        rho0 = np.stack([oracle.sample(lat.n_sites, nu, nd, 40 + k, m) for m in range(M)])
        refs.append(_oracle_run(lat, U, rho0, steps, every))
        P = ftwa.Plan(lat, U, n_up=nu, n_dn=nd, precision=1, out_every=every)
        plans.append(P)
        rhos.append(torch.from_numpy(rho0.astype(np.complex64)).cuda())
        snaps.append(torch.empty((steps // every + 1, M, 2 * lat.n_sites), dtype=torch.float32, device="cuda"))
    B = ftwa.Batch(plans, rhos, steps, snaps, persistent=True, tune=tune)
    B.launch()
    torch.cuda.synchronize()
    for P, rho, X, (fin_o, snap_o) in zip(plans, rhos, snaps, refs):
        assert P.status() == 0
        assert P.info()["variant"] == 3
        fin = rho.cpu().numpy().astype(np.complex128)
        for m in range(M):
            assert np.linalg.norm(fin[m] - fin_o[m]) / np.linalg.norm(fin_o[m]) <= 1e-4
            for sp in range(2):
                assert np.array_equal(fin[m, sp], fin[m, sp].conj().T)
        assert np.max(np.abs(X.cpu().numpy() - snap_o)) <= 1e-4
    B.close()
    for P in plans:
        P.close()


def test_persistent_batch_equals_individual_evolves(ftwa):
    """Many samples per problem (several slots per cluster for the small
    lattices, the 198-site flake split over a cluster) and a replay of the
    graph: the batch's states equal each plan's own ftwa_evolve to FP32
    rounding (the arithmetic per element is the same; the decomposition
    differs)."""
    specs = [(W.hexagonal_flake(2), 1.6, 700), (W.hexagonal_flake(4), 0.5, 150), (W.brick_wall_flake(), 2.5, 40),
             (W.hexagonal_flake(5), 1.0, 77)]
    steps = 30
    plans, rhos, refs = [], [], []
    for k, (lat, U, M) in enumerate(specs):
        nu, nd = W.neel_state(lat)
        P = ftwa.Plan(lat, U, n_up=nu, n_dn=nd, precision=1, out_every=10)
        rho = P.sample(70 + k, M)
        ref = rho.clone()
        P.evolve(ref, 2 * steps, snap=None)
        plans.append(P)
        rhos.append(rho)
        refs.append(ref)
    B = ftwa.Batch(plans, rhos, steps, persistent=True)
    B.launch()
    B.launch()                              # replay: continues from the new state
    torch.cuda.synchronize()
    for P, rho, ref in zip(plans, rhos, refs):
        assert P.status() == 0
        err = (torch.linalg.vector_norm(rho - ref) / torch.linalg.vector_norm(ref)).item()
        assert err <= 1e-5, err
    B.close()
    for P in plans:
        P.close()


def test_persistent_batch_rejects_unsupported(ftwa):
    lat = W.hexagonal_flake(2)
    nu, nd = W.neel_state(lat)
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=0) as P:      # FP64 plan
        rho = P.sample(1, 4)
        with pytest.raises(ftwa.FtwaError):
            ftwa.Batch([P], [rho], 10, persistent=True)
