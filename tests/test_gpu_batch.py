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
