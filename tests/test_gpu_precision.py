"""The FP32 precision gate on the 198-site flake: every reported observable of
the FP32 path (FP32 state, BF16x3 tensor-core Gram) against the FP64 path,
in units of its own statistical error bar.

The estimators are Eq. 5 (fTWA_moments: <n_k> = mean(Re rho_kk) + 1/2 and
the connected correlator C_kl) and Eq. 10 (g2_fTWA: g2_kl = <n_k n_l> /
(<n_k><n_l>)).  The FP64 path is pinned to the oracle trajectory by
trajectory (tests/test_gpu_parity.py, 1e-10 at T = 10), so it stands in for
the oracle's moments here; the tensor-core Gram is also compared directly
with the oracle's estimators on the same snapshots.

Gate (the reading of "10 % of the 1/sqrt(M) error bar"): for every output
time and entry,
  occupations  |d<n_k>|  <= 0.1 s_k / sqrt(M),
  correlator   |dC_kl|   <= 0.1 s_k s_l / sqrt(M),
  g2           |dg2_kl|  <= 0.1 se(g2_kl)   (delta-method standard error),
with s_k^2 = C_kk of the FP64 run, and an absolute floor of 1e-6 where the
error bar vanishes (deterministic diagonals at t = 0).
"""

import math

import numpy as np
import pytest

import oracle
import workloads as W
from tests.gate_stats import g2_standard_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FLOOR = 1e-6


@pytest.fixture(scope="module")
def ftwa():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_04352_gb300 as F
    F.load()
    return F


def _ratios(occ32, conn32, g32, occ64, conn64, g64, se_g2, M):
    s = torch.sqrt(torch.diagonal(conn64, dim1=1, dim2=2).clamp_min(0))
    bar_occ = (0.1 * s / math.sqrt(M)).clamp_min(FLOOR)
    bar_conn = (0.1 * s[:, :, None] * s[:, None, :] / math.sqrt(M)).clamp_min(FLOOR)
    r_occ = ((occ32 - occ64).abs() / bar_occ).max().item()
    r_conn = ((conn32 - conn64).abs() / bar_conn).max().item()
    nan32, nan64 = torch.isnan(g32), torch.isnan(g64)
    assert torch.equal(nan32, nan64)
    ok = ~nan64
    bar_g2 = (0.1 * se_g2).clamp_min(FLOOR)
    r_g2 = ((g32 - g64).abs()[ok] / bar_g2[ok]).max().item()
    return r_occ, r_conn, r_g2


@pytest.mark.parametrize("U", [1.0, 1.6])
def test_fp32_moments_within_tenth_of_error_bar(ftwa, U):
    """The 198-site flake workload (charge-imbalanced Fock start, T = 10,
    1000 RK4 steps, 101 output times) at U/t = 1.0 and 1.6: FP32 state with
    the BF16x3 Gram, and FP32 state with the FP64 Gram, against the FP64
    path on the same samples.  Every occupation, connected correlator and g2
    entry at every output time passes the gate."""
    lat = W.brick_wall_flake(11, 18)
    nu, nd = W.charge_imbalanced_state(lat)
    M, steps, seed = 2048, 1000, 41
    with ftwa.Plan(lat, U, n_up=nu, n_dn=nd, precision=ftwa.FTWA_FP64, out_every=10) as P64:
        X64 = P64.evolve(P64.sample(seed, M), steps)
        occ64, conn64, g64 = P64.moments(X64)
        assert P64.status() == 0
    with ftwa.Plan(lat, U, n_up=nu, n_dn=nd, precision=ftwa.FTWA_FP32, out_every=10) as P32:
        X32 = P32.evolve(P32.sample(seed, M), steps)
        res16 = P32.moments(X32, gram_mode=ftwa.FTWA_GRAM_BF16X3)
        res64 = P32.moments(X32, gram_mode=ftwa.FTWA_GRAM_FP64)
        assert P32.status() == 0
    se_g2 = g2_standard_error(X64)
    for occ32, conn32, g32 in (res16, res64):
        r_occ, r_conn, r_g2 = _ratios(occ32, conn32, g32, occ64, conn64, g64, se_g2, M)
        assert r_occ < 1.0, r_occ
        assert r_conn < 1.0, r_conn
        assert r_g2 < 1.0, r_g2


def test_bf16x3_gram_on_snapshots_against_oracle(ftwa):
    """The tensor-core correlator on real fTWA snapshots at the correlator
    workload's size (198-site flake, U/t = 1.6, M = 65536 samples, FP32
    state, outputs every 5 steps to T = 10: 201 times x 396 site-spins),
    against the oracle's estimators (Eqs. 5 and 10, FP64 C) on the same
    snapshots at the first, middle and last output times: occupations,
    connected correlator and g2 within 0.1 of their error bars (the oracle's
    standard deviations; delta-method error for g2)."""
    lat = W.brick_wall_flake(11, 18)
    nu, nd = W.charge_imbalanced_state(lat)
    M, steps = 65536, 1000
    with ftwa.Plan(lat, 1.6, n_up=nu, n_dn=nd, precision=ftwa.FTWA_FP32, out_every=5) as P:
        X = P.evolve(P.sample(51, M), steps)
        assert X.shape == (201, M, 396)
        occ, conn, g2 = P.moments(X, gram_mode=ftwa.FTWA_GRAM_BF16X3)
        assert P.status() == 0
    rows = [1, 100, 200]
    Xs = X[rows]
    occ_o, conn_o, g2_o = oracle.moments(Xs.cpu().numpy().astype(np.float64))
    dev = X.device
    occ_o, conn_o, g2_o = (torch.from_numpy(a).to(dev) for a in (occ_o, conn_o, g2_o))
    se_g2 = g2_standard_error(Xs)
    r_occ, r_conn, r_g2 = _ratios(occ[rows], conn[rows], g2[rows], occ_o, conn_o, g2_o, se_g2, M)
    assert r_occ < 1.0, r_occ
    assert r_conn < 1.0, r_conn
    assert r_g2 < 1.0, r_g2
