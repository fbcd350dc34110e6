"""The delta-method error bar of the precision gate (CPU)."""

import numpy as np
import torch

from tests.gate_stats import g2_standard_error


def test_g2_standard_error_formula():
    """The delta-method standard error used by the gate matches the spread of
    the g2 estimator over independent batches (CPU, synthetic correlated
    positive data), within 15 %."""
    rng = np.random.default_rng(5)
    T, M, K, R = 1, 4000, 3, 300
    L = np.array([[1.0, 0, 0], [0.5, 1.0, 0], [0.2, -0.3, 1.0]]) * 0.08
    vals, ses = [], []
    for r in range(R):
        z = rng.standard_normal((M, K)) @ L.T + np.array([0.1, -0.2, 0.3])
        X = torch.from_numpy(z[None])
        x = z + 0.5
        g = (x.T @ x / M) / np.outer(x.mean(0), x.mean(0))
        vals.append(g)
        ses.append(g2_standard_error(X)[0].numpy())
    spread = np.std(np.array(vals), axis=0)
    se = np.mean(np.array(ses), axis=0)
    assert np.all(np.abs(se / spread - 1) < 0.15)
