"""Error bars used by the precision gate of the GPU tests (test helper).

g2_standard_error gives the statistical error of the Eq. 10 estimator
g2_kl = mean(x_k x_l) / (mean(x_k) mean(x_l)), x = Re rho_kk + 1/2, from the
samples themselves (delta method).  It is the scale of a tolerance, not a
result under test; tests/test_gate_stats.py checks it against the spread of
the estimator over independent batches.
"""

import torch


def g2_standard_error(X):
    """Delta-method standard error of g2_kl = A/(B C), A = mean(x_k x_l),
    B = mean(x_k), C = mean(x_l), x = X + 1/2, from the samples X [T, M, K].

    With centred a = x_k - B, b = x_l - C and g = A/(BC), the per-sample
    influence is psi = (a b - E[a b])/(BC) + (1 - g)(a/B + b/C), whose
    variance needs E[a^2 b^2], E[a^2 b], E[a b^2] and the covariances
    (products of centred columns, taken in FP32 on the device: this is only
    the scale of a tolerance)."""
    X = X.to(torch.float64)
    T, M, K = X.shape
    out = torch.empty((T, K, K), dtype=torch.float64, device=X.device)
    for t in range(T):
        x = X[t] + 0.5
        mu = x.mean(0)
        xc = (x - mu).to(torch.float32)
        x2 = xc * xc
        cov = (xc.T @ xc).double() / M
        e22 = (x2.T @ x2).double() / M                 # E[a^2 b^2]
        e21 = (x2.T @ xc).double() / M                 # E[a^2 b]  (row k: a = x_k)
        B = mu[:, None]
        C = mu[None, :]
        g = (cov + B * C) / (B * C)
        var_u = e22 / (B * C) ** 2 - (cov / (B * C)) ** 2
        # cross term 2 E[u v], u = (a b - E ab)/(BC), v = (1 - g)(a/B + b/C)
        cross = 2 * (1 - g) * (e21 / B + e21.T / C) / (B * C)
        va = torch.diagonal(cov)
        var_v = (1 - g) ** 2 * (va[:, None] / B ** 2 + 2 * cov / (B * C) + va[None, :] / C ** 2)
        out[t] = torch.sqrt((var_u + cross + var_v).clamp_min(0) / M)
    return out
