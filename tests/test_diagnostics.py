"""The device ESS used for min-ESS/s agrees with the oracle's estimator
(run here on CPU tensors)."""
import numpy as np
import torch

from oracle import diagnostics as odiag
from paper_2002_01184_gb300 import diagnostics


def test_torch_ess_matches_oracle():
    rng = np.random.default_rng(0)
    n, C, D = 500, 6, 5
    z = np.empty((n, C, D))
    phi = np.linspace(0.0, 0.9, D)
    z[0] = rng.standard_normal((C, D))
    for t in range(1, n):
        z[t] = phi * z[t - 1] + rng.standard_normal((C, D))
    z[:, 3] += 0.3                         # one chain offset: between-chain variance
    a = diagnostics.ess(torch.tensor(z, dtype=torch.float32)).numpy()
    b = odiag.ess(z.astype(np.float32).astype(np.float64))
    np.testing.assert_allclose(a, b, rtol=1e-6)
