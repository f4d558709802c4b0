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


def test_batch_means_ess_matches_the_oracle():
    """The one-batch-per-chain figure the server reports equals the oracle's
    replicated batch means with batch_size = n (float32 samples, float64
    arithmetic on both sides)."""
    from oracle import diagnostics as odiag
    rng = np.random.default_rng(9)
    phi = 0.6
    e = rng.standard_normal((300, 40, 5))
    z = np.empty_like(e)
    z[0] = e[0] / np.sqrt(1 - phi * phi)
    for t in range(1, 300):
        z[t] = phi * z[t - 1] + e[t]
    z = z.astype(np.float32)
    got = diagnostics.ess_batch_means(torch.tensor(z)).numpy()
    np.testing.assert_allclose(got, odiag.batch_means_ess(z.astype(np.float64), 300), rtol=1e-9)
    sub = diagnostics.ess_batch_means(torch.tensor(z), max_dims=2).numpy()
    np.testing.assert_allclose(sub, got[[0, 4]], rtol=1e-12)
