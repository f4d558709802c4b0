"""The seeded synthetic inputs follow their stated recipes: shapes, value
laws, ranges and determinism (no dataset is used anywhere)."""
import math

import numpy as np
import pytest

from paper_2002_01184_gb300 import workloads


def test_initial_step_size_is_one_over_sqrt_dim_clipped():
    assert workloads.initial_step_size(1) == 1.0
    assert workloads.initial_step_size(256) == pytest.approx(1 / 16)
    assert workloads.initial_step_size(10 ** 8) == 1e-3


def test_log_uniform_integers_cover_the_range_with_log_uniform_mass():
    rng = np.random.default_rng(0)
    v = workloads.log_uniform_int(rng, 8, 512, size=200000)
    assert v.min() == 8 and v.max() == 512
    # log-uniform: equal mass per factor of two (8-16, 16-32, ..., 256-512)
    counts = np.array([np.sum((v >= 8 * 2 ** k) & (v < 16 * 2 ** k)) for k in range(6)])
    np.testing.assert_allclose(counts / counts.sum(), 1 / 6, atol=0.01)


def test_corr_gauss_precision_is_symmetric_positive_definite():
    p = workloads.corr_gauss(dim=32, num_chains=7)
    assert p.P.dtype == np.float32 and np.array_equal(p.P, p.P.T)
    ev = np.linalg.eigvalsh(p.P.astype(np.float64))
    assert ev.min() > 0.1 - 1e-5                       # A A^T / D + 0.1 I
    assert p.x0.shape == (7, 32) and p.adapt and p.target_accept == 0.65
    q = workloads.corr_gauss(dim=32, num_chains=7)
    assert np.array_equal(p.P, q.P) and np.array_equal(p.x0, q.x0)      # seeded


def test_logreg_labels_follow_the_true_weights():
    p = workloads.logreg(n_data=20000, dim=16, num_chains=3)
    assert p.X.shape == (20000, 16) and p.y.shape == (20000,)
    assert set(np.unique(p.y)) <= {0.0, 1.0}
    z = p.X.astype(np.float64) @ p.w_true.astype(np.float64)
    prob = 1 / (1 + np.exp(-z))
    # Bernoulli(sigmoid(X w)): the labels' mean matches the probabilities'
    assert abs(p.y.mean() - prob.mean()) < 4 * math.sqrt(0.25 / 20000)
    assert np.all(p.x0 == 0) and p.num_leapfrog == 10 and p.target_accept == 0.8


def test_uneven_batch_ranges():
    probs = workloads.uneven_batch(num_burnin=3, num_results=5)
    lr = [p for p in probs if p.kind == "logreg"]
    fu = [p for p in probs if p.kind == "funnel"]
    assert len(lr) == 64 and len(fu) == 16
    assert all(8 <= p.dim <= 512 and 500 <= p.X.shape[0] <= 20000 and 64 <= p.num_chains <= 4096
               for p in lr)
    assert all(10 <= p.dim <= 200 for p in fu)
    assert all(p.num_burnin == 3 and p.num_results == 5 for p in probs)


def test_serve_stream_is_poisson_with_half_burn_in():
    reqs = workloads.serve_stream(rate=50.0, duration=20.0, size_scale=0.05)
    times = np.array([t for t, _ in reqs])
    assert np.all(np.diff(times) > 0) and times[-1] <= 20.0
    assert len(reqs) == pytest.approx(1000, abs=4 * math.sqrt(1000))
    for _, p in reqs:
        assert p.num_burnin == (p.num_results + 1) // 2
    kinds = {p.kind for _, p in reqs}
    assert {"corr_gauss", "logreg"} <= kinds
