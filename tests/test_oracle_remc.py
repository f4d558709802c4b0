"""Pins for the replica-exchange oracle."""
import math

import numpy as np
import pytest

from oracle import diagnostics, hmc, philox, remc, targets


def test_swap_uniforms_are_distinct_from_other_streams():
    u = remc.swap_uniform(3, 5, 200, 4)
    assert u.shape == (200, 3)
    assert not np.allclose(u[:, 0], philox.accept_uniform(3, 5, 200))
    assert 0.0 < u.min() and u.max() < 1.0


def test_equal_temperatures_always_swap():
    """With beta_k == beta_{k+1} the exchange ratio is exactly 1."""
    rng = np.random.default_rng(0)
    x = rng.standard_normal((10, 4, 3))
    lp = -0.5 * (x ** 2).sum(axis=2)
    g = -x
    x2, lp2, g2, sw = remc.exchange(x, lp, g, np.ones(4), 1, 0)
    assert sw[:, 0].all() and sw[:, 2].all() and not sw[:, 1].any()
    np.testing.assert_array_equal(x2[:, 0], x[:, 1])
    np.testing.assert_array_equal(x2[:, 1], x[:, 0])
    np.testing.assert_array_equal(lp2[:, 2], lp[:, 3])
    # odd transitions pair (1, 2)
    _, _, _, sw = remc.exchange(x, lp, g, np.ones(4), 1, 1)
    assert sw[:, 1].all() and not sw[:, 0].any()


def test_swap_ratio_is_the_tempered_exchange_ratio():
    """The exchange acceptance equals the ratio of the tempered product
    densities after and before the swap, computed from its definition."""
    rng = np.random.default_rng(1)
    betas = np.array([1.0, 0.4])
    x = rng.standard_normal((5000, 2, 2))
    lp = -0.5 * (x ** 2).sum(axis=2)
    g = -x
    _, _, _, sw = remc.exchange(x, lp, g, betas, 7, 0)
    before = betas[0] * lp[:, 0] + betas[1] * lp[:, 1]
    after = betas[0] * lp[:, 1] + betas[1] * lp[:, 0]
    u = remc.swap_uniform(7, 0, 5000, 2)[:, 0]
    np.testing.assert_array_equal(sw[:, 0], np.log(u) < after - before)


@pytest.mark.slow
def test_tempered_replicas_have_the_tempered_marginals():
    """For a standard normal target replica k samples N(0, 1/beta_k); the
    cold replica's variance is 1 and every replica's is 1/beta_k within
    3 Monte Carlo standard errors."""
    betas = np.array([1.0, 0.5, 0.25])
    C, K, D = 400, 3, 1
    x0 = philox.momentum(5, 0, C * K, D).reshape(C, K, D) / np.sqrt(betas)[None, :, None]
    out = remc.sample_chain(x0, targets.std_normal, betas, 3, 0.8, 11, 50, 200)
    s = out["samples"]
    for k in range(K):
        sk2 = s[:, :, k, :] ** 2
        assert abs(sk2.mean() - 1.0 / betas[k]) < 3 * diagnostics.mcse_mean(sk2)[0]
    assert out["swaps"].mean() > 0.2
