"""Pins for the Metropolis-Hastings composition oracle (Section 4.1): the
random-walk and Langevin inner kernels."""
import math

import numpy as np

from oracle import hmc, mh, philox, targets


def test_random_walk_proposal_uses_the_momentum_stream():
    x = np.arange(12, dtype=np.float64).reshape(3, 4)
    x1, corr = mh.rw_propose(x, 0.25, 9, 4)
    np.testing.assert_allclose(x1, x + 0.25 * philox.momentum(9, 4, 3, 4), rtol=0, atol=0)
    assert np.all(corr == 0.0)


def test_random_walk_acceptance_matches_its_closed_form():
    """For the standard normal and x' = x + eps z started at stationarity,
    the acceptance probability E[min(1, p(x')/p(x))] is (2/pi) atan(2/eps):
    with a symmetric proposal it equals 2 P(|x'| < |x|) = 2 P(ab < 0) for
    a = x' - x, b = x' + x, jointly normal with correlation
    eps / sqrt(4 + eps^2), so 2 (1/2 - asin(.)/pi) = 1 - (2/pi) atan(eps/2).
    One transition of 200,000 chains."""
    C = 200_000
    for eps, t in ((0.6, 0), (2.4, 1), (5.0, 2)):
        x = philox.momentum(123, 1000 + t, C, 1)           # exact N(0, 1) draws
        lp, g = targets.std_normal(x)
        out = mh.rw_one_step(x, lp, g, eps, 7, t, targets.std_normal)
        a = np.where(np.isfinite(out["log_accept_ratio"]),
                     np.exp(np.minimum(out["log_accept_ratio"], 0.0)), 0.0)
        expect = 2.0 / math.pi * math.atan(2.0 / eps)
        se = a.std() / math.sqrt(C)
        assert abs(a.mean() - expect) < 5 * se, (eps, a.mean(), expect)
        # the decisions realise the same rate
        acc = out["is_accepted"].mean()
        assert abs(acc - expect) < 5 * math.sqrt(expect * (1 - expect) / C)


def test_random_walk_keeps_the_standard_normal_invariant():
    C, T = 20_000, 30
    x = philox.momentum(5, 999, C, 2)
    lp, g = targets.std_normal(x)
    for t in range(T):
        out = mh.rw_one_step(x, lp, g, 1.1, 3, t, targets.std_normal)
        x, lp, g = out["x"], out["lp"], out["g"]
    m, v = x.mean(axis=0), x.var(axis=0)
    assert np.all(np.abs(m) < 5 / math.sqrt(C))
    assert np.all(np.abs(v - 1.0) < 5 * math.sqrt(2.0 / C))


def test_rejected_chains_keep_state_and_cache():
    x = np.zeros((4, 3))
    lp, g = targets.std_normal(x)
    out = mh.rw_one_step(x, lp, g, 50.0, 1, 0, targets.std_normal)   # huge steps: all rejected
    assert not out["is_accepted"].any()
    np.testing.assert_array_equal(out["x"], x)
    np.testing.assert_array_equal(out["g"], g)


def test_mala_is_hmc_with_one_leapfrog_step():
    """One leapfrog step from momentum z proposes x + eps z + eps^2/2 g, the
    Langevin proposal; its energy difference H_0 - H_1 equals the Langevin
    log acceptance ratio written from the proposal density."""
    rng = np.random.default_rng(4)
    for kind, data, D in (("corr_gauss", None, 6), ("funnel", None, 5), ("logreg", None, 3)):
        if kind == "corr_gauss":
            A = rng.standard_normal((D, D))
            tgt = targets.make(kind, P=A @ A.T / D + 0.3 * np.eye(D))
        elif kind == "logreg":
            X = rng.standard_normal((40, D))
            y = (rng.random(40) < 0.5).astype(np.float64)
            tgt = targets.make(kind, X=X, y=y)
        else:
            tgt = targets.make(kind)
        x = 0.5 * rng.standard_normal((64, D))
        lp, g = tgt(x)
        eps = 0.17
        out = hmc.one_step(x, lp, g, eps, 1, 21, 3, tgt)
        z = philox.momentum(21, 3, 64, D)
        x1 = x + eps * z + 0.5 * eps * eps * g
        np.testing.assert_allclose(out["proposed_x"], x1, rtol=1e-13, atol=1e-13)
        lp1, g1 = tgt(x1)
        ref = mh.mala_log_accept(x, lp, g, x1, lp1, g1, eps)
        np.testing.assert_allclose(out["log_accept_ratio"], ref, rtol=1e-9, atol=1e-9)
