"""Pins for the unrolled NUTS oracle (Section 2.3)."""
import math

import numpy as np

from oracle import hmc, nuts, philox, targets


def test_depth_one_is_hmc_with_one_leapfrog_step():
    """With max_tree_depth = 1 the tree is the start and one leapfrog step of
    step v_0 eps; the step is taken iff log U <= H0 - H1, HMC's test with the
    same U, and the statistic is HMC's min(1, alpha)."""
    rng = np.random.default_rng(2)
    D, C, eps, seed, t = 5, 300, 0.45, 17, 4
    A = rng.standard_normal((D, D))
    tgt = targets.make("corr_gauss", P=A @ A.T / D + 0.5 * np.eye(D))
    x = rng.standard_normal((C, D))
    lp, g = tgt(x)
    out = nuts.one_step(x, lp, g, eps, 1, seed, t, tgt)
    dirs = np.array([nuts._word(seed, 0, c, t, nuts.TAG_DIRECTION) & 1 for c in range(C)])
    fwd = hmc.one_step(x, lp, g, eps, 1, seed, t, tgt)
    bwd = hmc.one_step(x, lp, g, -eps, 1, seed, t, tgt)
    for name in ("x", "is_accepted"):
        ref = np.where(dirs[:, None] if name == "x" else dirs, fwd[name], bwd[name])
        np.testing.assert_allclose(out[name], ref, rtol=1e-12, atol=1e-12)
    la = np.where(dirs == 1, fwd["log_accept_ratio"], bwd["log_accept_ratio"])
    np.testing.assert_allclose(out["stat"], np.exp(np.minimum(la, 0.0)), rtol=1e-12)
    assert np.all(out["leaves"] == 1) and np.all(out["depth"] == 1)
    assert 0.05 < out["is_accepted"].mean() < 0.995
    assert (dirs == 1).any() and (dirs == 0).any()


def test_draws_keep_a_correlated_gaussian_invariant():
    """Started at exact draws from N(0, Sigma), NUTS transitions leave the
    mean and covariance at 0 and Sigma = P^-1 within Monte Carlo error."""
    rng = np.random.default_rng(3)
    D, C = 3, 3000
    A = rng.standard_normal((D, D))
    P = A @ A.T / D + 0.4 * np.eye(D)
    S = np.linalg.inv(P)
    tgt = targets.make("corr_gauss", P=P)
    z = philox.momentum(99, 12345, C, D)                   # independent N(0, I)
    x = z @ np.linalg.cholesky(S).T
    lp, g = tgt(x)
    for t in range(6):
        out = nuts.one_step(x, lp, g, 0.3, 10, 5, t, tgt)
        x, lp, g = out["x"], out["lp"], out["g"]
    assert out["depth"].max() > 2                         # real trees were built
    m = x.mean(axis=0)
    cov = np.cov(x.T)
    se_m = np.sqrt(np.diag(S) / C)
    assert np.all(np.abs(m) < 5 * se_m)
    se_c = np.sqrt((S * S + np.outer(np.diag(S), np.diag(S))) / C)
    assert np.all(np.abs(cov - S) < 5 * se_c)


def test_u_turn_stops_the_harmonic_oscillator_near_half_a_period():
    """1-D standard normal from x = 0, p = 1: the exact orbit is (sin s, cos s).
    Whatever the directions, the trajectory cannot keep growing past a span
    of about a period (both ends' momenta then point inward); with eps = 0.05
    a period is about 126 steps, so the tree stops at depth <= 8 of 10 and
    holds at least a quarter period."""
    def tgt(x):
        return -0.5 * np.sum(x * x, axis=1), -x
    for t in range(12):
        o = nuts.one_chain(np.zeros(1), 0.0, np.zeros(1), np.ones(1), math.log(0.5), 0.05, 10, 8,
                           0, t, tgt)
        assert o["depth"] <= 8, o["depth"]
        assert o["leaves"] >= 2 ** 4, o["leaves"]


def test_divergence_stops_the_tree():
    """A step size far past the stability limit of a stiff Gaussian makes the
    energy explode; the first leaf is divergent, so nothing moves."""
    P = np.diag([1.0, 1e6])
    tgt = targets.make("corr_gauss", P=P)
    x = np.array([[0.3, 1e-3], [0.1, -2e-3]])
    lp, g = tgt(x)
    out = nuts.one_step(x, lp, g, 0.5, 10, 1, 0, tgt)
    assert not out["is_accepted"].any()
    assert np.all(out["leaves"] <= 2)
    np.testing.assert_array_equal(out["x"], x)


def test_integer_choice_rule():
    assert nuts._take(0, 1, 1) and nuts._take(2 ** 32 - 1, 1, 1)     # probability 1
    assert not nuts._take(0, 0, 5)                                   # probability 0
    # probability 1/2 splits the words at 2^31
    assert nuts._take(2 ** 31 - 1, 1, 2) and not nuts._take(2 ** 31, 1, 2)


def test_last_doubling_takes_the_candidate_uniformly_when_every_leaf_is_valid():
    """With a tiny step the energy is conserved to ~eps^2, so every leaf is in
    the slice, and a 3-level tree on a 1-D standard normal started at its mode
    never turns (the momentum keeps its sign over 7 steps of 1e-3).  The
    efficient NUTS then replaces the candidate with probability
    min(1, n'/n) = 1 at every doubling (n' = n = 2^j), and inside a subtree
    leaf k replaces it with probability 1/(k + 1): the new state is uniform
    over the four leaves of the last doubling and never an earlier state.
    Uniform progressive sampling over the whole trajectory, or keeping the
    subtree's first or last leaf, would fail this."""
    eps, depth, C, seed, t = 1e-3, 3, 4000, 21, 2

    def tgt(x):
        return -0.5 * np.sum(x * x, axis=1), -x

    x = np.zeros((C, 1))
    lp, g = tgt(x)
    out = nuts.one_step(x, lp, g, eps, depth, seed, t, tgt)
    assert out["is_accepted"].all() and np.all(out["leaves"] == 7) and np.all(out["depth"] == 3)
    p0 = philox.momentum(seed, t, C, 1)[:, 0]
    counts = np.zeros(4)
    for c in range(C):
        dirs = nuts._word(seed, 0, c, t, nuts.TAG_DIRECTION)
        ends = {+1: (0.0, p0[c]), -1: (0.0, p0[c])}
        for j in range(depth):
            v = 1 if (dirs >> j) & 1 else -1
            q, m = ends[v]
            leaves = []
            for _ in range(1 << j):          # velocity Verlet on -x^2/2, step v eps
                m = m - 0.5 * v * eps * q
                q = q + v * eps * m
                m = m - 0.5 * v * eps * q
                leaves.append(q)
            ends[v] = (q, m)
        hit = np.flatnonzero(np.abs(np.array(leaves) - out["x"][c, 0]) < 1e-12)
        assert hit.size == 1, (c, leaves, out["x"][c, 0])
        counts[hit[0]] += 1
    chi2 = np.sum((counts - C / 4) ** 2 / (C / 4))
    assert chi2 < 16.3, counts          # 3 degrees of freedom, p = 0.001
