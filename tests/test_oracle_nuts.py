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


# ---- the unrolled loop against the recursion it restates --------------------
#
# Hoffman and Gelman's efficient NUTS (their Algorithm 3) builds each
# doubling's subtree by recursion: BuildTree at height 0 takes one leapfrog
# step; at height j it builds a subtree of height j - 1, and only if that one
# did not stop, a second one from its far end, then tests the U-turn
# criterion on the ends of the whole height-j subtree.  The function below
# restates that recursion directly, in its own order, with nothing shared with
# oracle/nuts.py but the counter generator.  Its subtree candidate is drawn
# from the same words as the oracle's (the recursion's random merges with
# probability n''/(n' + n'') and the oracle's per-leaf 1/n' replacements give
# the same uniform law over the subtree's valid leaves but spend different
# random numbers, so the choice is made here by the per-leaf rule over the
# valid leaves the recursion returns).  Everything the recursion decides --
# how many leaves are built, where and why the tree stops, which leaves are
# valid -- is the recursion's own.

def _recursive_tree(x0, lp0, g0, p0, log_U, eps, max_depth, seed, chain, t, target):
    H0 = -lp0 + 0.5 * p0 @ p0

    def leapfrog(x, p, g, v):
        p = p + 0.5 * v * eps * g
        x = x + v * eps * p
        lpa, ga = target(x[None, :])
        g = ga[0]
        p = p + 0.5 * v * eps * g
        return x, p, g, float(lpa[0])

    def build(x, p, g, lp, v, j, k0):
        """Subtree of height j from (x, p) in direction v; its leaves are
        numbered k0, k0 + 1, ... in build order.  Returns a dict: first / last
        leaf states, the valid leaves [(k, x, g, lp)], whether it may go on
        (s), the leaves built with their energies, and the stop reason."""
        if j == 0:
            x, p, g, lp = leapfrog(x, p, g, v)
            H = -lp + 0.5 * p @ p
            finite = bool(np.isfinite(H))
            valid = finite and log_U <= H0 - H
            s = finite and (H - H0 < nuts.DELTA_MAX - log_U)
            return {"first": (x, p), "last": (x, p, g, lp),
                    "valid": [(k0, x, g, lp)] if valid else [], "s": s, "H": [H],
                    "stop": None if s else "divergence"}
        a = build(x, p, g, lp, v, j - 1, k0)
        if not a["s"]:
            return a
        b = build(*a["last"], v, j - 1, k0 + (1 << (j - 1)))
        out = {"first": a["first"], "last": b["last"], "valid": a["valid"] + b["valid"],
               "s": b["s"], "H": a["H"] + b["H"], "stop": b["stop"]}
        if b["s"]:
            xf, pf = a["first"]
            xl, pl = b["last"][0], b["last"][1]
            dx = v * (xl - xf)                 # x+ - x- in time order
            if dx @ pf < 0 or dx @ pl < 0:
                out["s"], out["stop"] = False, ("u_turn", j)
        return out

    ends = {+1: (x0, p0, g0, lp0), -1: (x0, p0, g0, lp0)}
    state = (x0, g0, lp0)
    n, moved, energies, depth, stop = 1, False, [], 0, "max_depth"
    dirs = nuts._word(seed, 0, chain, t, nuts.TAG_DIRECTION)
    for j in range(max_depth):
        v = 1 if (dirs >> j) & 1 else -1
        tree = build(*ends[v], v, j, 0)
        ends[v] = tree["last"]
        energies += tree["H"]
        depth = j + 1
        if not tree["s"]:
            stop = tree["stop"]
            break
        cand = None
        for m, (k, x, g, lp) in enumerate(tree["valid"], start=1):
            w = nuts._words(seed, k >> 2, chain, t, nuts.TAG_SUBTREE + j)[k & 3]
            if nuts._take(w, 1, m):
                cand = (x, g, lp)
        n_sub = len(tree["valid"])
        if n_sub and nuts._take(nuts._word(seed, j, chain, t, nuts.TAG_TOP), n_sub, n):
            state, moved = cand, True
        n += n_sub
        dx = ends[+1][0] - ends[-1][0]
        if dx @ ends[-1][1] < 0 or dx @ ends[+1][1] < 0:
            stop = "u_turn_top"
            break
    H = np.array(energies)
    stat = np.where(np.isfinite(H), np.exp(np.minimum(H0 - H, 0.0)), 0.0).mean()
    return {"x": state[0], "lp": state[2], "moved": moved, "depth": depth, "leaves": len(energies),
            "stop": stop, "stat": stat}


def _funnel_and_gauss_cases():
    """(name, target, states, step sizes) covering shallow and deep trees,
    divergences, and trees stopped by spans inside a subtree."""
    rng = np.random.default_rng(11)
    D = 6
    A = rng.standard_normal((D, D))
    gauss = targets.make("corr_gauss", P=A @ A.T / D + 0.05 * np.eye(D))
    funnel = targets.make("funnel")
    xg = rng.standard_normal((12, D)) * 2.0
    xf = np.concatenate([rng.normal(0.0, 3.0, (12, 1)), rng.standard_normal((12, 9))], axis=1)
    return [("corr_gauss", gauss, xg, (0.05, 0.2, 0.6, 1.9)),
            ("funnel", funnel, xf, (0.02, 0.15, 0.5, 1.5))]


def _compare_with_recursion(one_chain):
    seen = set()
    for name, tgt, x, steps in _funnel_and_gauss_cases():
        C, D = x.shape
        lp, g = tgt(x)
        for max_depth in (1, 3, 6, 10):
            for eps in steps:
                t = int(1000 * eps) + max_depth
                p0 = philox.momentum(5, t, C, D)
                log_U = np.log(philox.accept_uniform(5, t, C))
                for c in range(C):
                    args = (x[c], float(lp[c]), g[c], p0[c], float(log_U[c]), eps, max_depth, 5, c, t, tgt)
                    o = one_chain(*args)
                    r = _recursive_tree(*args)
                    for key in ("depth", "leaves", "moved", "stop"):
                        if o[key] != r[key]:
                            return False, (name, max_depth, eps, c, key, o[key], r[key]), seen
                    if not (np.allclose(o["x"], r["x"], rtol=1e-12, atol=1e-12)
                            and abs(o["stat"] - r["stat"]) <= 1e-12):
                        return False, (name, max_depth, eps, c, "state"), seen
                    stop = r["stop"]
                    seen.add(("inner_u_turn" if isinstance(stop, tuple) and stop[1] < r["depth"] - 1
                              else "subtree_u_turn" if isinstance(stop, tuple) else stop))
                    if r["depth"] >= 6:
                        seen.add("deep")
    return True, None, seen


def test_unrolled_loop_equals_the_recursive_build_tree():
    """Chain by chain, for depths 1-10 on a correlated Gaussian and the funnel:
    the same depth, leaf count, stop reason, statistic and new state as
    Hoffman and Gelman's recursive BuildTree.  The cases include trees stopped
    by a span strictly inside the last subtree, by the subtree's own span, by
    the whole trajectory, by divergence and by the depth cap."""
    ok, where, seen = _compare_with_recursion(nuts.one_chain)
    assert ok, where
    for kind in ("inner_u_turn", "subtree_u_turn", "u_turn_top", "divergence", "max_depth", "deep"):
        assert kind in seen, (kind, seen)


def _mutated_one_chain(old, new):
    """oracle/nuts.py's one_chain with one planted mistake (for the test below)."""
    import inspect
    src = inspect.getsource(nuts)
    assert old in src, old
    ns = {"__name__": "oracle.nuts_mutant", "__package__": "oracle"}
    exec(compile(src.replace(old, new), "nuts_mutant", "exec"), ns)
    return ns["one_chain"]


def test_the_comparison_catches_planted_span_mistakes():
    """Mistakes the other pins would miss -- spans closed one leaf early, or a
    span tested against the leaf after its first -- break the equality with
    the recursion (planted in a copy of the oracle, on the CPU)."""
    early = _mutated_one_chain("if (k + 1) % span == 0:", "if (k + 2) % span == 0:")
    assert not _compare_with_recursion(early)[0]
    shifted = _mutated_one_chain("if k % span == 0:", "if k % span == min(1, span - 1):")
    assert not _compare_with_recursion(shifted)[0]
