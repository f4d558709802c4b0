"""The No-U-Turn Sampler with the recursion unrolled, float64 (the paper's
Section 2.3).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 2.3: NUTS (Hoffman and Gelman 2014, which the paper cites) samples
from a Hamiltonian trajectory built by recursive doubling; the recursion is a
pre-order traversal that stops at a U-turn or a divergence, depth is capped
(max_tree_depth, default 10), and a vectorised implementation unrolls the
recursion into a loop over leapfrog steps that keeps O(max_tree_depth)
states instead of the O(2^depth) trajectory.  The transition here is
Hoffman and Gelman's efficient NUTS (their Algorithm 3, slice variable u),
unrolled:

  * p0 ~ N(0, I); H0 = -log p(x0) + |p0|^2/2; u = U exp(-H0) with U uniform;
    the candidate is x0 and n = 1.
  * Doubling j = 0, 1, ... (while no stop and j < max_depth): direction v_j
    = +/-1; a subtree of 2^j leapfrog steps of step v_j eps grows from the
    trajectory's end on that side.  Leaf k of it:
      - valid iff log u <= -H (its weight in n), divergent iff
        H - H0 >= Delta_max - log U (Delta_max = 1000), which stops the subtree;
      - the subtree's candidate becomes the leaf with probability 1/n'
        (n' = valid leaves so far): uniform over the subtree's valid leaves,
        as the recursion's n''/(n' + n'') merges give;
      - for every i >= 1 with 2^i | (k + 1), the span of the last 2^i leaves
        closes -- a node of the recursion -- and stops the subtree if
        (x+ - x-).p- < 0 or (x+ - x-).p+ < 0 for its ends in time order
        (x+ - x- = v (x_last - x_first)).  Only the first leaf of each open
        span is kept: O(max_depth) states.
  * A subtree that did not stop makes its candidate the transition's with
    probability min(1, n'/n); then n += n', and the whole trajectory stops
    if its ends make a U-turn.
  * The dual-averaging statistic is the mean of min(1, exp(H0 - H)) over all
    leaves built (their Algorithm 6).

Random numbers (readings; all from the counter generator, key = seed,
counter (word, chain, t, tag)): p0 from tag 0 as for HMC, U from tag 1 (the
accept uniform), the directions from tag 3 (bit j of word 0 of counter
(0, chain, t, 3): 1 is +1), the subtree choice at leaf k of doubling j from
word k mod 4 of counter (floor(k / 4), chain, t, 4 + j) -- four leaves per
generator call --, the top-level choice at doubling j from word 0 of counter
(j, chain, t, 14).  A choice with probability a / b
(integers) is taken iff (2 w + 1) b < a 2^33 for its word w -- exact integer
arithmetic, so both implementations take it identically.
"""
import numpy as np

from . import philox

TAG_DIRECTION = 3
TAG_SUBTREE = 4          # + doubling index j (< 10)
TAG_TOP = 14
DELTA_MAX = 1000.0
MAX_DEPTH_LIMIT = 10


def _words(seed, w0, chain, t, tag):
    """The four words of counter (w0, chain, t, tag)."""
    ctr = np.array([[w0, chain, t & 0xFFFFFFFF, tag]], dtype=np.uint64)
    return [int(w) for w in philox.philox4x32_10(ctr, philox.seed_key(seed))[0]]


def _word(seed, w0, chain, t, tag):
    return _words(seed, w0, chain, t, tag)[0]


def _take(w, a, b):
    """Probability a / b (non-negative integers, b > 0): (2w + 1) b < a 2^33."""
    return (2 * w + 1) * b < a * (1 << 33)


def one_chain(x0, lp0, g0, p0, log_U, eps, max_depth, seed, chain, t, target):
    """One NUTS transition of a single chain from (x0, p0).  ``target`` maps a
    (1, D) array to (log_prob[1], grad[1, D]).  Returns a dict with the new
    state, its log p and gradient, whether it moved, the statistic, the tree
    depth and leaf count, the smallest decision margin met and why the tree
    stopped (for tests: "max_depth", "divergence", ("u_turn", i) for a span
    of 2^i leaves inside a subtree, "u_turn_top" for the whole trajectory)."""
    x0 = np.asarray(x0, dtype=np.float64)
    p0 = np.asarray(p0, dtype=np.float64)
    H0 = -lp0 + 0.5 * p0 @ p0
    ends = {+1: [x0.copy(), p0.copy(), np.asarray(g0, dtype=np.float64).copy(), lp0],
            -1: [x0.copy(), p0.copy(), np.asarray(g0, dtype=np.float64).copy(), lp0]}
    xm, gm, lpm = x0.copy(), np.asarray(g0, dtype=np.float64).copy(), lp0
    n, moved = 1, False
    a_sum, n_a = 0.0, 0
    margin = np.inf
    dirs = _word(seed, 0, chain, t, TAG_DIRECTION)
    depth = 0
    stop = "max_depth"
    for j in range(max_depth):
        v = 1 if (dirs >> j) & 1 else -1
        x, p, g, lp = (e.copy() if isinstance(e, np.ndarray) else e for e in ends[v])
        n_sub, ok_sub = 0, True
        xs = gs = None
        lps = None
        first = {}                       # level i -> (x, p) at the first leaf of its open span
        for k in range(1 << j):
            # one leapfrog step of step v eps
            p = p + 0.5 * v * eps * g
            x = x + v * eps * p
            lpa, ga = target(x[None, :])
            lp, g = float(lpa[0]), ga[0]
            p = p + 0.5 * v * eps * g
            H = -lp + 0.5 * p @ p
            finite = np.isfinite(H)
            # divergence (Hoffman and Gelman: log u < Delta_max - H, else stop)
            if not finite or H - H0 >= DELTA_MAX - log_U:
                ok_sub = False
                stop = "divergence"
            a_sum += float(np.exp(min(H0 - H, 0.0))) if finite else 0.0
            n_a += 1
            if finite:
                margin = min(margin, abs((H0 - H) - log_U))
                if log_U <= H0 - H:
                    n_sub += 1
                    w = _words(seed, k >> 2, chain, t, TAG_SUBTREE + j)[k & 3]
                    if _take(w, 1, n_sub):
                        xs, gs, lps = x.copy(), g.copy(), lp
            for i in range(1, j + 1):
                span = 1 << i
                if k % span == 0:
                    first[i] = (x.copy(), p.copy())
                if (k + 1) % span == 0:
                    xf, pf = first[i]
                    dx = v * (x - xf)
                    d1, d2 = dx @ pf, dx @ p
                    scale = np.linalg.norm(dx) * max(np.linalg.norm(pf), np.linalg.norm(p))
                    margin = min(margin, abs(d1) / max(scale, 1e-300), abs(d2) / max(scale, 1e-300))
                    if d1 < 0 or d2 < 0:
                        if ok_sub:
                            stop = ("u_turn", i)       # the innermost span that turned
                        ok_sub = False
            if not ok_sub:
                break
        ends[v] = [x, p, g, lp]
        depth = j + 1
        if not ok_sub:
            break
        if n_sub > 0 and _take(_word(seed, j, chain, t, TAG_TOP), n_sub, n):
            xm, gm, lpm, moved = xs, gs, lps, True
        n += n_sub
        xr, pr = ends[+1][0], ends[+1][1]
        xl, pl = ends[-1][0], ends[-1][1]
        dx = xr - xl
        d1, d2 = dx @ pl, dx @ pr
        scale = np.linalg.norm(dx) * max(np.linalg.norm(pl), np.linalg.norm(pr))
        margin = min(margin, abs(d1) / max(scale, 1e-300), abs(d2) / max(scale, 1e-300))
        if d1 < 0 or d2 < 0:
            stop = "u_turn_top"
            break
    return {"x": xm, "lp": lpm, "g": gm, "moved": moved, "stat": a_sum / max(n_a, 1),
            "depth": depth, "leaves": n_a, "margin": margin, "stop": stop}


def one_step(x, lp, g, eps, max_depth, seed, t, target, chain_offset=0):
    """One NUTS transition for every chain (rows of x), the per-chain trees
    built independently; the momentum and U are the HMC streams."""
    x = np.asarray(x, dtype=np.float64)
    C, D = x.shape
    p0 = philox.momentum(seed, t, C, D, chain_offset)
    log_U = np.log(philox.accept_uniform(seed, t, C, chain_offset))
    outs = [one_chain(x[c], float(lp[c]), g[c], p0[c], float(log_U[c]), eps, max_depth, seed,
                      c + chain_offset, t, target) for c in range(C)]
    return {
        "x": np.stack([o["x"] for o in outs]),
        "lp": np.array([o["lp"] for o in outs]),
        "g": np.stack([o["g"] for o in outs]),
        "is_accepted": np.array([o["moved"] for o in outs]),
        "stat": np.array([o["stat"] for o in outs]),
        "depth": np.array([o["depth"] for o in outs]),
        "leaves": np.array([o["leaves"] for o in outs]),
        "margin": np.array([o["margin"] for o in outs]),
    }
