"""Metropolis-Hastings by composition, float64 (the paper's Section 4.1).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 4.1 builds a sampler as MetropolisHastings(Uncalibrated...(...)): the
inner kernel proposes a state and reports the log of its proposal-density
correction, the outer kernel accepts or rejects.  Two inner kernels besides
the leapfrog one:

  * random walk: x' = x + eps z with z ~ N(0, I) (symmetric, correction 0),
    log alpha = log p(x') - log p(x);
  * Langevin (MALA): x' = x + eps^2/2 grad log p(x) + eps z, with the
    correction log q(x | x') - log q(x' | x) of the Gaussian proposal
    q(a | b) = N(a; b + eps^2/2 grad log p(b), eps^2 I).  One leapfrog step
    with momentum z proposes the same x', and its energy difference equals
    this log alpha, so MALA is HMC with L = 1 (pinned in the tests).

Readings where the paper is silent:
  * z is the transition's momentum draw (counter tag 0) and u the accept
    uniform (tag 1), exactly as for HMC, so one generator serves all kernels;
  * the random walk's step size is the scalar eps of the context, adapted by
    dual averaging like HMC's;
  * the cached gradient is carried forward by the random walk too (computed
    at every proposal), so kernels can be swapped without a bootstrap.
"""
import numpy as np

from . import philox


def rw_propose(x, eps, seed, t, chain_offset=0):
    """The random-walk proposal x + eps z and its correction (0: symmetric)."""
    x = np.asarray(x, dtype=np.float64)
    C, D = x.shape
    z = philox.momentum(seed, t, C, D, chain_offset)
    return x + eps * z, np.zeros(C)


def mh_select(x, lp, g, x1, lp1, g1, log_correction, seed, t, chain_offset=0):
    """The Metropolis-Hastings step of the composition: accept x1 iff
    log u < log p(x1) - log p(x) + log_correction (strict); a non-finite ratio
    is a rejection."""
    x, x1 = np.asarray(x, dtype=np.float64), np.asarray(x1, dtype=np.float64)
    C = x.shape[0]
    with np.errstate(invalid="ignore"):
        log_alpha = np.asarray(lp1, dtype=np.float64) - np.asarray(lp, dtype=np.float64) + log_correction
    log_alpha = np.where(np.isfinite(log_alpha), log_alpha, -np.inf)
    log_u = np.log(philox.accept_uniform(seed, t, C, chain_offset))
    acc = log_u < log_alpha
    return {
        "x": np.where(acc[:, None], x1, x),
        "lp": np.where(acc, lp1, lp),
        "g": np.where(acc[:, None], g1, g),
        "is_accepted": acc,
        "log_accept_ratio": log_alpha,
        "log_u": log_u,
        "proposed_x": x1,
    }


def rw_one_step(x, lp, g, eps, seed, t, target, chain_offset=0):
    """One random-walk Metropolis-Hastings transition for every chain."""
    x1, corr = rw_propose(x, eps, seed, t, chain_offset)
    lp1, g1 = target(x1)
    return mh_select(x, lp, g, x1, lp1, g1, corr, seed, t, chain_offset)


def mala_log_accept(x, lp, g, x1, lp1, g1, eps):
    """log alpha of the Langevin proposal from x to x1, written from its
    proposal density (not through a Hamiltonian)."""
    x, x1 = np.asarray(x, dtype=np.float64), np.asarray(x1, dtype=np.float64)
    g, g1 = np.asarray(g, dtype=np.float64), np.asarray(g1, dtype=np.float64)

    def log_q(a, b, gb):          # log N(a; b + eps^2/2 gb, eps^2 I) up to a constant
        r = a - b - 0.5 * eps * eps * gb
        return -np.sum(r * r, axis=1) / (2.0 * eps * eps)

    return (np.asarray(lp1) - np.asarray(lp)) + log_q(x, x1, g1) - log_q(x1, x, g)
