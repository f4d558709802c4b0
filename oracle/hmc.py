"""Multi-chain Hamiltonian Monte Carlo in float64, step by step as the paper
describes it.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 2.1 ("Case Study: HMC"): draw one momentum per state variable per
chain, run a symplectic integrator for a fixed number of steps with the step
size broadcast over the state, then accept or reject by Metropolis-Hastings
with a per-chain select (the paper's tf.where, never a branch over chains).
Section 4.1 (TransitionKernel): bootstrap_results evaluates the target and its
gradient at the initial state once, and one_step carries the accepted
state's log-prob and gradient forward, so a transition costs L gradient
evaluations, not L + 1.  Section 4.2 (Driver): sample_chain runs burn-in
transitions whose states are not stored, then stores each kept state and
traces a kernel-result field (the worked example traces the step size).
Section 4.1 also names step-size tuning during burn-in by wrapping the inner
kernel; the adaptation rule used here is dual averaging (Hoffman and Gelman
2014, Section 3.2 and Algorithm 5), a reference the paper cites.

Readings where the paper is silent (each also listed in the design notes):
  * integrator: velocity Verlet (half kick, drift, half kick), identity mass;
  * H = -log p(x) + |p|^2 / 2; log alpha = H_0 - H_L; accept iff
    log u < log alpha (strict); a non-finite log alpha is a rejection;
  * dual averaging: gamma = 0.05, t0 = 10, kappa = 0.75, mu = log(10 eps0),
    one step size shared by all chains of a posterior, adapted on every
    burn-in transition with the statistic mean_c min(1, alpha_c) (non-finite
    alpha counts as 0); after burn-in the step size is frozen at eps_bar;
  * kept sample k is the state after transition num_burnin + k (0-based
    transition index t counts burn-in and kept transitions together).
"""
import math

import numpy as np

from . import philox

DA_GAMMA = 0.05
DA_T0 = 10.0
DA_KAPPA = 0.75


def bootstrap(x, target):
    """Log-prob and gradient at the initial state (Section 4.1,
    bootstrap_results)."""
    return target(np.asarray(x, dtype=np.float64))


def leapfrog(x, p, g, eps, num_steps, target):
    """``num_steps`` velocity-Verlet steps with identity mass:
    p <- p + eps/2 grad; x <- x + eps p; p <- p + eps/2 grad(x).
    ``g`` is the gradient of log p at ``x`` on entry.  Returns the final
    (x, p, log_prob, grad)."""
    x = np.array(x, dtype=np.float64)
    p = np.array(p, dtype=np.float64)
    g = np.array(g, dtype=np.float64)
    lp = None
    for _ in range(num_steps):
        p = p + 0.5 * eps * g
        x = x + eps * p
        lp, g = target(x)
        p = p + 0.5 * eps * g
    return x, p, lp, g


def hamiltonian(lp, p):
    """H = U(x) + K(p) with U = -log p(x) and K = |p|^2 / 2 per chain."""
    return -np.asarray(lp) + 0.5 * np.sum(np.asarray(p) ** 2, axis=1)


def one_step(x, lp, g, eps, num_leapfrog, seed, t, target, chain_offset=0):
    """One HMC transition for every chain (Section 2.1 and Section 4.1).

    ``(x, lp, g)`` is the current state with its cached log-prob and gradient.
    ``eps`` is a scalar step size broadcast over the state.  Random numbers
    come from the counter generator keyed by (seed, chain, t).  Returns a dict
    with the next state, its log-prob and gradient, ``is_accepted`` and
    ``log_accept_ratio``.
    """
    x = np.asarray(x, dtype=np.float64)
    lp = np.asarray(lp, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    C, D = x.shape
    p0 = philox.momentum(seed, t, C, D, chain_offset)
    h0 = hamiltonian(lp, p0)
    x1, p1, lp1, g1 = leapfrog(x, p0, g, eps, num_leapfrog, target)
    h1 = hamiltonian(lp1, p1)
    with np.errstate(invalid="ignore"):
        log_alpha = h0 - h1
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
        "h0": h0,
        "h1": h1,
    }


def accept_statistic(log_accept_ratio):
    """Mean over chains of min(1, alpha); a non-finite ratio counts as 0."""
    la = np.asarray(log_accept_ratio, dtype=np.float64)
    with np.errstate(over="ignore", invalid="ignore"):
        a = np.where(np.isfinite(la), np.exp(np.minimum(la, 0.0)), 0.0)
    return float(np.mean(a))


class DualAveraging:
    """Dual-averaging step-size adaptation (Hoffman and Gelman 2014,
    Section 3.2.1, Algorithm 5), with one step size per posterior.

    After m adaptation steps with statistics alpha_1..alpha_m:
      Hbar_m      = (1 - 1/(m + t0)) Hbar_{m-1} + (delta - alpha_m)/(m + t0)
      log eps_m   = mu - sqrt(m)/gamma * Hbar_m
      log ebar_m  = m^-kappa log eps_m + (1 - m^-kappa) log ebar_{m-1}
    with Hbar_0 = 0, log ebar_0 = 0 and mu = log(10 eps_0).
    """

    def __init__(self, eps0, target_accept, gamma=DA_GAMMA, t0=DA_T0, kappa=DA_KAPPA):
        self.delta = float(target_accept)
        self.gamma, self.t0, self.kappa = gamma, t0, kappa
        self.mu = math.log(10.0 * eps0)
        self.m = 0
        self.h_bar = 0.0
        self.log_eps = math.log(eps0)
        self.log_eps_bar = 0.0

    @property
    def step_size(self):
        return math.exp(self.log_eps)

    @property
    def final_step_size(self):
        return math.exp(self.log_eps_bar)

    def update(self, alpha):
        self.m += 1
        m = self.m
        w = 1.0 / (m + self.t0)
        self.h_bar = (1.0 - w) * self.h_bar + w * (self.delta - alpha)
        self.log_eps = self.mu - math.sqrt(m) / self.gamma * self.h_bar
        eta = m ** (-self.kappa)
        self.log_eps_bar = eta * self.log_eps + (1.0 - eta) * self.log_eps_bar
        return self.step_size


def initial_step_size(dim):
    """eps_0 = 1/sqrt(D) clipped to [1e-3, 1] (the configurations give none)."""
    return min(1.0, max(1e-3, 1.0 / math.sqrt(dim)))


def sample_chain(x0, target, num_leapfrog, step_size, seed, num_burnin, num_results,
                 adapt=False, target_accept=0.65, num_adapt_steps=None, chain_offset=0):
    """The sample_chain driver (Section 4.2): bootstrap, ``num_burnin``
    transitions whose states are discarded (the step size adapted on the first
    ``num_adapt_steps`` of them when ``adapt``), then ``num_results`` kept
    transitions.  Returns samples [K, C, D], the traced step size [K], the
    traced accept flags [K, C] and the final state and cached results."""
    x = np.array(x0, dtype=np.float64)
    C, D = x.shape
    lp, g = bootstrap(x, target)
    if num_adapt_steps is None:
        num_adapt_steps = num_burnin
    da = DualAveraging(step_size, target_accept) if adapt else None
    eps = float(step_size)
    samples = np.empty((num_results, C, D))
    trace_eps = np.empty(num_results)
    trace_acc = np.empty((num_results, C), dtype=bool)
    trace_stat = []
    for t in range(num_burnin + num_results):
        if da is not None and t == num_adapt_steps and da.m > 0:
            eps = da.final_step_size
        r = one_step(x, lp, g, eps, num_leapfrog, seed, t, target, chain_offset)
        x, lp, g = r["x"], r["lp"], r["g"]
        if da is not None and t < num_adapt_steps:
            stat = accept_statistic(r["log_accept_ratio"])
            trace_stat.append(stat)
            used = eps
            eps = da.update(stat)
        else:
            used = eps
        k = t - num_burnin
        if k >= 0:
            samples[k] = x
            trace_eps[k] = used
            trace_acc[k] = r["is_accepted"]
    return {"samples": samples, "step_size": trace_eps, "is_accepted": trace_acc,
            "x": x, "lp": lp, "g": g, "accept_stat": np.array(trace_stat),
            "final_step_size": eps}
