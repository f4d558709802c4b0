"""Seeded synthetic inputs shaped like the sampling workloads.

This module only draws and shapes input data (target parameters, initial
states, batch compositions).  It holds none of the sampler's arithmetic and
is the one module that both the CUDA path's callers and the float64 checker
use.  Everything is float32 on return, exactly as the device receives it; a
float64 consumer promotes these same values.

Workloads (sizes are defaults and can be shrunk for tests):
  std_normal   the 1-D N(0,1) worked example: 100 chains from x = 0, 3 leapfrog
               steps of size 1.5, 300 burn-in + 100 kept transitions, seed 0.
  corr_gauss   zero-mean Gaussian, D = 256, precision P = A A^T / D + 0.1 I
               with A[i, j] ~ N(0, 1) from seed 1; 4096 chains from N(0, 1);
               16 leapfrog steps, dual averaging to accept 0.65,
               1000 burn-in + 2000 kept.
  logreg       Bayesian logistic regression: X (20000 x 128) ~ N(0, 1),
               w ~ N(0, 1/D), y ~ Bernoulli(sigmoid(X w)), prior N(0, I);
               2048 chains from 0; 10 leapfrog steps, dual averaging to
               accept 0.8, 500 burn-in + 1000 kept.
  funnel       Neal's funnel of total dimension d (v and d - 1 x's).
  uneven_batch 64 logistic-regression posteriors with D, N and chain count
               log-uniform in [8, 512], [500, 20000], [64, 4096], plus 16
               funnels with d uniform in [10, 200].
"""
import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    kind: str                       # std_normal | corr_gauss | logreg | funnel
    dim: int
    num_chains: int
    x0: np.ndarray                  # [C, D] float32
    P: np.ndarray = None            # [D, D] float32 (corr_gauss)
    X: np.ndarray = None            # [N, D] float32 (logreg)
    y: np.ndarray = None            # [N] float32 in {0, 1} (logreg)
    w_true: np.ndarray = None       # [D] float32 (logreg)
    num_leapfrog: int = 1
    step_size: float = 0.1
    adapt: bool = False
    target_accept: float = 0.65
    num_burnin: int = 0
    num_results: int = 0
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n_data(self):
        return 0 if self.X is None else int(self.X.shape[0])

    def data(self):
        """Target parameters as keyword arguments (None entries dropped)."""
        out = {}
        if self.P is not None:
            out["P"] = self.P
        if self.X is not None:
            out["X"] = self.X
            out["y"] = self.y
        return out


def initial_step_size(dim):
    """1/sqrt(D) clipped to [1e-3, 1]; the configurations give no initial
    step size for the adapted runs."""
    return min(1.0, max(1e-3, 1.0 / math.sqrt(dim)))


def log_uniform_int(rng, lo, hi, size=None):
    """floor(exp(U(log lo, log(hi + 1)))), clipped to [lo, hi]."""
    v = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi + 1), size=size)))
    return np.clip(v, lo, hi).astype(np.int64)


def std_normal(num_chains=100, dim=1, num_burnin=300, num_results=100,
               num_leapfrog=3, step_size=1.5, seed=0):
    return Problem("std_normal", dim, num_chains,
                   np.zeros((num_chains, dim), np.float32),
                   num_leapfrog=num_leapfrog, step_size=step_size, adapt=False,
                   num_burnin=num_burnin, num_results=num_results, seed=seed)


def corr_gauss(dim=256, num_chains=4096, seed=1, num_burnin=1000, num_results=2000,
               num_leapfrog=16, target_accept=0.65):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((dim, dim))
    P = (A @ A.T / dim + 0.1 * np.eye(dim)).astype(np.float32)
    P = 0.5 * (P + P.T)                       # exactly symmetric after rounding
    x0 = rng.standard_normal((num_chains, dim)).astype(np.float32)
    return Problem("corr_gauss", dim, num_chains, x0, P=P,
                   num_leapfrog=num_leapfrog, step_size=initial_step_size(dim),
                   adapt=True, target_accept=target_accept, num_burnin=num_burnin,
                   num_results=num_results, seed=seed)


def logreg(n_data=20000, dim=128, num_chains=2048, seed=2, num_burnin=500,
           num_results=1000, num_leapfrog=10, target_accept=0.8):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n_data, dim)).astype(np.float32)
    w = (rng.standard_normal(dim) / math.sqrt(dim)).astype(np.float32)
    z = X.astype(np.float64) @ w.astype(np.float64)
    prob = 1.0 / (1.0 + np.exp(-z))
    y = (rng.uniform(size=n_data) < prob).astype(np.float32)
    x0 = np.zeros((num_chains, dim), np.float32)
    return Problem("logreg", dim, num_chains, x0, X=X, y=y, w_true=w,
                   num_leapfrog=num_leapfrog, step_size=initial_step_size(dim),
                   adapt=True, target_accept=target_accept, num_burnin=num_burnin,
                   num_results=num_results, seed=seed)


def funnel(dim=10, num_chains=256, seed=3, num_burnin=500, num_results=1000,
           num_leapfrog=10, target_accept=0.8):
    rng = np.random.default_rng(seed)
    x0 = rng.standard_normal((num_chains, dim)).astype(np.float32)
    return Problem("funnel", dim, num_chains, x0, num_leapfrog=num_leapfrog,
                   step_size=initial_step_size(dim), adapt=True,
                   target_accept=target_accept, num_burnin=num_burnin,
                   num_results=num_results, seed=seed)


def uneven_batch(seed=4, n_logreg=64, n_funnel=16, num_results=1000, num_burnin=500,
                 dim_range=(8, 512), n_range=(500, 20000), chain_range=(64, 4096),
                 funnel_dim_range=(10, 200), funnel_chains=None):
    """Posteriors of uneven dimension, data size and chain count."""
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(n_logreg):
        D = int(log_uniform_int(rng, *dim_range))
        N = int(log_uniform_int(rng, *n_range))
        C = int(log_uniform_int(rng, *chain_range))
        probs.append(logreg(n_data=N, dim=D, num_chains=C, seed=1000 + i,
                            num_burnin=num_burnin, num_results=num_results))
    for i in range(n_funnel):
        d = int(rng.integers(funnel_dim_range[0], funnel_dim_range[1] + 1))
        C = int(funnel_chains) if funnel_chains else int(log_uniform_int(rng, *chain_range))
        probs.append(funnel(dim=d, num_chains=C, seed=2000 + i,
                            num_burnin=num_burnin, num_results=num_results))
    return probs


def serve_stream(rate=50.0, duration=120.0, seed=6, size_scale=1.0, chain_range=(64, 4096),
                 sample_range=(200, 2000)):
    """Poisson arrivals of sampling requests, each a random posterior from the
    correlated-Gaussian, logistic-regression or uneven-batch families (sizes
    drawn as for those workloads), with chains and kept samples log-uniform in
    the given ranges and burn-in = ceil(samples / 2).  `size_scale` shrinks
    chains, samples and data rows together (for short test streams).
    Returns a list of (arrival_time_s, Problem)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    i = 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        fam = int(rng.integers(0, 3))
        C = max(8, int(log_uniform_int(rng, *chain_range) * size_scale))
        K = max(4, int(log_uniform_int(rng, *sample_range) * size_scale))
        B = (K + 1) // 2
        s = 10000 + i
        if fam == 0:
            p = corr_gauss(dim=256, num_chains=C, seed=s, num_burnin=B, num_results=K)
        elif fam == 1:
            p = logreg(n_data=max(64, int(20000 * size_scale)), dim=128, num_chains=C, seed=s,
                       num_burnin=B, num_results=K)
        else:
            if rng.uniform() < 0.8:
                D = int(log_uniform_int(rng, 8, 512))
                N = max(64, int(log_uniform_int(rng, 500, 20000) * size_scale))
                p = logreg(n_data=N, dim=D, num_chains=C, seed=s, num_burnin=B, num_results=K)
            else:
                d = int(rng.integers(10, 201))
                p = funnel(dim=d, num_chains=C, seed=s, num_burnin=B, num_results=K)
        p.meta["family"] = ["corr_gauss", "logreg", "uneven"][fam]
        out.append((t, p))
        i += 1
    return out
