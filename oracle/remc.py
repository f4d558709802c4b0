"""Replica exchange Monte Carlo over HMC, float64 (the paper's Section 2.2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper describes replica exchange as adding a batch dimension of K
temperatures: every chain carries K replicas whose target log-probabilities
are scaled by inverse temperatures beta_k (beta_0 = 1 is the distribution of
interest), all replicas advance by the ordinary transition kernel, and
adjacent replicas then swap states by a Metropolis-Hastings test.  Readings
where the paper is silent:
  * replica k of chain c is row c*K + k of the batched state, so its random
    streams are those of chain c*K + k;
  * tempered target log p_k(x) = beta_k log p(x), gradient beta_k grad log p;
  * after the transition with index t, the pairs (k, k+1) with k = t mod 2,
    t mod 2 + 2, ... are proposed for exchange (even / odd alternation);
  * the pair swaps iff log u < (beta_k - beta_{k+1}) (log p(x_{k+1}) - log p(x_k)),
    u from the counter generator with counter (k, chain c, t, tag 2);
  * kept states are taken after the exchange step.
"""
import numpy as np

from . import hmc, philox

TAG_SWAP = 2


def swap_uniform(seed, t, num_chains, num_replicas, chain_offset=0):
    """u[c, k] for the pair (k, k+1) of chain c at transition t."""
    K = num_replicas
    k, c = np.meshgrid(np.arange(K - 1), np.arange(num_chains) + chain_offset, indexing="xy")
    ctr = np.stack([k.ravel(), c.ravel(), np.full(k.size, t & 0xFFFFFFFF),
                    np.full(k.size, TAG_SWAP)], axis=1)
    w = philox.philox4x32_10(ctr, philox.seed_key(seed))
    return philox.words_to_uniform(w[:, 0]).reshape(num_chains, K - 1)


def tempered(target, betas):
    """Row r of a [C*K, D] batch uses beta_{r mod K}."""
    betas = np.asarray(betas, dtype=np.float64)

    def f(x):
        lp, g = target(x)
        b = np.tile(betas, x.shape[0] // betas.size)
        return b * lp, b[:, None] * g
    return f


def exchange(x, lp_raw, g_raw, betas, seed, t, chain_offset=0):
    """The exchange step after transition t on [C, K, D] states with their
    untempered log p and gradient.  Returns the new arrays and swapped[C, K-1]."""
    x, lp_raw, g_raw = x.copy(), lp_raw.copy(), g_raw.copy()
    C, K, _ = x.shape
    u = swap_uniform(seed, t, C, K, chain_offset)
    swapped = np.zeros((C, K - 1), dtype=bool)
    for k in range(t % 2, K - 1, 2):
        la = (betas[k] - betas[k + 1]) * (lp_raw[:, k + 1] - lp_raw[:, k])
        s = np.log(u[:, k]) < la
        swapped[:, k] = s
        for arr in (x, g_raw):
            a, b = arr[s, k].copy(), arr[s, k + 1].copy()
            arr[s, k], arr[s, k + 1] = b, a
        a, b = lp_raw[s, k].copy(), lp_raw[s, k + 1].copy()
        lp_raw[s, k], lp_raw[s, k + 1] = b, a
    return x, lp_raw, g_raw, swapped


def sample_chain(x0, target, betas, num_leapfrog, step_size, seed, num_burnin, num_results):
    """Replica exchange with a fixed step size: x0 [C, K, D]; returns kept
    states [num_results, C, K, D] and the swap indicators [num_results, C, K-1]."""
    betas = np.asarray(betas, dtype=np.float64)
    x = np.array(x0, dtype=np.float64)
    C, K, D = x.shape
    tt = tempered(target, betas)
    flat = x.reshape(C * K, D)
    lp, g = tt(flat)
    samples = np.empty((num_results, C, K, D))
    swaps = np.empty((num_results, C, K - 1), dtype=bool)
    for t in range(num_burnin + num_results):
        r = hmc.one_step(flat, lp, g, step_size, num_leapfrog, seed, t, tt)
        b = np.tile(betas, C)
        lp_raw = (r["lp"] / b).reshape(C, K)
        g_raw = (r["g"] / b[:, None]).reshape(C, K, D)
        x3, lp_raw, g_raw, sw = exchange(r["x"].reshape(C, K, D), lp_raw, g_raw, betas, seed, t)
        flat = x3.reshape(C * K, D)
        lp = (lp_raw.reshape(-1) * b)
        g = g_raw.reshape(C * K, D) * b[:, None]
        k = t - num_burnin
        if k >= 0:
            samples[k] = x3
            swaps[k] = sw
    return {"samples": samples, "swaps": swaps, "x": flat.reshape(C, K, D)}
