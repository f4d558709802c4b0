"""Multi-chain effective sample size and Monte Carlo standard error, float64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper names R-hat and effective sample size as what users monitor
(Section 5, "Discussion"); the estimator here is the multi-chain one of
Gelman et al., Bayesian Data Analysis 3rd ed. (Section 11.5): the
autocorrelation at lag t is rho_t = 1 - (W - mean_c acov_c(t)) / var_plus,
and the sum of autocorrelations is truncated with Geyer's initial monotone
sequence (Geyer 1992): adjacent pairs rho_{2k} + rho_{2k+1} are summed while
positive and forced to be non-increasing.  ESS = C n / tau with
tau = -1 + 2 sum_k P_k.
"""
import numpy as np


def _autocov(x):
    """Biased autocovariance of each series along axis 0 via FFT, all lags."""
    n = x.shape[0]
    xc = x - x.mean(axis=0, keepdims=True)
    m = 1 << int(np.ceil(np.log2(2 * n)))
    f = np.fft.rfft(xc, n=m, axis=0)
    ac = np.fft.irfft(f * np.conj(f), n=m, axis=0)[:n]
    return ac / n


def ess(samples):
    """Effective sample size per state dimension for samples [n, C, D]."""
    s = np.asarray(samples, dtype=np.float64)
    n, C = s.shape[0], s.shape[1]
    s = s.reshape(n, C, -1)
    acov = _autocov(s)                                  # [n, C, D]
    chain_var = acov[0] * n / (n - 1.0)                 # unbiased per chain
    W = chain_var.mean(axis=0)
    chain_mean = s.mean(axis=0)
    B_over_n = chain_mean.var(axis=0, ddof=1) if C > 1 else np.zeros_like(W)
    var_plus = (n - 1.0) / n * W + B_over_n
    rho = 1.0 - (W[None] - acov.mean(axis=1)) / var_plus[None]
    rho[0] = 1.0
    npairs = n // 2
    pairs = rho[0:2 * npairs:2] + rho[1:2 * npairs:2]  # [npairs, D]
    D = pairs.shape[1]
    tau = np.empty(D)
    for d in range(D):
        total = 0.0
        prev = np.inf
        for k in range(npairs):
            pk = pairs[k, d]
            if pk <= 0.0:
                break
            pk = min(pk, prev)
            total += pk
            prev = pk
        tau[d] = -1.0 + 2.0 * total
    tau = np.maximum(tau, 1.0 / np.log10(max(n * C, 10)))
    return n * C / tau


def mcse_mean(samples):
    """Monte Carlo standard error of the mean per dimension: sd / sqrt(ESS)."""
    s = np.asarray(samples, dtype=np.float64)
    n, C = s.shape[0], s.shape[1]
    flat = s.reshape(n * C, -1)
    return flat.std(axis=0, ddof=1) / np.sqrt(ess(s))


def batch_means_ess(samples, batch_size):
    """Replicated batch-means effective sample size per state dimension for
    samples [n, C, D] (the streaming-expectations driver's estimate, Section
    4.2's planned driver that keeps no trace).

    Each chain's n draws are cut into nb = n // batch_size consecutive batches
    of batch_size draws (a last partial batch is left out of the batch means;
    every draw counts in the variance).  The C nb batch means are pooled
    about their grand mean (Gupta and Vats 2020, replicated batch means;
    batch means after Geyer 1992):
      W    = mean over chains of the sample variance of the chain's n draws
             (divisor n - 1),
      sig2 = batch_size x sum over chains and batches of (batch mean - grand
             mean)^2 / (C nb - 1), the estimate of n x the variance of a
             chain mean,
      ESS  = C n W / sig2.
    batch_size = n makes one batch per chain: the spread of the chain means
    across chains estimates the variance directly."""
    s = np.asarray(samples, dtype=np.float64)
    n, C = s.shape[0], s.shape[1]
    s = s.reshape(n, C, -1)
    b = int(batch_size)
    nb = n // b if b >= 1 else 0
    if b < 1 or nb < 1 or C * nb < 2:
        raise ValueError("need batch_size >= 1, one complete batch and at least two batches in all")
    W = s.var(axis=0, ddof=1).mean(axis=0)                         # [D]
    bmeans = s[: nb * b].reshape(nb, b, C, -1).mean(axis=1)        # [nb, C, D]
    grand = bmeans.mean(axis=(0, 1))
    sig2 = b * ((bmeans - grand) ** 2).sum(axis=(0, 1)) / (C * nb - 1)
    return C * n * W / sig2
