"""Target log-densities and their gradients, float64, one row per chain.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Every function follows the paper's "batch semantics" (Section 2, the
batch-friendly target log-prob listing): the leading axis indexes chains and
only the event axis is reduced, so chain i's value never depends on chain j.
Log-densities are given up to an additive constant, which cancels in the
Metropolis-Hastings ratio.  Each function returns (log_prob [C], grad [C, D]).
"""
import numpy as np


def std_normal(x):
    """Standard normal, the worked example's target (Section 1 listing):
    log p(x) = -x^2 / 2 summed over the event axis; gradient -x."""
    x = np.asarray(x, dtype=np.float64)
    return -0.5 * np.sum(x * x, axis=1), -x


def corr_gauss(x, P):
    """Zero-mean Gaussian with precision P: log p(x) = -x^T P x / 2 and
    gradient -P x.  With chains as rows this is one C x D x D product
    G = -X P (P symmetric)."""
    x = np.asarray(x, dtype=np.float64)
    P = np.asarray(P, dtype=np.float64)
    g = -(x @ P)
    return 0.5 * np.sum(x * g, axis=1), g


def softplus(z):
    """log(1 + e^z) in the overflow-free form max(z, 0) + log1p(e^-|z|)."""
    return np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))


def sigmoid(z):
    """1 / (1 + e^-z), evaluated without overflow for either sign of z."""
    e = np.exp(-np.abs(z))
    return np.where(z >= 0, 1.0 / (1.0 + e), e / (1.0 + e))


def logreg(theta, X, y):
    """Bayesian logistic regression with prior theta ~ N(0, I):
    log p(theta | X, y) = sum_i [y_i z_i - softplus(z_i)] - |theta|^2 / 2,
    z = X theta.  Gradient X^T (y - sigmoid(z)) - theta.  With chains as rows,
    Z = Theta X^T (C x N) and G = (y - sigmoid(Z)) X - Theta (C x D)."""
    th = np.asarray(theta, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    z = th @ X.T
    lp = np.sum(y[None, :] * z - softplus(z), axis=1) - 0.5 * np.sum(th * th, axis=1)
    g = (y[None, :] - sigmoid(z)) @ X - th
    return lp, g


def funnel(s):
    """Neal's funnel with state (v, x_1..x_n), n = D - 1: v ~ N(0, 9) and
    x_i | v ~ N(0, e^v).  log p = -v^2/18 - (n/2) v - e^-v |x|^2 / 2;
    d/dv = -v/9 - n/2 + e^-v |x|^2 / 2, d/dx_i = -e^-v x_i."""
    s = np.asarray(s, dtype=np.float64)
    v = s[:, 0]
    xs = s[:, 1:]
    n = xs.shape[1]
    q = np.sum(xs * xs, axis=1)
    ev = np.exp(-v)
    lp = -v * v / 18.0 - 0.5 * n * v - 0.5 * ev * q
    g = np.empty_like(s)
    g[:, 0] = -v / 9.0 - 0.5 * n + 0.5 * ev * q
    g[:, 1:] = -ev[:, None] * xs
    return lp, g


def make(kind, **data):
    """Bind a target family to its data; returns x -> (log_prob, grad)."""
    if kind == "std_normal":
        return std_normal
    if kind == "corr_gauss":
        P = np.asarray(data["P"], dtype=np.float64)
        return lambda x: corr_gauss(x, P)
    if kind == "logreg":
        X = np.asarray(data["X"], dtype=np.float64)
        y = np.asarray(data["y"], dtype=np.float64)
        return lambda x: logreg(x, X, y)
    if kind == "funnel":
        return funnel
    raise ValueError(f"unknown target {kind!r}")
