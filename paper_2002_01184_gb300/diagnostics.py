"""Post-run measurement on the device: multi-chain effective sample size.

Same estimator as the float64 checker (Gelman et al., BDA3 Section 11.5 with
Geyer's initial monotone sequence), written with torch so that ESS of an
8 GB sample buffer is computed where it lives.  Not part of the sampler.
"""
import torch


def ess(samples, max_dims=None, chunk_dims=16):
    """ESS per dimension of samples [n, C, D] (float32 device tensor);
    computed in float64 over chunks of dimensions.  Returns a float64 tensor."""
    n, C, D = samples.shape
    dims = torch.arange(D) if max_dims is None or max_dims >= D else \
        torch.linspace(0, D - 1, max_dims).round().long().unique()
    out = []
    m = 1 << (2 * n - 1).bit_length()
    for i in range(0, len(dims), chunk_dims):
        idx = dims[i:i + chunk_dims].to(samples.device)
        s = samples.index_select(2, idx).double()           # [n, C, d]
        xc = s - s.mean(dim=0, keepdim=True)
        f = torch.fft.rfft(xc, n=m, dim=0)
        acov = torch.fft.irfft(f * f.conj(), n=m, dim=0)[:n] / n
        chain_var = acov[0] * n / (n - 1.0)
        W = chain_var.mean(dim=0)
        B_over_n = s.mean(dim=0).var(dim=0, unbiased=True) if C > 1 else torch.zeros_like(W)
        var_plus = (n - 1.0) / n * W + B_over_n
        rho = 1.0 - (W[None] - acov.mean(dim=1)) / var_plus[None]
        rho[0] = 1.0
        npairs = n // 2
        pairs = rho[0:2 * npairs:2] + rho[1:2 * npairs:2]   # [npairs, d]
        # Geyer: keep the initial positive run, then force it non-increasing
        positive = (pairs > 0).double().cumprod(dim=0)
        mono = torch.cummin(torch.where(positive > 0, pairs, torch.zeros_like(pairs)), dim=0).values
        tau = -1.0 + 2.0 * (mono * positive).sum(dim=0)
        tau = torch.clamp(tau, min=1.0 / torch.log10(torch.tensor(float(max(n * C, 10)))).item())
        out.append(n * C / tau)
    return torch.cat(out).cpu()


def ess_batch_means(samples, max_dims=None):
    """Replicated batch-means ESS with one batch per chain (the estimator of
    the streaming driver with batch_size = n): per dimension
    C n W / (n var_c(chain mean)), W the mean within-chain variance.  A few
    reductions and no FFT, for callers that need a cheap figure per request.
    Returns a float64 tensor on the host."""
    n, C, D = samples.shape
    s = samples if max_dims is None or max_dims >= D else samples[:, :, torch.linspace(
        0, D - 1, max_dims).round().long().unique().to(samples.device)]
    s = s.double()
    W = s.var(dim=0, unbiased=True).mean(dim=0)
    V = n * s.mean(dim=0).var(dim=0, unbiased=True)
    return (C * n * W / V).cpu()
