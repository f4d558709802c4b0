"""The streaming-expectations driver (Welford moments instead of a stored
trace) against the definition applied to the stored trace of the same run:
the two drivers draw the same transitions, so the running mean and sum of
squared deviations must equal the mean and centred sum of squares of the
stored samples."""
import numpy as np
import pytest

from paper_2002_01184_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2002_01184_gb300 import build
    build.build()
    from paper_2002_01184_gb300 import hmc
    return hmc


@pytest.mark.parametrize("kind", ["corr_gauss", "funnel", "nuts_corr_gauss"])
def test_streaming_moments_equal_stored_trace_moments(H, kind):
    from paper_2002_01184_gb300.sampler import Sampler
    prop = H.HMC_PROPOSAL_LEAPFROG
    if kind == "corr_gauss":
        p = workloads.corr_gauss(dim=64, num_chains=300, num_burnin=20, num_results=40)
    elif kind == "nuts_corr_gauss":
        # NUTS on a dense target: the moment updates ride in the captured graph
        p = workloads.corr_gauss(dim=32, num_chains=150, num_burnin=10, num_results=20, num_leapfrog=6)
        prop = H.HMC_PROPOSAL_NUTS
    else:
        p = workloads.funnel(dim=17, num_chains=100, num_burnin=20, num_results=40)
    s = Sampler(p, proposal=prop)
    x = torch.as_tensor(p.x0).cuda().contiguous()
    samples, eps, acc = s.sample_chain(x, p.num_burnin, p.num_results)
    x2 = torch.as_tensor(p.x0).cuda().contiguous()
    mean = torch.empty_like(x2)
    m2 = torch.empty_like(x2)
    eps2 = torch.empty_like(eps)
    H.hmc_sample_chain_streaming(s.ctx, x2, p.num_burnin, p.num_results, mean, m2, eps2)
    torch.cuda.synchronize()
    smp = samples.double().cpu().numpy()
    np.testing.assert_array_equal(x2.cpu().numpy(), x.cpu().numpy())
    np.testing.assert_array_equal(eps2.cpu().numpy(), eps.cpu().numpy())
    ref_mean = smp.mean(axis=0)
    ref_m2 = ((smp - ref_mean) ** 2).sum(axis=0)
    scale = np.abs(smp).max(axis=0) + 1e-6
    assert np.max(np.abs(mean.double().cpu().numpy() - ref_mean) / scale) < 1e-5
    assert np.max(np.abs(m2.double().cpu().numpy() - ref_m2) / (scale ** 2 * p.num_results)) < 1e-5
    s.close()


@pytest.mark.parametrize("kind,bsize", [("corr_gauss", 10), ("funnel", 7), ("corr_gauss", 60)])
def test_streaming_batch_means_ess_equals_oracle_on_stored_trace(H, kind, bsize):
    """Batch-means ESS from the streaming driver against the oracle's
    estimator applied to the stored trace of the same run (60 kept draws: six
    batches of 10, eight of 7 with 4 draws left out of the batch means, or
    one batch per chain)."""
    from oracle import diagnostics as odiag
    from paper_2002_01184_gb300.sampler import Sampler
    if kind == "corr_gauss":
        p = workloads.corr_gauss(dim=64, num_chains=300, num_burnin=20, num_results=60)
    else:
        p = workloads.funnel(dim=17, num_chains=100, num_burnin=20, num_results=60)
    s = Sampler(p)
    x = torch.as_tensor(p.x0).cuda().contiguous()
    samples, eps, acc = s.sample_chain(x, p.num_burnin, p.num_results)
    x2 = torch.as_tensor(p.x0).cuda().contiguous()
    mean = torch.empty_like(x2)
    m2 = torch.empty_like(x2)
    ess = torch.empty(p.dim, device="cuda")
    H.hmc_sample_chain_streaming_ess(s.ctx, x2, p.num_burnin, p.num_results, bsize, mean, m2, ess)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(x2.cpu().numpy(), x.cpu().numpy())
    ref = odiag.batch_means_ess(samples.double().cpu().numpy(), bsize)
    got = ess.double().cpu().numpy()
    assert np.all(np.isfinite(got)) and np.all(got > 0)
    np.testing.assert_allclose(got, ref, rtol=1e-3)
    # the plain streaming call afterwards is unaffected (same moments)
    x3 = torch.as_tensor(p.x0).cuda().contiguous()
    mean3, m23 = torch.empty_like(x3), torch.empty_like(x3)
    H.hmc_sample_chain_streaming(s.ctx, x3, p.num_burnin, p.num_results, mean3, m23)
    torch.cuda.synchronize()
    assert torch.equal(mean3, mean) and torch.equal(m23, m2)
    s.close()


@pytest.mark.parametrize("C,bsize", [(8, 0), (8, 10), (1, 5), (1, 9)])
def test_streaming_ess_rejects_too_few_batches(H, C, bsize):
    """9 kept draws: no batch of 0 or 10 draws; one chain needs two batches."""
    from paper_2002_01184_gb300.sampler import Sampler
    p = workloads.funnel(dim=5, num_chains=C, num_burnin=2, num_results=9)
    s = Sampler(p)
    x = torch.as_tensor(p.x0).cuda().contiguous()
    mean, m2 = torch.empty_like(x), torch.empty_like(x)
    ess = torch.empty(5, device="cuda")
    with pytest.raises(H.HMCError) as ei:
        H.hmc_sample_chain_streaming_ess(s.ctx, x, 2, 9, bsize, mean, m2, ess)
    assert ei.value.status == H.HMC_E_INVALID
    s.close()
