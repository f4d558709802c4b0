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


@pytest.mark.parametrize("kind", ["corr_gauss", "funnel"])
def test_streaming_moments_equal_stored_trace_moments(H, kind):
    from paper_2002_01184_gb300.sampler import Sampler
    if kind == "corr_gauss":
        p = workloads.corr_gauss(dim=64, num_chains=300, num_burnin=20, num_results=40)
    else:
        p = workloads.funnel(dim=17, num_chains=100, num_burnin=20, num_results=40)
    s = Sampler(p)
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
