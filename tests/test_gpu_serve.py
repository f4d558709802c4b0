"""Continuous batching: requests admitted while others run overlap on the
device, and each result is the same alone and in the mix."""
import numpy as np
import pytest

from paper_2002_01184_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2002_01184_gb300 import build
    build.build()
    from paper_2002_01184_gb300 import serve
    return serve


def test_results_alone_equal_results_in_the_mix(S):
    reqs = workloads.serve_stream(rate=200.0, duration=0.05, seed=3, size_scale=0.02)
    assert len(reqs) >= 4
    mixed = S.Server(hbm_budget_bytes=8 * 2 ** 30, slots=8).run(reqs, max_wall=600)
    assert all(j.finished is not None for j in mixed)
    overlapped = sum(1 for a in mixed for b in mixed
                     if a.id < b.id and a.admitted < b.finished and b.admitted < a.finished)
    assert overlapped > 0                      # jobs really ran concurrently
    for job in mixed:
        alone = S.Server(hbm_budget_bytes=8 * 2 ** 30, slots=1).run([(0.0, job.problem)])[0]
        np.testing.assert_array_equal(alone.result["x"], job.result["x"])
        np.testing.assert_array_equal(alone.result["step_size"], job.result["step_size"])


def test_admission_respects_the_budget(S):
    reqs = workloads.serve_stream(rate=500.0, duration=0.02, seed=4, size_scale=0.02)
    need = max(S.job_bytes(p) for _, p in reqs)
    server = S.Server(hbm_budget_bytes=need, slots=8)
    peak = []
    orig = server.admit

    def admit(job, now):
        orig(job, now)
        peak.append(server.used)
    server.admit = admit
    jobs = server.run(reqs, max_wall=600)
    assert all(j.finished is not None for j in jobs)
    assert max(peak) <= need


CASES = [
    ("corr_gauss", dict(dim=256, num_chains=512), "fused", "leapfrog"),
    ("corr_gauss", dict(dim=256, num_chains=512), "single", "leapfrog"),
    ("corr_gauss", dict(dim=256, num_chains=512), "plain", "leapfrog"),
    ("corr_gauss", dict(dim=384, num_chains=300), "fused", "leapfrog"),
    ("logreg", dict(n_data=2500, dim=64, num_chains=256), "fused", "leapfrog"),
    ("logreg", dict(n_data=3000, dim=160, num_chains=200), "fused", "leapfrog"),
    ("logreg", dict(n_data=500, dim=16, num_chains=64), "fused", "leapfrog"),
    ("funnel", dict(dim=50, num_chains=1000), "fused", "leapfrog"),
    ("funnel", dict(dim=50, num_chains=1000), "fused", "nuts"),
    ("std_normal", dict(dim=3, num_chains=100), "fused", "random_walk"),
]


@pytest.mark.parametrize("kind,kw,impl,proposal", CASES)
def test_create_device_bytes_equal_what_a_context_allocates(S, kind, kw, impl, proposal):
    """Admission by HBM budget relies on the library's size query: for every
    path a configuration can select, hmc_create_device_bytes (computed
    without creating anything, from the target's family and sizes alone)
    equals the bytes the created context requested from the device, and the
    server's job_bytes covers it plus the job's own buffers."""
    from paper_2002_01184_gb300 import hmc
    from paper_2002_01184_gb300.sampler import Sampler
    p = getattr(workloads, kind)(**kw)
    impl_id = {"fused": hmc.HMC_IMPL_FUSED, "single": hmc.HMC_IMPL_FUSED_SINGLE_CTA, "plain": hmc.HMC_IMPL_PLAIN}[impl]
    prop = {"leapfrog": hmc.HMC_PROPOSAL_LEAPFROG, "nuts": hmc.HMC_PROPOSAL_NUTS,
            "random_walk": hmc.HMC_PROPOSAL_RANDOM_WALK}[proposal]
    if proposal == "nuts":
        p.num_leapfrog = 10
    s = Sampler(p, impl=impl_id, proposal=prop)
    n_data = 0 if p.X is None else p.X.shape[0]
    shape_only = hmc.hmc_target(hmc.TARGET_IDS[kind], p.dim, n_data, None, None, None)
    predicted = hmc.hmc_create_device_bytes(shape_only, p.num_chains, s.config)
    assert predicted == hmc.hmc_context_device_bytes(s.ctx)
    assert predicted >= 4 * p.num_chains * p.dim            # at least the cached gradient
    if impl == "fused" and proposal == "leapfrog":
        own = 4 * p.num_chains * p.dim * (1 + p.num_results)
        assert S.job_bytes(p) >= predicted + own
    s.close()
