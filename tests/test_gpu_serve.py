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
