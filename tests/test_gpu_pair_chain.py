"""The dense-Gaussian pair kernel runs a whole sample_chain in one
(cooperative) launch -- P resident across transitions, momenta drawn in the
kernel, dual averaging over a grid barrier (Section 2.1's transition under
Section 4.2's driver).  Its arithmetic is the one-transition launch's, so a
chain through hmc_sample_chain must equal, bit for bit, the same transitions
taken one hmc_step at a time; the per-transition parity with the float64
oracle is covered by test_gpu_tensor_core.py."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2002_01184_gb300 import build
    build.build()
    from paper_2002_01184_gb300 import hmc
    return hmc


# (chains, dim, leapfrog steps, burn-in, kept): ragged chains and dims, the
# full workload size
@pytest.mark.parametrize("C,D,L,B,K", [(256, 256, 8, 6, 5), (200, 100, 5, 4, 3), (4096, 256, 16, 3, 2)])
def test_one_launch_chain_equals_single_transitions(H, C, D, L, B, K):
    from paper_2002_01184_gb300 import workloads
    from paper_2002_01184_gb300.sampler import Sampler
    p = workloads.corr_gauss(dim=D, num_chains=C, num_burnin=B, num_results=K, num_leapfrog=L)
    x0 = torch.as_tensor(p.x0).cuda().contiguous()
    one = Sampler(p, adapt=True)
    x1 = x0.clone()
    samples, eps, acc = one.sample_chain(x1, B, K)
    name, per = H.hmc_dominant_kernel_info(one.ctx)
    assert name == "k_gauss_pair"
    assert per == C * L * (B + K)            # every transition in one launch
    each = Sampler(p, adapt=True)
    x2 = x0.clone()
    each.bootstrap(x2)
    for t in range(B + K):
        r = each.results(each.step(x2, t))
        if t >= B:
            k = t - B
            torch.cuda.synchronize()
            assert torch.equal(samples[k], x2), f"sample {k}"
            assert torch.equal(acc[k], r["is_accepted"]), f"accept {k}"
    H.hmc_synchronize(one.ctx)
    H.hmc_synchronize(each.ctx)
    assert torch.equal(x1, x2)
    assert one.adaptation() == each.adaptation()
    assert 0.0 < float(acc.float().mean()) <= 1.0
    one.close()
    each.close()


@pytest.mark.parametrize("cap", [1, 3])
def test_launch_cap_splits_the_chain_without_changing_it(H, cap):
    from paper_2002_01184_gb300 import workloads
    from paper_2002_01184_gb300.sampler import Sampler
    C, D, L, B, K = 192, 128, 6, 4, 4
    p = workloads.corr_gauss(dim=D, num_chains=C, num_burnin=B, num_results=K, num_leapfrog=L)
    x0 = torch.as_tensor(p.x0).cuda().contiguous()
    whole = Sampler(p, adapt=True)
    x1 = x0.clone()
    s1, e1, a1 = whole.sample_chain(x1, B, K)
    split = Sampler(p, adapt=True, max_transitions_per_launch=cap)
    x2 = x0.clone()
    s2, e2, a2 = split.sample_chain(x2, B, K)
    assert H.hmc_dominant_kernel_info(split.ctx)[1] == C * L * cap
    H.hmc_synchronize(whole.ctx)
    H.hmc_synchronize(split.ctx)
    assert torch.equal(x1, x2) and torch.equal(s1, s2) and torch.equal(e1, e2) and torch.equal(a1, a2)
    assert whole.adaptation() == split.adaptation()
    whole.close()
    split.close()


def test_trace_without_16_byte_alignment_matches(H):
    """The pair kernel streams kept samples to the trace by bulk copies,
    which need a 16-byte-aligned destination; a trace that starts one float
    into a buffer takes the kernel's plain-store path and must hold the same
    samples, bit for bit."""
    from paper_2002_01184_gb300 import workloads
    from paper_2002_01184_gb300.sampler import Sampler
    C, D, L, B, K = 160, 132, 4, 3, 3
    p = workloads.corr_gauss(dim=D, num_chains=C, num_burnin=B, num_results=K, num_leapfrog=L)
    x0 = torch.as_tensor(p.x0).cuda().contiguous()
    s = Sampler(p, adapt=True)
    aligned = torch.empty((K, C, D), device="cuda")
    x1 = x0.clone()
    H.hmc_sample_chain(s.ctx, x1, B, K, aligned, None, None)
    buf = torch.zeros(K * C * D + 1, device="cuda")
    offset = buf[1:]
    assert offset.data_ptr() % 16 == 4
    x2 = x0.clone()
    H.hmc_sample_chain(s.ctx, x2, B, K, offset, None, None)
    H.hmc_synchronize(s.ctx)
    assert torch.equal(x1, x2)
    assert torch.equal(offset.view(K, C, D), aligned)
    assert H.hmc_dominant_kernel_info(s.ctx)[0] == "k_gauss_pair"
    s.close()
