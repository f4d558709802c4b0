"""Checkpoint / resume and the bounded-wait failure path on the GPU.

A transition is a pure function of (state, kernel results) and the counter
generator's key (Section 4.1), so a chain split at transition k -- its kernel
results and step-size adaptation saved to host memory, restored into a fresh
context -- must continue bit for bit as if it had never stopped.  The second
test makes the dense-Gaussian pair kernel's grid barrier wait run out on
purpose (a barrier generation that can never complete, set through the
library's test knob): the kernel must give up, unwind and return, the host
must see HMC_E_TIMEOUT, and the GPU must stay usable."""
import numpy as np
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


def problems():
    from paper_2002_01184_gb300 import workloads
    return {
        # the CTA-pair kernel, whole ranges in one cooperative launch
        "corr_gauss": workloads.corr_gauss(dim=256, num_chains=320, num_burnin=6, num_results=5, num_leapfrog=6),
        # the fused elementwise transition
        "funnel": workloads.funnel(dim=20, num_chains=300, num_burnin=6, num_results=5),
        # the tensor-core logistic regression (long data pass)
        "logreg": workloads.logreg(n_data=2500, dim=64, num_chains=256, num_burnin=4, num_results=4,
                                   num_leapfrog=5),
        # NUTS on the dense targets: every range is captured with its leaf
        # loops (num_leapfrog is the maximum tree depth)
        "nuts_corr_gauss": workloads.corr_gauss(dim=64, num_chains=200, num_burnin=6, num_results=5,
                                                num_leapfrog=6),
        "nuts_logreg": workloads.logreg(n_data=1500, dim=24, num_chains=150, num_burnin=5, num_results=4,
                                        num_leapfrog=6),
    }


def proposal(H, kind):
    return H.HMC_PROPOSAL_NUTS if kind.startswith("nuts") else H.HMC_PROPOSAL_LEAPFROG


def run_whole(H, p, prop):
    from paper_2002_01184_gb300.sampler import Sampler
    s = Sampler(p, adapt=True, proposal=prop)
    x = torch.as_tensor(p.x0).cuda().contiguous()
    samples, eps, acc = s.sample_chain(x, p.num_burnin, p.num_results)
    H.hmc_synchronize(s.ctx)
    out = (x, samples, eps, acc, H.hmc_read_adaptation(s.ctx))
    s.close()
    return out


@pytest.mark.parametrize("kind", ["corr_gauss", "funnel", "logreg", "nuts_corr_gauss", "nuts_logreg"])
@pytest.mark.parametrize("where", ["burn-in", "sampling"])
def test_split_run_resumed_in_a_fresh_context_is_bit_identical(H, kind, where):
    from paper_2002_01184_gb300.sampler import Sampler
    p = problems()[kind]
    prop = proposal(H, kind)
    B, K = p.num_burnin, p.num_results
    n = B + K
    k = B - 2 if where == "burn-in" else B + 2
    x_ref, s_ref, e_ref, a_ref, da_ref = run_whole(H, p, prop)
    C, D = p.num_chains, p.dim
    x = torch.as_tensor(p.x0).cuda().contiguous()
    first = Sampler(p, adapt=True, proposal=prop)
    k1 = max(0, k - B)                         # kept transitions of the first piece
    s1 = torch.empty((max(k1, 1), C, D), device="cuda")
    e1 = torch.empty(max(k1, 1), device="cuda")
    a1 = torch.empty((max(k1, 1), C), dtype=torch.uint8, device="cuda")
    H.hmc_sample_chain_range(first.ctx, x, B, 0, k, s1, e1, a1)
    state = H.hmc_save_state(first.ctx)
    first.close()
    second = Sampler(p, adapt=True, proposal=prop)
    H.hmc_restore_state(second.ctx, state)
    k2 = K - k1
    s2 = torch.empty((k2, C, D), device="cuda")
    e2 = torch.empty(k2, device="cuda")
    a2 = torch.empty((k2, C), dtype=torch.uint8, device="cuda")
    H.hmc_sample_chain_range(second.ctx, x, B, k, n, s2, e2, a2)
    H.hmc_synchronize(second.ctx)
    assert torch.equal(x, x_ref)
    samples = torch.cat([s1[:k1], s2]) if k1 else s2
    assert torch.equal(samples, s_ref)
    assert torch.equal(torch.cat([e1[:k1], e2]) if k1 else e2, e_ref)
    assert torch.equal(torch.cat([a1[:k1], a2]) if k1 else a2, a_ref)
    assert H.hmc_read_adaptation(second.ctx) == da_ref
    second.close()


def test_restore_rejects_a_state_of_another_shape(H):
    from paper_2002_01184_gb300 import workloads
    from paper_2002_01184_gb300.sampler import Sampler
    p = workloads.funnel(dim=10, num_chains=64, num_burnin=2, num_results=2)
    s = Sampler(p, adapt=True)
    x = torch.as_tensor(p.x0).cuda().contiguous()
    H.hmc_sample_chain_range(s.ctx, x, 2, 0, 2)
    state = H.hmc_save_state(s.ctx)
    other = Sampler(workloads.funnel(dim=12, num_chains=64, num_burnin=2, num_results=2), adapt=True)
    with pytest.raises(H.HMCError) as err:
        H.hmc_restore_state(other.ctx, state)
    assert err.value.status == H.HMC_E_INVALID
    with pytest.raises(H.HMCError):
        H.hmc_sample_chain_range(other.ctx, x, 2, 1, 2)     # no state to continue from
    s.close()
    other.close()


def test_grid_barrier_wait_runs_out_and_reports_timeout(H):
    from paper_2002_01184_gb300 import workloads
    from paper_2002_01184_gb300.sampler import Sampler
    p = workloads.corr_gauss(dim=128, num_chains=256, num_burnin=4, num_results=3, num_leapfrog=4)
    x0 = torch.as_tensor(p.x0).cuda().contiguous()
    try:
        # generation 2 (the second adapting transition) can never complete
        H.hmc_debug_set_grid_barrier(20_000_000, 2)
        s = Sampler(p, adapt=True, use_graph=False)
        x = x0.clone()
        H.hmc_sample_chain(s.ctx, x, p.num_burnin, p.num_results, None, None, None)
        with pytest.raises(H.HMCError) as err:
            H.hmc_synchronize(s.ctx)
        assert err.value.status == H.HMC_E_TIMEOUT
        assert "site 7" in str(err.value)                  # the grid barrier gave up
        assert H.hmc_dominant_kernel_info(s.ctx)[0] == "k_gauss_pair"
        s.close()
    finally:
        H.hmc_debug_set_grid_barrier()                     # defaults for everything after
    # the GPU is still usable: a fresh run matches a second fresh run bit for bit
    a = Sampler(p, adapt=True)
    xa = x0.clone()
    sa, _, _ = a.sample_chain(xa, p.num_burnin, p.num_results)
    b = Sampler(p, adapt=True)
    xb = x0.clone()
    sb, _, _ = b.sample_chain(xb, p.num_burnin, p.num_results)
    H.hmc_synchronize(a.ctx)
    H.hmc_synchronize(b.ctx)
    assert torch.equal(xa, xb) and torch.equal(sa, sb)
    assert np.isfinite(xa.cpu().numpy()).all()
    a.close()
    b.close()
