"""The Metropolis-Hastings composition on the GPU (Section 4.1): the random-
walk inner kernel, the Langevin proposal as one leapfrog step, and the
propose / select split of the ABI, against the float64 oracle."""
import math

import numpy as np
import pytest

from oracle import hmc as ohmc, mh as omh, targets as otargets
from paper_2002_01184_gb300 import workloads
from tests.parity import compare_transition

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


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda().contiguous()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def problem(kind, C, D, eps, N=300, L=1):
    if kind == "std_normal":
        p = workloads.std_normal(num_chains=C, dim=D, step_size=eps, num_leapfrog=L)
    elif kind == "funnel":
        p = workloads.funnel(dim=D, num_chains=C)
    elif kind == "corr_gauss":
        p = workloads.corr_gauss(dim=D, num_chains=C)
    else:
        p = workloads.logreg(n_data=N, dim=D, num_chains=C)
        p.x0 = (0.1 * np.random.default_rng(0).standard_normal(p.x0.shape)).astype(np.float32)
    p.step_size = eps
    p.num_leapfrog = L
    p.adapt = False
    return p


# (target, chains, dim, step size): one warp-tile and ragged shapes
RW_CASES = [("std_normal", 100, 1, 2.4), ("std_normal", 45, 13, 0.7), ("funnel", 37, 50, 0.08),
            ("corr_gauss", 130, 70, 0.15), ("logreg", 70, 20, 0.03)]


@pytest.mark.parametrize("kind,C,D,eps", RW_CASES)
def test_random_walk_transition_matches_oracle(H, kind, C, D, eps):
    from paper_2002_01184_gb300.sampler import Sampler
    p = problem(kind, C, D, eps)
    s = Sampler(p, adapt=False, proposal=H.HMC_PROPOSAL_RANDOM_WALK)
    assert not H.hmc_uses_tensor_cores(s.ctx)
    x = dev(p.x0)
    s.bootstrap(x)
    tgt = otargets.make(p.kind, **p.data())
    n_acc = 0
    for t in range(5):
        xin = host(x).astype(np.float64)
        lp, g = tgt(xin)
        r = s.results(s.step(x, t))
        ref = omh.rw_one_step(xin, lp, g, np.float32(eps), p.seed, t, tgt)
        compare_transition(xin, host(x), host(r["is_accepted"]), host(r["log_accept_ratio"]), ref,
                           label=f"rw {kind} t={t}")
        n_acc += int(host(r["is_accepted"]).sum())
    assert 0 < n_acc < 5 * C          # both decisions occur
    s.close()


@pytest.mark.parametrize("proposal", [0, 1], ids=["leapfrog", "random_walk"])
def test_propose_then_select_equals_step(H, proposal):
    """hmc_propose + hmc_mh_select is hmc_step, bit for bit, and the proposal
    the split exposes is the oracle's."""
    from paper_2002_01184_gb300.sampler import Sampler, device_view
    p = problem("corr_gauss", 96, 40, 0.1 if proposal == 0 else 0.2, L=4 if proposal == 0 else 1)
    a = Sampler(p, adapt=False, impl=H.HMC_IMPL_PLAIN, proposal=proposal)
    b = Sampler(p, adapt=False, impl=H.HMC_IMPL_PLAIN, proposal=proposal)
    xa, xb = dev(p.x0), dev(p.x0)
    a.bootstrap(xa)
    b.bootstrap(xb)
    tgt = otargets.make(p.kind, **p.data())
    for t in range(4):
        xin = host(xb).astype(np.float64)
        ra = a.results(a.step(xa, t))
        prop = H.hmc_propose(b.ctx, xb, t)
        xp = device_view(prop.x, (96, 40), "<f4").clone()
        lap = device_view(prop.log_accept_ratio, (96,), "<f4").clone()
        rb = b.results(H.hmc_mh_select(b.ctx, xb, t))
        assert torch.equal(xa, xb)
        assert torch.equal(ra["is_accepted"], rb["is_accepted"])
        assert torch.equal(ra["log_accept_ratio"], lap)
        lp, g = tgt(xin)
        ref = (ohmc.one_step(xin, lp, g, np.float32(p.step_size), p.num_leapfrog, p.seed, t, tgt)
               if proposal == 0 else omh.rw_one_step(xin, lp, g, np.float32(p.step_size), p.seed, t, tgt))
        err = np.max(np.abs(host(xp) - ref["proposed_x"]), axis=1) / np.maximum(
            np.max(np.abs(ref["proposed_x"]), axis=1), 1e-3)
        assert err.max() < 1e-4
    a.close()
    b.close()


def test_split_needs_the_plain_path(H):
    from paper_2002_01184_gb300.sampler import Sampler
    p = problem("corr_gauss", 64, 32, 0.1, L=2)
    s = Sampler(p, adapt=False)                       # tensor-core path
    x = dev(p.x0)
    s.bootstrap(x)
    with pytest.raises(H.HMCError) as ei:
        H.hmc_propose(s.ctx, x, 0)
    assert ei.value.status == H.HMC_E_UNSUPPORTED
    s.close()


def test_mala_acceptance_matches_the_langevin_formula(H):
    """Leapfrog with L = 1 is MALA: the GPU's log alpha against the Langevin
    proposal density evaluated by the oracle at the GPU's own proposal."""
    from paper_2002_01184_gb300.sampler import Sampler, device_view
    p = problem("funnel", 77, 30, 0.06, L=1)
    s = Sampler(p, adapt=False, impl=H.HMC_IMPL_PLAIN)
    x = dev(p.x0)
    s.bootstrap(x)
    tgt = otargets.make(p.kind, **p.data())
    for t in range(3):
        xin = host(x).astype(np.float64)
        lp, g = tgt(xin)
        prop = H.hmc_propose(s.ctx, x, t)
        xp = device_view(prop.x, (77, 30), "<f4").clone()
        la = host(device_view(prop.log_accept_ratio, (77,), "<f4").clone()).astype(np.float64)
        x1 = host(xp).astype(np.float64)
        lp1, g1 = tgt(x1)
        ref = omh.mala_log_accept(xin, lp, g, x1, lp1, g1, float(np.float32(p.step_size)))
        # float32 energies of O(|log p|) magnitude against float64
        tol = 1e-4 * np.maximum(1.0, np.abs(lp) + np.abs(lp1))
        assert np.all(np.abs(la - ref) < tol), np.max(np.abs(la - ref) / tol)
        H.hmc_mh_select(s.ctx, x, t)
    s.close()


def test_random_walk_chain_adapts_and_samples_the_normal(H):
    """sample_chain with the random walk and dual averaging on a 4-D standard
    normal: the kept acceptance rate is near the target and the moments are
    those of N(0, I) within Monte Carlo error."""
    from paper_2002_01184_gb300.sampler import Sampler
    p = workloads.std_normal(num_chains=2048, dim=4, step_size=0.5, num_leapfrog=1)
    p.adapt, p.target_accept, p.num_burnin, p.num_results = True, 0.35, 400, 400
    s = Sampler(p, adapt=True, proposal=H.HMC_PROPOSAL_RANDOM_WALK)
    x = torch.zeros((2048, 4), device="cuda")
    samples, eps, acc = s.sample_chain(x, p.num_burnin, p.num_results)
    H.hmc_synchronize(s.ctx)
    rate = float(acc.float().mean())
    assert abs(rate - 0.35) < 0.05, rate
    xs = host(samples)[100:].reshape(-1, 4)
    # 300 draws x 2048 independent chains; random-walk autocorrelation
    # inflates the variance of the mean by at most ~20x here
    se = math.sqrt(20.0 / xs.shape[0])
    assert np.all(np.abs(xs.mean(axis=0)) < 5 * se)
    assert np.all(np.abs(xs.var(axis=0) - 1.0) < 5 * math.sqrt(2.0) * se)
    s.close()
