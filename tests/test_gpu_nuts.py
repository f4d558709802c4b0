"""NUTS on the GPU (Section 2.3, the recursion unrolled) against the float64
oracle: teacher-forced transitions on the elementwise targets, and the
moments of a chain with step-size adaptation."""
import math

import numpy as np
import pytest

from oracle import nuts as onuts, targets as otargets
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


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda().contiguous()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


# (target, chains, dim, step size, max depth): a warp-tile, ragged dims, the
# three register widths (dim <= 128, 256, 512); span starts in shared memory
# except the last case, whose 2 x 9 span rows of 500 floats per chain exceed
# the shared-memory budget and live in the per-chain scratch
CASES = [("std_normal", 64, 5, 0.3, 6), ("std_normal", 37, 130, 0.25, 5),
         ("funnel", 40, 10, 0.1, 6), ("funnel", 19, 300, 0.03, 4),
         ("std_normal", 21, 500, 0.08, 10)]

# a decision closer than this (relative) to its threshold may go either way
# in float32
BAND = 1e-4


@pytest.mark.parametrize("kind,C,D,eps,depth", CASES)
def test_nuts_transition_matches_oracle(H, kind, C, D, eps, depth):
    from paper_2002_01184_gb300.sampler import Sampler
    if kind == "std_normal":
        p = workloads.std_normal(num_chains=C, dim=D, step_size=eps, num_leapfrog=depth)
        p.x0 = np.random.default_rng(1).standard_normal((C, D)).astype(np.float32)
    else:
        p = workloads.funnel(dim=D, num_chains=C)
    p.step_size, p.num_leapfrog, p.adapt = eps, depth, False
    s = Sampler(p, adapt=False, proposal=H.HMC_PROPOSAL_NUTS)
    name, _ = H.hmc_dominant_kernel_info(s.ctx)
    assert name == "k_nuts"
    x = dev(p.x0)
    s.bootstrap(x)
    tgt = otargets.make(kind)
    n_checked = n_moved = leaves = 0
    for t in range(4):
        xin = host(x).astype(np.float64)
        lp, g = tgt(xin)
        r = s.results(s.step(x, t))
        ref = onuts.one_step(xin, lp, g, float(np.float32(eps)), depth, p.seed, t, tgt)
        leaves += int(ref["leaves"].sum())
        xg = host(x).astype(np.float64)
        sure = ref["margin"] > BAND
        assert sure.sum() >= C - 3, (t, np.sort(ref["margin"])[:5])
        mv = host(r["is_accepted"]).astype(bool)
        np.testing.assert_array_equal(mv[sure], ref["is_accepted"][sure])
        err = np.max(np.abs(xg - ref["x"]), axis=1) / np.maximum(np.max(np.abs(ref["x"]), axis=1), 1e-3)
        assert err[sure].max() < 1e-4, err[sure].max()
        stat = np.exp(host(r["log_accept_ratio"]).astype(np.float64))
        np.testing.assert_allclose(stat[sure], ref["stat"][sure], rtol=1e-4, atol=1e-5)
        n_checked += int(sure.sum())
        n_moved += int(mv.sum())
        # teacher forcing: continue from the oracle's state where the two may differ
        if not sure.all():
            xg[~sure] = ref["x"][~sure]
            x.copy_(dev(xg.astype(np.float32)))
            s.close()
            s = Sampler(p, adapt=False, proposal=H.HMC_PROPOSAL_NUTS)
            s.bootstrap(x)
    assert n_moved > 0 and n_checked >= 4 * C - 12
    s.close()


def test_leapfrog_count_matches_the_trees(H):
    from paper_2002_01184_gb300.sampler import Sampler
    C, D, eps, depth = 50, 3, 0.2, 8
    p = workloads.std_normal(num_chains=C, dim=D, step_size=eps, num_leapfrog=depth)
    p.x0 = np.random.default_rng(2).standard_normal((C, D)).astype(np.float32)
    s = Sampler(p, adapt=False, proposal=H.HMC_PROPOSAL_NUTS)
    x = dev(p.x0)
    s.bootstrap(x)
    xin = host(x).astype(np.float64)
    lp, g = otargets.std_normal(xin)
    s.results(s.step(x, 0))
    ref = onuts.one_step(xin, lp, g, float(np.float32(eps)), depth, p.seed, 0, otargets.std_normal)
    got = H.hmc_nuts_leapfrog_count(s.ctx)
    if (ref["margin"] > BAND).all():
        assert got == int(ref["leaves"].sum())
    else:
        assert abs(got - int(ref["leaves"].sum())) <= 2 ** depth
    assert ref["depth"].max() >= 3
    s.close()


def test_nuts_chain_samples_the_standard_normal(H):
    """sample_chain with NUTS and dual averaging (target 0.8) on a 10-D
    standard normal: moments of N(0, I) within Monte Carlo error, step size
    adapted to the statistic."""
    from paper_2002_01184_gb300.sampler import Sampler
    C, D = 1024, 10
    p = workloads.std_normal(num_chains=C, dim=D, step_size=0.5, num_leapfrog=10)
    p.adapt, p.target_accept, p.num_burnin, p.num_results = True, 0.8, 200, 200
    s = Sampler(p, adapt=True, proposal=H.HMC_PROPOSAL_NUTS)
    x = torch.zeros((C, D), device="cuda")
    samples, eps, acc = s.sample_chain(x, p.num_burnin, p.num_results)
    H.hmc_synchronize(s.ctx)
    stat_eps = float(eps[-1])
    assert 0.1 < stat_eps < 2.0
    xs = host(samples)[50:].reshape(-1, D)
    se = math.sqrt(3.0 / xs.shape[0])        # NUTS draws are nearly independent
    assert np.all(np.abs(xs.mean(axis=0)) < 5 * se)
    assert np.all(np.abs(xs.var(axis=0) - 1.0) < 5 * math.sqrt(2.0) * se)
    assert float(acc.float().mean()) > 0.5
    s.close()


@pytest.mark.parametrize("adapt", [False, True], ids=["fixed", "adapted"])
def test_multi_transition_launch_is_bit_identical(H, adapt):
    """The transitions that do not adapt run in one launch (or launches of at
    most max_transitions_per_launch): the same samples, traces, final state
    and leapfrog count as one launch per transition."""
    from paper_2002_01184_gb300.sampler import Sampler
    C, D, B, K = 150, 70, 12, 30
    runs = []
    for cap in (1, 7, 0):
        p = workloads.funnel(dim=D, num_chains=C)
        p.num_leapfrog, p.adapt, p.num_burnin, p.num_results = 6, adapt, B, K
        p.step_size = 0.05
        s = Sampler(p, adapt=adapt, proposal=H.HMC_PROPOSAL_NUTS, max_transitions_per_launch=cap)
        x = dev(p.x0)
        samples, eps, acc = s.sample_chain(x, B, K)
        H.hmc_synchronize(s.ctx)
        runs.append((host(samples), host(eps), host(acc), host(x), H.hmc_nuts_leapfrog_count(s.ctx)))
        s.close()
    for other in runs[1:]:
        for u, w in zip(runs[0], other):
            np.testing.assert_array_equal(u, w)
    assert runs[0][2].any() and not runs[0][2].all()
    assert np.unique(runs[0][0][:, 0, 0]).size > K // 2         # the chain moved


@pytest.mark.parametrize("C,D,depth", [(1, 1, 1), (1, 1, 4), (33, 1, 3), (2, 4, 10)])
def test_nuts_edge_sizes_match_oracle(H, C, D, depth):
    """One chain, one dimension, depth 1 (a single leapfrog step) and the
    maximum depth, against the oracle transition by transition."""
    from paper_2002_01184_gb300.sampler import Sampler
    p = workloads.std_normal(num_chains=C, dim=D, step_size=0.7, num_leapfrog=depth)
    p.x0 = np.random.default_rng(C + D).standard_normal((C, D)).astype(np.float32)
    s = Sampler(p, adapt=False, proposal=H.HMC_PROPOSAL_NUTS)
    x = dev(p.x0)
    s.bootstrap(x)
    tgt = otargets.std_normal
    for t in range(6):
        xin = host(x).astype(np.float64)
        lp, g = tgt(xin)
        r = s.results(s.step(x, t))
        ref = onuts.one_step(xin, lp, g, float(np.float32(0.7)), depth, p.seed, t, tgt)
        sure = ref["margin"] > BAND
        xg = host(x).astype(np.float64)
        np.testing.assert_array_equal(host(r["is_accepted"]).astype(bool)[sure], ref["is_accepted"][sure])
        err = np.max(np.abs(xg - ref["x"]), axis=1) / np.maximum(np.max(np.abs(ref["x"]), axis=1), 1e-3)
        assert err[sure].max(initial=0.0) < 1e-4
        if not sure.all():                 # teacher forcing where float32 may decide otherwise
            xg[~sure] = ref["x"][~sure]
            x.copy_(dev(xg.astype(np.float32)))
            s.close()
            s = Sampler(p, adapt=False, proposal=H.HMC_PROPOSAL_NUTS)
            s.bootstrap(x)
    s.close()


def test_nuts_chain_is_independent_of_the_batch(H):
    """Chain c's transitions depend only on (seed, chain index, t): chain 5 of
    a 64-chain run equals a one-chain run with chain_offset 5."""
    from paper_2002_01184_gb300.sampler import Sampler
    p = workloads.funnel(dim=20, num_chains=64)
    p.step_size, p.num_leapfrog, p.adapt = 0.1, 7, False
    full = Sampler(p, adapt=False, proposal=H.HMC_PROPOSAL_NUTS)
    x = dev(p.x0)
    full.bootstrap(x)
    p1 = workloads.funnel(dim=20, num_chains=1)
    p1.x0 = p.x0[5:6].copy()
    p1.step_size, p1.num_leapfrog, p1.adapt = 0.1, 7, False
    one = Sampler(p1, adapt=False, proposal=H.HMC_PROPOSAL_NUTS, chain_offset=5)
    x1 = dev(p1.x0)
    one.bootstrap(x1)
    for t in range(5):
        full.step(x, t)
        one.step(x1, t)
        np.testing.assert_array_equal(host(x1)[0], host(x)[5])
    full.close()
    one.close()
