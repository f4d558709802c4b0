"""NUTS on the dense targets (Section 2.3 over the correlated Gaussian and
the Bayesian logistic regression): the chains advance in lockstep, one leaf
per iteration whose gradients are tensor-core products (a persistent launch
for the Gaussian, a CUDA-graph loop for the logistic regression).
Teacher-forced transitions against the float64 oracle, the loop's length,
independence of the batch, the graph path against single steps, and the
moments of an adapted chain."""
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


# a decision closer than this to its threshold may go either way in float32
# (energies of a few hundred carry rounding of order 1e-5; U-turn margins are
# relative).  A tree of tens of leaves meets hundreds of decisions, so a few
# per cent of the chains meet one inside the band.
BAND = 2e-4


def gauss_problem(C, D, eps, depth, seed=11):
    p = workloads.corr_gauss(dim=D, num_chains=C, seed=seed)
    p.step_size, p.num_leapfrog, p.adapt = eps, depth, False
    return p


def logreg_problem(C, D, N, eps, depth, seed=12):
    p = workloads.logreg(n_data=N, dim=D, num_chains=C, seed=seed)
    # start near the posterior: N(w_true, 0.1^2)
    rng = np.random.default_rng(seed + 100)
    p.x0 = (p.w_true[None, :] + 0.1 * rng.standard_normal((C, D))).astype(np.float32)
    p.step_size, p.num_leapfrog, p.adapt = eps, depth, False
    return p


# (kind, chains, dim, data rows, step size, max depth): several 128-chain
# tiles with a ragged last tile; dims with one and two 128-float lane blocks;
# logistic regressions on the CTA-pair kernel (dim a multiple of 4, <= 128:
# two pairs, the second ragged, data rows split over ranges) and on the
# one-CTA tile products (rows padded, dim 5 -> 8; dim 130; ragged data tiles)
CASES = [("corr_gauss", 300, 64, 0, 0.3, 6), ("corr_gauss", 130, 256, 0, 0.25, 5),
         ("corr_gauss", 37, 8, 0, 0.5, 10),
         ("logreg", 300, 32, 1000, 0.03, 6), ("logreg", 280, 128, 2000, 0.01, 5),
         ("logreg", 200, 5, 300, 0.06, 6), ("logreg", 130, 130, 257, 0.02, 5)]


def make(kind, C, D, N, eps, depth):
    if kind == "corr_gauss":
        p = gauss_problem(C, D, eps, depth)
        tgt = otargets.make("corr_gauss", P=p.P)
    else:
        p = logreg_problem(C, D, N, eps, depth)
        tgt = otargets.make("logreg", X=p.X, y=p.y)
    return p, tgt


@pytest.mark.parametrize("kind,C,D,N,eps,depth", CASES)
def test_dense_nuts_transition_matches_oracle(H, kind, C, D, N, eps, depth):
    from paper_2002_01184_gb300.sampler import Sampler
    p, tgt = make(kind, C, D, N, eps, depth)
    s = Sampler(p, adapt=False, proposal=H.HMC_PROPOSAL_NUTS)
    name, _ = H.hmc_dominant_kernel_info(s.ctx)
    assert name == "nuts_dense_transition"
    assert H.hmc_uses_tensor_cores(s.ctx)
    x = dev(p.x0)
    s.bootstrap(x)
    n_checked = n_moved = 0
    worst = 0.0
    it0 = H.hmc_nuts_leaf_iterations(s.ctx)
    for t in range(3):
        xin = host(x).astype(np.float64)
        lp, g = tgt(xin)
        r = s.results(s.step(x, t))
        ref = onuts.one_step(xin, lp, g, float(np.float32(eps)), depth, p.seed, t, tgt)
        xg = host(x).astype(np.float64)
        sure = ref["margin"] > BAND
        assert sure.sum() >= 0.9 * C, (t, np.sort(ref["margin"])[:5])
        mv = host(r["is_accepted"]).astype(bool)
        np.testing.assert_array_equal(mv[sure], ref["is_accepted"][sure])
        err = np.max(np.abs(xg - ref["x"]), axis=1) / np.maximum(np.max(np.abs(ref["x"]), axis=1), 1e-3)
        worst = max(worst, float(err[sure].max()))
        assert err[sure].max() < 1e-4, err[sure].max()
        stat = np.exp(host(r["log_accept_ratio"]).astype(np.float64))
        np.testing.assert_allclose(stat[sure], ref["stat"][sure], rtol=1e-3, atol=1e-4)
        # the kernel results: log p and gradient of the new state
        lpn, gn = tgt(xg)
        np.testing.assert_allclose(host(r["target_log_prob"])[sure], lpn[sure],
                                   rtol=1e-4, atol=1e-4 * np.abs(lpn).max())
        gg = host(r["grad"]).astype(np.float64)
        gerr = np.max(np.abs(gg - gn), axis=1) / np.maximum(np.max(np.abs(gn), axis=1), 1e-3)
        assert gerr[sure].max() < 1e-4
        # the loop ran as many iterations as the deepest tree had leaves
        it1 = H.hmc_nuts_leaf_iterations(s.ctx)
        if sure.all():
            assert it1 - it0 == int(ref["leaves"].max())
        it0 = it1
        n_checked += int(sure.sum())
        n_moved += int(mv.sum())
        if not sure.all():           # teacher forcing where float32 may decide otherwise
            xg[~sure] = ref["x"][~sure]
            x.copy_(dev(xg.astype(np.float32)))
            s.bootstrap(x)
    assert n_moved > 0 and n_checked >= 0.9 * 3 * C
    print(f"{kind} C={C} D={D}: largest per-chain position error {worst:.2e}")
    s.close()


def test_leapfrog_count_and_depths(H):
    """The leapfrog count is the sum of the trees' leaves and the loop length
    the largest tree, with trees of several depths in one batch."""
    from paper_2002_01184_gb300.sampler import Sampler
    p, tgt = make("corr_gauss", 260, 32, 0, 0.35, 7)
    s = Sampler(p, adapt=False, proposal=H.HMC_PROPOSAL_NUTS)
    x = dev(p.x0)
    s.bootstrap(x)
    xin = host(x).astype(np.float64)
    lp, g = tgt(xin)
    l0 = H.hmc_nuts_leapfrog_count(s.ctx)
    s.results(s.step(x, 0))
    ref = onuts.one_step(xin, lp, g, float(np.float32(0.35)), 7, p.seed, 0, tgt)
    got = H.hmc_nuts_leapfrog_count(s.ctx) - l0
    if (ref["margin"] > BAND).all():
        assert got == int(ref["leaves"].sum())
        assert H.hmc_nuts_leaf_iterations(s.ctx) == int(ref["leaves"].max())
    else:
        assert abs(got - int(ref["leaves"].sum())) <= 2 ** 7
    assert np.unique(ref["depth"]).size >= 2
    s.close()


@pytest.mark.parametrize("kind", ["corr_gauss", "logreg"])
def test_dense_chain_is_independent_of_the_batch(H, kind):
    """Chain 150 of a 200-chain run equals a one-chain run with chain_offset
    150, bit for bit: its row of every product and its tree are its own."""
    from paper_2002_01184_gb300.sampler import Sampler
    p, _ = make(kind, 200, 24, 400, 0.3 if kind == "corr_gauss" else 0.05, 6)
    full = Sampler(p, adapt=False, proposal=H.HMC_PROPOSAL_NUTS)
    x = dev(p.x0)
    full.bootstrap(x)
    p1, _ = make(kind, 1, 24, 400, 0.3 if kind == "corr_gauss" else 0.05, 6)
    p1.x0 = p.x0[150:151].copy()
    one = Sampler(p1, adapt=False, proposal=H.HMC_PROPOSAL_NUTS, chain_offset=150)
    x1 = dev(p1.x0)
    one.bootstrap(x1)
    for t in range(4):
        full.step(x, t)
        one.step(x1, t)
        np.testing.assert_array_equal(host(x1)[0], host(x)[150])
    full.close()
    one.close()


@pytest.mark.parametrize("kind", ["corr_gauss", "logreg"])
def test_sample_chain_graph_equals_steps(H, kind):
    """sample_chain (one graph with a loop node per transition, adaptation
    included) equals the same transitions enqueued one hmc_step at a time."""
    from paper_2002_01184_gb300.sampler import Sampler
    B, K = 6, 5
    runs = []
    for graph in (True, False):
        p, _ = make(kind, 140, 16, 300, 0.4 if kind == "corr_gauss" else 0.08, 6)
        p.adapt, p.num_burnin, p.num_results, p.target_accept = True, B, K, 0.8
        s = Sampler(p, adapt=True, proposal=H.HMC_PROPOSAL_NUTS, use_graph=graph)
        x = dev(p.x0)
        if graph:
            samples, eps, acc = s.sample_chain(x, B, K)
            out = (host(samples), host(eps), host(acc), host(x))
        else:
            s.bootstrap(x)
            keep, eps, acc = [], [], []
            for t in range(B + K):
                r = s.results(s.step(x, t))
                if t >= B:
                    keep.append(host(x).copy())
                    eps.append(float(r["step_size"][0]))
                    acc.append(host(r["is_accepted"]).copy())
            out = (np.stack(keep), None, np.stack(acc), host(x))
        H.hmc_synchronize(s.ctx)
        runs.append((out, H.hmc_nuts_leapfrog_count(s.ctx), H.hmc_nuts_leaf_iterations(s.ctx)))
        s.close()
    (a, la, ia), (b, lb, ib) = runs
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[2], b[2])
    np.testing.assert_array_equal(a[3], b[3])
    assert la == lb and ia == ib


@pytest.mark.parametrize("kind", ["corr_gauss", "logreg"])
def test_host_entry_point_equals_device_entry_point(H, kind):
    """hmc_sample_chain_host (state and traces in pinned host memory) runs
    the same transitions as the device entry point."""
    from paper_2002_01184_gb300.sampler import Sampler
    p, _ = make(kind, 130, 16, 400, 0.4 if kind == "corr_gauss" else 0.08, 6)
    p.adapt, p.num_burnin, p.num_results, p.target_accept = True, 5, 6, 0.8
    s = Sampler(p, adapt=True, proposal=H.HMC_PROPOSAL_NUTS)
    x = dev(p.x0)
    samples, eps, acc = s.sample_chain(x, p.num_burnin, p.num_results)
    torch.cuda.synchronize()
    C, D, K = p.num_chains, p.dim, p.num_results
    xh = torch.as_tensor(p.x0).clone().pin_memory()
    sh = torch.empty((K, C, D), dtype=torch.float32).pin_memory()
    eh = torch.empty(K, dtype=torch.float32).pin_memory()
    ah = torch.empty((K, C), dtype=torch.uint8).pin_memory()
    H.hmc_sample_chain_host(s.ctx, xh, p.num_burnin, K, sh, eh, ah)
    H.hmc_synchronize(s.ctx)
    np.testing.assert_array_equal(xh.numpy(), host(x))
    np.testing.assert_array_equal(sh.numpy(), host(samples))
    np.testing.assert_array_equal(eh.numpy(), host(eps))
    np.testing.assert_array_equal(ah.numpy(), host(acc))
    s.close()


def test_dense_nuts_samples_the_gaussian(H):
    """sample_chain with NUTS and dual averaging on a 16-D correlated
    Gaussian: means and marginal variances of N(0, P^-1) within Monte Carlo
    error; the step size adapts to the statistic."""
    from paper_2002_01184_gb300.sampler import Sampler
    C, D = 1024, 16
    p = workloads.corr_gauss(dim=D, num_chains=C, seed=7, num_burnin=150, num_results=150)
    p.num_leapfrog, p.target_accept = 8, 0.8
    s = Sampler(p, adapt=True, proposal=H.HMC_PROPOSAL_NUTS)
    x = dev(p.x0)
    samples, eps, acc = s.sample_chain(x, p.num_burnin, p.num_results)
    H.hmc_synchronize(s.ctx)
    assert 0.05 < float(eps[-1]) < 2.0
    xs = host(samples)[20:].reshape(-1, D).astype(np.float64)
    cov = np.linalg.inv(p.P.astype(np.float64))
    var = np.diag(cov)
    n = xs.shape[0] / 3.0                   # NUTS draws: a conservative effective size
    assert np.all(np.abs(xs.mean(axis=0)) < 5 * np.sqrt(var / n))
    assert np.all(np.abs(xs.var(axis=0) / var - 1.0) < 5 * math.sqrt(2.0 / n))
    assert float(acc.float().mean()) > 0.5
    s.close()


def test_dense_nuts_shape_limits(H):
    """The tensor-core products' row stride needs a multiple of 4 floats for
    the Gaussian; dims above 512 are refused for both dense targets."""
    from paper_2002_01184_gb300.sampler import Sampler
    p = gauss_problem(8, 6, 0.3, 4)
    with pytest.raises(H.HMCError) as e:
        Sampler(p, adapt=False, proposal=H.HMC_PROPOSAL_NUTS)
    assert e.value.status == H.HMC_E_UNSUPPORTED
    p = logreg_problem(8, 520, 64, 0.01, 3)
    with pytest.raises(H.HMCError) as e:
        Sampler(p, adapt=False, proposal=H.HMC_PROPOSAL_NUTS)
    assert e.value.status == H.HMC_E_UNSUPPORTED
