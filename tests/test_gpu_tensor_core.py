"""The tensor-core (tcgen05, 3xTF32) transition for the dense Gaussian
target against the float64 oracle, teacher-forced transition by transition,
on sizes that span several tiles with ragged edges in every dimension."""
import numpy as np
import pytest

from oracle import hmc as ohmc, targets as otargets
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


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


# (chains, dim, step size, leapfrog steps): one tile; ragged K/N/M tails;
# several tiles in every direction; the full dimension of the workload
CASES = [(128, 64, 0.1, 3), (130, 100, 0.08, 5), (257, 196, 0.06, 4), (512, 256, 0.05, 16),
         (33, 32, 0.2, 1), (4096, 256, 0.05, 2),
         # dimensions past 256 take the one-launch-per-leapfrog-step kernel
         (100, 320, 0.04, 3)]


@pytest.mark.parametrize("impl", [0, 2], ids=["pair", "single"])
@pytest.mark.parametrize("C,D,eps,L", CASES)
def test_tensor_core_transition_matches_oracle(H, C, D, eps, L, impl):
    from paper_2002_01184_gb300.sampler import Sampler
    if D > 256 and impl == 2:
        pytest.skip("one variant past dim 256")
    p = workloads.corr_gauss(dim=D, num_chains=C, num_burnin=0, num_results=0, num_leapfrog=L)
    p.step_size = eps
    s = Sampler(p, adapt=False, impl=impl)
    assert H.hmc_uses_tensor_cores(s.ctx)
    name, per_launch = H.hmc_dominant_kernel_info(s.ctx)
    expect = "k_gauss_tc_step" if D > 256 else ("k_gauss_pair" if impl == 0 else "k_gauss_fused")
    assert name == expect
    x = torch.as_tensor(p.x0).cuda().contiguous()
    s.bootstrap(x)
    tgt = otargets.make("corr_gauss", P=p.P)
    n_same = 0
    for t in range(4):
        xin = host(x).astype(np.float64)
        lp, g = tgt(xin)
        r = s.results(s.step(x, t))
        H.hmc_synchronize(s.ctx)
        ref = ohmc.one_step(xin, lp, g, np.float32(eps), L, p.seed, t, tgt)
        a, _ = compare_transition(xin, host(x), host(r["is_accepted"]), host(r["log_accept_ratio"]),
                                  ref, label=f"tc C={C} D={D} t={t}")
        n_same += a
        lp_new, g_new = tgt(host(x).astype(np.float64))
        np.testing.assert_allclose(host(r["target_log_prob"]), lp_new, rtol=1e-4,
                                   atol=1e-4 * max(1.0, np.abs(lp_new).max()))
        gg = host(r["grad"])
        row = np.max(np.abs(g_new), axis=1, keepdims=True)
        assert np.max(np.abs(gg - g_new) / np.maximum(row, 1e-6)) < 1e-4
    assert n_same >= 4 * C - 2
    s.close()


def test_tensor_core_and_plain_paths_agree(H):
    """Same seeds through both implementations, transition by transition
    with step-size adaptation: identical accept decisions away from the
    decision band, positions within the tolerance, and step sizes equal to
    1e-4 for as long as every decision so far has agreed.  Each update then
    sees the same acceptance statistics up to float32 rounding: energies of
    about 10^2 carry about 1e-5 of rounding in log alpha, so each chain's
    acceptance probability differs by up to about 1e-5, and dual averaging
    scales the mean's difference by sqrt(t) / (gamma (t + t0)) <= 3 over
    these transitions (gamma 0.05, t0 10).  After a decision differs, the
    two chains' states, and with them the later statistics, part: the step
    sizes then only agree to 1e-3."""
    from paper_2002_01184_gb300.sampler import Sampler
    p = workloads.corr_gauss(dim=64, num_chains=200, num_burnin=5, num_results=5, num_leapfrog=6)
    T = p.num_burnin + p.num_results
    sf, sp = Sampler(p, impl=H.HMC_IMPL_FUSED), Sampler(p, impl=H.HMC_IMPL_PLAIN)
    xf = torch.as_tensor(p.x0).cuda().contiguous()
    xp = xf.clone()
    sf.bootstrap(xf)
    sp.bootstrap(xp)
    parted = False
    agree = []
    ever = np.zeros(p.num_chains, dtype=bool)      # chains whose decisions differed at some step
    for t in range(T):
        rf, rp = sf.results(sf.step(xf, t)), sp.results(sp.step(xp, t))
        af, ap = host(rf["is_accepted"]).astype(bool), host(rp["is_accepted"]).astype(bool)
        ef, ep = float(rf["step_size"][0]), float(rp["step_size"][0])
        if not parted:
            assert abs(ef - ep) <= 1e-4 * abs(ep), (t, ef, ep)
        else:
            assert abs(ef - ep) <= 1e-3 * abs(ep), (t, ef, ep)
        parted = parted or bool((af != ap).any())
        agree.append((af == ap).mean())
        ever |= af != ap
        np.testing.assert_allclose(host(xf)[~ever], host(xp)[~ever], rtol=1e-3, atol=1e-3)
    assert np.mean(agree) > 0.99
    sf.close()
    sp.close()


# logistic regression on tensor cores: (chains, dim, data rows, step, L) --
# ragged chain groups, ragged last data tile, dims below / at the 128 limit
LOGREG_CASES = [(130, 64, 2500, 0.01, 3), (200, 128, 4100, 0.005, 2), (64, 20, 2049, 0.02, 4),
                # dims past the pair kernel's 128: one-CTA tile products (dim 260 leaves a
                # ragged K-chunk, 2500 a ragged data tile)
                (150, 160, 2500, 0.008, 3), (70, 260, 3001, 0.005, 2), (300, 512, 2100, 0.003, 2),
                # rows padded to a multiple of 4 inside the workspace: one-CTA
                # tiles (203), CTA pairs (37, 63, 127 over two ragged pairs)
                (90, 203, 2300, 0.005, 2), (40, 37, 2100, 0.01, 3), (300, 63, 2200, 0.01, 2),
                (140, 127, 2400, 0.006, 2),
                # 38 x 8 = 304 tiles of G = R X fill two waves of the SMs: no K-split
                # (the cases above split K and sum the splits)
                (4864, 452, 2100, 0.003, 1),
                # short data passes with much work per gradient (chains x rows x dim > 2^22)
                (600, 100, 1500, 0.005, 2), (500, 90, 1000, 0.006, 2),
                # CTA pairs whose ranges of (chain group, data tile) items cross
                # from one group into the next (3 groups x 157 tiles over the pairs)
                (600, 64, 20000, 0.002, 2)]


@pytest.mark.parametrize("C,D,N,eps,L", LOGREG_CASES)
def test_tensor_core_logreg_transition_matches_oracle(H, C, D, N, eps, L):
    from paper_2002_01184_gb300.sampler import Sampler
    p = workloads.logreg(n_data=N, dim=D, num_chains=C, num_burnin=0, num_results=0, num_leapfrog=L)
    p.step_size = eps
    p.x0 = (0.05 * np.random.default_rng(D).standard_normal((C, D))).astype(np.float32)
    s = Sampler(p, adapt=False)
    assert H.hmc_uses_tensor_cores(s.ctx)
    pair = D <= 128
    assert H.hmc_dominant_kernel_info(s.ctx)[0] == ("k_lr_grad" if pair else "k_gauss_tc_step<logreg>")
    x = torch.as_tensor(p.x0).cuda().contiguous()
    s.bootstrap(x)
    tgt = otargets.make("logreg", X=p.X, y=p.y)
    n_same = 0
    for t in range(3):
        xin = host(x).astype(np.float64)
        lp, g = tgt(xin)
        r = s.results(s.step(x, t))
        H.hmc_synchronize(s.ctx)
        ref = ohmc.one_step(xin, lp, g, np.float32(eps), L, p.seed, t, tgt)
        a, _ = compare_transition(xin, host(x), host(r["is_accepted"]), host(r["log_accept_ratio"]),
                                  ref, label=f"lr-tc C={C} D={D} N={N} t={t}")
        n_same += a
        lp_new, g_new = tgt(host(x).astype(np.float64))
        np.testing.assert_allclose(host(r["target_log_prob"]), lp_new, rtol=1e-4,
                                   atol=1e-4 * max(1.0, np.abs(lp_new).max()))
        gg = host(r["grad"])
        row = np.max(np.abs(g_new), axis=1, keepdims=True)
        assert np.max(np.abs(gg - g_new) / np.maximum(row, 1e-6)) < 1e-4
    assert n_same >= 3 * C - max(2, C // 500)      # decisions inside the float32 band
    s.close()


def test_full_size_logreg_transition_matches_oracle(H):
    """The logistic-regression workload at its full size (2048 chains, 20000
    rows, dim 128, L = 10), in the launch configuration the bench times (the
    CTA-pair tensor-core products, 9 data ranges x 8 chain groups), teacher-
    forced against the float64 oracle for one transition on every chain (the
    oracle's transition at this size takes about half a minute on the host).
    Chains start near the posterior mode (a few Newton steps of the float64
    log-density) so that the trajectories are the posterior's, not a
    divergence from the prior mean."""
    from paper_2002_01184_gb300.sampler import Sampler
    C, D, N, L, eps = 2048, 128, 20000, 10, 0.004
    p = workloads.logreg(n_data=N, dim=D, num_chains=C, num_burnin=0, num_results=0, num_leapfrog=L)
    X, y = p.X.astype(np.float64), p.y.astype(np.float64)
    w = np.zeros(D)
    for _ in range(8):                         # Newton on y.z - softplus(z) - |w|^2/2
        z = X @ w
        s_ = 1.0 / (1.0 + np.exp(-z))
        grad = X.T @ (y - s_) - w
        hess = -(X.T * (s_ * (1 - s_))) @ X - np.eye(D)
        w = w - np.linalg.solve(hess, grad)
    rng = np.random.default_rng(5)
    p.x0 = (w + rng.standard_normal((C, D)) * (0.5 / np.sqrt(N))).astype(np.float32)
    p.step_size = eps
    s = Sampler(p, adapt=False)
    assert H.hmc_dominant_kernel_info(s.ctx)[0] == "k_lr_grad"
    x = torch.as_tensor(p.x0).cuda().contiguous()
    s.bootstrap(x)
    tgt = otargets.make("logreg", X=p.X, y=p.y)
    xin = host(x).astype(np.float64)
    lp, g = tgt(xin)
    r = s.results(s.step(x, 0))
    H.hmc_synchronize(s.ctx)
    ref = ohmc.one_step(xin, lp, g, np.float32(eps), L, p.seed, 0, tgt)
    n_same, _ = compare_transition(xin, host(x), host(r["is_accepted"]), host(r["log_accept_ratio"]),
                                   ref, label="lr-tc full size")
    gg = host(r["grad"])
    _, g_new = tgt(host(x).astype(np.float64))
    row = np.max(np.abs(g_new), axis=1, keepdims=True)
    assert np.max(np.abs(gg - g_new) / np.maximum(row, 1e-6)) < 1e-4
    assert n_same >= C - 2
    assert 0.3 < float(host(r["is_accepted"]).mean()) < 1.0     # real proposals, mostly accepted
    s.close()
