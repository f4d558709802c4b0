"""Replica exchange on the GPU against the float64 oracle: each transition
(tempered HMC for every replica, then the exchange step) teacher-forced from
the GPU's state, and the tempered marginals of a long run."""
import numpy as np
import pytest

from oracle import diagnostics, hmc as ohmc, philox, remc, targets as otargets
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


# the dense Gaussian cases run the CTA-pair tensor-core kernel, tempered:
# one K-chunk, several, and all eight (chunk 7 read from shared memory)
@pytest.mark.parametrize("kind,C,K,D,eps,L", [("std_normal", 40, 4, 3, 0.5, 3),
                                              ("funnel", 24, 3, 12, 0.05, 5),
                                              ("corr_gauss", 20, 3, 8, 0.1, 4),
                                              ("corr_gauss", 50, 4, 64, 0.08, 6),
                                              ("corr_gauss", 17, 3, 256, 0.05, 3)])
def test_replica_exchange_transition_matches_oracle(H, kind, C, K, D, eps, L):
    from paper_2002_01184_gb300.sampler import _CudaArray
    betas = np.array([1.0, 0.6, 0.35, 0.2][:K], dtype=np.float32)
    if D >= 64:
        # adjacent log-densities differ by ~ D dbeta / 2 in high dimension: keep
        # the spacing near sqrt(0.6 / D) so that swaps happen
        betas = (1.0 - np.sqrt(0.6 / D) * np.arange(K)).astype(np.float32)
    P = None
    if kind == "corr_gauss":
        prob = workloads.corr_gauss(dim=D, num_chains=C * K)
        P = torch.as_tensor(prob.P).cuda()
        tgt = otargets.make("corr_gauss", P=prob.P)
    else:
        tgt = otargets.std_normal if kind == "std_normal" else otargets.funnel
    target = H.make_target(kind, D, P)
    cfg = H.make_config(L, eps, seed=5, use_graph=False)
    ctx = H.hmc_remc_create(target, C, betas, cfg)
    if kind == "corr_gauss":
        assert H.hmc_dominant_kernel_info(ctx)[0] == "k_gauss_pair"
    x0 = (np.random.default_rng(1).standard_normal((C * K, D)) /
          np.sqrt(np.tile(betas, C))[:, None]).astype(np.float32)
    x = torch.as_tensor(x0).cuda().contiguous()
    H.hmc_bootstrap(ctx, x)
    tt = remc.tempered(tgt, betas.astype(np.float64))
    b = np.tile(betas.astype(np.float64), C)
    swaps_seen = 0
    for t in range(4):
        xin = host(x).astype(np.float64)
        lp, g = tt(xin)
        r = H.hmc_step(ctx, x, t)
        ref = ohmc.one_step(xin, lp, g, np.float32(eps), L, 5, t, tt)
        # the exchange step applied to the oracle's post-transition state
        lp_raw = (ref["lp"] / b).reshape(C, K)
        g_raw = (ref["g"] / b[:, None]).reshape(C, K, D)
        x3, _, _, sw = remc.exchange(ref["x"].reshape(C, K, D), lp_raw, g_raw, betas.astype(np.float64),
                                     5, t)
        swp = torch.as_tensor(_CudaArray(H.hmc_remc_swaps(ctx), (C, K - 1), "|u1"), device="cuda")
        sw_gpu = host(swp).astype(bool)
        acc = host(torch.as_tensor(_CudaArray(r.is_accepted, (C * K,), "|u1"), device="cuda"))
        la = host(torch.as_tensor(_CudaArray(r.log_accept_ratio, (C * K,), "<f4"), device="cuda"))
        # undo the GPU's exchange to compare the transition itself, then the swaps
        xg = host(x).astype(np.float64).reshape(C, K, D)
        if np.array_equal(sw_gpu, sw):
            np.testing.assert_allclose(xg, x3, rtol=1e-4, atol=1e-4)
        else:
            # a swap decision may differ only when its ratio is within float32 noise
            u = remc.swap_uniform(5, t, C, K)
            lr = (betas[:-1] - betas[1:]) * (lp_raw[:, 1:] - lp_raw[:, :-1])
            diff = sw_gpu != sw
            assert np.all(np.abs(np.log(u) - lr)[diff] < 1e-4)
        swaps_seen += int(sw_gpu.sum())
        pre = xg.copy()
        for c in range(C):
            for k in range(t % 2, K - 1, 2):
                if sw_gpu[c, k]:
                    pre[c, [k, k + 1]] = pre[c, [k + 1, k]]
        compare_transition(xin, pre.reshape(C * K, D), acc, la, ref, label=f"remc {kind} t={t}")
    assert swaps_seen > 0
    H.hmc_destroy(ctx)


def test_tempered_marginals_on_gpu(H):
    """Standard normal, betas 1, 0.5, 0.25: replica k's draws have variance
    1 / beta_k within 3 Monte Carlo standard errors."""
    betas = np.array([1.0, 0.5, 0.25], dtype=np.float32)
    C, K, D = 2000, 3, 1
    cfg = H.make_config(3, 0.8, seed=13)
    ctx = H.hmc_remc_create(H.make_target("std_normal", D), C, betas, cfg)
    x = torch.as_tensor((philox.momentum(5, 0, C * K, D) /
                         np.sqrt(np.tile(betas, C))[:, None]).astype(np.float32)).cuda().contiguous()
    Kr = 200
    samples = torch.empty((Kr, C * K, D), device="cuda")
    H.hmc_sample_chain(ctx, x, 50, Kr, samples)
    s = host(samples).astype(np.float64).reshape(Kr, C, K, D)
    for k in range(K):
        sk2 = s[:, :, k, :] ** 2
        assert abs(sk2.mean() - 1.0 / betas[k]) < 3 * diagnostics.mcse_mean(sk2)[0]
    H.hmc_destroy(ctx)


@pytest.mark.parametrize("K,C", [(4, 48), (32, 8)])
@pytest.mark.parametrize("cap", [0, 1, 7])
def test_replica_exchange_in_the_pair_launch_equals_step_by_step(H, cap, K, C):
    """sample_chain of a dense-Gaussian replica set runs the exchange step
    inside the CTA-pair launch (all transitions in one launch, one per launch,
    or launches of 7): the same kept states, final state and last swap flags
    as hmc_step followed by the exchange kernel, transition by transition.
    With 4 replicas both rows of every swapped pair belong to one epilogue
    thread (swapped in registers); with 32 a pair can straddle two threads
    (swapped through the [C x D] gradient cache)."""
    from paper_2002_01184_gb300.sampler import _CudaArray
    D, L, eps, B, Kk = 64, 5, 0.08, 6, 9
    if K == 4:
        betas = (1.0 - np.sqrt(0.6 / D) * np.arange(K)).astype(np.float32)
    else:
        betas = (0.97 ** np.arange(K)).astype(np.float32)
    prob = workloads.corr_gauss(dim=D, num_chains=C * K)
    P = torch.as_tensor(prob.P).cuda()
    target = H.make_target("corr_gauss", D, P)
    x0 = (np.random.default_rng(3).standard_normal((C * K, D)) /
          np.sqrt(np.tile(betas, C))[:, None]).astype(np.float32)
    ctx1 = H.hmc_remc_create(target, C, betas, H.make_config(L, eps, seed=5, use_graph=False))
    x1 = torch.as_tensor(x0).cuda().contiguous()
    H.hmc_bootstrap(ctx1, x1)
    ref = []
    for t in range(B + Kk):
        H.hmc_step(ctx1, x1, t)
        if t >= B:
            ref.append(host(x1).copy())
    sw1 = host(torch.as_tensor(_CudaArray(H.hmc_remc_swaps(ctx1), (C, K - 1), "|u1"), device="cuda")).copy()
    ctx2 = H.hmc_remc_create(target, C, betas,
                             H.make_config(L, eps, seed=5, max_transitions_per_launch=cap))
    x2 = torch.as_tensor(x0).cuda().contiguous()
    samples = torch.empty((Kk, C * K, D), dtype=torch.float32, device="cuda")
    H.hmc_sample_chain(ctx2, x2, B, Kk, samples, None, None)
    sw2 = host(torch.as_tensor(_CudaArray(H.hmc_remc_swaps(ctx2), (C, K - 1), "|u1"), device="cuda"))
    np.testing.assert_array_equal(host(samples), np.stack(ref))
    np.testing.assert_array_equal(host(x2), host(x1))
    np.testing.assert_array_equal(sw2, sw1)
    assert sw1.any()
    H.hmc_destroy(ctx1)
    H.hmc_destroy(ctx2)


def test_replica_set_host_entry_point_segments_large_pinned_sample_sets(H):
    """A replica set's kept samples (629 MB, bound for pinned host memory)
    leave the device in segments while the later transitions, exchange step
    included, run: the same samples, state and last swap flags as the device
    entry point."""
    from paper_2002_01184_gb300.sampler import _CudaArray
    C, K, D, L, eps, B, Kk = 1024, 4, 256, 4, 0.3, 10, 150
    betas = (1.0 - np.sqrt(0.6 / D) * np.arange(K)).astype(np.float32)
    prob = workloads.corr_gauss(dim=D, num_chains=C * K)
    P = torch.as_tensor(prob.P).cuda()
    target = H.make_target("corr_gauss", D, P)
    x0 = (np.random.default_rng(4).standard_normal((C * K, D)) /
          np.sqrt(np.tile(betas, C))[:, None]).astype(np.float32)
    ctx = H.hmc_remc_create(target, C, betas, H.make_config(L, eps, seed=6))
    x = torch.as_tensor(x0).cuda().contiguous()
    samples = torch.empty((Kk, C * K, D), dtype=torch.float32, device="cuda")
    H.hmc_sample_chain(ctx, x, B, Kk, samples, None, None)
    ref_s, ref_x = host(samples), host(x)
    ref_sw = host(torch.as_tensor(_CudaArray(H.hmc_remc_swaps(ctx), (C, K - 1), "|u1"), device="cuda")).copy()
    del samples
    xh = torch.from_numpy(x0.copy()).pin_memory()
    sh = torch.empty((Kk, C * K, D), dtype=torch.float32, pin_memory=True)
    H.hmc_sample_chain_host(ctx, xh, B, Kk, sh, None, None)
    sw = host(torch.as_tensor(_CudaArray(H.hmc_remc_swaps(ctx), (C, K - 1), "|u1"), device="cuda"))
    np.testing.assert_array_equal(sh.numpy(), ref_s)
    np.testing.assert_array_equal(xh.numpy(), ref_x)
    np.testing.assert_array_equal(sw, ref_sw)
    assert ref_sw.any()
    H.hmc_destroy(ctx)

