"""Batched posteriors of uneven size, the small ones in one persistent
launch for all their transitions: every posterior's chains must follow
exactly the transitions they follow when the posterior is sampled alone
(same seeds, same kernels), each posterior adapts its own step size, and a
grouped member's transition matches the float64 oracle."""
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


def small_batch():
    probs = workloads.uneven_batch(seed=5, n_logreg=5, n_funnel=3, num_burnin=15, num_results=10,
                                   dim_range=(8, 64), n_range=(50, 400), chain_range=(9, 70),
                                   funnel_dim_range=(10, 40))
    # members with long data passes run on side streams: one on the tensor
    # cores (dim <= 128), one on the tiled SIMT products (dim > 128)
    probs.append(workloads.logreg(n_data=2500, dim=16, num_chains=33, seed=77, num_burnin=15,
                                  num_results=10))
    probs.append(workloads.logreg(n_data=600, dim=200, num_chains=40, seed=78, num_burnin=15,
                                  num_results=10))
    return probs


def test_batch_equals_each_posterior_alone(H):
    from paper_2002_01184_gb300.sampler import Sampler
    probs = small_batch()
    probs[1].num_burnin, probs[1].num_results = 5, 4      # uneven schedules too
    dev = lambda a: torch.as_tensor(a).cuda().contiguous()
    keep = []
    targets, chains, configs = [], [], []
    for p in probs:
        Xd = dev(p.X) if p.X is not None else None
        yd = dev(p.y) if p.y is not None else None
        keep.append((Xd, yd))
        targets.append(H.make_target(p.kind, p.dim, None, Xd, yd))
        chains.append(p.num_chains)
        configs.append(H.make_config(p.num_leapfrog, p.step_size, p.seed, p.adapt, p.target_accept,
                                     p.num_burnin))
    batch = H.hmc_batch_create(targets, chains, configs)
    xs = [dev(p.x0) for p in probs]
    samples = [torch.empty((p.num_results, p.num_chains, p.dim), device="cuda") for p in probs]
    eps = [torch.empty(p.num_results, device="cuda") for p in probs]
    acc = [torch.empty((p.num_results, p.num_chains), dtype=torch.uint8, device="cuda") for p in probs]
    for rep in range(2):                    # capture, then replay the graph
        xs = [dev(p.x0) for p in probs] if rep == 0 else xs
        if rep == 1:
            for x, p in zip(xs, probs):
                x.copy_(dev(p.x0))
        H.hmc_batch_sample_chain(batch, xs, [p.num_burnin for p in probs],
                                 [p.num_results for p in probs], samples, eps, acc)
        H.hmc_batch_synchronize(batch)
        for i, p in enumerate(probs):
            # a grouped logistic regression runs the shared-memory SIMT tile;
            # alone, the same path is HMC_IMPL_FUSED_SIMT (the default picks
            # the tensor cores for a narrow grid with a long data pass)
            path, _, _ = H.hmc_batch_member_path(batch, i)
            grouped_lr = p.kind == "logreg" and path == 0
            s = Sampler(p, impl=H.HMC_IMPL_FUSED_SIMT if grouped_lr else H.HMC_IMPL_FUSED)
            x = dev(p.x0)
            smp, e, a = s.sample_chain(x, p.num_burnin, p.num_results)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(xs[i].cpu().numpy(), x.cpu().numpy())
            np.testing.assert_array_equal(samples[i].cpu().numpy(), smp.cpu().numpy())
            np.testing.assert_array_equal(eps[i].cpu().numpy(), e.cpu().numpy())
            np.testing.assert_array_equal(acc[i].cpu().numpy(), a.cpu().numpy())
            s.close()
    H.hmc_batch_destroy(batch)


def test_batch_rejects_unsupported_targets(H):
    p = workloads.corr_gauss(dim=8, num_chains=4)
    P = torch.as_tensor(p.P).cuda()
    with pytest.raises(H.HMCError) as ei:
        H.hmc_batch_create([H.make_target("corr_gauss", 8, P)], [4], [H.make_config(2, 0.1)])
    assert ei.value.status == H.HMC_E_UNSUPPORTED


def test_grouped_members_transitions_match_oracle(H):
    """Teacher-forced through the batch: with a fixed step size, each call
    runs one transition (index 0) of every posterior from the state the
    previous call left, and the float64 oracle takes the same transition from
    the same float32 state: positions within 1e-4 per chain, accept decisions
    equal outside the 1e-5 band (tests/parity.py's reading)."""
    from oracle import hmc as ohmc, targets as otargets
    from tests.parity import DECISION_BAND, POS_RTOL, chain_error
    probs = workloads.uneven_batch(seed=9, n_logreg=3, n_funnel=2, num_burnin=0, num_results=1,
                                   dim_range=(8, 48), n_range=(60, 300), chain_range=(9, 40),
                                   funnel_dim_range=(10, 30))
    dev = lambda a: torch.as_tensor(a).cuda().contiguous()
    keep, targets, chains, configs = [], [], [], []
    for p in probs:
        p.adapt = False
        p.step_size = 0.02 if p.kind == "logreg" else 0.1
        if p.kind == "logreg":
            p.x0 = (0.1 * np.random.default_rng(p.seed).standard_normal(p.x0.shape)).astype(np.float32)
        Xd = dev(p.X) if p.X is not None else None
        yd = dev(p.y) if p.y is not None else None
        keep.append((Xd, yd))
        targets.append(H.make_target(p.kind, p.dim, None, Xd, yd))
        chains.append(p.num_chains)
        configs.append(H.make_config(p.num_leapfrog, p.step_size, p.seed, False, p.target_accept, 0))
    batch = H.hmc_batch_create(targets, chains, configs)
    xs = [dev(p.x0) for p in probs]
    acc = [torch.empty((1, p.num_chains), dtype=torch.uint8, device="cuda") for p in probs]
    for rep in range(3):
        before = [x.double().cpu().numpy() for x in xs]
        H.hmc_batch_sample_chain(batch, xs, [0] * len(probs), [1] * len(probs), None, None, acc)
        H.hmc_batch_synchronize(batch)
        for i, p in enumerate(probs):
            tgt = otargets.make(p.kind, **p.data())
            lp, g = tgt(before[i])
            ref = ohmc.one_step(before[i], lp, g, float(np.float32(p.step_size)), p.num_leapfrog, p.seed, 0, tgt)
            a_gpu = acc[i][0].cpu().numpy().astype(bool)
            near = np.abs(ref["log_u"] - ref["log_accept_ratio"]) < DECISION_BAND
            assert np.all((a_gpu == ref["is_accepted"]) | near), (p.kind, rep)
            same = a_gpu == ref["is_accepted"]
            err = chain_error(xs[i].double().cpu().numpy(), ref["x"])
            assert err[same].max() <= POS_RTOL, (p.kind, rep, err[same].max())
    H.hmc_batch_destroy(batch)


def test_autotuned_batch_equals_each_posterior_alone_on_its_chosen_path(H):
    """The autotuner times each logistic regression's two paths (grouped SIMT
    tiles, tensor-core products in a context of its own) and the batch runs
    each on the faster: a member then equals sampling it alone with the
    matching impl, bit for bit.  A second batch of the same shapes reuses
    the cached choices."""
    from paper_2002_01184_gb300.sampler import Sampler
    probs = small_batch()
    dev = lambda a: torch.as_tensor(a).cuda().contiguous()
    keep, targets, chains, configs = [], [], [], []
    for p in probs:
        Xd = dev(p.X) if p.X is not None else None
        yd = dev(p.y) if p.y is not None else None
        keep.append((Xd, yd))
        targets.append(H.make_target(p.kind, p.dim, None, Xd, yd))
        chains.append(p.num_chains)
        configs.append(H.make_config(p.num_leapfrog, p.step_size, p.seed, p.adapt, p.target_accept,
                                     p.num_burnin))
    batch = H.hmc_batch_create_autotuned(targets, chains, configs)
    paths = [H.hmc_batch_member_path(batch, i) for i in range(len(probs))]
    for p, (path, mg, mt) in zip(probs, paths):
        if p.kind == "logreg":
            assert path in (0, 1)
            assert np.isfinite(min(mg, mt)) and (mt < mg) == (path == 1)
        else:
            assert path == 0
    xs = [dev(p.x0) for p in probs]
    samples = [torch.empty((p.num_results, p.num_chains, p.dim), device="cuda") for p in probs]
    H.hmc_batch_sample_chain(batch, xs, [p.num_burnin for p in probs], [p.num_results for p in probs], samples)
    H.hmc_batch_synchronize(batch)
    for i, (p, (path, _, _)) in enumerate(zip(probs, paths)):
        impl = H.HMC_IMPL_FUSED
        if p.kind == "logreg":
            impl = H.HMC_IMPL_FUSED_TENSOR if path == 1 else H.HMC_IMPL_FUSED_SIMT
        s = Sampler(p, impl=impl)
        x = dev(p.x0)
        smp, _, _ = s.sample_chain(x, p.num_burnin, p.num_results)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(xs[i].cpu().numpy(), x.cpu().numpy())
        np.testing.assert_array_equal(samples[i].cpu().numpy(), smp.cpu().numpy())
        s.close()
    again = H.hmc_batch_create_autotuned(targets, chains, configs)
    cached = [H.hmc_batch_member_path(again, i) for i in range(len(probs))]
    np.testing.assert_array_equal(np.array(cached), np.array(paths))    # NaN-aware: untimed members
    H.hmc_batch_destroy(again)
    H.hmc_batch_destroy(batch)
