"""The no-allocation gradient entry point, for callers that may not allocate
device memory (a host that owns the whole HBM budget, or a latency-critical
loop that cannot afford cudaMalloc's synchronisation): through the C ABI it
must give the same log-prob and gradient as the regular entry point, which
takes caller-provided scratch, on two calls in a row (the second call must
not be affected by what the first left in the shared scratch array).

This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes alone in a fresh process, where its
first call performs the per-device set-up.

It is also compared with the float64 oracle directly, for every target
(Section 3's log-densities and their gradients), so that it does not rest
only on the regular entry point's own parity."""
import numpy as np
import pytest

from oracle import targets as otargets
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


def evaluate_both(H, prob, x):
    C, D = x.shape
    dev = lambda a: torch.as_tensor(a).cuda().contiguous()
    Pd = dev(prob.P) if prob.P is not None else None
    Xd = dev(prob.X) if prob.X is not None else None
    yd = dev(prob.y) if prob.y is not None else None
    t = H.make_target(prob.kind, D, Pd, Xd, yd)
    xd = dev(x)
    nbytes = H.hmc_grad_workspace_bytes(t, C)
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device="cuda")
    lp_ref = torch.empty(C, device="cuda")
    g_ref = torch.empty((C, D), device="cuda")
    H.hmc_target_log_prob_and_grad(t, C, xd, lp_ref, g_ref, ws, nbytes)
    lp = torch.full((C,), float("nan"), device="cuda")
    g = torch.full((C, D), float("nan"), device="cuda")
    H.hmc_target_log_prob_and_grad_noalloc(t, C, xd, lp, g)
    torch.cuda.synchronize()
    return (lp.cpu().numpy(), g.cpu().numpy(), lp_ref.cpu().numpy(), g_ref.cpu().numpy(),
            nbytes, (t, Pd, Xd, yd))


def assert_same(lp, g, lp_ref, g_ref):
    # the gradient tolerance of the parity tests (normwise per chain, 1e-5)
    row = np.max(np.abs(g_ref), axis=1, keepdims=True)
    assert np.max(np.abs(g - g_ref) / np.maximum(row, 1e-6)) < 1e-5
    np.testing.assert_allclose(lp, lp_ref, rtol=1e-5, atol=1e-5)


def test_no_alloc_entry_point_matches_workspace_entry_point(H):
    rng = np.random.default_rng(0)
    # logistic regression needs scratch (residuals and split-K partial sums)
    first = workloads.logreg(n_data=700, dim=20, num_chains=96)
    x1 = (0.2 * rng.standard_normal((96, 20))).astype(np.float32)
    lp, g, lp_ref, g_ref, nbytes, _ = evaluate_both(H, first, x1)
    assert nbytes > 0
    assert_same(lp, g, lp_ref, g_ref)
    # a second call in a row, different sizes and data, same shared array
    second = workloads.logreg(n_data=1500, dim=33, num_chains=64, seed=9)
    x2 = (0.2 * rng.standard_normal((64, 33))).astype(np.float32)
    lp, g, lp_ref, g_ref, _, _ = evaluate_both(H, second, x2)
    assert_same(lp, g, lp_ref, g_ref)


def test_no_alloc_entry_point_rejects_oversized_requests(H):
    prob = workloads.logreg(n_data=20000, dim=8, num_chains=1024)
    x = np.zeros((1024, 8), np.float32)
    dev = lambda a: torch.as_tensor(a).cuda().contiguous()
    Xd, yd = dev(prob.X), dev(prob.y)
    t = H.make_target("logreg", 8, None, Xd, yd)
    assert H.hmc_grad_workspace_bytes(t, 1024) > 64 << 20
    lp = torch.empty(1024, device="cuda")
    g = torch.empty((1024, 8), device="cuda")
    with pytest.raises(H.HMCError) as ei:
        H.hmc_target_log_prob_and_grad_noalloc(t, 1024, dev(x), lp, g)
    assert ei.value.status == H.HMC_E_INVALID
    assert "scratch" in str(ei.value)


ORACLE_CASES = [
    ("std_normal", workloads.std_normal, dict(num_chains=37, dim=13)),
    ("funnel", workloads.funnel, dict(num_chains=41, dim=50)),
    ("corr_gauss", workloads.corr_gauss, dict(num_chains=130, dim=70)),
    ("corr_gauss", workloads.corr_gauss, dict(num_chains=300, dim=256)),
    ("logreg", workloads.logreg, dict(n_data=1000, dim=65, num_chains=129)),
]


@pytest.mark.parametrize("kind,make,kw", ORACLE_CASES)
def test_no_alloc_entry_point_matches_oracle(H, kind, make, kw):
    prob = make(**kw)
    C, D = prob.num_chains, prob.dim
    x = (0.3 * np.random.default_rng(5).standard_normal((C, D))).astype(np.float32)
    lp, g, _, _, _, _ = evaluate_both(H, prob, x)
    lp_ref, g_ref = otargets.make(kind, **prob.data())(x.astype(np.float64))
    assert_same(lp, g, lp_ref, g_ref)
