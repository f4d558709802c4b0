"""The autograd binding's hand-written adjoints against float64 central
differences of the oracle's log-density and against the oracle gradient."""
import numpy as np
import pytest

from oracle import targets as otargets
from paper_2002_01184_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2002_01184_gb300 import build
    build.build()
    from paper_2002_01184_gb300 import autograd
    return autograd


CASES = [("std_normal", 17, None), ("funnel", 23, None), ("corr_gauss", 40, None),
         ("logreg", 12, 500)]


@pytest.mark.parametrize("kind,D,N", CASES)
def test_adjoint_matches_finite_differences_and_oracle(A, kind, D, N):
    C = 33
    if kind == "corr_gauss":
        p = workloads.corr_gauss(dim=D, num_chains=C)
    elif kind == "logreg":
        p = workloads.logreg(n_data=N, dim=D, num_chains=C)
    elif kind == "funnel":
        p = workloads.funnel(dim=D, num_chains=C)
    else:
        p = workloads.std_normal(num_chains=C, dim=D)
    rng = np.random.default_rng(3)
    x = (0.5 * rng.standard_normal((C, D))).astype(np.float32)
    w = rng.standard_normal(C).astype(np.float32)
    target = A.Target(kind, D, p.P, p.X, p.y)
    xt = torch.tensor(x, device="cuda", requires_grad=True)
    lp = A.log_prob(xt, target)
    (lp * torch.tensor(w, device="cuda")).sum().backward()
    dx = xt.grad.cpu().numpy().astype(np.float64)
    f = otargets.make(kind, **p.data())
    x64 = x.astype(np.float64)
    lp_ref, g_ref = f(x64)
    np.testing.assert_allclose(lp.detach().cpu().numpy(), lp_ref, rtol=1e-5, atol=1e-5)
    expect = w[:, None].astype(np.float64) * g_ref
    row = np.maximum(np.max(np.abs(expect), axis=1, keepdims=True), 1e-6)
    assert np.max(np.abs(dx - expect) / row) < 1e-4
    # float64 central differences of the oracle's log p on a few coordinates
    for d in rng.choice(D, size=min(D, 6), replace=False):
        h = 1e-6 * np.maximum(1.0, np.abs(x64[:, d]))
        xp, xm = x64.copy(), x64.copy()
        xp[:, d] += h
        xm[:, d] -= h
        fd = w * (f(xp)[0] - f(xm)[0]) / (2 * h)
        assert np.max(np.abs(dx[:, d] - fd) / row[:, 0]) < 1e-4
