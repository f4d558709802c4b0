"""Pins for the float64 oracle against facts that do not come from the oracle.

Each test checks the oracle against a closed form, an invariant, an
independent implementation, brute force or a library routine, chosen so that
a plausible slip (a dropped half-kick, a wrong sign, a transposed operand, a
wrong index into the random stream) fails at least one of them.
"""
import json
import math
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import diagnostics, hmc, philox, targets
from paper_2002_01184_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def worked_example():
    with open(os.path.join(GOLDEN, "worked_example.json")) as f:
        return json.load(f)


def one_step_matrix(eps, lam=1.0):
    """Transfer matrix of one velocity-Verlet step on U = lam x^2 / 2, acting
    on (x, p): derived by composing kick(-eps lam/2), drift(eps), kick."""
    return np.array([[1.0 - eps * eps * lam / 2.0, eps],
                     [-eps * lam * (1.0 - eps * eps * lam / 4.0), 1.0 - eps * eps * lam / 2.0]])


# ---------------------------------------------------------------- Philox ----

TRITON_CHECK = textwrap.dedent("""
    import os, sys
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def k(out_ptr, ctr_ptr, seed, N: tl.constexpr):
        off = tl.arange(0, N)
        c0 = tl.load(ctr_ptr + off * 4 + 0)
        c1 = tl.load(ctr_ptr + off * 4 + 1)
        c2 = tl.load(ctr_ptr + off * 4 + 2)
        c3 = tl.load(ctr_ptr + off * 4 + 3)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
        tl.store(out_ptr + off * 4 + 0, a)
        tl.store(out_ptr + off * 4 + 1, b)
        tl.store(out_ptr + off * 4 + 2, c)
        tl.store(out_ptr + off * 4 + 3, d)

    ctr = np.load(sys.argv[1])
    seed = int(sys.argv[2])
    out = torch.zeros(ctr.size, dtype=torch.int32)
    k[(1,)](out, torch.from_numpy(ctr.view(np.int32).ravel().copy()), seed, N=ctr.shape[0])
    np.save(sys.argv[3], out.numpy().view(np.uint32).reshape(-1, 4))
""")


def test_philox_matches_independent_implementation(tmp_path):
    """Triton ships its own Philox4x32-10 (run here on the CPU interpreter);
    the oracle's words must equal it for arbitrary counters and 64-bit keys."""
    pytest.importorskip("triton")
    rng = np.random.default_rng(7)
    ctr = rng.integers(0, 2 ** 32, size=(128, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [1, 0, 0, 0], [0xFFFFFFFF] * 4, [0, 5, 300, 1]]
    np.save(tmp_path / "ctr.npy", ctr)
    script = tmp_path / "tri.py"
    script.write_text(TRITON_CHECK)
    for seed in (0, 1, 2 ** 32 + 3, 0xDEADBEEFCAFEF00D):
        out = tmp_path / f"out_{seed}.npy"
        env = dict(os.environ, TRITON_INTERPRET="1")
        subprocess.run([sys.executable, str(script), str(tmp_path / "ctr.npy"), str(seed), str(out)],
                       check=True, env=env, timeout=300, capture_output=True)
        ref = np.load(out)
        mine = philox.philox4x32_10(ctr, philox.seed_key(seed))
        np.testing.assert_array_equal(mine, ref)


def test_philox_is_a_bijection_on_counters():
    ctr = np.zeros((1 << 18, 4), np.uint32)
    ctr[:, 0] = np.arange(1 << 18)
    ctr[:, 2] = 77
    w = philox.philox4x32_10(ctr, (123, 456))
    packed = w.view(np.dtype((np.void, 16))).ravel()
    assert np.unique(packed).size == packed.size


def test_uniforms_and_normals_have_the_right_law():
    u = philox.accept_uniform(seed=11, transition=3, num_chains=400000)
    assert u.min() > 0.0 and u.max() < 1.0
    counts, _ = np.histogram(u, bins=64, range=(0, 1))
    chi2 = stats.chisquare(counts)
    assert chi2.pvalue > 1e-4
    z = philox.momentum(seed=5, transition=9, num_chains=50000, dim=7).ravel()
    ks = stats.kstest(z, "norm")
    assert ks.pvalue > 1e-4
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / z.size)


def test_momentum_stream_layout_is_per_chain_and_transition():
    """Chain c's draw depends only on (seed, c, t): taking it alone (with a
    chain offset) gives the same numbers; other transitions and seeds differ."""
    full = philox.momentum(3, 17, 64, 10)
    alone = philox.momentum(3, 17, 1, 10, chain_offset=41)
    np.testing.assert_array_equal(full[41], alone[0])
    assert not np.allclose(full, philox.momentum(3, 18, 64, 10))
    assert not np.allclose(full, philox.momentum(4, 17, 64, 10))
    # dims 4j..4j+3 come from block j: a 7-dim draw is a prefix of an 8-dim one
    np.testing.assert_array_equal(philox.momentum(3, 17, 64, 8)[:, :7],
                                  philox.momentum(3, 17, 64, 7))


# -------------------------------------------------------------- leapfrog ----

def test_worked_example_leapfrog_map_is_exact():
    """Worked example (eps = 1.5, L = 3 on N(0,1)): the leapfrog map is linear
    with dyadic entries, so float64 must reproduce M^3 exactly."""
    ex = worked_example()
    eps, L = ex["step_size"], ex["num_leapfrog_steps"]
    M = one_step_matrix(eps)
    np.testing.assert_array_equal(M, [[-0.125, 1.5], [-0.65625, -0.125]])
    M3 = np.linalg.matrix_power(M, L)
    np.testing.assert_array_equal(M3, [[0.3671875, -1.40625], [0.615234375, 0.3671875]])
    assert np.linalg.det(M3) == pytest.approx(1.0, abs=1e-15)
    for x0, p0 in [(1.0, 0.0), (0.0, 1.0), (0.75, -2.5)]:
        x = np.array([[x0]])
        lp, g = targets.std_normal(x)
        x1, p1, _, _ = hmc.leapfrog(x, np.array([[p0]]), g, eps, L, targets.std_normal)
        exp = M3 @ np.array([x0, p0])
        assert x1[0, 0] == exp[0] and p1[0, 0] == exp[1]


def test_worked_example_log_accept_ratio_closed_form():
    """From x = 0, H_L - H_0 = p^2 (1.40625^2 + 0.3671875^2 - 1) / 2 for the
    drawn momentum p, so log alpha is known exactly per chain; averaged over
    p ~ N(0,1), E[alpha] = 1/sqrt(1 + 2 q) with that q."""
    ex = worked_example()
    C = 200000
    x = np.zeros((C, 1))
    lp, g = targets.std_normal(x)
    r = hmc.one_step(x, lp, g, ex["step_size"], ex["num_leapfrog_steps"], 0, 0, targets.std_normal)
    p = philox.momentum(0, 0, C, 1)[:, 0]
    q = 0.5 * (1.40625 ** 2 + 0.3671875 ** 2 - 1.0)
    np.testing.assert_allclose(r["log_accept_ratio"], -q * p * p, rtol=1e-13, atol=1e-15)
    mean_alpha = hmc.accept_statistic(r["log_accept_ratio"])
    assert mean_alpha == pytest.approx(1.0 / math.sqrt(1.0 + 2.0 * q), abs=4e-3)
    # accepted iff log u < log alpha for this chain's uniform
    u = philox.accept_uniform(0, 0, C)
    np.testing.assert_array_equal(r["is_accepted"], np.log(u) < -q * p * p)
    np.testing.assert_allclose(r["x"][:, 0], np.where(r["is_accepted"], -1.40625 * p, 0.0),
                               rtol=1e-14, atol=0)


def stationary_acceptance(eps, L):
    """E over (x, p) ~ N(0, I_2) of min(1, exp(-dH)), dH = z^T Q z with
    Q = (M^T M - I)/2; in polar form (1/2pi) int [q<=0 ? 1 : 1/(1+2q)]."""
    M = np.linalg.matrix_power(one_step_matrix(eps), L)
    Q = 0.5 * (M.T @ M - np.eye(2))

    def f(th):
        c, s = math.cos(th), math.sin(th)
        q = Q[0, 0] * c * c + 2 * Q[0, 1] * c * s + Q[1, 1] * s * s
        return 1.0 if q <= 0 else 1.0 / (1.0 + 2.0 * q)

    val, _ = integrate.quad(f, 0.0, 2 * math.pi, limit=400, epsabs=1e-12)
    return val / (2 * math.pi)


def test_worked_example_stationary_acceptance():
    """Started at stationarity, the mean acceptance probability of the worked
    example's kernel is a closed-form integral (about 0.760231)."""
    ex = worked_example()
    expect = stationary_acceptance(ex["step_size"], ex["num_leapfrog_steps"])
    assert expect == pytest.approx(0.760231, abs=2e-6)
    C = 100000
    x = philox.momentum(99, 0, C, 1)       # an N(0,1) start drawn from a spare stream
    lp, g = targets.std_normal(x)
    stats_ = []
    for t in range(6):
        r = hmc.one_step(x, lp, g, ex["step_size"], ex["num_leapfrog_steps"], 1, t, targets.std_normal)
        x, lp, g = r["x"], r["lp"], r["g"]
        stats_.append(hmc.accept_statistic(r["log_accept_ratio"]))
    assert np.mean(stats_) == pytest.approx(expect, abs=3e-3)


def test_worked_example_stationary_moments():
    """The chain leaves N(0,1) invariant: kept samples of the worked example
    (and of a 100k-chain variant) have mean 0 and variance 1 within 3 MCSE."""
    ex = worked_example()
    for C, B, K in [(ex["num_chains"], ex["num_burnin_steps"], ex["num_results"]), (100000, 20, 20)]:
        x0 = np.full((C, 1), ex["initial_state"])
        out = hmc.sample_chain(x0, targets.std_normal, ex["num_leapfrog_steps"], ex["step_size"],
                               0, B, K)
        s = out["samples"]
        assert np.all(out["step_size"] == ex["step_size"])
        m = s.mean()
        assert abs(m) < 3 * diagnostics.mcse_mean(s)[0]
        s2 = s ** 2
        assert abs(s2.mean() - 1.0) < 3 * diagnostics.mcse_mean(s2)[0]


def test_gaussian_leapfrog_matches_eigenbasis_closed_form():
    """For a Gaussian target each eigenmode of P is a 1-D oscillator with
    lam_i; the oracle's L-step map must equal the product of per-mode
    transfer matrices."""
    prob = workloads.corr_gauss(dim=8, num_chains=5, num_burnin=0, num_results=0)
    P = prob.P.astype(np.float64)
    lam, V = np.linalg.eigh(P)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((5, 8))
    p = rng.standard_normal((5, 8))
    eps, L = 0.3, 7
    tgt = targets.make("corr_gauss", P=P)
    _, g = tgt(x)
    x1, p1, _, _ = hmc.leapfrog(x, p, g, eps, L, tgt)
    xt, pt = x @ V, p @ V
    for i in range(8):
        Mi = np.linalg.matrix_power(one_step_matrix(eps, lam[i]), L)
        xe = Mi[0, 0] * xt[:, i] + Mi[0, 1] * pt[:, i]
        pe = Mi[1, 0] * xt[:, i] + Mi[1, 1] * pt[:, i]
        np.testing.assert_allclose((x1 @ V)[:, i], xe, rtol=0, atol=1e-12)
        np.testing.assert_allclose((p1 @ V)[:, i], pe, rtol=0, atol=1e-12)


def small_targets():
    cg = workloads.corr_gauss(dim=6, num_chains=4, num_burnin=0, num_results=0)
    lr = workloads.logreg(n_data=40, dim=5, num_chains=4, num_burnin=0, num_results=0)
    return {
        "std_normal": (targets.std_normal, 3),
        "corr_gauss": (targets.make("corr_gauss", P=cg.P), 6),
        "logreg": (targets.make("logreg", X=lr.X, y=lr.y), 5),
        "funnel": (targets.funnel, 7),
    }


@pytest.mark.parametrize("name", ["std_normal", "corr_gauss", "logreg", "funnel"])
def test_leapfrog_is_time_reversible(name):
    tgt, D = small_targets()[name]
    rng = np.random.default_rng(1)
    x = 0.5 * rng.standard_normal((4, D))
    p = rng.standard_normal((4, D))
    _, g = tgt(x)
    x1, p1, _, g1 = hmc.leapfrog(x, p, g, 0.05, 9, tgt)
    x2, p2, _, _ = hmc.leapfrog(x1, -p1, g1, 0.05, 9, tgt)
    np.testing.assert_allclose(x2, x, rtol=0, atol=1e-12)
    np.testing.assert_allclose(-p2, p, rtol=0, atol=1e-12)


@pytest.mark.parametrize("name", ["logreg", "funnel"])
def test_energy_error_is_second_order(name):
    """Over a fixed integration time, halving eps quarters the energy error."""
    tgt, D = small_targets()[name]
    rng = np.random.default_rng(2)
    x = 0.3 * rng.standard_normal((4, D))
    p = rng.standard_normal((4, D))
    errs = []
    T = 0.4
    for eps in (0.02, 0.01, 0.005):
        lp, g = tgt(x)
        x1, p1, lp1, _ = hmc.leapfrog(x, p, g, eps, int(round(T / eps)), tgt)
        errs.append(np.max(np.abs(hmc.hamiltonian(lp1, p1) - hmc.hamiltonian(lp, p))))
    slopes = np.diff(np.log(errs)) / np.diff(np.log([0.02, 0.01, 0.005]))
    assert np.all(np.abs(slopes - 2.0) < 0.1), slopes


@pytest.mark.parametrize("name", ["std_normal", "corr_gauss", "logreg", "funnel"])
def test_gradient_matches_central_differences(name):
    tgt, D = small_targets()[name]
    rng = np.random.default_rng(3)
    x = 0.7 * rng.standard_normal((4, D))
    lp, g = tgt(x)
    fd = np.empty_like(x)
    for d in range(D):
        h = 1e-6 * np.maximum(1.0, np.abs(x[:, d]))
        xp, xm = x.copy(), x.copy()
        xp[:, d] += h
        xm[:, d] -= h
        fd[:, d] = (tgt(xp)[0] - tgt(xm)[0]) / (2 * h)
    scale = np.maximum(1.0, np.abs(lp))[:, None]
    np.testing.assert_allclose(g, fd, rtol=0, atol=1e-7 * scale.max() * 10)


def test_log_densities_against_library_routines():
    """Values (not just gradients) against scipy's densities, up to the
    constant that the oracle drops."""
    rng = np.random.default_rng(4)
    cg = workloads.corr_gauss(dim=6, num_chains=3, num_burnin=0, num_results=0)
    P = cg.P.astype(np.float64)
    x = rng.standard_normal((3, 6))
    ref = stats.multivariate_normal(mean=np.zeros(6), cov=np.linalg.inv(P)).logpdf(x)
    lp, _ = targets.corr_gauss(x, P)
    d = ref - lp
    np.testing.assert_allclose(d, d[0], atol=1e-10)
    s = rng.standard_normal((3, 5))
    ref = stats.norm(0, 3).logpdf(s[:, 0]) + np.sum(
        stats.norm(0, np.exp(s[:, 0] / 2)[:, None]).logpdf(s[:, 1:]), axis=1)
    d = ref - targets.funnel(s)[0]
    np.testing.assert_allclose(d, d[0], atol=1e-10)
    lr = workloads.logreg(n_data=30, dim=4, num_chains=3, num_burnin=0, num_results=0)
    th = rng.standard_normal((3, 4))
    z = th @ lr.X.astype(np.float64).T
    ref = np.sum(stats.bernoulli.logpmf(lr.y[None, :], 1 / (1 + np.exp(-z))), axis=1) + \
        np.sum(stats.norm.logpdf(th), axis=1)
    d = ref - targets.logreg(th, lr.X, lr.y)[0]
    np.testing.assert_allclose(d, d[0], atol=1e-9)


def test_nonfinite_proposals_are_rejected():
    def bad(x):
        lp, g = targets.std_normal(x)
        return np.where(np.abs(x[:, 0]) > 0.5, np.nan, lp), g
    x = np.zeros((500, 1))
    lp, g = bad(x)
    r = hmc.one_step(x, lp, g, 1.0, 2, 0, 0, bad)
    moved = np.abs(r["proposed_x"][:, 0]) > 0.5
    assert moved.any() and np.all(~r["is_accepted"][moved])
    assert np.all(r["log_accept_ratio"][moved] == -np.inf)
    np.testing.assert_array_equal(r["x"][moved], x[moved])


def test_chain_isolation_in_the_oracle():
    """A chain's transition depends only on its own state and (seed, c, t):
    simulating it alone with its chain offset gives the same result."""
    rng = np.random.default_rng(5)
    x = rng.standard_normal((16, 6))
    lp, g = targets.funnel(x)
    full = hmc.one_step(x, lp, g, 0.2, 5, 9, 4, targets.funnel)
    for c in (0, 7, 15):
        one = hmc.one_step(x[c:c + 1], lp[c:c + 1], g[c:c + 1], 0.2, 5, 9, 4, targets.funnel,
                           chain_offset=c)
        np.testing.assert_array_equal(one["x"][0], full["x"][c])
        assert one["is_accepted"][0] == full["is_accepted"][c]


# ------------------------------------------------------ dual averaging ----

def test_dual_averaging_fixed_point_and_direction():
    da = hmc.DualAveraging(0.3, 0.65)
    for _ in range(50):
        da.update(0.65)
    assert da.log_eps == pytest.approx(math.log(3.0), abs=1e-15)
    assert da.log_eps_bar == pytest.approx(math.log(3.0), abs=1e-12)
    hi = hmc.DualAveraging(0.3, 0.65)
    lo = hmc.DualAveraging(0.3, 0.65)
    for _ in range(20):
        hi.update(0.95)
        lo.update(0.2)
    assert hi.step_size > 3.0 > lo.step_size


def test_dual_averaging_reaches_target_acceptance():
    """Adapting on N(0, 1) in D = 10 drives the frozen step size to an
    acceptance close to the target."""
    C, D = 512, 10
    x0 = philox.momentum(77, 0, C, D)
    out = hmc.sample_chain(x0, targets.std_normal, 5, 1.0, 123, 400, 100,
                           adapt=True, target_accept=0.7)
    lp, g = targets.std_normal(out["x"])
    x = out["x"]
    st = []
    for t in range(1000, 1010):
        r = hmc.one_step(x, lp, g, out["final_step_size"], 5, 123, t, targets.std_normal)
        x, lp, g = r["x"], r["lp"], r["g"]
        st.append(hmc.accept_statistic(r["log_accept_ratio"]))
    assert np.mean(st) == pytest.approx(0.7, abs=0.03)
    assert np.all(out["step_size"] == out["final_step_size"])


# --------------------------------------------------------- diagnostics ----

def test_ess_of_iid_draws_is_the_draw_count():
    z = np.random.default_rng(6).standard_normal((1000, 8, 3))
    e = diagnostics.ess(z)
    np.testing.assert_allclose(e, 8000, rtol=0.12)


def test_ess_of_ar1_matches_closed_form():
    """For AR(1) with coefficient phi, tau = (1 + phi) / (1 - phi)."""
    rng = np.random.default_rng(7)
    phi, n, C = 0.8, 4000, 8
    e = rng.standard_normal((n, C, 2))
    z = np.empty_like(e)
    z[0] = e[0] / math.sqrt(1 - phi * phi)
    for t in range(1, n):
        z[t] = phi * z[t - 1] + e[t]
    np.testing.assert_allclose(diagnostics.ess(z), n * C * (1 - phi) / (1 + phi), rtol=0.15)


def test_mcse_of_the_mean_matches_the_spread_of_replicated_means():
    """The Monte Carlo standard error of the mean is its sampling spread: over
    400 independent AR(1) runs (phi = 0.5, 8 chains x 500 draws) the standard
    deviation of the runs' means agrees with the average reported MCSE, and
    with the closed form sqrt(tau / (C n)) sigma, tau = (1 + phi) / (1 - phi)."""
    rng = np.random.default_rng(14)
    phi, n, C, R = 0.5, 500, 8, 400
    e = rng.standard_normal((n, R * C))
    z = np.empty_like(e)
    z[0] = e[0] / math.sqrt(1 - phi * phi)
    for t in range(1, n):
        z[t] = phi * z[t - 1] + e[t]
    z = z.reshape(n, R, C)
    means = z.mean(axis=(0, 2))
    mcse = np.array([diagnostics.mcse_mean(z[:, r, :, None])[0] for r in range(R)])
    sigma = 1.0 / math.sqrt(1 - phi * phi)
    closed = sigma * math.sqrt((1 + phi) / (1 - phi) / (C * n))
    assert means.std(ddof=1) == pytest.approx(closed, rel=0.12)
    assert mcse.mean() == pytest.approx(closed, rel=0.06)


def test_batch_means_ess_worked_by_hand():
    """One chain, draws 1, 3, 2, 6 in batches of 2: s2 = (4 + 0 + 1 + 9) / 3 =
    14/3; batch means 2 and 4 (grand mean 3) give sig2 = 2 x (1 + 1) / 1 = 4
    and ESS = 4 x (14/3) / 4 = 14/3.  A fifth draw beyond the last complete
    batch enters the variance only: 1, 3, 2, 6, 3 have mean 3 and
    s2 = 14/4, so ESS = 5 x 3.5 / 4 = 4.375.  Two chains (1, 3) and (2, 6)
    with one batch each (batch_size = n = 2): W = (2 + 8) / 2 = 5, chain means
    2 and 4 about 3 give sig2 = 2 x 2 / 1 = 4, ESS = 2 x 2 x 5 / 4 = 5."""
    z = np.array([1.0, 3.0, 2.0, 6.0]).reshape(4, 1, 1)
    assert diagnostics.batch_means_ess(z, 2)[0] == pytest.approx(14.0 / 3.0, rel=1e-15)
    z5 = np.array([1.0, 3.0, 2.0, 6.0, 3.0]).reshape(5, 1, 1)
    assert diagnostics.batch_means_ess(z5, 2)[0] == pytest.approx(4.375, rel=1e-15)
    z2 = np.array([[1.0, 2.0], [3.0, 6.0]]).reshape(2, 2, 1)
    assert diagnostics.batch_means_ess(z2, 2)[0] == pytest.approx(5.0, rel=1e-15)
    with pytest.raises(ValueError):
        diagnostics.batch_means_ess(z, 3)                # one batch in all
    with pytest.raises(ValueError):
        diagnostics.batch_means_ess(z2, 3)               # no complete batch


def test_batch_means_ess_of_iid_draws_is_the_draw_count():
    """Independent draws: sig2 estimates the variance itself; pooled over 200
    chains of 20 batches the estimate's relative spread is about
    sqrt(2 / (200 x 19)) = 2.3 %."""
    z = np.random.default_rng(11).standard_normal((1000, 200, 2))
    np.testing.assert_allclose(diagnostics.batch_means_ess(z, 50), 200 * 1000, rtol=0.1)


def test_batch_means_ess_of_ar1_matches_closed_form():
    """AR(1) with coefficient phi: the asymptotic variance is
    (1 + phi) / (1 - phi) times the marginal variance, so ESS / (C n) ->
    (1 - phi) / (1 + phi); batches of 400 draws (>> 1 / (1 - phi)) leave a
    bias of order 2 phi / (b (1 - phi)^2) / 9 ~ 2 %."""
    rng = np.random.default_rng(12)
    phi, n, C = 0.8, 8000, 100
    e = rng.standard_normal((n, C, 1))
    z = np.empty_like(e)
    z[0] = e[0] / math.sqrt(1 - phi * phi)
    for t in range(1, n):
        z[t] = phi * z[t - 1] + e[t]
    np.testing.assert_allclose(diagnostics.batch_means_ess(z, 400), n * C * (1 - phi) / (1 + phi),
                               rtol=0.1)


def test_batch_means_ess_with_one_batch_per_chain_is_the_between_chain_estimate():
    """batch_size = n: each chain is one batch, and sig2 = n x the variance of
    the chain means across chains.  For stationary AR(1) chains that variance
    is about sigma^2 tau / n with tau = (1 + phi) / (1 - phi), so ESS / (C n)
    -> (1 - phi) / (1 + phi); 400 chains leave a relative spread of about
    sqrt(2 / 399) = 7 %."""
    rng = np.random.default_rng(13)
    phi, n, C = 0.8, 2000, 400
    e = rng.standard_normal((n, C, 1))
    z = np.empty_like(e)
    z[0] = e[0] / math.sqrt(1 - phi * phi)
    for t in range(1, n):
        z[t] = phi * z[t - 1] + e[t]
    np.testing.assert_allclose(diagnostics.batch_means_ess(z, n), n * C * (1 - phi) / (1 + phi),
                               rtol=0.25)


def test_logreg_posterior_mean_is_near_truth():
    prob = workloads.logreg(n_data=2000, dim=6, num_chains=32, num_burnin=150, num_results=150)
    tgt = targets.make("logreg", X=prob.X, y=prob.y)
    out = hmc.sample_chain(prob.x0, tgt, prob.num_leapfrog, prob.step_size, prob.seed,
                           prob.num_burnin, prob.num_results, adapt=True, target_accept=0.8)
    mean = out["samples"].reshape(-1, 6).mean(axis=0)
    assert np.linalg.norm(mean - prob.w_true) < 4 * math.sqrt(6 / (0.2 * 2000))
