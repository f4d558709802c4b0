"""Teacher-forced comparison of one GPU transition with the float64 oracle.

HMC is exact only in distribution and trajectories of float32 and float64
chains separate after many transitions, so the element-by-element check is
per transition: the oracle starts from the GPU's float32 state (promoted),
uses the same (seed, chain, t) streams and the step size the GPU used, and
the two outcomes are compared with these tolerances:
  * positions: 1e-4 relative, read per chain in the max norm:
    max_d |x_gpu - x_ref| / max(max_d |x_ref|, 1e-3) <= 1e-4.  (Read
    elementwise, the bound fails for correct float32 arithmetic: a component
    of size 1e-3 carries the absolute rounding error of the O(1) components
    it was computed with -- a float32 emulation of the funnel on the CPU shows
    1.5e-4 elementwise against 2.6e-7 per chain.);
  * accept decisions identical except where |log u - log alpha| < 1e-5
    (log u and log alpha both from the oracle); such chains are only checked
    to hold one of the two valid states.
"""
import numpy as np

POS_RTOL = 1e-4
POS_FLOOR = 1e-3
DECISION_BAND = 1e-5
# float32 energies of magnitude |H| carry rounding of order 1e-7 |H| per
# operation and about sqrt(n) 1e-7 |H| over a sum of n terms: decisions closer
# than 1e-6 (|H0| + |H_L|) to their threshold may go either way
DECISION_REL = 1e-6

# |log alpha_gpu - log alpha_oracle| of every compared transition, for the
# record the suite can write (HMC_PARITY_LOG, see conftest.py): label, the
# largest absolute difference, the largest difference relative to
# |H0| + |H_L|, and the number of finite chains compared
MARGINS = []


def chain_error(x, ref):
    """Per-chain max-norm relative error, floor 1e-3."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.maximum(np.max(np.abs(ref), axis=1), POS_FLOOR)
    return np.max(np.abs(x - ref), axis=1) / scale


def compare_transition(x_before, x_after_gpu, acc_gpu, la_gpu, ref, label=""):
    acc_gpu = np.asarray(acc_gpu).astype(bool)
    acc_ref = np.asarray(ref["is_accepted"]).astype(bool)
    band = DECISION_BAND
    if "h0" in ref:
        band = np.maximum(DECISION_BAND, DECISION_REL * (np.abs(ref["h0"]) + np.abs(ref["h1"])))
    near = np.abs(ref["log_u"] - ref["log_accept_ratio"]) < band
    bad = (acc_gpu != acc_ref) & ~near
    if bad.any():
        i = np.nonzero(bad)[0][:10]
        raise AssertionError(f"{label}: accept decisions differ for chains {i}; |log u - log alpha| = "
                             f"{np.abs(ref['log_u'] - ref['log_accept_ratio'])[i]}")
    same = acc_gpu == acc_ref
    xg = np.asarray(x_after_gpu, dtype=np.float64)
    err = chain_error(xg, ref["x"])
    if same.any():
        worst = err[same].max()
        assert worst <= POS_RTOL, f"{label}: position error {worst:.3e} > {POS_RTOL}"
    # chains inside the decision band hold either the old state or the proposal
    for c in np.nonzero(~same)[0]:
        alt = ref["proposed_x"][c] if acc_gpu[c] else x_before[c]
        e = chain_error(xg[c:c + 1], np.asarray(alt)[None])
        assert e.max() <= POS_RTOL, f"{label}: chain {c} holds neither valid state"
    # rejected chains keep their state bit for bit
    rej = ~acc_gpu
    assert np.array_equal(xg[rej], np.asarray(x_before, dtype=np.float64)[rej])
    # divergences: a float64 non-finite energy is non-finite in float32 too;
    # float32 may also overflow where float64 only reaches a huge energy
    # error (float32's range ends near 3e38) -- both reject those chains
    la_ref = ref["log_accept_ratio"]
    la_gpu = np.asarray(la_gpu, dtype=np.float64)
    fin = np.isfinite(la_ref) & np.isfinite(la_gpu)
    if fin.any():
        d = np.abs(la_gpu[fin] - la_ref[fin])
        rel = d / np.maximum(np.abs(ref["h0"][fin]) + np.abs(ref["h1"][fin]), 1e-30) if "h0" in ref else d * np.nan
        MARGINS.append((label, float(d.max()), float(np.nanmax(rel)) if "h0" in ref else None, int(fin.sum())))
    assert np.all(~np.isfinite(la_gpu[~np.isfinite(la_ref)])), f"{label}: missed divergence"
    extra = ~np.isfinite(la_gpu) & np.isfinite(la_ref)
    assert np.all(la_ref[extra] < -1e30), f"{label}: spurious divergence"
    return int(same.sum()), int((~same).sum())
