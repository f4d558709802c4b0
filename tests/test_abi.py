"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function declared in include/hmc.h, and rejects bad arguments before
touching the device."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def binding():
    from paper_2002_01184_gb300 import build
    build.build()
    from paper_2002_01184_gb300 import hmc
    return hmc


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:hmc_status|const char\*|uint64_t|int32_t|hmc_ctx\*|void)\s+(hmc_\w+)\s*\(",
                                    text, re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["hmc_create", "hmc_bootstrap", "hmc_step", "hmc_sample_chain",
                     "hmc_destroy", "hmc_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(binding):
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(hmc_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(binding.LIB_PATH)
    for n in declared_functions():
        assert getattr(lib, n) is not None


def test_invalid_arguments_are_rejected_on_the_host(binding):
    h = binding
    good_t = h.make_target("std_normal", 4)
    good_c = h.make_config(3, 0.5)
    bad_cases = [
        (h.make_target("std_normal", 0), 8, good_c, "dim"),
        (good_t, 0, good_c, "num_chains"),
        (h.make_target("funnel", 1), 8, good_c, "funnel"),
        (h.make_target("corr_gauss", 4), 8, good_c, "P"),
        (h.make_target("logreg", 4), 8, good_c, "X"),
        (h.make_target(7, 4), 8, good_c, "unknown target"),
        (good_t, 8, h.make_config(0, 0.5), "num_leapfrog"),
        (good_t, 8, h.make_config(3, 0.0), "step_size"),
        (good_t, 8, h.make_config(3, float("nan")), "step_size"),
        (good_t, 8, h.make_config(3, float("inf")), "step_size"),
        (good_t, 8, h.make_config(3, 0.5, adapt=True, target_accept=1.0), "target_accept"),
        (good_t, 8, h.make_config(3, 0.5, impl=9), "impl"),
        (good_t, 8, h.make_config(3, 0.5, chain_offset=-1), "chain_offset"),
        (good_t, 8, h.make_config(3, 0.5, proposal=5), "proposal"),
        (good_t, 8, h.make_config(11, 0.5, proposal=h.HMC_PROPOSAL_NUTS), "tree depth"),
        (good_t, 8, h.make_config(3, 0.5, max_transitions_per_launch=-1), "max_transitions_per_launch"),
    ]
    for t, C, c, word in bad_cases:
        with pytest.raises(h.HMCError) as ei:
            h.hmc_create(t, C, c, stream=0)
        assert ei.value.status == h.HMC_E_INVALID
        assert word in str(ei.value), (word, str(ei.value))
        assert word in h.hmc_last_error(None)


def test_null_context_and_workspace_queries(binding):
    h = binding
    assert h.lib.hmc_bootstrap(None, None) == h.HMC_E_INVALID
    assert h.lib.hmc_step(None, None, 0, None) == h.HMC_E_INVALID
    assert h.lib.hmc_sample_chain(None, None, 0, 0, None, None, None) == h.HMC_E_INVALID
    assert h.lib.hmc_propose(None, None, 0, None) == h.HMC_E_INVALID
    assert h.lib.hmc_nuts_leapfrog_count(None, None) == h.HMC_E_INVALID
    # NUTS runs the elementwise targets only
    with pytest.raises(h.HMCError) as ei:
        h.hmc_create(h.hmc_target(h.HMC_T_LOGREG, 4, 10, 16, 16, 16), 8,
                     h.make_config(5, 0.1, proposal=h.HMC_PROPOSAL_NUTS), stream=0)
    assert ei.value.status == h.HMC_E_UNSUPPORTED
    assert h.lib.hmc_mh_select(None, None, 0, None) == h.HMC_E_INVALID
    assert h.lib.hmc_destroy(None) == h.HMC_OK
    assert h.hmc_grad_workspace_bytes(h.make_target("std_normal", 5), 10) == 0
    # logistic regression: C x N residuals + split partials + per-tile sums
    t = h.hmc_target(h.HMC_T_LOGREG, 128, 20000, 16, 16, 16)
    b = h.hmc_grad_workspace_bytes(t, 2048)
    assert b >= 2048 * 20000 * 4
    with pytest.raises(h.HMCError):
        h.hmc_target_log_prob_and_grad(t, 2048, 16, 16, 16, None, 0, stream=0)


def test_create_device_bytes_needs_no_device_and_checks_its_arguments(binding):
    h = binding
    cfg = h.make_config(4, 0.1)
    shape_only = h.hmc_target(h.TARGET_IDS["logreg"], 32, 1000, None, None, None)
    assert h.hmc_create_device_bytes(shape_only, 64, cfg) >= 4 * 64 * 32
    for bad in (h.hmc_target(h.TARGET_IDS["logreg"], 32, 0, None, None, None),
                h.hmc_target(9, 32, 0, None, None, None),
                h.hmc_target(h.TARGET_IDS["funnel"], 1, 0, None, None, None)):
        with pytest.raises(h.HMCError):
            h.hmc_create_device_bytes(bad, 64, cfg)
    with pytest.raises(h.HMCError):
        h.hmc_create_device_bytes(shape_only, 0, cfg)
