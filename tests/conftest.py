import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libhmc.so")
    config.addinivalue_line("markers", "slow: long-running statistical test")


def pytest_sessionfinish(session, exitstatus):
    """With HMC_PARITY_LOG set, write the log-alpha differences the parity
    comparisons measured (tests/parity.py) to that file as JSON lines."""
    path = os.environ.get("HMC_PARITY_LOG")
    if not path:
        return
    try:
        from tests.parity import MARGINS
    except ImportError:
        return
    import json
    with open(path, "w") as f:
        for label, dmax, rel, n in MARGINS:
            f.write(json.dumps({"label": label, "max_abs_dlogalpha": dmax, "max_rel_dlogalpha": rel,
                                "chains": n}) + "\n")
