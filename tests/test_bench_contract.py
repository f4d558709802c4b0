"""The benchmark's reference arm (the float64 oracle on the host cores) keeps
the JSON contract: one line from rank 0, the metric and unit of the GPU arm,
a cpu_baseline describing the run and an e2e object with no copies."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


@pytest.mark.parametrize("extra", [["--workload", "funnel"], ["--workload", "funnel", "--proposal", "nuts"]],
                         ids=["hmc", "nuts"])
def test_reference_arm_line(extra):
    lines = run(["--impl", "reference", "--steps", "1", "--warmup", "1", "--cpu-seconds", "0.5", *extra])
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "leapfrog grad-evals/s" and d["unit"] == "grad-evals/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    if "nuts" in extra:
        assert "NUTS" in d["config"]["workload"] and "NUTS" in d["cpu_baseline"]["sample"]


def test_reference_arm_prints_only_on_rank_zero():
    assert run(["--impl", "reference", "--steps", "1", "--warmup", "1", "--cpu-seconds", "0.2",
                "--workload", "funnel"], {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []
