"""The benchmark's reference arm (the FP64 oracle on the host cores) reports the metric of the
mode it stands beside: Gibbs sweeps/s for the plain sweep and for the PP workload (one PP sweep
per step), gradient evaluations/s for the adjoint workload, and an 'unavailable' line for the
partition experiment, whose metric needs 3 x 1200 sweeps per grid."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*extra):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--cpu-seconds", "0.2", "--steps", "2", *extra], capture_output=True,
                       text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


@pytest.mark.parametrize("workload,scale,metric,unit", [
    ("planted-1000x500-k10", "1.0", "Gibbs sweeps/s", "sweeps/s"),
    ("pp4x4-100000x20000-20M-k16", "0.03", "Gibbs sweeps/s", "sweeps/s"),
    ("uniform-200000x50000-50M-k64", "0.03", "log-joint gradient evaluations/s (adjoint, K=64)",
     "grad evals/s"),
])
def test_reference_arm_metric_follows_the_mode(workload, scale, metric, unit):
    out = _run("--workload", workload, "--scale", scale, "--warmup", "1")
    assert out["impl"] == "reference" and out["metric"] == metric and out["unit"] == unit
    assert out["value"] > 0 and out["cpu_baseline"]["kind"].startswith("oracle")
    assert out["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_partition_experiment_is_unavailable():
    out = _run("--workload", "sim-6040x3706-k5")
    assert out["impl"] == "reference" and "unavailable" in out


def test_reference_arm_pp_takes_the_requested_steps_and_warmup():
    out = _run("--workload", "pp4x4-100000x20000-20M-k16", "--scale", "0.03", "--warmup", "2")
    assert out["steps"] == 2 and out["warmup"] == 2
    assert out["config"]["grid"] == "4x4"
