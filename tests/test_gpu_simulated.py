"""The paper's simulated-data experiment (Section 5.3) end to end on the GPU at a tenth of its
size: PP on an r x r grid against the full-posterior (1 x 1) chain on the same data, and the
benchmark's partition mode.  With K and tau at their true values the test RMSE sits just above
the unit noise floor, and PP stays close to the full chain (the paper: 1.008 against 1.008 up to
5 x 5, 1.018 at 30 x 30 on the full-size data)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_1703_00734_gb300 import synth
from pairing import Pair, assert_rows_close

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rmse(d, g, order="decreasing", sweeps=120, burnin=80):
    from paper_1703_00734_gb300 import bmf
    m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], d["K"], d["tau"], "fp64", I=g, J=g,
                X0=d["X0"], W0=d["W0"], order=order, burnin=burnin, thin=2, seed=3)
    for stage in ((1,) if g == 1 else (1, 2, 3)):
        m.stage(stage, sweeps)
    _, r = m.predict(d["test_row"], d["test_col"], d["test_val"])
    m.close()
    return r


@pytest.mark.parametrize("name", ["sim-6040x3706-k5", "sim-6040x3706-k5-structured"])
def test_pp_matches_the_full_chain_on_simulated_data(name):
    d = synth.make_workload(name, scale=0.1)
    full = _rmse(d, 1)
    pp = _rmse(d, 3)
    assert 1.0 < full < 1.3 and 1.0 < pp < 1.3
    assert abs(pp - full) < 0.05


@pytest.mark.parametrize("name", ["sim-6040x3706-k5", "sim-6040x3706-k5-structured"])
def test_fine_grid_pp_matches_the_oracle_per_state(name):
    """A 10 x 10 grid (100 subsets, 81 in stage 3) on a tenth-size simulated data set: every
    subset chain of the three stages against the oracle on the same generated draws, the
    moment-matched summaries, and the aggregated posterior means."""
    d = synth.make_workload(name, scale=0.1)
    pr = Pair(d, 5, I=10, J=10, burnin=10, thin=2, gen=True, seed=21)
    for stage in (1, 2, 3):
        pr.run_stage(stage, 40)
        for s in pr.p.stage_subsets(stage):
            pr.compare_subset(s.sid, rel=1e-7)
        pr.finish_stage(stage)
    Xo, Wo, nco = oracle.aggregate_plan(pr.p, pr.finals, 5)
    Xm, Wm, nc = pr.m.posterior_means()
    assert nc == nco
    assert_rows_close(Xm, Xo[np.argsort(pr.p.row_perm)], 1e-6, "aggregated X")
    assert_rows_close(Wm, Wo[np.argsort(pr.p.col_perm)], 1e-6, "aggregated W")
    pr.m.close()


def test_partition_mode_of_the_benchmark():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload",
                        "sim-6040x3706-k5", "--scale", "0.1", "--datasets", "2"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    grids = {(q["grid"], q["order"]) for q in out["table"]}
    assert grids == {(f"{g}x{g}", o) for g in (1, 3, 5, 10, 30) for o in ("decreasing", "none")}
    assert all(q["datasets"] == 2 for q in out["table"])
    assert {q["dataset"] for q in out["runs"]} == {0, 1}
    table = [(q["grid"], q["order"], round(q["rmse"], 4)) for q in out["runs"]]
    assert all(np.isfinite(q["rmse"]) and q["rmse"] > 1.0 for q in out["runs"]), table
    # at a tenth of the size a 10 x 10 grid leaves about 7 training cells per row and subset
    # (30 x 30: about 2, and the predictions fall back to the mean), so only the coarse grids
    # are held to the full chain's neighbourhood here; the full-size runs are the experiment
    assert all(q["rmse"] < 1.2 for q in out["runs"] if q["grid"] in ("1x1", "3x3")), table
    assert out["gpu_launches"] > 0


def test_correlation_experiment_of_the_benchmark():
    """Section 5.6 at a tenth of the size: PP's subset posterior means correlate across subsets
    sharing rows or columns more strongly than those of independent subsets (without the
    alignment the baseline's latent dimensions disagree)."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload",
                        "sim-6040x3706-k5", "--scale", "0.1", "--experiment", "correlations"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert [g["grid"] for g in out["grids"]] == ["3x3", "5x5", "10x10"]
    for g in out["grids"]:
        assert g["pp"]["raw"]["mean"] > g["independent"]["raw"]["mean"], g
        assert g["pp"]["raw"]["mean"] > g["independent"]["aligned"]["mean"], g
