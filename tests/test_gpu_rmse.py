"""Test RMSE of whole runs on the benchmark workloads: the CUDA path (reduced precision where the
workload says so) against the FP64 oracle on the same draws must agree within 0.002 (the
accuracy target of the method's reduced-precision and batched forms); the FP64 path agrees to
rounding.  Sizes: the 1000 x 500 planted workload in full (200 sweeps, burn-in 100), the
69,878 x 10,677 Zipf workload for 20 sweeps, and the 4 x 4 posterior-propagation workload at a
quarter of its rows and columns (1/16 of its observations) for 40 sweeps per stage."""
import numpy as np
import pytest

import oracle
from paper_1703_00734_gb300 import synth
from pairing import Pair

pytestmark = pytest.mark.gpu


def plain_rmse(pr, d):
    """Test RMSE of the oracle's posterior-mean prediction (1 x 1 grid)."""
    st = pr.chains[0]
    rr, cr = np.argsort(pr.p.row_perm), np.argsort(pr.p.col_perm)
    Xm, Wm = st.S1X / st.n_kept, st.S1W / st.n_kept
    yo = oracle.predict(d["test_row"], d["test_col"], Xm[rr], Wm[cr], pr.p.offset)
    return oracle.rmse(yo, d["test_val"])


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 2e-3)])
def test_planted_full_run(precision, tol):
    d = synth.make_workload("planted-1000x500-k10")
    pr = Pair(d, 10, precision=precision, burnin=100, moments="full")
    pr.run_stage(1, 200)
    _, r_gpu = pr.m.predict(d["test_row"], d["test_col"], d["test_val"])
    r_cpu = plain_rmse(pr, d)
    print(f"planted {precision}: rmse gpu {r_gpu:.6f} oracle {r_cpu:.6f}")
    assert abs(r_gpu - r_cpu) <= tol


def test_zipf_rating_workload_fp32():
    d = synth.make_workload("zipf-69878x10677-10M-k10")
    pr = Pair(d, 10, precision="fp32", burnin=10, moments="full")
    pr.run_stage(1, 20)
    _, r_gpu = pr.m.predict(d["test_row"], d["test_col"], d["test_val"])
    r_cpu = plain_rmse(pr, d)
    print(f"zipf 10M fp32: rmse gpu {r_gpu:.6f} oracle {r_cpu:.6f}")
    assert abs(r_gpu - r_cpu) <= 2e-3


def test_pp_stages_reduced_workload_fp32():
    d = synth.make_workload("pp4x4-100000x20000-20M-k16", scale=0.25)
    pr = Pair(d, 16, I=4, J=4, precision="fp32", burnin=20)
    for stage in (1, 2, 3):
        pr.run_stage(stage, 40)
        pr.finish_stage(stage)
    Xm, Wm, _ = oracle.aggregate_plan(pr.p, pr.finals, 16)
    rr, cr = np.argsort(pr.p.row_perm), np.argsort(pr.p.col_perm)
    yo = oracle.predict(d["test_row"], d["test_col"], Xm[rr], Wm[cr], pr.p.offset)
    r_cpu = oracle.rmse(yo, d["test_val"])
    _, r_gpu = pr.m.predict(d["test_row"], d["test_col"], d["test_val"])
    print(f"pp 4x4 fp32: rmse gpu {r_gpu:.6f} oracle {r_cpu:.6f}")
    assert abs(r_gpu - r_cpu) <= 2e-3
