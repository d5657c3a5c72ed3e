"""K > 16: the warp-per-row conditional and the tensor-core / FP64 Gram kernels against the
oracle.  FP64 mode to the 1e-9 per-row tolerance; BF16 (mma m16n8k16, y split into high and low
BF16 parts: u_y = 2^-16) and FP32 (split TF32, three products: u_in = 2^-21) under the
first-order bound of test_gpu_precision.py."""
import numpy as np
import pytest

import oracle
from paper_1703_00734_gb300 import synth
from pairing import Pair, assert_rows_close
from test_gpu_precision import run_reduced

pytestmark = pytest.mark.gpu


def data(K, N=260, D=200, M=20_000, seed=0, pattern="uniform", ratings=False):
    return synth.make_workload(None, N=N, D=D, M=M, pattern=pattern, K=K, sigma=0.5, tau=4.0,
                               seed=seed, s_row=1.1, s_col=1.1, ratings=ratings)


@pytest.mark.parametrize("K", [17, 20, 32, 33, 64])
def test_wide_fp64_single_transition(K):
    pr = Pair(data(K, seed=K), K)
    pr.run_stage(1, 1)
    pr.compare_subset(0)


def test_wide_fp64_split_rows_and_sweeps():
    d = data(32, N=300, D=2500, M=70_000, seed=3, pattern="zipf")
    assert np.bincount(d["row"], minlength=d["N"]).max() > 2048
    pr = Pair(d, 32, burnin=1)
    pr.run_stage(1, 3)
    pr.compare_subset(0, rel=1e-8)


@pytest.mark.parametrize("K", [32, 64])
def test_wide_bf16_within_bound(K):
    d = data(K, N=400, D=300, M=40_000, seed=10 + K, pattern="zipf", ratings=True)
    d["tau"] = 1.5625
    qx, qw = run_reduced(d, K, "bf16", 2.0 ** -8, u_y=2.0 ** -16)
    print(f"bf16 K={K}: worst err/bound X {qx:.3f} W {qw:.3f}")


@pytest.mark.parametrize("K", [24, 32, 64])
def test_wide_fp32_split_tf32_within_bound(K):
    d = data(K, N=400, D=300, M=40_000, seed=20 + K, pattern="zipf", ratings=True)
    d["tau"] = 1.5625
    qx, qw = run_reduced(d, K, "fp32", 2.0 ** -21)
    print(f"fp32 (split TF32) K={K}: worst err/bound X {qx:.3f} W {qw:.3f}")


@pytest.mark.parametrize("K", [20, 40])
def test_wide_pp_stages_moment_matching_and_aggregation(K):
    """Three PP stages at K > 16 (tensor-core Gram path, team conditional, moment matching and
    Algorithm 2 with fewer rows per block) against the oracle, FP64."""
    d = synth.make_workload(None, N=240, D=160, M=9000, pattern="uniform", K=K, sigma=0.5,
                            tau=4.0, seed=100 + K)
    pr = Pair(d, K, I=2, J=2, burnin=3)
    T = 3 + 2 * K
    for stage in (1, 2, 3):
        pr.run_stage(stage, T)
        for s in pr.p.stage_subsets(stage):
            pr.compare_subset(s.sid, rel=1e-7)
        pr.finish_stage(stage)
        for s in pr.p.stage_subsets(stage):
            for f in (0, 1):
                mu, Lam = pr.m.get_posterior(s.sid, f)
                fm = pr.finals[s.sid]
                assert_rows_close(mu, fm[2 * f], 1e-6, f"MM mean {s.sid}/{f}")
                assert_rows_close(Lam.reshape(len(Lam), -1), fm[2 * f + 1].reshape(len(Lam), -1),
                                  1e-6, f"MM precision {s.sid}/{f}")
    Xm_o, Wm_o, nc_o = oracle.aggregate_plan(pr.p, pr.finals, K)
    Xm, Wm, nc = pr.m.posterior_means()
    assert nc == nc_o
    rr, cr = np.argsort(pr.p.row_perm), np.argsort(pr.p.col_perm)
    assert_rows_close(Xm, Xm_o[rr], 1e-6, "aggregated X")
    assert_rows_close(Wm, Wm_o[cr], 1e-6, "aggregated W")
