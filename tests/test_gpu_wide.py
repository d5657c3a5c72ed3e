"""K > 16: the warp-per-row conditional and the tensor-core / FP64 Gram kernels against the
oracle.  FP64 mode to the 1e-9 per-row tolerance; BF16 (mma m16n8k16, y split into high and low
BF16 parts: u_y = 2^-16) and FP32 (split TF32, three products: u_in = 2^-21) under the
first-order bound of test_gpu_precision.py."""
import numpy as np
import pytest

from paper_1703_00734_gb300 import synth
from pairing import Pair
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
