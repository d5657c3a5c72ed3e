"""The simulated data sets of the paper's Section 5.3 (inputs only, no sampler arithmetic):
Y = X W^T + E with standard-normal X, W, E, K = 5, every cell present before the split;
80% of the cells held out at random, or kept for training with probability w_n w_d (w equally
spaced from 0.9 to 0.005 over rows and over columns) in the structured scenario."""
import numpy as np

from paper_1703_00734_gb300 import synth


def test_random_missingness_holds_out_eighty_percent():
    d = synth.make_workload("sim-6040x3706-k5", scale=0.1)
    N, D = d["N"], d["D"]
    n_train, n_test = len(d["row"]), len(d["test_row"])
    assert n_train + n_test == N * D
    assert n_test == int(round(0.8 * N * D))
    keys = np.concatenate([d["row"].astype(np.int64) * D + d["col"],
                           d["test_row"].astype(np.int64) * D + d["test_col"]])
    assert np.array_equal(np.sort(keys), np.arange(N * D))      # every cell exactly once
    assert d["K"] == 5 and d["tau"] == 1.0


def test_values_are_low_rank_plus_unit_noise():
    d = synth.make_workload("sim-6040x3706-k5", scale=0.1)
    X, W = d["X_true"], d["W_true"]
    y = np.concatenate([d["val"], d["test_val"]])
    r = np.concatenate([d["row"], d["test_row"]])
    c = np.concatenate([d["col"], d["test_col"]])
    resid = y - np.einsum("ij,ij->i", X[r], W[c])
    assert abs(resid.mean()) < 0.02 and abs(resid.var() - 1.0) < 0.03   # E ~ N(0, 1)
    assert abs(y.var() - 6.0) < 0.6                                      # K + 1


def test_structured_missingness_follows_row_and_column_weights():
    d = synth.make_workload("sim-6040x3706-k5-structured", scale=0.2)
    N, D = d["N"], d["D"]
    frac_missing = len(d["test_row"]) / (N * D)
    mean_w = (0.9 + 0.005) / 2
    assert abs(frac_missing - (1 - mean_w ** 2)) < 0.01                  # about 80% missing
    keep_rows = np.bincount(d["row"], minlength=N) / D
    wn = np.linspace(0.9, 0.005, N)
    # expected keep rate of row n is w_n * mean(w_d)
    assert np.abs(keep_rows - wn * mean_w).max() < 0.12
    assert keep_rows[: N // 10].mean() > 5 * keep_rows[-N // 10:].mean()
