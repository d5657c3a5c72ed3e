"""The subset-posterior correlation statistics of Section 5.6 (bench.py): the latent-dimension
alignment applied to the embarrassingly parallel baseline recovers a permuted, sign-flipped copy,
the block correlation is Pearson's r over all entries, and the pairs are the blocks that subsets
sharing rows or columns estimate."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_alignment_recovers_permutation_and_signs():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((400, 6)) * np.arange(1, 7)
    perm = rng.permutation(6)
    sign = np.where(rng.random(6) < 0.5, -1.0, 1.0)
    B = (A * sign)[:, perm] + 0.05 * rng.standard_normal((400, 6))
    raw = bench.block_correlation(A, B)
    al = bench.block_correlation(A, bench.align_latent(A, B))
    assert abs(raw) < 0.5 and al > 0.999


def test_block_correlation_is_pearson_over_entries():
    rng = np.random.default_rng(1)
    A, B = rng.standard_normal((30, 4)), rng.standard_normal((30, 4))
    B = 0.7 * A + B
    np.testing.assert_allclose(bench.block_correlation(A, B),
                               np.corrcoef(A.ravel(), B.ravel())[0, 1], rtol=1e-12)


def test_pairs_of_subsets_sharing_rows_or_columns():
    rng = np.random.default_rng(2)
    I, J = 3, 4
    means = {s: (rng.standard_normal((5, 2)), rng.standard_normal((6, 2))) for s in range(I * J)}
    out = bench.subset_correlations(means, I, J)
    assert out["raw"]["pairs"] == I * (J - 1) + J * (I - 1)
    # identical blocks correlate perfectly
    same = {s: (np.ones((5, 2)) * np.arange(2) + np.arange(5)[:, None], np.eye(6, 2))
            for s in range(I * J)}
    assert bench.subset_correlations(same, I, J)["raw"]["min"] > 0.999999
