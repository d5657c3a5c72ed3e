"""The benchmark's roofline arithmetic: algorithmic work per launch from the per-unit figures
(per observation-side: 4-byte index + value + gathered row; per row: assembly K(K+1)/2 + K,
Cholesky (K^3 - K)/6, two solves K(K - 1) FMA, 2 flops each), and the committed ncu traffic
lookups."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _fake(N, D, M):
    return {"N": N, "D": D, "row": np.zeros(M, np.int32)}


def test_gram_and_conditional_work_of_the_bench_workload():
    d = _fake(69878, 10677, 9_000_000)
    a = bench.algorithmic(d, 10, "fp32")
    assert a["gram_x"] == ("hbm", 9_000_000 * (4 + 4 + 40), "GB/s")       # 432 MB
    assert a["gram_w"][1] == 432_000_000
    fma_row = 55 + 10 + 165 + 90
    assert a["cond_x"] == ("alu", 2.0 * fma_row * 69878, "TFLOP/s")
    assert a["cond_w"][1] == 2.0 * fma_row * 10677
    # precision changes the gathered bytes only
    assert bench.algorithmic(d, 10, "bf16")["gram_x"][1] == 9_000_000 * (4 + 4 + 20)
    assert bench.algorithmic(d, 10, "fp64")["gram_x"][1] == 9_000_000 * (4 + 8 + 80)


def test_cholesky_term_matches_a_direct_count():
    for K in (1, 3, 10, 16, 32):
        d = _fake(1, 1, 1)
        got = bench.algorithmic(d, K, "fp32")["cond_x"][1] / 2.0
        # direct count: Crout column j costs j FMA for the pivot and j for each of the K-1-j
        # entries below it
        chol = sum(j + (K - 1 - j) * j for j in range(K))
        assert got == K * (K + 1) // 2 + K + chol + K * (K - 1)


def test_committed_traffic_lookups():
    t = bench.traffic_for("gram_x", "fp32", "zipf-69878x10677-10M-k10")
    assert t is not None and 5e7 < t < 1e8                  # the observation stream, ~78 MB
    assert bench.traffic_for("adjoint", "fp32", "uniform-200000x50000-50M-k64") > 1e9
    assert bench.traffic_for("gram_x", "fp32", "no-such-workload") is None
    assert bench.traffic_for("cond_x", "bf16", "zipf-69878x10677-10M-k10") is None


def test_pp_work_per_launch_by_stage():
    """Per stage, the Gram classes move entries x (index + value + gathered row) bytes and the
    conditional classes do rows x 2 x (assembly + Cholesky + solves) flops."""
    K = 16
    geom = {1: [25_000, 5_000, 6_000_000], 2: [150_000, 30_000, 7_000_000],
            3: [225_000, 45_000, 5_000_000]}
    a = bench.pp_algorithmic(geom, K, "fp32")
    fma_row = 136 + 16 + (K ** 3 - K) // 6 + K * (K - 1)
    assert fma_row == 1072
    for st, (nx, nw, nnz) in geom.items():
        assert a[(st, "gram_x")] == ("hbm", nnz * (4 + 4 + 64), "GB/s")
        assert a[(st, "gram_w")][1] == nnz * 72
        assert a[(st, "cond_x")] == ("alu", 2.0 * fma_row * nx, "TFLOP/s")
        assert a[(st, "cond_w")][1] == 2.0 * fma_row * nw


def test_pp_kernel_table_shares_and_roofline():
    algo = bench.pp_algorithmic({1: [100, 50, 1000], 2: [0, 0, 0], 3: [0, 0, 0]}, 4, "fp32")
    prof = {1: {"cond_x": (10, 2.0), "gram_x": (10, 1.0), "hyper": (20, 1.0)}, 2: {}, 3: {}}
    t = bench.pp_kernel_table(prof, algo, 6000.0)
    assert abs(sum(v["stream_time_share"] for v in t.values()) - 1.0) < 1e-12
    c = t["s1.cond_x"]
    assert c["launches"] == 10 and abs(c["avg_us"] - 200.0) < 1e-9
    assert abs(c["achieved"] - algo[(1, "cond_x")][1] / 200e-6 / 1e12) < 1e-12
    assert "bound" not in t["s1.hyper"]
