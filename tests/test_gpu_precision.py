"""Reduced-precision parity: the FP32 and BF16 gather paths against the FP64 oracle under a
per-result error bound, and the FP64 path on the full 69,878 x 10,677 Zipf workload in the
launch configuration the benchmark times.

Bound (first-order perturbation of the conditional draw x = Lambda^{-1} b + L^{-T} z):
  |dLambda| <= tau (m u_acc + 2 u_in) |P|^T |P| + tau (|P|^T |dP| + |dP|^T |P|)   entrywise,
  |db|      <= tau (m u_acc + u_in + u_y) |P|^T |y| + tau |dP|^T |y|,
  |dx|_2    <= ||Lambda^{-1}||_2 (|db|_2 + ||dLambda||_F (|mu|_2 + 2 |L^{-T} z|_2)),
with u_in the rounding of the gathered partner rows (2^-24 FP32, 2^-8 BF16), u_y = 2^-24 the
rounding of the values, u_acc = 2^-24 the FP32 accumulation, m = the longest sequential sum of one
lane (ceil(deg / lanes) + log2(lanes) + 2), and dP the difference of the partner rows the two
sides used (zero for the first half of a sweep).  The test requires |dx|_inf <= 2 * bound per
row."""
import math

import numpy as np
import pytest

import oracle
from paper_1703_00734_gb300 import synth
from pairing import Pair, assert_rows_close

pytestmark = pytest.mark.gpu

U_ACC = 2.0 ** -24


def lanes_for(count):
    """Lanes per row of the K <= 16 Gram pass (8 up to 64 observations, 16 up to 256)."""
    return 8 if count <= 64 else (16 if count <= 256 else 32)


def seq_len(n, K):
    """Longest sequential FP32 sum behind one accumulated entry: lanes x iterations for the
    CUDA-core kernels (K <= 16); tensor-core accumulation steps of 16 (or 8) observations plus
    the products summed inside one instruction for K > 16; every observation in list order for
    a row that forms its own Gram sums in the conditional (13 <= K <= 16, at most 64)."""
    c = min(n, 1024)
    if 13 <= K <= 16 and n <= 64:
        return n + 2
    if K > 16:
        return math.ceil(c / 8) + 16 + 2
    lanes = lanes_for(c)
    return math.ceil(c / lanes) + math.log2(lanes) + 2


def row_bounds(ptr, idx, val, P, dP, tau, mu_p, Lam_p, z, u_in, rows, u_y=U_ACC):
    out = np.zeros(len(rows))
    b_p = Lam_p @ mu_p
    K = P.shape[1]
    for k, r in enumerate(rows):
        sl = slice(ptr[r], ptr[r + 1])
        Pr, yr, dPr = P[idx[sl]], val[sl], dP[idx[sl]]
        n = len(yr)
        m = seq_len(n, K)
        aP, ay, adP = np.abs(Pr), np.abs(yr), np.abs(dPr)
        Lam = Lam_p + tau * Pr.T @ Pr
        E = tau * ((m * U_ACC + 2 * u_in) * aP.T @ aP + aP.T @ adP + adP.T @ aP)
        eb = tau * ((m * U_ACC + u_in + u_y) * aP.T @ ay + adP.T @ ay)
        b = b_p + tau * Pr.T @ yr
        mu = np.linalg.solve(Lam, b)
        L = np.linalg.cholesky(Lam)
        w = np.linalg.solve(L.T, z[r])
        out[k] = (np.linalg.norm(eb) + np.linalg.norm(E) * (np.linalg.norm(mu) + 2 * np.linalg.norm(w))) \
            / np.linalg.eigvalsh(Lam)[0]
    return out


def check_half(gpu_rows, cpu_rows, bound, what, factor=2.0):
    """|dx|_inf <= factor * bound per row, plus the FP64 rounding level of the factorisation
    (the reduced-precision modes refine the pivot reciprocal square root to a relative error
    below 1e-12): a row without observations has a zero Gram bound."""
    err = np.abs(gpu_rows - cpu_rows).max(1)
    floor = 1e-11 * (np.abs(cpu_rows).max(1) + 1e-3)
    ratio = err / (factor * bound + floor)
    assert ratio.max() <= 1.0, f"{what}: worst |dx| {err.max():.3e}, worst err/bound {ratio.max():.3f}"
    return ratio.max()


def run_reduced(d, K, precision, u_in, rows_x=None, rows_w=None, u_y=U_ACC):
    pr = Pair(d, K, precision=precision)
    s = pr.p.subsets[0]
    H = oracle.hyper_block_len(K)
    dr = pr.draws(1, 0)
    lay = oracle.stage_draw_layout([s], K)
    zx = dr[lay[(0, "zx")]:lay[(0, "zx")] + s.n * K].reshape(s.n, K)
    zw = dr[lay[(0, "zw")]:lay[(0, "zw")] + s.d * K].reshape(s.d, K)
    X0, W0 = pr.X0.copy(), pr.W0.copy()
    pr.run_stage(1, 1)
    X, W, hyp = pr.m.get_state(0)
    st = pr.chains[0]
    # the hyperparameter draw is FP64 on both sides from identical inputs
    assert_rows_close(hyp["LamX"], st.LamX, 1e-9, "Lambda_X")
    assert_rows_close(hyp["LamW"], st.LamW, 1e-9, "Lambda_W")
    rx = np.arange(s.n) if rows_x is None else rows_x
    rw = np.arange(s.d) if rows_w is None else rows_w
    bx = row_bounds(s.rptr, s.ridx, s.rval, W0, np.zeros_like(W0), d["tau"], st.muX, st.LamX, zx,
                    u_in, rx, u_y)
    qx = check_half(X[rx], st.X[rx], bx, f"{precision} X half")
    dX = np.abs(X - st.X)
    bw = row_bounds(s.cptr, s.cidx, s.cval, st.X, dX, d["tau"], st.muW, st.LamW, zw, u_in, rw, u_y)
    qw = check_half(W[rw], st.W[rw], bw, f"{precision} W half")
    return qx, qw


@pytest.mark.parametrize("K,pattern", [(10, "zipf"), (16, "zipf"), (5, "uniform")])
def test_fp32_single_transition_within_bound(K, pattern):
    d = synth.make_workload(None, N=500, D=320, M=40_000, pattern=pattern, K=K, sigma=0.8,
                            tau=1.5625, seed=40 + K, s_row=1.2, s_col=1.2, ratings=True)
    qx, qw = run_reduced(d, K, "fp32", 2.0 ** -24)
    print(f"fp32 K={K}: worst err/bound X {qx:.3f} W {qw:.3f}")


@pytest.mark.parametrize("K", [24, 40])
def test_tf32_single_transition_within_bound(K):
    """BMF_TF32 at K > 16: one TF32 tensor-core product per Gram tile, partner rows and values
    rounded to 10-bit mantissas (2^-11)."""
    d = synth.make_workload(None, N=500, D=320, M=40_000, pattern="zipf", K=K, sigma=0.8,
                            tau=1.5625, seed=60 + K, s_row=1.2, s_col=1.2, ratings=True)
    qx, qw = run_reduced(d, K, "tf32", 2.0 ** -11, u_y=2.0 ** -11)
    print(f"tf32 K={K}: worst err/bound X {qx:.3f} W {qw:.3f}")


@pytest.mark.parametrize("K", [10, 16])
def test_bf16_single_transition_within_bound(K):
    d = synth.make_workload(None, N=500, D=320, M=40_000, pattern="zipf", K=K, sigma=0.8,
                            tau=1.5625, seed=50 + K, s_row=1.2, s_col=1.2, ratings=True)
    qx, qw = run_reduced(d, K, "bf16", 2.0 ** -8)
    print(f"bf16 K={K}: worst err/bound X {qx:.3f} W {qw:.3f}")


def test_full_size_workload_one_sweep():
    """The 69,878 x 10,677 Zipf workload with 9M training entries (the benchmark's), in the
    benchmark's launch configuration: FP64 path on every row to the FP64 tolerance, FP32 path
    on sampled rows within the bound."""
    d = synth.make_workload("zipf-69878x10677-10M-k10")
    pr = Pair(d, 10, precision="fp64", burnin=2)
    pr.run_stage(1, 1)
    pr.compare_subset(0, rel=1e-9)
    rng = np.random.default_rng(0)
    s = pr.p.subsets[0]
    rows_x = np.unique(np.concatenate([np.arange(40), rng.choice(s.n, 400, replace=False)]))
    rows_w = np.unique(np.concatenate([np.arange(40), rng.choice(s.d, 400, replace=False)]))
    pr.m.close()
    qx, qw = run_reduced(d, 10, "fp32", 2.0 ** -24, rows_x, rows_w)
    print(f"full-size fp32: worst err/bound X {qx:.3f} W {qw:.3f}")
