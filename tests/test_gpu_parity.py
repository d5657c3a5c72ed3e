"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, same inputs, same
draws.  FP64 mode: every sampled state agrees per row to 1e-9 relative (|x_gpu - x_cpu|_inf <=
1e-9 (|x_cpu|_inf + 1e-3 rms)) after one transition from an identical state, and over a few
sweeps; integer work (ordering, grid) is bit-exact."""
import numpy as np
import pytest

import oracle
from paper_1703_00734_gb300 import synth
from pairing import Pair, assert_rows_close

pytestmark = pytest.mark.gpu


def small(N=300, D=170, M=6000, K=5, seed=0, pattern="uniform", **kw):
    return synth.make_workload(None, N=N, D=D, M=M, pattern=pattern, K=K, sigma=0.5,
                               tau=kw.pop("tau", 4.0), seed=seed, s_row=1.2, s_col=1.2, **kw)


def test_ordering_and_grid_are_bit_exact():
    d = small(pattern="zipf", seed=3)
    pr = Pair(d, 5, I=3, J=2)
    rp, cp = pr.m.perm()
    np.testing.assert_array_equal(rp, pr.p.row_perm)
    np.testing.assert_array_equal(cp, pr.p.col_perm)
    for s in pr.p.subsets:
        info = pr.m.subset_info(s.sid)
        assert (info["row0"], info["row1"], info["col0"], info["col1"]) == (s.r0, s.r1, s.c0, s.c1)
        assert info["nnz"] == s.nnz and info["stage"] == s.stage


@pytest.mark.parametrize("K", [1, 3, 5, 10, 16])
def test_single_transition_fp64(K):
    d = small(K=K, seed=K)
    pr = Pair(d, K)
    pr.run_stage(1, 1)
    pr.compare_subset(0)


@pytest.mark.parametrize("K,prec,rel", [(16, "fp64", 1e-9), (13, "fp64", 1e-9), (16, "fp32", 1e-3)])
def test_rows_forming_their_own_gram_sums(K, prec, rel):
    """13 <= K <= 16: rows with at most 64 observations form G_n, r_n inside the conditional
    draw, longer rows come from the Gram pass; both kinds against the oracle, over sweeps that
    keep moments (FP32: one transition, within the error of its FP32 Gram sums)."""
    d = small(N=600, D=250, M=30_000, K=K, pattern="zipf", seed=40 + K)
    for side, n in (("row", d["N"]), ("col", d["D"])):
        counts = np.bincount(d[side], minlength=n)
        assert (counts > 64).any() and ((counts > 0) & (counts <= 64)).any(), side
    pr = Pair(d, K, precision=prec, burnin=1, moments="full")
    pr.run_stage(1, 1)
    pr.compare_subset(0, rel=rel)
    if prec != "fp64":
        return
    pr.run_stage(1, 3, t0=1)
    pr.compare_subset(0, rel=10 * rel)
    S1, S2, kept = pr.m.get_moments(0, 0)
    assert kept == 3
    assert_rows_close(S2.reshape(len(S2), -1), pr.chains[0].S2X.reshape(len(S2), -1), 10 * rel, "S2X")


def test_multi_sweep_fp64_with_moments():
    d = small(K=4, N=257, D=129, M=5000, seed=7)
    pr = Pair(d, 4, burnin=2, thin=2, moments="full")
    stats = pr.run_stage(1, 8)
    pr.compare_subset(0, rel=1e-8)
    S1, S2, kept = pr.m.get_moments(0, 0)
    st = pr.chains[0]
    assert kept == st.n_kept == 3
    assert_rows_close(S1, st.S1X, 1e-8, "S1X")
    assert_rows_close(S2.reshape(len(S2), -1), st.S2X.reshape(len(S2), -1), 1e-8, "S2X")
    assert np.isfinite(stats["rmse_sample"]) and np.isfinite(stats["rmse_mean"])


def test_zipf_heavy_rows_split_across_work_items():
    """Rows longer than one Gram work item (1024 observations) are split; the partial sums
    must combine to the same conditional."""
    d = small(N=400, D=3000, M=90_000, K=6, pattern="zipf", seed=5)
    counts = np.bincount(d["row"], minlength=d["N"])
    assert counts.max() > 2048
    pr = Pair(d, 6)
    pr.run_stage(1, 2)
    pr.compare_subset(0, rel=1e-8)


def test_empty_rows_and_columns():
    d = small(N=50, D=40, M=300, K=3, seed=9)
    keep = (d["row"] != 7) & (d["col"] != 11)
    for k in ("row", "col", "val"):
        d[k] = d[k][keep]
    pr = Pair(d, 3)
    pr.run_stage(1, 1)
    pr.compare_subset(0)


def test_pp_stages_fp64_parity_and_aggregation():
    """Three stages of Algorithm 1 on a 3 x 2 grid, both sides fed the same draws; then the
    moment-matched summaries and the Algorithm 2 aggregate."""
    d = small(N=240, D=160, M=9000, K=4, seed=13)
    pr = Pair(d, 4, I=3, J=2, burnin=3)
    T = 12
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
    Xm_o, Wm_o, nc_o = oracle.aggregate_plan(pr.p, pr.finals, 4)
    Xm, Wm, nc = pr.m.posterior_means()
    assert nc == nc_o
    rr, cr = np.argsort(pr.p.row_perm), np.argsort(pr.p.col_perm)
    assert_rows_close(Xm, Xm_o[rr], 1e-6, "aggregated X")
    assert_rows_close(Wm, Wm_o[cr], 1e-6, "aggregated W")
    yh, r = pr.m.predict(d["test_row"], d["test_col"], d["test_val"])
    yo = oracle.predict(d["test_row"], d["test_col"], Xm_o[rr], Wm_o[cr], pr.p.offset)
    np.testing.assert_allclose(yh, yo, rtol=1e-6, atol=1e-8)
    assert abs(r - oracle.rmse(yo, d["test_val"])) < 1e-8
    # Eq. 14 with Algorithm 2 on identical inputs: the library's own moment-matched subset
    # posteriors fed to the oracle's aggregation.  The eigenvalue correction must have run on
    # the device (an indefinite difference Lambda^(j) - Lambda^(1) in some rows).
    gfin = {}
    for s in pr.p.subsets:
        mx, Lx = pr.m.get_posterior(s.sid, 0)
        mw, Lw = pr.m.get_posterior(s.sid, 1)
        gfin[s.sid] = (mx, Lx, mw, Lw)
    Xg_o, Wg_o, nc_g = oracle.aggregate_plan(pr.p, gfin, 4)
    assert nc > 0 and nc_g == nc
    assert_rows_close(Xm, Xg_o[rr], 1e-9, "aggregated X, identical inputs")
    assert_rows_close(Wm, Wg_o[cr], 1e-9, "aggregated W, identical inputs")


def test_error_paths():
    from paper_1703_00734_gb300 import bmf
    d = small(N=30, D=20, M=200, K=2, seed=21)
    row = np.concatenate([d["row"], d["row"][:1]])
    col = np.concatenate([d["col"], d["col"][:1]])
    val = np.concatenate([d["val"], d["val"][:1]])
    with pytest.raises(bmf.BmfError) as e:
        bmf.BMF(d["N"], d["D"], row, col, val, 2, 1.0, X0=d["X0"], W0=d["W0"])
    assert e.value.status == 1
    v = d["val"].copy()
    v[3] = np.nan
    with pytest.raises(bmf.BmfError) as e:
        bmf.BMF(d["N"], d["D"], d["row"], d["col"], v, 2, 1.0, X0=d["X0"], W0=d["W0"])
    assert e.value.status == 4
    m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], 2, 1.0, X0=d["X0"], W0=d["W0"],
                I=2, J=2)
    with pytest.raises(bmf.BmfError) as e:
        m.stage(1, 1, np.zeros(5))
    assert e.value.status == 2
    with pytest.raises(bmf.BmfError) as e:
        m.stage(3, 1, np.zeros(m.draws_per_sweep(3)))
    assert e.value.status == 8


@pytest.mark.parametrize("K", [3, 7, 12])
def test_thread_per_row_conditional_on_large_halves(K):
    """The thread-per-row conditional (K <= 12) on halves of thousands of rows: FP64 parity."""
    d = small(N=9000, D=8300, M=120_000, K=K, seed=90 + K, pattern="zipf")
    pr = Pair(d, K)
    pr.run_stage(1, 1)
    pr.compare_subset(0)


def test_fault_injection_on_the_host():
    """Faults made on the host give their documented status and leave the GPU usable: an
    out-of-range index, a forced non-positive-definite prior (BMF_E_NOT_PD, then BMF_E_STATE
    until bmf_set_state), and a tuner call on a stage that is not open."""
    from paper_1703_00734_gb300 import bmf
    d = small(N=60, D=40, M=800, K=3, seed=23)
    for bad in (d["N"], -1):
        row = d["row"].copy()
        row[5] = bad
        with pytest.raises(bmf.BmfError) as e:
            bmf.BMF(d["N"], d["D"], row, d["col"], d["val"], 3, 1.0, X0=d["X0"], W0=d["W0"])
        assert e.value.status == 1
    m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], 3, 4.0, X0=d["X0"], W0=d["W0"],
                seed=2)
    n = d["N"]
    mu = np.zeros((n, 3))
    m.set_prior(0, bmf.FACTOR_X, mu, np.tile(-np.eye(3) * 1e3, (n, 1, 1)))
    with pytest.raises(bmf.BmfError) as e:
        m.sweep(0, 1, None)
    assert e.value.status == 3 and "arena row" in str(e.value)
    with pytest.raises(bmf.BmfError) as e:
        m.sweep(0, 1, None)
    assert e.value.status == 8
    X0 = d["X0"][m.perm()[0]]
    W0 = d["W0"][m.perm()[1]]
    m.set_state(0, X0, W0)
    m.set_prior(0, bmf.FACTOR_X, mu, np.tile(np.eye(3), (n, 1, 1)))
    st = m.sweep(0, 2, None)
    assert st["sweeps"] >= 2
    X, W, _ = m.get_state(0)
    assert np.all(np.isfinite(X)) and np.all(np.isfinite(W))
    m.close()
    m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], 3, 4.0, I=2, J=2)
    with pytest.raises(bmf.BmfError) as e:
        m.autotune(2, -1, 1)
    assert e.value.status == 8
    m.close()


def test_pp_with_empty_subsets_and_zero_sweep_calls():
    """A 2 x 2 grid whose off-diagonal blocks hold no observations (their chains sample the
    prior and the propagated summaries), and calls of zero sweeps, against the oracle."""
    d = small(N=120, D=100, M=3000, K=3, seed=31)
    rb, cb = np.array([0, 60, 120]), np.array([0, 50, 100])
    # keep only observations in the diagonal blocks of the original order, no reordering
    keep = ((d["row"] < 60) & (d["col"] < 50)) | ((d["row"] >= 60) & (d["col"] >= 50))
    for k in ("row", "col", "val"):
        d[k] = d[k][keep]
    tk = ((d["test_row"] < 60) & (d["test_col"] < 50)) | ((d["test_row"] >= 60) & (d["test_col"] >= 50))
    for k in ("test_row", "test_col", "test_val"):
        d[k] = d[k][tk]
    pr = Pair(d, 3, I=2, J=2, burnin=2, order="none", row_bounds=rb, col_bounds=cb)
    for s in pr.p.subsets:
        if s.i != s.j:
            assert s.nnz == 0
    for stage in (1, 2, 3):
        pr.m.stage(stage, 0, None)
        pr.run_stage(stage, 8)
        for s in pr.p.stage_subsets(stage):
            pr.compare_subset(s.sid, rel=1e-7)
        pr.finish_stage(stage)
    Xm_o, Wm_o, nc_o = oracle.aggregate_plan(pr.p, pr.finals, 3)
    Xm, Wm, nc = pr.m.posterior_means()
    assert nc == nc_o
    assert_rows_close(Xm, Xm_o, 1e-6, "aggregated X")
    assert_rows_close(Wm, Wm_o, 1e-6, "aggregated W")


def test_restart_reproduces_a_run_and_test_rmse_matches_predict():
    """bmf_restart: a restarted context with the same seed repeats a whole PP run bit for bit
    (device generator), equals a freshly initialised context, and a new seed gives a new run;
    bmf_test_rmse equals the RMSE of bmf_predict on the same held-out entries."""
    from paper_1703_00734_gb300 import bmf
    d = small(N=240, D=160, M=9000, K=4, seed=13)
    test = (d["test_row"], d["test_col"], d["test_val"])

    def ctx(seed):
        return bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], 4, d["tau"], "fp32",
                       I=2, J=3, X0=d["X0"], W0=d["W0"], test=test, burnin=3, seed=seed)

    def run(m):
        for stage in (1, 2, 3):
            m.stage(stage, 10, None)
        Xm, Wm, nc = m.posterior_means()
        return m.test_rmse(), Xm, Wm

    m = ctx(5)
    r1, X1, W1 = run(m)
    _, rp = m.predict(*test)
    assert abs(r1 - rp) < 1e-12 * max(1.0, r1)
    m.restart(5)
    r2, X2, W2 = run(m)
    assert r2 == r1
    np.testing.assert_array_equal(X2, X1)
    np.testing.assert_array_equal(W2, W1)
    m.restart(6)
    r3, X3, _ = run(m)
    assert r3 != r1 and not np.array_equal(X3, X1)
    m.restart(5, X0=d["X0"], W0=d["W0"])
    r4, X4, _ = run(m)
    assert r4 == r1
    np.testing.assert_array_equal(X4, X1)
    with pytest.raises(bmf.BmfError) as e:
        m.restart(5, X0=np.full_like(d["X0"], np.nan))
    assert e.value.status == 4
    m.close()
    f = ctx(5)
    r5, X5, _ = run(f)
    assert r5 == r1
    np.testing.assert_array_equal(X5, X1)
    f.close()


def test_independent_subsets_fp64_parity():
    """The embarrassingly parallel baseline (no propagation: standard priors and hyperparameter
    draws in every subset, chains from the initial state) against the oracle with the same
    draws, through the three stages, and the aggregation of its subset posteriors."""
    d = small(N=240, D=160, M=9000, K=4, seed=17)
    pr = Pair(d, 4, I=3, J=2, burnin=3, propagate=False)
    for stage in (1, 2, 3):
        pr.run_stage(stage, 12)
        for s in pr.p.stage_subsets(stage):
            pr.compare_subset(s.sid, rel=1e-7)
            st = pr.chains[s.sid]
            assert not st.prior_x and not st.prior_w
        pr.finish_stage(stage)
    Xm_o, Wm_o, nc_o = oracle.aggregate_plan(pr.p, pr.finals, 4)
    Xm, Wm, nc = pr.m.posterior_means()
    assert nc == nc_o
    assert_rows_close(Xm, Xm_o[np.argsort(pr.p.row_perm)], 1e-6, "aggregated X")
    assert_rows_close(Wm, Wm_o[np.argsort(pr.p.col_perm)], 1e-6, "aggregated W")
