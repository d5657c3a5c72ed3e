"""Whole-chain pins of the oracle: planted low-rank recovery (the paper's simulated-data
protocol, Section 5.3), the column-mean baseline (Section 5.2), sign-flip invariance of the
predictions (Section 2.1.1) and a small posterior-propagation run (Algorithm 1)."""
import numpy as np
import pytest

from paper_1703_00734_gb300 import synth


def _run_plain(orc, d, K, T, burnin, seed=0):
    p = orc.plan(d["N"], d["D"], d["row"], d["col"], d["val"], 1, 1)
    s = p.subsets[0]
    prior = orc.NWPrior(K)
    st = orc.new_chain(d["X0"][p.row_perm], d["W0"][p.col_perm], K)
    chains = {0: st}
    orc.run_stage(p, 1, chains, K, d["tau"], prior,
                  lambda t: synth.sweep_draws([(s.n, s.d)], K, prior.nu0,
                                              synth.rng_for(seed, t)), T, burnin, 1)
    Xm, Wm = st.S1X / st.n_kept, st.S1W / st.n_kept
    rr = np.argsort(p.row_perm)
    cr = np.argsort(p.col_perm)
    return p, Xm[rr], Wm[cr]


def test_planted_recovery_beats_column_means_and_nears_noise_floor(orc):
    d = synth.make_workload("planted-1000x500-k10", scale=0.4, M=12_000)
    # 400 x 200, 12k entries (15% observed), sigma = 0.5
    p, Xm, Wm = _run_plain(orc, d, 10, T=60, burnin=30)
    yhat = orc.predict(d["test_row"], d["test_col"], Xm, Wm, p.offset)
    r = orc.rmse(yhat, d["test_val"])
    cm = np.zeros(d["D"])
    cnt = np.bincount(d["col"], minlength=d["D"])
    np.add.at(cm, d["col"], d["val"])
    cm = np.where(cnt > 0, cm / np.maximum(cnt, 1), d["val"].mean())
    r_cm = orc.rmse(cm[d["test_col"]], d["test_val"])
    assert r < 0.35 * r_cm, (r, r_cm)
    assert r < 2.0 * d["sigma"], r
    # sign flips of latent columns leave predictions unchanged
    f = np.array([1, -1, 1, 1, -1, -1, 1, 1, 1, -1], float)
    np.testing.assert_allclose(orc.predict(d["test_row"], d["test_col"], Xm * f, Wm * f, p.offset),
                               yhat, rtol=1e-12, atol=1e-12)


def test_pp_run_matches_full_posterior_accuracy(orc):
    """A 2 x 2 grid run of Algorithm 1 on planted data predicts about as well as the plain
    sampler (the paper's finding that PP costs little accuracy, Section 5.4)."""
    d = synth.make_workload("planted-1000x500-k10", scale=0.3, M=8_000, K=4)
    K, T, B = 4, 40, 20
    prior = orc.NWPrior(K)
    p = orc.plan(d["N"], d["D"], d["row"], d["col"], d["val"], 2, 2)

    def draws_fn(stage, t):
        subs = p.stage_subsets(stage)
        return synth.sweep_draws([(s.n, s.d) for s in subs], K, prior.nu0,
                                 synth.rng_for(9, stage, t))

    res = orc.pp_run(p, K, d["tau"], prior, d["X0"][p.row_perm], d["W0"][p.col_perm], draws_fn,
                     T, B, 1)
    rr, cr = np.argsort(p.row_perm), np.argsort(p.col_perm)
    y_pp = orc.predict(d["test_row"], d["test_col"], res["Xm"][rr], res["Wm"][cr], p.offset)
    _, Xm, Wm = _run_plain(orc, d, K, T, B)
    y_full = orc.predict(d["test_row"], d["test_col"], Xm, Wm, p.offset)
    r_pp, r_full = orc.rmse(y_pp, d["test_val"]), orc.rmse(y_full, d["test_val"])
    assert r_pp < 1.25 * r_full + 0.05, (r_pp, r_full)
    # stage wiring: stage-2 subset (1,0) propagated W^(0) from (0,0) and starts there
    st = res["chains"][2]
    assert st.prior_w == 1 and st.prior_x == 0
    st3 = res["chains"][3]
    assert st3.prior_x == 1 and st3.prior_w == 1
