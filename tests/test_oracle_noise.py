"""Pins of the oracle's sampled noise precision (Section 2.1: one precision per column, tau_d, or
one per chain, with conjugate Gamma priors): the Gamma update against scipy's Gamma law, the
per-column precisions in the row and column conditionals against weighted least squares, the
generator's chi-square variates against their law, and recovery of planted per-column noise."""
import numpy as np
import pytest

import oracle
from paper_1703_00734_gb300 import synth

stats = pytest.importorskip("scipy.stats")


def _column_block(rng, D, K, n_per):
    """A CSC block of D columns with n_per[d] entries each, its X, W and values."""
    N = 40
    X = rng.standard_normal((N, K))
    W = rng.standard_normal((D, K))
    cptr = np.concatenate([[0], np.cumsum(n_per)]).astype(np.int64)
    cidx = np.concatenate([rng.choice(N, n, replace=False) for n in n_per]).astype(np.int32)
    cval = rng.standard_normal(len(cidx)) * 2.0
    return X, W, cptr, cidx, cval


def test_gamma_update_matches_scipy():
    """tau_d = c / (2 b0 + SSE_d) with c ~ chi^2(2 a0 + n_d) is Gamma(a0 + n_d/2, rate
    b0 + SSE_d/2): at the chi-square quantile q the update equals scipy's Gamma quantile q."""
    rng = np.random.default_rng(1)
    K, a0, b0 = 3, 1.5, 0.7
    n_per = [5, 1, 9, 3]
    X, W, cptr, cidx, cval = _column_block(rng, len(n_per), K, n_per)
    sse = np.array([np.sum((cval[cptr[d]:cptr[d + 1]] - X[cidx[cptr[d]:cptr[d + 1]]] @ W[d]) ** 2)
                    for d in range(len(n_per))])
    for q in (0.05, 0.5, 0.93):
        c = stats.chi2.ppf(q, 2 * a0 + np.array(n_per))
        tau = oracle.noise_update(cptr, cidx, cval, X, W, "column", a0, b0, c)
        want = stats.gamma.ppf(q, a0 + np.array(n_per) / 2, scale=1 / (b0 + sse / 2))
        np.testing.assert_allclose(tau, want, rtol=1e-9)
        # one precision: shape a0 + |Omega|/2, rate b0 + SSE/2 over every column
        cg = stats.chi2.ppf(q, 2 * a0 + sum(n_per))
        tg = oracle.noise_update(cptr, cidx, cval, X, W, "global", a0, b0, [cg])
        wg = stats.gamma.ppf(q, a0 + sum(n_per) / 2, scale=1 / (b0 + sse.sum() / 2))
        np.testing.assert_allclose(tg, np.full(len(n_per), wg), rtol=1e-9)


def test_per_column_precisions_weight_the_conditionals():
    """With z = 0 a row's draw is its posterior mean, the minimiser of
    sum_d tau_d (y_d - x^T w_d)^2 + (x - mu)^T Lambda (x - mu): weighted least squares."""
    rng = np.random.default_rng(2)
    K, D = 4, 12
    W = rng.standard_normal((D, K))
    tau = rng.uniform(0.2, 5.0, D)
    mu = rng.standard_normal(K)
    A = rng.standard_normal((K, K))
    Lam = A @ A.T + np.eye(K)
    cols = np.sort(rng.choice(D, 8, replace=False))
    y = rng.standard_normal(8)
    ptr = np.array([0, 8], np.int64)
    x = oracle.update_rows(ptr, cols.astype(np.int32), y, W, 99.0, mu, Lam, np.zeros((1, K)),
                           tau_partner=tau)[0]
    Lc = np.linalg.cholesky(Lam)
    Amat = np.vstack([np.sqrt(tau[cols])[:, None] * W[cols], Lc.T])
    bvec = np.concatenate([np.sqrt(tau[cols]) * y, Lc.T @ mu])
    np.testing.assert_allclose(x, np.linalg.lstsq(Amat, bvec, rcond=None)[0], rtol=1e-10)
    # column side: every entry of row r has that row's precision
    xr = oracle.update_rows(ptr, cols.astype(np.int32), y, W, 99.0, mu, Lam, np.zeros((1, K)),
                            tau_row=np.array([tau[3]]))[0]
    Amat = np.vstack([np.sqrt(tau[3]) * W[cols], Lc.T])
    bvec = np.concatenate([np.sqrt(tau[3]) * y, Lc.T @ mu])
    np.testing.assert_allclose(xr, np.linalg.lstsq(Amat, bvec, rcond=None)[0], rtol=1e-10)


def test_generated_noise_variates_follow_their_chi_square_laws():
    dof = np.array([2.0 * 1.5 + 4, 2.0 * 1.5 + 40, 2.0 * 1.5 + 400])
    v = np.stack([oracle.gen_noise(7, t, 3, dof) for t in range(1, 3001)])
    for k, nu in enumerate(dof):
        assert stats.kstest(v[:, k], stats.chi2(nu).cdf).pvalue > 1e-3
    # a different subset, sweep or seed gives different numbers
    assert not np.array_equal(oracle.gen_noise(7, 1, 3, dof), oracle.gen_noise(7, 1, 4, dof))
    assert not np.array_equal(oracle.gen_noise(7, 1, 3, dof), oracle.gen_noise(8, 1, 3, dof))


def test_planted_per_column_noise_is_recovered():
    """Columns with noise sd 0.25 and 1.0: the sampled tau_d settle near 16 and 1."""
    rng = np.random.default_rng(4)
    N, D, K = 300, 40, 2
    Xt, Wt = rng.standard_normal((N, K)), rng.standard_normal((D, K))
    sd = np.where(np.arange(D) < D // 2, 0.25, 1.0)
    keys = rng.choice(N * D, 6000, replace=False)
    row, col = (keys // D).astype(np.int32), (keys % D).astype(np.int32)
    val = np.einsum("ij,ij->i", Xt[row], Wt[col]) + sd[col] * rng.standard_normal(len(row))
    p = oracle.plan(N, D, row, col, val, 1, 1, order="none", center=False)
    s = p.subsets[0]
    prior = oracle.NWPrior(K)
    noise = oracle.NoiseModel("column", 1.0, 1.0, 1.0)
    st = oracle.new_chain(0.1 * rng.standard_normal((N, K)), 0.1 * rng.standard_normal((D, K)), K)
    lay = oracle.stage_draw_layout([s], K, noise)
    H = oracle.hyper_block_len(K)
    taus = []
    for t in range(1, 301):
        dr = oracle.gen_batch_draws([s], K, prior.nu0, 5, t, noise)
        oracle.sweep_subset(s, st, K, 1.0, prior, dr[0:H], dr[H:2 * H],
                            dr[lay[(0, "zx")]:lay[(0, "zx")] + N * K],
                            dr[lay[(0, "zw")]:lay[(0, "zw")] + D * K], noise,
                            dr[lay[(0, "nz")]:lay[(0, "nz")] + D])
        if t > 100:
            taus.append(st.tau_col.copy())
    tm = np.mean(taus, 0)
    assert 8.0 < np.median(tm[: D // 2]) < 32.0
    assert 0.5 < np.median(tm[D // 2:]) < 2.0
