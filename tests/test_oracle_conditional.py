"""Pins of the oracle's row conditional (the Gibbs update of x_n given W, Eqs. 2-4) against
routes that do not share its formula: a least-squares solve for the mean, the Hessian of the
log-posterior assembled from scipy log-densities for the precision, and the sweep wiring."""
import numpy as np
import pytest
from scipy import stats

from paper_1703_00734_gb300 import synth


def _tiny(rng, R=5, Dp=7, K=3, fill=0.6):
    P = rng.standard_normal((Dp, K))
    mask = rng.random((R, Dp)) < fill
    mask[0, :] = False            # an empty row: prior-only draw
    mask[1, :] = True             # a full row
    Y = rng.standard_normal((R, Dp)) * 2.0
    ptr = np.concatenate([[0], np.cumsum(mask.sum(1))]).astype(np.int64)
    idx = np.concatenate([np.nonzero(mask[r])[0] for r in range(R)]).astype(np.int32)
    val = np.concatenate([Y[r, mask[r]] for r in range(R)])
    A = rng.standard_normal((K, K))
    Lam_p = A @ A.T + K * np.eye(K)
    mu_p = rng.standard_normal(K)
    return P, mask, Y, ptr, idx, val, Lam_p, mu_p


def test_mean_is_regularised_least_squares(orc):
    """z = 0 gives the posterior mean, the minimiser of
    tau |y - P_Omega x|^2 + (x - mu_p)^T Lambda_p (x - mu_p): solved here by lstsq on the
    stacked system [sqrt(tau) P_Omega; C^T] x = [sqrt(tau) y; C^T mu_p], Lambda_p = C C^T."""
    rng = np.random.default_rng(1)
    P, mask, Y, ptr, idx, val, Lam_p, mu_p = _tiny(rng)
    tau = 2.5
    R, K = mask.shape[0], P.shape[1]
    X = orc.update_rows(ptr, idx, val, P, tau, mu_p, Lam_p, np.zeros((R, K)))
    C = np.linalg.cholesky(Lam_p)
    for r in range(R):
        A = np.vstack([np.sqrt(tau) * P[mask[r]], C.T])
        b = np.concatenate([np.sqrt(tau) * Y[r, mask[r]], C.T @ mu_p])
        x_ls = np.linalg.lstsq(A, b, rcond=None)[0]
        np.testing.assert_allclose(X[r], x_ls, rtol=1e-12, atol=1e-12)


def _logpost(x, prow, yrow, tau, mu_p, Lam_p):
    """log p(y | x) + log p(x) from scipy densities (constants do not matter)."""
    lp = stats.multivariate_normal.logpdf(x, mean=mu_p, cov=np.linalg.inv(Lam_p))
    if len(yrow):
        lp += stats.norm.logpdf(yrow, loc=prow @ x, scale=1.0 / np.sqrt(tau)).sum()
    return lp


def _hessian(f, x0, h=1.0):
    K = len(x0)
    H = np.zeros((K, K))
    E = np.eye(K) * h
    for i in range(K):
        for j in range(K):
            H[i, j] = (f(x0 + E[i] + E[j]) - f(x0 + E[i] - E[j]) - f(x0 - E[i] + E[j])
                       + f(x0 - E[i] - E[j])) / (4 * h * h)
    return H


def test_draw_uses_precision_cholesky(orc):
    """x = mu + L^{-T} z with L L^T the conditional precision: the precision is read off the
    Hessian of the log-posterior (exact for a quadratic), L from numpy's Cholesky."""
    rng = np.random.default_rng(2)
    P, mask, Y, ptr, idx, val, Lam_p, mu_p = _tiny(rng)
    tau = 1.7
    R, K = mask.shape[0], P.shape[1]
    z = rng.standard_normal((R, K))
    Xmu = orc.update_rows(ptr, idx, val, P, tau, mu_p, Lam_p, np.zeros((R, K)))
    Xz = orc.update_rows(ptr, idx, val, P, tau, mu_p, Lam_p, z)
    for r in range(R):
        f = lambda x: _logpost(x, P[mask[r]], Y[r, mask[r]], tau, mu_p, Lam_p)
        Lam_r = -_hessian(f, Xmu[r])
        L = np.linalg.cholesky(0.5 * (Lam_r + Lam_r.T))
        np.testing.assert_allclose(L.T @ (Xz[r] - Xmu[r]), z[r], rtol=1e-7, atol=1e-7)
        # the mean is the mode: zero gradient of the log-posterior
        g = np.array([(f(Xmu[r] + e) - f(Xmu[r] - e)) / 2 for e in np.eye(K) * 1e-3])
        assert np.abs(g).max() < 1e-6


def test_per_row_prior_and_scalar_case(orc):
    """K = 1: the textbook conjugate normal update, precision lam + tau sum p^2 and mean
    (lam mu + tau sum y p) / precision; per-row priors are honoured."""
    rng = np.random.default_rng(3)
    R, Dp = 4, 6
    P = rng.standard_normal((Dp, 1))
    ptr = np.array([0, 0, 2, 5, 6], np.int64)
    idx = np.array([1, 4, 0, 2, 5, 3], np.int32)
    val = rng.standard_normal(6)
    mu_p = rng.standard_normal((R, 1))
    lam = (rng.random(R) + 0.5).reshape(R, 1, 1)
    z = rng.standard_normal((R, 1))
    X = orc.update_rows(ptr, idx, val, P, 0.8, mu_p, lam, z, per_row_prior=True)
    for r in range(R):
        p = P[idx[ptr[r]:ptr[r + 1]], 0]
        y = val[ptr[r]:ptr[r + 1]]
        prec = lam[r, 0, 0] + 0.8 * (p * p).sum()
        mean = (lam[r, 0, 0] * mu_p[r, 0] + 0.8 * (y * p).sum()) / prec
        assert X[r, 0] == pytest.approx(mean + z[r, 0] / np.sqrt(prec), rel=1e-13, abs=1e-14)


def test_sweep_wiring(orc):
    """A sweep is: hyperparameters of X from the old X, of W from the old W, then X given the
    old W, then W given the NEW X (Section 5.1 / BPMF order)."""
    data = synth.make_workload("planted-1000x500-k10", scale=0.03)
    K = 3
    p = orc.plan(data["N"], data["D"], data["row"], data["col"], data["val"], 1, 1)
    s = p.subsets[0]
    prior = orc.NWPrior(K)
    rng = np.random.default_rng(5)
    X0 = rng.standard_normal((s.n, K))
    W0 = rng.standard_normal((s.d, K))
    dr = synth.sweep_draws([(s.n, s.d)], K, prior.nu0, rng)
    lay = orc.stage_draw_layout([s], K)
    H = orc.hyper_block_len(K)
    st = orc.new_chain(X0, W0, K)
    orc.sweep_subset(s, st, K, 2.0, prior, dr[0:H], dr[H:2 * H],
                     dr[lay[(0, "zx")]:lay[(0, "zx")] + s.n * K],
                     dr[lay[(0, "zw")]:lay[(0, "zw")] + s.d * K])
    muX, LamX = orc.nw_draw(orc.nw_posterior(X0, prior), dr[0:H], K)
    muW, LamW = orc.nw_draw(orc.nw_posterior(W0, prior), dr[H:2 * H], K)
    zx = dr[lay[(0, "zx")]:lay[(0, "zx")] + s.n * K].reshape(s.n, K)
    zw = dr[lay[(0, "zw")]:lay[(0, "zw")] + s.d * K].reshape(s.d, K)
    X1 = orc.update_rows(s.rptr, s.ridx, s.rval, W0, 2.0, muX, LamX, zx)
    W1 = orc.update_rows(s.cptr, s.cidx, s.cval, X1, 2.0, muW, LamW, zw)
    np.testing.assert_array_equal(st.X, X1)
    np.testing.assert_array_equal(st.W, W1)
    np.testing.assert_array_equal(st.LamX, LamX)
    np.testing.assert_array_equal(st.muW, muW)
