"""Pins of the oracle's dominant-mode (PP DM) and mixture (PP GMM) summaries (Section 4.1,
Section 5.1): lambda-means clustering, the per-row Gaussian fits, the pooled moments the
aggregation takes, and the responsibility choice of a mixture prior's component."""
import numpy as np
import pytest

import oracle
from paper_1703_00734_gb300 import synth

scipy_stats = pytest.importorskip("scipy.stats")


def _blobs(rng, sizes, centres, sd):
    x = np.concatenate([c + sd * rng.standard_normal((n, len(c))) for n, c in zip(sizes, centres)])
    truth = np.concatenate([np.full(n, g) for g, n in enumerate(sizes)])
    return x, truth


def test_lambda_means_recovers_separated_clusters():
    rng = np.random.default_rng(1)
    centres = [np.array([0.0, 0.0, 0.0]), np.array([8.0, 0.0, 0.0]), np.array([0.0, 8.0, 0.0])]
    x, truth = _blobs(rng, [40, 25, 15], centres, 0.3)
    perm = rng.permutation(len(x))
    x, truth = x[perm], truth[perm]
    assign, n = oracle.lambda_means(x, lam=9.0)
    assert n == 3
    # same partition up to relabelling
    pairs = {(a, t) for a, t in zip(assign, truth)}
    assert len(pairs) == 3
    for a, t in pairs:
        np.testing.assert_allclose(x[assign == a].mean(0), x[truth == t].mean(0), rtol=1e-12)


def test_lambda_means_limits_and_fixed_point():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((30, 4))
    a_big, n_big = oracle.lambda_means(x, lam=1e9)
    assert n_big == 1 and np.all(a_big == 0)
    a0, n0 = oracle.lambda_means(x, lam=0.0)
    assert n0 == 30 and len(set(a0.tolist())) == 30          # distinct points: one each
    # at convergence every point sits with its nearest centre (centres = cluster means), or
    # no centre is within lam of it
    for lam in (0.5, 2.0, 6.0):
        a, n = oracle.lambda_means(x, lam=lam, max_iter=1000)
        cen = np.stack([x[a == c].mean(0) for c in range(n)])
        d = ((x[:, None, :] - cen[None]) ** 2).sum(-1)
        nearest = d.argmin(1)
        ok = (nearest == a) | (d.min(1) > lam)
        assert ok.all()


def test_moment_matching_and_dominant_mode_fits():
    rng = np.random.default_rng(3)
    K, R = 3, 4
    # per row: 70% of the samples near +a, 30% near -a (the sign ambiguity of BMF)
    samples = np.zeros((100, R, K))
    groups = []
    for r in range(R):
        a = rng.standard_normal(K) * 2 + 3.0
        x, truth = _blobs(rng, [70, 30], [a, -a], 0.4)
        perm = rng.permutation(100)
        samples[:, r] = x[perm]
        groups.append(truth[perm])
    mm = oracle.fit_summaries(samples, "mm")
    dm = oracle.fit_summaries(samples, "dm", lam=16.0)
    for r in range(R):
        xs = samples[:, r]
        np.testing.assert_allclose(mm["mu"][r, 0], xs.mean(0), rtol=1e-12)
        np.testing.assert_allclose(mm["Lam"][r, 0], np.linalg.inv(np.cov(xs.T, bias=True)),
                                   rtol=1e-9)
        big = xs[groups[r] == 0]
        np.testing.assert_allclose(dm["mu"][r, 0], big.mean(0), rtol=1e-12)
        np.testing.assert_allclose(dm["Lam"][r, 0], np.linalg.inv(np.cov(big.T, bias=True)),
                                   rtol=1e-9)
        assert dm["pi"][r, 0] == 1.0


def test_mixture_weights_components_and_pooled_moments():
    """Top-3 modes with weights by size; the pooled moments of a mixture fitted to every
    sample are the plain mean and ML covariance of all samples (law of total covariance), so
    a pooled formula without the between-component term fails."""
    rng = np.random.default_rng(4)
    K = 2
    x, truth = _blobs(rng, [50, 30, 20], [np.zeros(K), np.array([9.0, 0]), np.array([0, 9.0])],
                      0.5)
    samples = x[rng.permutation(len(x))][:, None, :]
    g = oracle.fit_summaries(samples, "gmm", lam=16.0, C=3)
    np.testing.assert_allclose(np.sort(g["pi"][0])[::-1], [0.5, 0.3, 0.2], rtol=1e-14)
    xs = samples[:, 0]
    np.testing.assert_allclose(g["pooled_mu"][0], xs.mean(0), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(np.linalg.inv(g["pooled_Lam"][0]), np.cov(xs.T, bias=True),
                               rtol=1e-10)


def test_small_modes_are_skipped_and_dm_falls_back_to_moment_matching():
    rng = np.random.default_rng(5)
    K = 2
    x, _ = _blobs(rng, [60, 36, 2], [np.zeros(K), np.array([9.0, 0]), np.array([0, 9.0])], 0.5)
    s = x[rng.permutation(len(x))][:, None, :]
    g = oracle.fit_summaries(s, "gmm", lam=16.0, C=3)
    np.testing.assert_allclose(np.sort(g["pi"][0])[::-1], [60 / 96, 36 / 96, 0.0], rtol=1e-14)
    # every cluster below K + 1 samples: the dominant mode falls back to moment matching
    y = rng.standard_normal((6, 3)) * 10.0                    # six far-apart points, K = 3
    s2 = y[:, None, :]
    dm = oracle.fit_summaries(s2, "dm", lam=1e-3)
    mm = oracle.fit_summaries(s2, "mm")
    np.testing.assert_allclose(dm["mu"], mm["mu"], rtol=1e-14)
    np.testing.assert_allclose(dm["Lam"], mm["Lam"], rtol=1e-12)


def test_mixture_prior_component_choice_matches_scipy():
    """argmax_c log pi_c + log N(x; mu_c, Lam_c^{-1}), checked against scipy's densities."""
    rng = np.random.default_rng(6)
    K, R, C = 3, 200, 3
    pi = rng.dirichlet(np.ones(C), size=R)
    pi[::7, 2] = 0.0                                           # unused components
    pi /= pi.sum(1, keepdims=True)
    mu = rng.standard_normal((R, C, K)) * 2
    A = rng.standard_normal((R, C, K, K))
    Lam = A @ A.transpose(0, 1, 3, 2) + 0.5 * np.eye(K)
    X = rng.standard_normal((R, K)) * 2
    chosen, mu_r, Lam_r = oracle.mix_choose(dict(pi=pi, mu=mu, Lam=Lam), X)
    for r in range(R):
        scores = [np.log(pi[r, c]) + scipy_stats.multivariate_normal.logpdf(
                      X[r], mu[r, c], np.linalg.inv(Lam[r, c])) if pi[r, c] > 0 else -np.inf
                  for c in range(C)]
        assert chosen[r] == int(np.argmax(scores))
        np.testing.assert_array_equal(mu_r[r], mu[r, chosen[r]])
        np.testing.assert_array_equal(Lam_r[r], Lam[r, chosen[r]])


def _small_pp(summary, lam, T=40, burnin=20):
    d = synth.make_workload(None, N=90, D=70, M=3200, pattern="uniform", K=3, sigma=0.3,
                            tau=1 / 0.09, seed=8)
    K = d["K"]
    p = oracle.plan(d["N"], d["D"], d["row"], d["col"], d["val"], 2, 2)
    prior = oracle.NWPrior(K)

    def draws(stage, t):
        return synth.sweep_draws([(s.n, s.d) for s in p.stage_subsets(stage)], K, prior.nu0,
                                 synth.rng_for(30, stage, t))

    out = oracle.pp_run(p, K, d["tau"], prior, d["X0"][p.row_perm], d["W0"][p.col_perm], draws,
                        T, burnin, 1, summary=summary, lam=lam)
    inv_r, inv_c = np.argsort(p.row_perm), np.argsort(p.col_perm)
    yhat = oracle.predict(d["test_row"], d["test_col"], out["Xm"][inv_r], out["Wm"][inv_c],
                          p.offset)
    return out, oracle.rmse(yhat, d["test_val"])


def test_one_mode_reduces_dm_and_gmm_to_moment_matching():
    """With a penalty larger than any squared distance every row has one cluster: DM and GMM
    propagate and aggregate the moment-matched Gaussians (same draws, so the same chains up to
    rounding)."""
    mm, r_mm = _small_pp("mm", 0.0)
    for summary in ("dm", "gmm"):
        out, r = _small_pp(summary, 1e12)
        np.testing.assert_allclose(out["Xm"], mm["Xm"], rtol=1e-7, atol=1e-9)
        np.testing.assert_allclose(out["Wm"], mm["Wm"], rtol=1e-7, atol=1e-9)
        assert abs(r - r_mm) < 1e-8


def test_dm_and_gmm_predict_like_moment_matching():
    _, r_mm = _small_pp("mm", 0.0)
    for summary in ("dm", "gmm"):
        _, r = _small_pp(summary, 0.05)
        assert np.isfinite(r) and abs(r - r_mm) < 0.03, (summary, r, r_mm)
