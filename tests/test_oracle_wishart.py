"""Pins of the oracle's Normal-Wishart hyperparameter step (Section 5.1 and its footnote)."""
import numpy as np

from paper_1703_00734_gb300 import synth


def _prior(orc, K, rng):
    A = rng.standard_normal((K, K))
    return orc.NWPrior(K, mu0=rng.standard_normal(K), beta0=1.7, nu0=K + 2.5,
                       W0=A @ A.T / K + np.eye(K))


def test_three_equivalent_forms_of_the_scale_update(orc):
    """The footnote gives two alternatives to the corrected (centred) update, both written with
    the uncentred S = (1/N) sum x x^T:
      W0^{-1} + N S + (b0 N/(b0+N)) (mu0 - xbar)(mu0 - xbar)^T - N xbar xbar^T
      W0^{-1} + N S + b0 mu0 mu0^T - b* mu* mu*^T.
    All three must agree; an oracle using the uncentred S in the first form fails."""
    rng = np.random.default_rng(11)
    for K, N in [(1, 5), (3, 40), (6, 200)]:
        pr = _prior(orc, K, rng)
        X = rng.standard_normal((N, K)) * 1.3 + rng.standard_normal(K) * 2.0
        post = orc.nw_posterior(X, pr)
        W0i = np.linalg.inv(pr.W0)
        xbar = X.mean(0)
        S_unc = X.T @ X / N
        b0 = pr.beta0
        form2 = W0i + N * S_unc + (b0 * N / (b0 + N)) * np.outer(pr.mu0 - xbar, pr.mu0 - xbar) \
            - N * np.outer(xbar, xbar)
        mus = post["mu_star"]
        form3 = W0i + N * S_unc + b0 * np.outer(pr.mu0, pr.mu0) - (b0 + N) * np.outer(mus, mus)
        scale = np.abs(post["Wstar_inv"]).max()
        np.testing.assert_allclose(post["Wstar_inv"], form2, atol=1e-11 * scale)
        np.testing.assert_allclose(post["Wstar_inv"], form3, atol=1e-11 * scale)
        assert post["beta_star"] == b0 + N and post["nu_star"] == pr.nu0 + N


def test_posterior_mean_minimises_regularised_squares(orc):
    """mu* minimises b0 |mu - mu0|^2 + sum_i |x_i - mu|^2 (the Gaussian part of the conjugate
    update); solved by lstsq on the stacked system."""
    rng = np.random.default_rng(12)
    K, N = 4, 25
    pr = _prior(orc, K, rng)
    X = rng.standard_normal((N, K)) + 3.0
    post = orc.nw_posterior(X, pr)
    A = np.vstack([np.sqrt(pr.beta0) * np.eye(K)] + [np.eye(K)] * N)
    b = np.concatenate([np.sqrt(pr.beta0) * pr.mu0] + list(X))
    np.testing.assert_allclose(post["mu_star"], np.linalg.lstsq(A, b, rcond=None)[0],
                               rtol=1e-12, atol=1e-12)


def test_empty_factor_keeps_the_prior(orc):
    rng = np.random.default_rng(13)
    K = 3
    pr = _prior(orc, K, rng)
    post = orc.nw_posterior(np.zeros((0, K)), pr)
    np.testing.assert_allclose(post["Wstar_inv"], np.linalg.inv(pr.W0), rtol=1e-12)
    np.testing.assert_allclose(post["mu_star"], pr.mu0, rtol=1e-14)


def test_bartlett_convention(orc):
    """Lambda = (L A)(L A)^T with L = chol(W*) (lower) and A the Bartlett factor built from the
    draw block; mu = mu* + chol(beta* Lambda)^{-T} z_mu."""
    rng = np.random.default_rng(14)
    K = 4
    pr = _prior(orc, K, rng)
    post = orc.nw_posterior(rng.standard_normal((30, K)), pr)
    h = synth.hyper_block(K, post["nu_star"], rng)
    mu, Lam = orc.nw_draw(post, h, K)
    L = np.linalg.cholesky(np.linalg.inv(post["Wstar_inv"]))
    A = np.zeros((K, K))
    A[np.diag_indices(K)] = np.sqrt(h[:K])
    A[np.tril_indices(K, -1)] = h[K:K + K * (K - 1) // 2]   # row-major below diagonal
    B = L @ A
    np.testing.assert_allclose(Lam, B @ B.T, rtol=1e-11)
    Lp = np.linalg.cholesky(post["beta_star"] * Lam)
    np.testing.assert_allclose(Lp.T @ (mu - post["mu_star"]), h[-K:], rtol=1e-9, atol=1e-10)


def test_wishart_and_mean_moments(orc):
    """Monte Carlo: E[Lambda] = nu* W*, Var(Lambda_ij) = nu* (W*_ij^2 + W*_ii W*_jj),
    E[mu] = mu*, Cov(mu) = (W*)^{-1} / (beta* (nu* - K - 1)) (textbook Normal-Wishart)."""
    rng = np.random.default_rng(15)
    K = 3
    pr = orc.NWPrior(K, mu0=np.array([0.5, -1.0, 2.0]), beta0=3.0, nu0=4.0,
                     W0=np.array([[1.0, 0.3, 0.0], [0.3, 0.8, -0.2], [0.0, -0.2, 0.5]]))
    post = orc.nw_posterior(rng.standard_normal((6, K)), pr)
    nu, bs = post["nu_star"], post["beta_star"]
    Ws = np.linalg.inv(post["Wstar_inv"])
    S = 40000
    Lams = np.empty((S, K, K))
    mus = np.empty((S, K))
    for s in range(S):
        mus[s], Lams[s] = orc.nw_draw(post, synth.hyper_block(K, nu, rng), K)
    mean = Lams.mean(0)
    var = nu * (Ws ** 2 + np.outer(np.diag(Ws), np.diag(Ws)))
    se = np.sqrt(var / S)
    assert np.all(np.abs(mean - nu * Ws) < 5 * se), (mean, nu * Ws)
    np.testing.assert_allclose(Lams.var(0), var, rtol=0.08)
    cov_mu = post["Wstar_inv"] / (bs * (nu - K - 1))
    assert np.all(np.abs(mus.mean(0) - post["mu_star"]) < 5 * np.sqrt(np.diag(cov_mu) / S))
    np.testing.assert_allclose(np.cov(mus.T), cov_mu, rtol=0.1, atol=0.05 * np.abs(cov_mu).max())


def test_factor_identities_of_the_kernel_route(orc):
    """The CUDA hyperparameter step reaches the oracle's factors by another route (equal up to
    rounding): with P the order reversal and P [W*]^{-1} P = R R^T (R lower), the lower Cholesky
    factor of W* = ([W*]^{-1})^{-1} is P R^{-T} P; and since L A is lower with a positive
    diagonal, chol(beta* Lambda) = sqrt(beta*) L A.  Checked against the oracle's explicit
    inverse-then-factor route and its draw of (mu, Lambda)."""
    rng = np.random.default_rng(15)
    for K, N in [(1, 7), (4, 30), (10, 200), (16, 500)]:
        pr = _prior(orc, K, rng)
        post = orc.nw_posterior(rng.standard_normal((N, K)) * 0.8 + 1.0, pr)
        C = post["Wstar_inv"]
        Pm = np.eye(K)[::-1]
        R = np.linalg.cholesky(Pm @ C @ Pm)
        L_route = Pm @ np.linalg.inv(R).T @ Pm
        L_oracle = np.linalg.cholesky(np.linalg.inv(C))
        assert np.allclose(np.triu(L_route, 1), 0.0)
        np.testing.assert_allclose(L_route, L_oracle, rtol=1e-10, atol=1e-12 * np.abs(L_oracle).max())
        h = synth.hyper_block(K, post["nu_star"], rng)
        mu, Lam = orc.nw_draw(post, h, K)
        A = np.zeros((K, K))
        A[np.diag_indices(K)] = np.sqrt(h[:K])
        A[np.tril_indices(K, -1)] = h[K:K + K * (K - 1) // 2]
        LA = L_route @ A
        np.testing.assert_allclose(LA @ LA.T, Lam, rtol=1e-9, atol=1e-12 * np.abs(Lam).max())
        np.testing.assert_allclose(np.sqrt(post["beta_star"]) * LA,
                                   np.linalg.cholesky(post["beta_star"] * Lam), rtol=1e-8,
                                   atol=1e-10 * np.sqrt(post["beta_star"]) * np.abs(LA).max())
        # mu = mu* + (L A)^{-T} z_mu / sqrt(beta*), the kernel's form
        v = np.linalg.solve(LA.T, h[-K:]) / np.sqrt(post["beta_star"])
        np.testing.assert_allclose(post["mu_star"] + v, mu, rtol=1e-8, atol=1e-10)
