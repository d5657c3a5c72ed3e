"""Pins of the oracle's masked log-joint and its gradient (the differentiation extension):
the value against scipy densities up to the normalising constants, the gradient against central
finite differences."""
import numpy as np
from scipy import stats


def _problem(rng, K=3, N=7, D=5, M=20):
    cells = rng.choice(N * D, M, replace=False)
    row, col = (cells // D).astype(np.int32), (cells % D).astype(np.int32)
    val = rng.standard_normal(M) * 2.0
    X, W = rng.standard_normal((N, K)), rng.standard_normal((D, K))
    A = rng.standard_normal((K, K))
    LamX = A @ A.T + np.eye(K)
    B = rng.standard_normal((K, K))
    LamW = B @ B.T + 0.5 * np.eye(K)
    return row, col, val, X, W, rng.standard_normal(K), LamX, rng.standard_normal(K), LamW


def test_value_is_the_log_joint_up_to_constants(orc):
    rng = np.random.default_rng(61)
    row, col, val, X, W, muX, LamX, muW, LamW = _problem(rng)
    N, K = X.shape
    D = W.shape[0]
    la = 0.4
    a = np.exp(la)
    _, _, _, v = orc.logjoint_grad(row, col, val, X, W, la, muX, LamX, muW, LamW)
    ref = stats.norm.logpdf(val, np.einsum("ij,ij->i", X[row], W[col]), 1 / np.sqrt(a)).sum()
    ref += stats.multivariate_normal.logpdf(X, muX, np.linalg.inv(LamX)).sum()
    ref += stats.multivariate_normal.logpdf(W, muW, np.linalg.inv(LamW)).sum()
    const = -0.5 * len(val) * np.log(2 * np.pi)
    const += N * (-0.5 * K * np.log(2 * np.pi) + 0.5 * np.linalg.slogdet(LamX)[1])
    const += D * (-0.5 * K * np.log(2 * np.pi) + 0.5 * np.linalg.slogdet(LamW)[1])
    assert abs(v + const - ref) < 1e-10 * max(1.0, abs(ref))


def test_gradient_matches_central_differences(orc):
    rng = np.random.default_rng(62)
    row, col, val, X, W, muX, LamX, muW, LamW = _problem(rng)
    la = -0.3
    gX, gW, ga, _ = orc.logjoint_grad(row, col, val, X, W, la, muX, LamX, muW, LamW)
    f = lambda X_, W_, la_: orc.logjoint_grad(row, col, val, X_, W_, la_, muX, LamX, muW, LamW)[3]
    h = 1e-6
    for (M, G, which) in ((X, gX, 0), (W, gW, 1)):
        for idx in np.ndindex(M.shape):
            P, Q = M.copy(), M.copy()
            P[idx] += h
            Q[idx] -= h
            fd = (f(P, W, la) - f(Q, W, la)) / (2 * h) if which == 0 else \
                (f(X, P, la) - f(X, Q, la)) / (2 * h)
            assert abs(fd - G[idx]) < 1e-6 * max(1.0, abs(G[idx])), (which, idx, fd, G[idx])
    fd = (f(X, W, la + h) - f(X, W, la - h)) / (2 * h)
    assert abs(fd - ga) < 1e-6 * max(1.0, abs(ga))
