"""GPU parity of the log-joint adjoint (bmf_logjoint_grad), the Langevin moves and the autograd
wrapper against the FP64 oracle, whose gradient is pinned by central finite differences
(test_oracle_adjoint.py).  The CUDA adjoint computes in FP32: gradients must agree with the
oracle to 1e-4 relative (per row, relative to the row's largest gradient entry), the scalar
parts to 1e-5 relative."""
import numpy as np
import pytest

import oracle
from paper_1703_00734_gb300 import synth

pytestmark = pytest.mark.gpu


def _setup(K, with_sweep=True, seed=70):
    torch = pytest.importorskip("torch")
    from paper_1703_00734_gb300 import bmf
    d = synth.make_workload(None, N=160, D=130, M=7000, pattern="zipf", K=K, sigma=0.3,
                            tau=1 / 0.09, seed=seed + K, s_row=1.1, s_col=1.1)
    m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], K, d["tau"], "fp32", X0=d["X0"],
                W0=d["W0"])
    p = oracle.plan(d["N"], d["D"], d["row"], d["col"], d["val"], 1, 1)
    s = p.subsets[0]
    rng = np.random.default_rng(seed)
    if with_sweep:
        dr = synth.sweep_draws([(s.n, s.d)], K, float(K), rng)
        m.sweep(0, 1, dr)
        _, _, hyp = m.get_state(0)
        prior = dict(muX=hyp["muX"], LamX=hyp["LamX"], muW=hyp["muW"], LamW=hyp["LamW"])
    else:
        # per-row priors installed on both factors
        def rows(n):
            A = rng.standard_normal((n, K, K)) * 0.3
            return rng.standard_normal((n, K)), A @ A.transpose(0, 2, 1) + np.eye(K)
        muX, LX = rows(s.n)
        muW, LW = rows(s.d)
        m.set_prior(0, bmf.FACTOR_X, muX, LX)
        m.set_prior(0, bmf.FACTOR_W, muW, LW)
        prior = dict(muXr=muX, LamXr=LX, muWr=muW, LamWr=LW)
    ld = (K + 3) // 4 * 4
    X = (rng.standard_normal((s.n, K)) * 0.7).astype(np.float32)
    W = (rng.standard_normal((s.d, K)) * 0.7).astype(np.float32)
    return torch, bmf, m, s, X, W, ld, prior


def _dev(torch, A, ld):
    out = torch.zeros((A.shape[0], ld), dtype=torch.float32, device="cuda")
    out[:, :A.shape[1]] = torch.from_numpy(A).cuda()
    return out


def _oracle_grad(s, X, W, la, prior):
    rows = np.repeat(np.arange(s.n), np.diff(s.rptr)).astype(np.int32)
    K = X.shape[1]
    X64, W64 = X.astype(np.float64), W.astype(np.float64)
    if "muX" in prior:
        return oracle.logjoint_grad(rows, s.ridx, s.rval, X64, W64, la, prior["muX"],
                                    prior["LamX"], prior["muW"], prior["LamW"])
    # per-row priors: gradient -L_n (x_n - mu_n); evaluate the data part with a zero-precision
    # shared prior and add the per-row prior part here
    Z = np.zeros((K, K))
    gX, gW, ga, v = oracle.logjoint_grad(rows, s.ridx, s.rval, X64, W64, la, np.zeros(K), Z,
                                         np.zeros(K), Z)
    dx = X64 - prior["muXr"]
    dw = W64 - prior["muWr"]
    gX = gX - np.einsum("nij,nj->ni", prior["LamXr"], dx)
    gW = gW - np.einsum("nij,nj->ni", prior["LamWr"], dw)
    v = v - 0.5 * np.einsum("ni,nij,nj->", dx, prior["LamXr"], dx) \
        - 0.5 * np.einsum("ni,nij,nj->", dw, prior["LamWr"], dw)
    return gX, gW, ga, v


def _const(s, prior):
    """The dropped terms: 1/2 sum mu^T L mu over rows."""
    if "muX" in prior:
        return 0.5 * (s.n * prior["muX"] @ prior["LamX"] @ prior["muX"]
                      + s.d * prior["muW"] @ prior["LamW"] @ prior["muW"])
    return 0.5 * (np.einsum("ni,nij,nj->", prior["muXr"], prior["LamXr"], prior["muXr"])
                  + np.einsum("ni,nij,nj->", prior["muWr"], prior["LamWr"], prior["muWr"]))


def _close_rows(g, ref, rel, what):
    scale = np.abs(ref).max(1, keepdims=True) + 1e-3 * np.abs(ref).max()
    err = (np.abs(g - ref) / scale).max()
    assert err < rel, f"{what}: worst relative error {err:.2e}"


@pytest.mark.parametrize("K,with_sweep", [(5, True), (16, True), (10, False), (20, True), (40, False),
                                           (64, False), (64, True)])
def test_logjoint_grad_matches_oracle(K, with_sweep):
    torch, bmf, m, s, X, W, ld, prior = _setup(K, with_sweep)
    la = np.log(1 / 0.09)
    dX, dW = _dev(torch, X, ld), _dev(torch, W, ld)
    gX, gW = torch.empty_like(dX), torch.empty_like(dW)
    v, ga = m.logjoint_grad(0, dX.data_ptr(), dW.data_ptr(), ld, la, gX.data_ptr(), gW.data_ptr())
    gXo, gWo, gao, vo = _oracle_grad(s, X, W, la, prior)
    _close_rows(gX.cpu().numpy()[:, :K], gXo, 1e-4, "grad X")
    _close_rows(gW.cpu().numpy()[:, :K], gWo, 1e-4, "grad W")
    assert np.all(gX.cpu().numpy()[:, K:] == 0)
    assert abs(ga - gao) <= 1e-5 * max(1.0, abs(gao))
    assert abs(v - (vo + _const(s, prior))) <= 1e-5 * max(1.0, abs(vo))
    m.close()


def test_autograd_function_returns_the_adjoint():
    torch, bmf, m, s, X, W, ld, prior = _setup(8)
    from paper_1703_00734_gb300.autograd import LogJoint
    dX = _dev(torch, X, ld).requires_grad_(True)
    dW = _dev(torch, W, ld).requires_grad_(True)
    la = torch.tensor(0.3, dtype=torch.float64, device="cuda", requires_grad=True)
    val = LogJoint.apply(m, 0, dX, dW, la)
    (2.0 * val).backward()
    gXo, gWo, gao, _ = _oracle_grad(s, X, W, 0.3, prior)
    _close_rows(dX.grad.cpu().numpy()[:, :8] / 2.0, gXo, 1e-4, "autograd X")
    _close_rows(dW.grad.cpu().numpy()[:, :8] / 2.0, gWo, 1e-4, "autograd W")
    assert abs(la.grad.item() / 2.0 - gao) <= 1e-5 * max(1.0, abs(gao))
    m.close()


def test_langevin_ula_and_mala_steps():
    torch, bmf, m, s, X, W, ld, prior = _setup(6)
    la, eps = np.log(1 / 0.09), 1e-4
    rng = np.random.default_rng(5)
    K = 6
    xi = rng.standard_normal((2, (s.n + s.d) * K)).astype(np.float32)
    dxi = torch.from_numpy(xi).cuda()
    # one unadjusted step
    dX, dW = _dev(torch, X, ld), _dev(torch, W, ld)
    acc, _ = m.langevin(0, 1, dX.data_ptr(), dW.data_ptr(), ld, la, eps, dxi.data_ptr())
    assert acc == 1
    gXo, gWo, _, v0 = _oracle_grad(s, X, W, la, prior)
    Xn = X + 0.5 * eps * gXo + np.sqrt(eps) * xi[0, :s.n * K].reshape(s.n, K)
    Wn = W + 0.5 * eps * gWo + np.sqrt(eps) * xi[0, s.n * K:].reshape(s.d, K)
    _close_rows(dX.cpu().numpy()[:, :K], Xn, 1e-5, "ULA X")
    _close_rows(dW.cpu().numpy()[:, :K], Wn, 1e-5, "ULA W")
    # MALA: the acceptance log-ratio from oracle quantities decides; uniforms far from it
    Xp, Wp = Xn.astype(np.float32), Wn.astype(np.float32)
    gXp, gWp, _, v1 = _oracle_grad(s, Xp, Wp, la, prior)
    back = ((X - Xp - 0.5 * eps * gXp) ** 2).sum() + ((W - Wp - 0.5 * eps * gWp) ** 2).sum()
    fwd = ((Xp - X - 0.5 * eps * gXo) ** 2).sum() + ((Wp - W - 0.5 * eps * gWo) ** 2).sum()
    logA = v1 - v0 - back / (2 * eps) + fwd / (2 * eps)
    cases = [(np.exp(min(logA, 0.0) - 1.0), 1)]          # log u < log A: accepted
    if logA < -0.01:                                          # log u > log A: rejected
        cases.append((min(1.0, np.exp(logA + 1.0)), 0))
    for u, expect in cases:
        dX, dW = _dev(torch, X, ld), _dev(torch, W, ld)
        acc, _ = m.langevin(0, 1, dX.data_ptr(), dW.data_ptr(), ld, la, eps, dxi.data_ptr(),
                            uniforms=[u])
        assert acc == expect, (u, logA)
        ref = (Xn, Wn) if expect else (X, W)
        _close_rows(dX.cpu().numpy()[:, :K], ref[0], 1e-5, "MALA X")
    m.close()
