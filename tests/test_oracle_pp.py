"""Pins of the oracle's moment matching (Section 4.1), aggregation (Eq. 14, Algorithm 2) and
stage wiring (Algorithm 1, Theorem 1)."""
import numpy as np
import pytest

from paper_1703_00734_gb300 import synth


def _spd(rng, K, scale=1.0):
    A = rng.standard_normal((K, K))
    return scale * (A @ A.T / K + 0.5 * np.eye(K))


def test_mm_finalize_is_sample_mean_and_inverse_ml_covariance(orc):
    rng = np.random.default_rng(21)
    K, R, S = 4, 6, 50
    samples = rng.standard_normal((S, R, K)) @ np.triu(np.ones((K, K))) + 2.0
    S1 = samples.sum(0)
    S2 = np.einsum("sri,srj->rij", samples, samples)
    mu, Lam = orc.mm_finalize(S1, S2, S)
    for r in range(R):
        np.testing.assert_allclose(mu[r], samples[:, r].mean(0), rtol=1e-13)
        cov = np.cov(samples[:, r].T, bias=True)
        np.testing.assert_allclose(Lam[r], np.linalg.inv(cov), rtol=1e-9)


def test_moments_accumulate(orc):
    rng = np.random.default_rng(22)
    st = orc.new_chain(rng.standard_normal((5, 3)), rng.standard_normal((4, 3)), 3)
    orc.accumulate(st)
    orc.accumulate(st)
    np.testing.assert_allclose(st.S1X, 2 * st.X)
    np.testing.assert_allclose(st.S2W, 2 * np.einsum("ri,rj->rij", st.W, st.W))
    assert st.n_kept == 2


def test_algorithm2_equals_eq14_when_differences_are_pd(orc):
    """Without corrections Algorithm 2 is Eq. 14:
    Lambda* = L1 + sum_j (Lj - L1),  mu* = Lambda*^{-1}(L1 m1 + sum_j (Lj mj - L1 m1))."""
    rng = np.random.default_rng(23)
    K, R, J = 5, 7, 4
    L1 = np.stack([_spd(rng, K) for _ in range(R)])
    Lam = [L1] + [L1 + np.stack([_spd(rng, K, 0.3) for _ in range(R)]) for _ in range(J - 1)]
    mu = rng.standard_normal((J, R, K))
    mus, Ls, nc = orc.aggregate(mu, np.stack(Lam))
    assert nc == 0
    for r in range(R):
        Lstar = L1[r] + sum(Lam[j][r] - L1[r] for j in range(1, J))
        h = L1[r] @ mu[0, r] + sum(Lam[j][r] @ mu[j, r] - L1[r] @ mu[0, r] for j in range(1, J))
        np.testing.assert_allclose(Ls[r], Lstar, rtol=1e-12)
        np.testing.assert_allclose(mus[r], np.linalg.solve(Lstar, h), rtol=1e-10)


def test_eigenvalue_correction(orc):
    """A non-PD difference Lj - L1 is shifted so that its smallest eigenvalue becomes eps
    (|lambda_min| + eps added to the diagonal); with J = 2, Lambda* = corrected + L1."""
    rng = np.random.default_rng(24)
    K = 4
    L1 = _spd(rng, K, 2.0)
    Q = np.linalg.qr(rng.standard_normal((K, K)))[0]
    diff = Q @ np.diag([0.7, 0.2, -0.15, 0.4]) @ Q.T
    Lam = np.stack([L1[None], (L1 + diff)[None]])
    mu = rng.standard_normal((2, 1, K))
    mus, Ls, nc = orc.aggregate(mu, Lam, eps_rel=1e-6)
    assert nc == 1
    eps = 1e-6 * max(1.0, np.trace(L1) / K)
    ev = np.linalg.eigvalsh(Ls[0] - L1)
    assert ev.min() == pytest.approx(eps, abs=1e-12)
    np.testing.assert_allclose(np.sort(ev), np.sort(np.linalg.eigvalsh(diff) + 0.15 + eps),
                               atol=1e-11)
    # mu* = Lambda*^{-1} (0 * L1 m1 + Lambda*^(2) m2) = m2 when J = 2
    np.testing.assert_allclose(mus[0], mu[1, 0], rtol=1e-10)


def test_min_eig_matches_lapack(orc):
    rng = np.random.default_rng(25)
    for K in (1, 2, 5, 16, 33):
        A = rng.standard_normal((K, K))
        A = A + A.T
        assert orc.min_eig(A) == pytest.approx(np.linalg.eigvalsh(A).min(), abs=1e-10)


def test_theorem1_gaussian_case_is_exact(orc):
    """W clamped: every subset posterior of x_n is exactly Gaussian.  Stage I on block (0,0),
    stage II on (0,j) with the stage-I posterior as prior, then Eq. 14 must reproduce the
    full-data conditional exactly (Theorem 1 restricted to X)."""
    rng = np.random.default_rng(26)
    K, N, D, J = 3, 9, 28, 4
    W = rng.standard_normal((D, K))
    mask = rng.random((N, D)) < 0.85   # every row sees >= K columns of every block: G_j PD
    Y = rng.standard_normal((N, D))
    tau = 1.3
    A = rng.standard_normal((K, K))
    Lp, mp = A @ A.T + np.eye(K), rng.standard_normal(K)
    cb = orc.equal_bounds(D, J)

    def block(c0, c1):
        m = mask[:, c0:c1]
        ptr = np.concatenate([[0], np.cumsum(m.sum(1))]).astype(np.int64)
        idx = np.concatenate([np.nonzero(m[n])[0] for n in range(N)]).astype(np.int32)
        val = np.concatenate([Y[n, c0:c1][m[n]] for n in range(N)])
        G = np.einsum("nd,di,dj->nij", m, W[c0:c1], W[c0:c1])
        return ptr, idx, val, G

    z0 = np.zeros((N, K))
    ptr, idx, val, G = block(cb[0], cb[1])
    m1 = orc.update_rows(ptr, idx, val, W[cb[0]:cb[1]], tau, mp, Lp, z0)
    L1 = Lp + tau * G
    mus, Lams = [m1], [L1]
    for j in range(1, J):
        ptr, idx, val, G = block(cb[j], cb[j + 1])
        mus.append(orc.update_rows(ptr, idx, val, W[cb[j]:cb[j + 1]], tau, m1, L1, z0,
                                   per_row_prior=True))
        Lams.append(L1 + tau * G)
    mstar, Lstar, nc = orc.aggregate(np.stack(mus), np.stack(Lams))
    assert nc == 0
    ptr, idx, val, G = block(0, D)
    full = orc.update_rows(ptr, idx, val, W, tau, mp, Lp, z0)
    np.testing.assert_allclose(mstar, full, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(Lstar, Lp + tau * G, rtol=1e-12)


def test_grid_plan(orc):
    """Every observation lands in exactly one subset; CSR and CSC are transposes; the
    decreasing order sorts counts with ties by index; stages follow Eqs. 10-12."""
    d = synth.make_workload("zipf-69878x10677-10M-k10", scale=0.01)
    p = orc.plan(d["N"], d["D"], d["row"], d["col"], d["val"], I=3, J=4)
    assert sum(s.nnz for s in p.subsets) == len(d["row"])
    rc = np.bincount(d["row"], minlength=d["N"])[p.row_perm]
    assert np.all(np.diff(rc) <= 0)
    ties = np.nonzero(np.diff(rc) == 0)[0]
    assert np.all(p.row_perm[ties] < p.row_perm[ties + 1])
    stages = {(s.i, s.j): s.stage for s in p.subsets}
    assert stages[(0, 0)] == 1 and stages[(0, 2)] == 2 and stages[(2, 0)] == 2
    assert stages[(1, 1)] == 3
    for s in p.subsets:
        rows = np.repeat(np.arange(s.n), np.diff(s.rptr))
        cols = np.repeat(np.arange(s.d), np.diff(s.cptr))
        a = set(zip(rows.tolist(), s.ridx.tolist(), s.rval.tolist()))
        b = set(zip(s.cidx.tolist(), cols.tolist(), s.cval.tolist()))
        assert a == b
    # values are centred by the training mean
    assert p.offset == pytest.approx(d["val"].mean())


def test_theorem1_with_singular_differences_stays_close(orc):
    """With one observation per row block the differences Lambda^(j) - Lambda^(1) = tau G_j
    are only semidefinite; Algorithm 2 then shifts them by |lambda_min| + eps, which moves the
    aggregate by O(eps) only."""
    rng = np.random.default_rng(27)
    K, N, J = 2, 5, 3
    D = J
    W = rng.standard_normal((D, K))
    Y = rng.standard_normal((N, D))
    tau = 2.0
    Lp, mp = np.eye(K), np.zeros(K)
    z0 = np.zeros((N, K))
    ptr1 = np.arange(N + 1, dtype=np.int64)
    zeros = np.zeros(N, np.int32)
    m1 = orc.update_rows(ptr1, zeros, Y[:, 0], W[0:1], tau, mp, Lp, z0)
    L1 = Lp + tau * np.outer(W[0], W[0])
    mus, Lams = [m1], [np.repeat(L1[None], N, 0)]
    for j in range(1, J):
        mus.append(orc.update_rows(ptr1, zeros, Y[:, j], W[j:j + 1], tau, m1,
                                   np.repeat(L1[None], N, 0), z0, per_row_prior=True))
        Lams.append(np.repeat((L1 + tau * np.outer(W[j], W[j]))[None], N, 0))
    mstar, _, nc = orc.aggregate(np.stack(mus), np.stack(Lams), eps_rel=1e-9)
    assert nc > 0
    full = orc.update_rows(np.arange(0, N * D + 1, D, dtype=np.int64),
                           np.tile(np.arange(D, dtype=np.int32), N), Y.ravel(), W, tau, mp, Lp,
                           z0)
    np.testing.assert_allclose(mstar, full, atol=1e-6)


def test_stage_sources_and_hyperparameter_rule(orc):
    """Algorithm 1's propagation sources and the stage-wise rule of Section 5.1: stage 2 (i,0)
    takes W^(0) from (0,0), (0,j) takes X^(0) from (0,0); stage 3 (i,j) takes X from (i,0) and
    W from (0,j); a propagated factor starts at the propagated mean and draws no
    hyperparameters, a non-propagated one draws them (its mu, Lambda move off the start)."""
    rng = np.random.default_rng(21)
    K, I, J = 2, 3, 3
    d = synth.make_workload(None, N=60, D=45, M=1500, pattern="uniform", K=K, sigma=0.5,
                            tau=4.0, seed=22)
    p = orc.plan(d["N"], d["D"], d["row"], d["col"], d["val"], I, J)
    # recognisable per-subset summaries: subset s has mean 10 s + 1 (X) and -(10 s + 1) (W)
    finals = {s.sid: (np.full((s.n, K), 10.0 * s.sid + 1), np.tile(np.eye(K), (s.n, 1, 1)),
                      np.full((s.d, K), -(10.0 * s.sid + 1)), np.tile(np.eye(K), (s.d, 1, 1)))
              for s in p.subsets}
    X0, W0 = d["X0"][p.row_perm], d["W0"][p.col_perm]
    prior = orc.NWPrior(K)
    for stage in (2, 3):
        chains = orc.setup_stage_chains(p, stage, X0, W0, K, finals)
        for s in p.stage_subsets(stage):
            st = chains[s.sid]
            if stage == 2:
                src_x = None if s.j == 0 else 0
                src_w = 0 if s.j == 0 else None
            else:
                src_x, src_w = s.i * J, s.j
            assert st.prior_x == (src_x is not None) and st.prior_w == (src_w is not None)
            if src_x is not None:
                np.testing.assert_array_equal(st.muX_row, finals[src_x][0])
                np.testing.assert_array_equal(st.X, finals[src_x][0])
            if src_w is not None:
                np.testing.assert_array_equal(st.muW_row, finals[src_w][2])
                np.testing.assert_array_equal(st.W, finals[src_w][2])
        subs = p.stage_subsets(stage)
        before = {sid: (st.muX.copy(), st.muW.copy()) for sid, st in chains.items()}
        dr = synth.sweep_draws([(s.n, s.d) for s in subs], K, prior.nu0, rng)
        orc.run_stage(p, stage, chains, K, d["tau"], prior, lambda t: dr, 1)
        for s in subs:
            st = chains[s.sid]
            mx0, mw0 = before[s.sid]
            assert np.array_equal(st.muX, mx0) == bool(st.prior_x)   # drawn iff not propagated
            assert np.array_equal(st.muW, mw0) == bool(st.prior_w)


def test_independent_subsets_are_standalone_chains(orc):
    """Without propagation (the embarrassingly parallel baseline of Sections 5.4 and 5.6) every
    subset's chain is the plain sampler on that subset's data alone: a 1 x 1 plan built from
    the block's entries, its own hyperparameter draws and z's taken from the stage's buffer,
    the initial state of the block."""
    K, I, J, T = 3, 3, 2, 4
    d = synth.make_workload(None, N=54, D=40, M=1300, pattern="uniform", K=K, sigma=0.5,
                            tau=4.0, seed=23)
    p = orc.plan(d["N"], d["D"], d["row"], d["col"], d["val"], I, J)
    prior = orc.NWPrior(K)
    X0, W0 = d["X0"][p.row_perm], d["W0"][p.col_perm]
    rrank, crank = np.argsort(p.row_perm), np.argsort(p.col_perm)
    nr, nc = rrank[d["row"]], crank[d["col"]]
    vc = d["val"] - p.offset
    H = orc.hyper_block_len(K)
    for stage in (1, 2, 3):
        subs = p.stage_subsets(stage)
        chains = orc.setup_stage_chains(p, stage, X0, W0, K, {}, propagate=False)
        rng = np.random.default_rng(100 + stage)
        bufs = [synth.sweep_draws([(s.n, s.d) for s in subs], K, prior.nu0, rng) for _ in range(T)]
        orc.run_stage(p, stage, chains, K, d["tau"], prior, lambda t: bufs[t], T)
        lay = orc.stage_draw_layout(subs, K)
        for s in subs:
            st = chains[s.sid]
            assert not st.prior_x and not st.prior_w
            m = (nr >= s.r0) & (nr < s.r1) & (nc >= s.c0) & (nc < s.c1)
            q = orc.plan(s.n, s.d, nr[m] - s.r0, nc[m] - s.c0, vc[m], 1, 1, order="none",
                         center=False)
            alone = orc.new_chain(X0[s.r0:s.r1], W0[s.c0:s.c1], K)
            for t in range(T):
                b = bufs[t]
                orc.sweep_subset(q.subsets[0], alone, K, d["tau"], prior,
                                 b[lay[(s.sid, "hx")]:lay[(s.sid, "hx")] + H],
                                 b[lay[(s.sid, "hw")]:lay[(s.sid, "hw")] + H],
                                 b[lay[(s.sid, "zx")]:lay[(s.sid, "zx")] + s.n * K],
                                 b[lay[(s.sid, "zw")]:lay[(s.sid, "zw")] + s.d * K])
            np.testing.assert_array_equal(st.X, alone.X)
            np.testing.assert_array_equal(st.W, alone.W)
            np.testing.assert_array_equal(st.LamX, alone.LamX)
