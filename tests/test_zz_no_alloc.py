"""bmf_aggregate_static, the aggregation entry point that allocates nothing (for callers that
cannot let a library call cudaMalloc, such as a runtime that owns all device memory through its
own pool allocator, or a service whose device footprint is fixed at start-up).

It must give the same posterior means as the context's own aggregation (bmf_posterior_means) on
the same moment-matched subset posteriors, on two calls in a row (the second call finds the
previous call's data in the shared static array), at K = 4 and at K = 16 (where the kernel's
shared memory exceeds 48 KiB); with one submodel it returns the submodel's mean; and on inputs
built so that the eigenvalue correction of Algorithm 2 runs, it matches the oracle's Eq. 14 /
Algorithm 2 with the same number of corrected pairs.  This file is collected last."""
import numpy as np
import pytest

import oracle
from paper_1703_00734_gb300 import synth
from pairing import assert_rows_close

pytestmark = pytest.mark.gpu


def _posteriors(m, sids, factor):
    mus, lams = [], []
    for s in sids:
        mu, lam = m.get_posterior(s, factor)
        mus.append(mu)
        lams.append(lam)
    return np.stack(mus), np.stack(lams)


def _aggregate_static(bmf, torch, mu, lam, eps_rel):
    J, R, K = mu.shape
    dmu = torch.from_numpy(np.ascontiguousarray(mu)).cuda()
    dlam = torch.from_numpy(np.ascontiguousarray(lam)).cuda()
    out = torch.full((R, K), float("nan"), dtype=torch.float64, device="cuda")
    nc = bmf.aggregate_static(K, R, J, dmu.data_ptr(), dlam.data_ptr(), out.data_ptr(), eps_rel,
                              torch.cuda.current_stream().cuda_stream)
    return out.cpu().numpy(), nc


@pytest.mark.parametrize("K,I,J,T,burnin", [(4, 2, 3, 14, 4), (16, 2, 2, 30, 6)])
def test_static_aggregation_matches_context_aggregation_twice(K, I, J, T, burnin):
    torch = pytest.importorskip("torch")
    from paper_1703_00734_gb300 import bmf
    eps = 1e-6
    d = synth.make_workload(None, N=180, D=150, M=9000, pattern="uniform", K=K, sigma=0.5,
                            tau=4.0, seed=31 + K)
    m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], K, d["tau"], "fp64", I=I, J=J,
                X0=d["X0"], W0=d["W0"], burnin=burnin, eps_rel=eps)
    nu0 = float(K)
    for stage in (1, 2, 3):
        per = m.draws_per_sweep(stage)
        sizes = []
        for s in range(I * J):
            info = m.subset_info(s)
            if info["stage"] == stage:
                sizes.append((info["row1"] - info["row0"], info["col1"] - info["col0"]))
        dr = np.concatenate([synth.sweep_draws(sizes, K, nu0, synth.rng_for(7, stage, t))
                             for t in range(T)])
        assert dr.size == per * T
        m.stage(stage, T, dr)
    Xm, Wm, nc_ctx = m.posterior_means()
    rp, cp = m.perm()
    for call in range(2):
        nc_total = 0
        for i in range(I):
            info = m.subset_info(i * J)
            mu, lam = _posteriors(m, [i * J + j for j in range(J)], bmf.FACTOR_X)
            out, nc = _aggregate_static(bmf, torch, mu, lam, eps)
            nc_total += nc
            assert_rows_close(out, Xm[rp[info["row0"]:info["row1"]]], 1e-9,
                              f"call {call}: X block {i}")
        for j in range(J):
            info = m.subset_info(j)
            mu, lam = _posteriors(m, [i * J + j for i in range(I)], bmf.FACTOR_W)
            out, nc = _aggregate_static(bmf, torch, mu, lam, eps)
            nc_total += nc
            assert_rows_close(out, Wm[cp[info["col0"]:info["col1"]]], 1e-9,
                              f"call {call}: W block {j}")
        assert nc_total == nc_ctx
    m.close()


def _submodels(R, J, K, seed):
    """J per-row Gaussians whose differences Lambda^(j) - Lambda^(1) are indefinite in most
    rows (a random symmetric perturbation), every Lambda^(j) itself positive definite."""
    rng = np.random.default_rng(seed)
    mu = rng.standard_normal((J, R, K))
    A = rng.standard_normal((R, K, K))
    L1 = A @ A.transpose(0, 2, 1) / K + np.eye(K)
    lam = [L1]
    for _ in range(1, J):
        B = rng.standard_normal((R, K, K))
        Lj = L1 + 0.3 * (B + B.transpose(0, 2, 1)) / 2
        lo = np.linalg.eigvalsh(Lj)[:, 0]
        Lj = Lj + np.maximum(0.1 - lo, 0.0)[:, None, None] * np.eye(K)
        lam.append(Lj)
    return mu, np.stack(lam)


@pytest.mark.parametrize("K,J", [(4, 3), (16, 2), (16, 4)])
def test_static_aggregation_with_corrections_matches_the_oracle_twice(K, J):
    torch = pytest.importorskip("torch")
    from paper_1703_00734_gb300 import bmf
    R, eps = 300, 1e-6
    mu, lam = _submodels(R, J, K, seed=100 + K + J)
    want, _, nc_o = oracle.aggregate(mu, lam, eps)
    assert nc_o > R // 2
    for call in range(2):
        out, nc = _aggregate_static(bmf, torch, mu, lam, eps)
        assert nc == nc_o, (call, nc, nc_o)
        assert_rows_close(out, want, 1e-9, f"call {call}")


def test_static_aggregation_of_one_submodel_returns_its_mean():
    """J = 1: Lambda* = (2 - 1) Lambda^(1), so mu* = mu^(1)."""
    torch = pytest.importorskip("torch")
    from paper_1703_00734_gb300 import bmf
    mu, lam = _submodels(250, 1, 16, seed=7)
    for call in range(2):
        out, nc = _aggregate_static(bmf, torch, mu, lam, 1e-6)
        assert nc == 0
        assert_rows_close(out, mu[0], 1e-9, f"call {call}")


def test_static_aggregation_rejects_sizes_beyond_its_array():
    from paper_1703_00734_gb300 import bmf
    L = bmf.load()
    with pytest.raises(bmf.BmfError) as e:
        bmf.aggregate_static(16, 20000, 2, None, None, None)
    assert e.value.status == 2
    assert b"exceeds the static scratch" in L.bmf_last_error(None)
