"""GPU parity of the dominant-mode (PP DM) and mixture (PP GMM) summaries (Section 4.1, Section
5.1) against the oracle: the context-free fits (bmf_fit_summaries) with lambda-means cluster
assignments bit-identical and the fitted Gaussians at 1e-9, and three-stage PP runs with each
summary (propagated dominant modes; propagated mixtures with the per-draw component choice;
pooled moments in the aggregation) per state at 1e-7, on the same draws."""
import numpy as np
import pytest

import oracle
from paper_1703_00734_gb300 import synth
from pairing import assert_rows_close

pytestmark = pytest.mark.gpu


def _multimodal(rng, R, S, K, spread):
    """R rows of S samples in R^K from two or three well separated blobs of random sizes."""
    x = np.zeros((S, R, K))
    for r in range(R):
        ncl = 2 + r % 2
        sizes = rng.multinomial(S, rng.dirichlet(np.ones(ncl) * 2))
        centres = rng.standard_normal((ncl, K)) * spread
        pts = np.concatenate([c + 0.3 * rng.standard_normal((n, K)) for n, c in zip(sizes, centres)])
        x[:, r] = pts[rng.permutation(S)]
    return x


@pytest.mark.parametrize("K,S,R", [(3, 100, 60), (16, 37, 40), (16, 120, 24), (32, 64, 12)])
@pytest.mark.parametrize("mode,lam", [("mm", 1.0), ("dm", 4.0), ("gmm", 4.0), ("gmm", 0.5)])
def test_fit_summaries_match_the_oracle(K, S, R, mode, lam):
    torch = pytest.importorskip("torch")
    from paper_1703_00734_gb300 import bmf
    rng = np.random.default_rng(K * 1000 + S)
    x = _multimodal(rng, R, S, K, spread=3.0)
    got = bmf.fit_summaries(torch.from_numpy(x).cuda(), mode, lam, C=3)
    want = oracle.fit_summaries(x, mode, lam=lam, C=3)
    g = {k: v.cpu().numpy() for k, v in got.items()}
    if mode != "mm":
        for r in range(R):
            a, _ = oracle.lambda_means(x[:, r], lam)
            np.testing.assert_array_equal(g["assign"][r], a, err_msg=f"row {r}")
    np.testing.assert_array_equal(g["pi"], want["pi"])
    C = want["pi"].shape[1]
    assert_rows_close(g["mu"].reshape(R * C, K), want["mu"].reshape(R * C, K), 1e-9, "mu")
    assert_rows_close(g["Lam"].reshape(R * C, K * K), want["Lam"].reshape(R * C, K * K), 1e-9, "Lam")
    assert_rows_close(g["pooled_mu"], want["pooled_mu"], 1e-9, "pooled mu")
    assert_rows_close(g["pooled_Lam"].reshape(R, K * K), want["pooled_Lam"].reshape(R, K * K), 1e-9,
                      "pooled Lambda")


def test_fit_summaries_reject_bad_shapes():
    torch = pytest.importorskip("torch")
    from paper_1703_00734_gb300 import bmf
    x = torch.zeros((300, 2, 32), dtype=torch.float64, device="cuda")
    with pytest.raises(bmf.BmfError) as e:
        bmf.fit_summaries(x, "gmm", 1.0)                      # S * K > 8192
    assert e.value.status == 2


@pytest.mark.parametrize("summary,lam", [("dm", 0.05), ("gmm", 0.05), ("gmm", 1e12)])
def test_pp_with_dm_and_gmm_summaries_matches_the_oracle(summary, lam):
    from paper_1703_00734_gb300 import bmf
    d = synth.make_workload(None, N=90, D=70, M=3200, pattern="uniform", K=3, sigma=0.3,
                            tau=1 / 0.09, seed=8)
    K, T, B, C = d["K"], 40, 20, 3
    p = oracle.plan(d["N"], d["D"], d["row"], d["col"], d["val"], 2, 2)
    prior = oracle.NWPrior(K)

    def draws(stage, t):
        return synth.sweep_draws([(s.n, s.d) for s in p.stage_subsets(stage)], K, prior.nu0,
                                 synth.rng_for(30, stage, t))

    m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], K, d["tau"], "fp64", I=2, J=2,
                X0=d["X0"], W0=d["W0"], burnin=B, summary=summary, lam=lam, components=C,
                max_samples=T - B)
    X0, W0 = d["X0"][p.row_perm], d["W0"][p.col_perm]
    finals = {}
    n_mix = 0
    for stage in (1, 2, 3):
        chains = oracle.setup_stage_chains(p, stage, X0, W0, K, finals, summary)
        oracle.run_stage(p, stage, chains, K, d["tau"], prior, lambda t: draws(stage, t), T, B, 1)
        m.stage(stage, T, np.concatenate([draws(stage, t) for t in range(T)]))
        for s in p.stage_subsets(stage):
            X, W, _ = m.get_state(s.sid)
            assert_rows_close(X, chains[s.sid].X, 1e-7, f"{summary}: X of subset {s.sid}")
            assert_rows_close(W, chains[s.sid].W, 1e-7, f"{summary}: W of subset {s.sid}")
            finals[s.sid] = oracle.finalize(chains[s.sid], summary, lam, C)
            n_mix += int(chains[s.sid].mixX is not None) + int(chains[s.sid].mixW is not None)
            for f in (0, 1):
                mu, Lam = m.get_posterior(s.sid, f)
                assert_rows_close(mu, finals[s.sid][2 * f], 1e-7, f"{summary}: summary mean {s.sid}/{f}")
                assert_rows_close(Lam.reshape(len(Lam), -1),
                                  finals[s.sid][2 * f + 1].reshape(len(Lam), -1), 1e-7,
                                  f"{summary}: summary precision {s.sid}/{f}")
    if summary == "gmm":
        assert n_mix > 0           # stages 2 and 3 ran with propagated mixtures
    Xo, Wo, nco = oracle.aggregate_plan(p, finals, K)
    Xm, Wm, nc = m.posterior_means()
    assert nc == nco
    assert_rows_close(Xm, Xo[np.argsort(p.row_perm)], 1e-7, f"{summary}: aggregated X")
    assert_rows_close(Wm, Wo[np.argsort(p.col_perm)], 1e-7, f"{summary}: aggregated W")
    m.close()


def test_summary_ring_capacity_is_enforced():
    from paper_1703_00734_gb300 import bmf
    d = synth.make_workload(None, N=60, D=40, M=900, pattern="uniform", K=3, sigma=0.3,
                            tau=4.0, seed=9)
    m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], 3, d["tau"], "fp64", I=2, J=2,
                X0=d["X0"], W0=d["W0"], burnin=2, summary="dm", lam=1.0, max_samples=5)
    m.stage(1, 7, None)                       # 5 retained samples: fills the ring
    with pytest.raises(bmf.BmfError) as e:
        m.stage(1, 1, None)
    assert e.value.status == 8
    m.close()
    with pytest.raises(bmf.BmfError) as e:
        bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], 3, d["tau"], "fp64", summary="gmm",
                lam=0.0, max_samples=5)
    assert e.value.status == 1
