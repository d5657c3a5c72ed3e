"""GPU parity of the sampled noise precision (Section 2.1: one precision per column, tau_d, or one
per chain, Gamma priors) against the oracle on the same counter-based draws: the generated
draw buffers with the noise chi-squares, and three PP stages per state (X, W, the precisions),
on the CUDA-core Gram (K = 4) and the tensor-core path (K = 20)."""
import numpy as np
import pytest

import oracle
from paper_1703_00734_gb300 import synth
from pairing import assert_rows_close

pytestmark = pytest.mark.gpu


def _data(K, seed):
    return synth.make_workload(None, N=160, D=90, M=6000, pattern="zipf", K=K, sigma=0.5,
                               tau=4.0, seed=seed, s_row=1.2, s_col=1.2)


@pytest.mark.parametrize("mode", ["column", "global"])
def test_generated_draws_include_the_noise_variates(mode):
    from paper_1703_00734_gb300 import bmf
    d = _data(4, 3)
    K, seed = 4, 17
    m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], K, d["tau"], "fp64", I=2, J=2,
                X0=d["X0"], W0=d["W0"], seed=seed, noise=mode, noise_a0=1.5, noise_b0=0.5)
    p = oracle.plan(d["N"], d["D"], d["row"], d["col"], d["val"], 2, 2)
    noise = oracle.NoiseModel(mode, 1.5, 0.5, d["tau"])
    for stage in (1, 2, 3):
        got = m.generate_draws(3, 2, stage=stage)
        want = np.concatenate([oracle.gen_batch_draws(p.stage_subsets(stage), K, float(K), seed, t,
                                                      noise) for t in (3, 4)])
        assert got.shape == want.shape
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-13)
    m.close()


@pytest.mark.parametrize("K,mode,prec", [(4, "column", "fp64"), (4, "global", "fp64"),
                                         (20, "column", "fp64"), (4, "column", "fp32")])
def test_pp_with_sampled_noise_matches_the_oracle(K, mode, prec):
    from paper_1703_00734_gb300 import bmf
    d = _data(K, 5 + K)
    T, B, seed, a0, b0 = K + 10, 3, 23, 2.0, 0.5
    m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], K, d["tau"], prec, I=2, J=2,
                X0=d["X0"], W0=d["W0"], burnin=B, seed=seed, noise=mode, noise_a0=a0,
                noise_b0=b0)
    p = oracle.plan(d["N"], d["D"], d["row"], d["col"], d["val"], 2, 2)
    prior = oracle.NWPrior(K)
    noise = oracle.NoiseModel(mode, a0, b0, d["tau"])
    X0, W0 = d["X0"][p.row_perm], d["W0"][p.col_perm]
    finals = {}
    # FP64 agrees to rounding; FP32 gathers leave differences of the order of the FP32 Gram
    # (compared on stage 1, before moment matching amplifies them)
    rel = 1e-7 if prec == "fp64" else 1e-3
    for stage in ((1, 2, 3) if prec == "fp64" else (1,)):
        subs = p.stage_subsets(stage)
        chains = oracle.setup_stage_chains(p, stage, X0, W0, K, finals)
        oracle.run_stage(p, stage, chains, K, d["tau"], prior,
                         lambda t: oracle.gen_batch_draws(subs, K, float(K), seed, t + 1, noise),
                         T, B, 1, noise)
        m.stage(stage, T, None)
        for s in subs:
            X, W, _ = m.get_state(s.sid)
            st = chains[s.sid]
            assert_rows_close(X, st.X, rel, f"{mode}: X of subset {s.sid}")
            assert_rows_close(W, st.W, rel, f"{mode}: W of subset {s.sid}")
            tau = m.get_noise(s.sid)
            assert_rows_close(tau[:, None], st.tau_col[:, None], rel, f"{mode}: tau of {s.sid}")
            if mode == "global":
                assert np.all(tau == tau[0])
            finals[s.sid] = oracle.finalize(st)
    assert not np.allclose(m.get_noise(0), d["tau"])      # the precisions moved
    m.close()
