"""GPU parity of the device generator (draws == NULL): the generated buffers against the
oracle's implementation of the same counter-based generator (Philox4x64-10, Box-Muller,
Marsaglia-Tsang; pinned in test_oracle_rng.py), and whole sweeps and PP stages driven by it
against the oracle fed with its own generated draws.

Tolerance of the buffers: the two sides evaluate log, sqrt, sin, cos and pow with different
libraries (each within a few units in the last place), so values agree to
1e-12 (|x| + 1); the integer part of the generator (Philox words, acceptance decisions) is the
same on both sides.  Sweeps: the FP64 per-row bound of the other parity tests."""
import numpy as np
import pytest

import oracle
from paper_1703_00734_gb300 import synth
from pairing import Pair, assert_rows_close

pytestmark = pytest.mark.gpu


def small(N=300, D=170, M=6000, K=5, seed=0, pattern="uniform", **kw):
    return synth.make_workload(None, N=N, D=D, M=M, pattern=pattern, K=K, sigma=0.5,
                               tau=kw.pop("tau", 4.0), seed=seed, s_row=1.2, s_col=1.2, **kw)


def close_draws(gpu, cpu):
    err = np.abs(gpu - cpu)
    tol = 1e-12 * (np.abs(cpu) + 1.0)
    assert np.all(np.isfinite(gpu))
    assert np.all(err <= tol), f"worst |diff| {err.max():.3e} at {np.argmax(err / tol)}"


@pytest.mark.parametrize("K,I,J", [(5, 1, 1), (1, 1, 1), (10, 2, 3), (32, 2, 2), (64, 1, 1)])
def test_generated_buffers_match_oracle(K, I, J):
    from paper_1703_00734_gb300 import bmf
    d = small(K=min(K, 10), seed=K)
    seed = 1234 + K
    m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], K, d["tau"], "fp64", I=I, J=J,
                seed=seed)
    p = oracle.plan(d["N"], d["D"], d["row"], d["col"], d["val"], I, J)
    for stage in sorted({s.stage for s in p.subsets}):
        subs = p.stage_subsets(stage)
        got = m.generate_draws(3, 2, stage=stage)
        per = m.draws_per_sweep(stage)
        for i in range(2):
            ref = oracle.gen_batch_draws(subs, K, float(K), seed, 3 + i)
            close_draws(got[i * per:(i + 1) * per], ref)
        # one subset alone: the same numbers as its part of the batch
        s = subs[-1]
        one = m.generate_draws(4, 1, subset=s.sid)
        close_draws(one, oracle.gen_batch_draws([s], K, float(K), seed, 4))
    m.close()


def test_device_output_equals_host_output():
    torch = pytest.importorskip("torch")
    from paper_1703_00734_gb300 import bmf
    d = small(K=6, seed=2)
    m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], 6, d["tau"], "fp32", seed=99)
    per = m.draws_per_sweep(1)
    host = m.generate_draws(1, 3)
    dev = m.generate_draws(1, 3, out=torch.empty(3 * per, dtype=torch.float64, device="cuda"))
    assert np.array_equal(host, dev.cpu().numpy())
    m.close()


@pytest.mark.parametrize("K", [3, 10, 24])
def test_sweeps_with_device_generator_match_oracle(K):
    d = small(K=K, seed=40 + K)
    pr = Pair(d, K, gen=True, burnin=1)
    pr.run_stage(1, 1)
    pr.compare_subset(0)
    pr.run_stage(1, 3, t0=1)
    pr.compare_subset(0, rel=1e-8)


def test_pp_stages_with_device_generator():
    d = small(N=240, D=160, M=9000, K=4, seed=13)
    pr = Pair(d, 4, I=3, J=2, burnin=3, gen=True)
    for stage in (1, 2, 3):
        pr.run_stage(stage, 8)
        for s in pr.p.stage_subsets(stage):
            pr.compare_subset(s.sid, rel=1e-7)
        pr.finish_stage(stage)
    Xm_o, Wm_o, nc_o = oracle.aggregate_plan(pr.p, pr.finals, 4)
    Xm, Wm, nc = pr.m.posterior_means()
    rr, cr = np.argsort(pr.p.row_perm), np.argsort(pr.p.col_perm)
    assert nc == nc_o
    assert_rows_close(Xm, Xm_o[rr], 1e-6, "aggregated X")
    assert_rows_close(Wm, Wm_o[cr], 1e-6, "aggregated W")


def test_split_calls_equal_one_call():
    from paper_1703_00734_gb300 import bmf
    d = small(K=8, seed=77, pattern="zipf")
    states = []
    for split in ([5], [2, 3], [1, 1, 3]):
        m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], 8, d["tau"], "fp32",
                    X0=d["X0"], W0=d["W0"], seed=5)
        for n in split:
            m.sweep(0, n, None)
        states.append(m.get_state(0))
        m.close()
    for X, W, h in states[1:]:
        assert np.array_equal(X, states[0][0]) and np.array_equal(W, states[0][1])
        assert np.array_equal(h["LamW"], states[0][2]["LamW"])


def test_generator_argument_errors():
    from paper_1703_00734_gb300 import bmf
    d = small(N=40, D=30, M=300, K=2, seed=3)
    m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], 2, d["tau"], I=2, J=2)
    with pytest.raises(bmf.BmfError) as e:
        m.generate_draws(0, 1)
    assert e.value.status == 1
    with pytest.raises(bmf.BmfError) as e:
        m.generate_draws(1, 1, subset=9)
    assert e.value.status == 1
    m.close()


def test_moment_matching_needs_k_plus_one_samples():
    from paper_1703_00734_gb300 import bmf
    d = small(N=60, D=40, M=1200, K=3, seed=4)
    m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], 3, d["tau"], I=2, J=2,
                X0=d["X0"], W0=d["W0"], seed=8)
    m.stage(1, 3, None)                       # 3 retained samples < K + 1
    with pytest.raises(bmf.BmfError) as e:
        m.stage(2, 1, None)
    assert e.value.status == 8
    m.stage(1, 1, None)                       # the chain continues; now 4 samples
    m.stage(2, 4, None)
    m.close()
