"""The launch schedule (bmf_set_schedule: row chunks per sweep half, Gram grid) changes only
how the work is launched: the sampled states must be bit-identical under every schedule, and
the chunked path must keep FP64 parity with the oracle."""
import numpy as np
import pytest

from paper_1703_00734_gb300 import synth
from pairing import Pair

pytestmark = pytest.mark.gpu

SCHEDULES = [(1, 1, 4, 0.0, 0, 0), (2, 3, 2, 0.0, 0, 2), (8, 8, 1, 0.0, 0, 8),
             (4, 2, 4, 500.0, 0, 4), (1, 1, 4, 0.0, 1, 16), (3, 2, 8, 0.0, 1, 2),
             (1, 1, 4, 0.0, 0, 32)]


def run(d, K, prec, sched, I=1, J=1, sweeps=3):
    from paper_1703_00734_gb300 import bmf
    m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], K, d["tau"], prec, I=I, J=J,
                X0=d["X0"], W0=d["W0"], seed=3, burnin=1,
                test=(d["test_row"], d["test_col"], d["test_val"]))
    m.set_schedule(*sched)
    assert m.get_schedule()["chunks_x"] == sched[0]
    out = []
    stages = (1,) if I * J == 1 else (1, 2, 3)
    for stage in stages:
        st = m.stage(stage, sweeps, None)
        out.append(st["rmse_sample"])
        for sid in range(I * J):
            if m.subset_info(sid)["stage"] == stage:
                X, W, h = m.get_state(sid)
                out += [X, W, h["LamX"], h["LamW"]]
    m.close()
    return out


@pytest.mark.parametrize("K,prec,I,J", [(5, "fp32", 1, 1), (10, "fp64", 1, 1), (16, "bf16", 1, 1),
                                        (24, "fp32", 1, 1), (4, "fp32", 2, 3), (16, "fp32", 2, 2),
                                        (13, "fp64", 1, 1)])
def test_states_identical_under_every_schedule(K, prec, I, J):
    d = synth.make_workload(None, N=900, D=500, M=40_000, pattern="zipf", K=K, sigma=0.5,
                            tau=4.0, seed=60 + K, s_row=1.2, s_col=1.2)
    # a PP grid keeps at least 2K samples per chain, so that the moment-matched precisions
    # are well conditioned
    sweeps = 2 * K + 2 if I * J > 1 else 3
    ref = run(d, K, prec, SCHEDULES[0], I, J, sweeps=sweeps)
    for sc in SCHEDULES[1:]:
        got = run(d, K, prec, sc, I, J, sweeps=sweeps)
        for a, b in zip(ref, got):
            assert np.array_equal(a, b, equal_nan=True), sc


def test_chunked_schedule_fp64_parity():
    d = synth.make_workload(None, N=700, D=300, M=30_000, pattern="zipf", K=6, sigma=0.5,
                            tau=4.0, seed=71, s_row=1.2, s_col=1.2)
    pr = Pair(d, 6)
    pr.m.set_schedule(4, 3, 2)
    pr.run_stage(1, 2)
    pr.compare_subset(0, rel=1e-8)
    pr.m.set_schedule(2, 2, 4, graph=1)      # and the graph-captured launch, twice (update path)
    pr.run_stage(1, 2, t0=2)
    pr.run_stage(1, 2, t0=4)
    pr.compare_subset(0, rel=1e-7)


def test_schedule_argument_errors():
    from paper_1703_00734_gb300 import bmf
    d = synth.make_workload(None, N=40, D=30, M=300, pattern="uniform", K=2, sigma=0.5,
                            tau=4.0, seed=1)
    m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], 2, d["tau"])
    for bad in [(0, 1, 4, 0.0), (1, 9, 4, 0.0), (1, 1, 0, 0.0), (1, 1, 4, -1.0), (1, 1, 4, 0.0, 2)]:
        with pytest.raises(bmf.BmfError) as e:
            m.set_schedule(*bad)
        assert e.value.status == 1
    m.close()


def test_lanes_that_do_not_fit_are_rejected_and_the_tuner_skips_them():
    """Two lanes per row exist only for 13 <= K <= 16 and a team's rows must fit in shared
    memory: at K = 64 a team of 8 lanes would need 291 KB per block."""
    from paper_1703_00734_gb300 import bmf
    for K, bad, good in [(32, 2, 16), (64, 8, 32)]:
        d = synth.make_workload(None, N=300, D=200, M=6000, pattern="zipf", K=min(K, 10),
                                sigma=0.5, tau=4.0, seed=K, s_row=1.2, s_col=1.2)
        m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], K, d["tau"], "bf16",
                    X0=None, W0=None, seed=2, burnin=1)
        with pytest.raises(bmf.BmfError) as e:
            m.set_schedule(1, 1, 4, 0.0, 0, bad)
        assert e.value.status == 1
        m.set_schedule(1, 1, 4, 0.0, 0, good)
        m.sweep(0, 1, None)
        sc = m.autotune(1, -1, 1)
        assert sc["cond_lanes"] in (0, 8, 16, 32)
        m.sweep(0, 1, None)
        m.close()


@pytest.mark.parametrize("I,J,stage", [(1, 1, 1), (2, 3, 2)])
def test_autotune_restores_the_chain(I, J, stage):
    from paper_1703_00734_gb300 import bmf
    d = synth.make_workload(None, N=800, D=400, M=30_000, pattern="zipf", K=6, sigma=0.5,
                            tau=4.0, seed=81, s_row=1.2, s_col=1.2)
    test = (d["test_row"], d["test_col"], d["test_val"])

    def chain(tune):
        m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], 6, d["tau"], "fp32", I=I, J=J,
                    X0=d["X0"], W0=d["W0"], seed=4, burnin=1, test=test, moments="full")
        for s in range(1, stage):
            m.stage(s, 8, None)
        m.stage(stage, 2, None)
        sc = m.autotune(stage, -1, 2) if tune else None
        st = m.stage(stage, 3, None)
        out = [st["rmse_sample"], st["rmse_mean"], st["sweeps"], st["kept"]]
        for sid in range(I * J):
            if m.subset_info(sid)["stage"] == stage:
                X, W, h = m.get_state(sid)
                out += [X, W, h["LamX"], h["LamW"], *m.get_moments(sid, 0)[:2]]
        m.close()
        return out, sc

    ref, _ = chain(False)
    got, sc = chain(True)
    assert 1 <= sc["chunks_x"] <= 8 and sc["gram_blocks_per_sm"] in (2, 4, 8)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b, equal_nan=True)
