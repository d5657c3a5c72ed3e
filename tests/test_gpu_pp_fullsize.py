"""The PP benchmark workload at full size (100,000 x 20,000 Zipf(1.2), 18M training entries,
K = 16, a 4 x 4 grid) batched as the benchmark runs it (all subsets of a stage in the same
launches): stages 1 and 2 on the device generator, then one stage-3 sweep (nine subsets, every X
and W row forming its own Gram sums) checked on sampled rows against the oracle's conditional draw (Eqs. 2-4) given the same
partner states, propagated per-row priors (the stage-2 moment-matched posteriors, Algorithm 1)
and draws: the FP64 path to the FP64 tolerance, the FP32 path within the first-order bound of
its reduced-precision Gram sums."""
import numpy as np
import pytest

import oracle
from paper_1703_00734_gb300 import synth
from pairing import assert_rows_close
from test_gpu_precision import check_half, row_bounds

pytestmark = pytest.mark.gpu

T12, B12 = 40, 6            # stage 1 and 2 sweeps, burn-in: 34 retained samples = 2K + 2


def _rows_csr(ptr, idx, val, rows):
    """CSR of the selected rows of a block."""
    sl = [slice(ptr[r], ptr[r + 1]) for r in rows]
    cnt = np.array([s.stop - s.start for s in sl], np.int64)
    p = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
    return p, np.concatenate([idx[s] for s in sl]), np.concatenate([val[s] for s in sl])


@pytest.fixture(scope="module")
def workload():
    return synth.make_workload("pp4x4-100000x20000-20M-k16")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_stage3_sweep_on_sampled_rows(workload, precision):
    from paper_1703_00734_gb300 import bmf
    d = workload
    K, tau, I, J = d["K"], d["tau"], d["I"], d["J"]
    m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], K, tau, precision, I=I, J=J,
                X0=d["X0"], W0=d["W0"], burnin=B12, seed=21)
    m.set_monitor(False)
    m.stage(1, T12, None)
    m.stage(2, T12, None)
    m.stage(3, 0, None)                          # installs the propagated priors
    p = oracle.plan(d["N"], d["D"], d["row"], d["col"], d["val"], I, J)
    subs = p.stage_subsets(3)
    before = {s.sid: m.get_state(s.sid)[:2] for s in subs}
    draws = synth.sweep_draws([(s.n, s.d) for s in subs], K, float(K), synth.rng_for(77, 3))
    lay = oracle.stage_draw_layout(subs, K)
    m.stage(3, 1, draws)
    rng = np.random.default_rng(5)
    qmax = 0.0
    for s in subs[:3]:
        i, j = divmod(s.sid, J)
        X0s, W0s = before[s.sid]
        X1, W1 = m.get_state(s.sid)[:2]
        # X | W: prior from subset (i, 0), partners the subset's W before the sweep
        mu_x, Lam_x = m.get_posterior(i * J, bmf.FACTOR_X)
        zx = draws[lay[(s.sid, "zx")]:lay[(s.sid, "zx")] + s.n * K].reshape(s.n, K)
        rx = np.unique(np.concatenate([np.arange(20), rng.choice(s.n, 300, replace=False)]))
        ptr, idx, val = _rows_csr(s.rptr, s.ridx, s.rval, rx)
        want_x = oracle.update_rows(ptr, idx, val, W0s, tau, mu_x[rx], Lam_x[rx], zx[rx],
                                    per_row_prior=True)
        # W | X: prior from subset (0, j), partners the subset's new X (the GPU's)
        mu_w, Lam_w = m.get_posterior(j, bmf.FACTOR_W)
        zw = draws[lay[(s.sid, "zw")]:lay[(s.sid, "zw")] + s.d * K].reshape(s.d, K)
        rw = np.unique(np.concatenate([np.arange(20), rng.choice(s.d, 300, replace=False)]))
        ptr, idx, val = _rows_csr(s.cptr, s.cidx, s.cval, rw)
        want_w = oracle.update_rows(ptr, idx, val, X1, tau, mu_w[rw], Lam_w[rw], zw[rw],
                                    per_row_prior=True)
        assert (np.diff(s.rptr)[rx] <= 64).all()      # rows forming their own Gram sums
        if precision == "fp64":
            assert_rows_close(X1[rx], want_x, 1e-9, f"X of subset {s.sid}")
            assert_rows_close(W1[rw], want_w, 1e-9, f"W of subset {s.sid}")
        else:
            u_in = 2.0 ** -24
            for rows, ptr_, idx_, val_, P, mu, Lam, z, got, want, what in (
                    (rx, s.rptr, s.ridx, s.rval, W0s, mu_x, Lam_x, zx, X1[rx], want_x, "X"),
                    (rw, s.cptr, s.cidx, s.cval, X1, mu_w, Lam_w, zw, W1[rw], want_w, "W")):
                bounds = np.array([row_bounds(ptr_, idx_, val_, P, np.zeros_like(P), tau, mu[r],
                                              Lam[r], z, u_in, [r])[0] for r in rows])
                qmax = max(qmax, check_half(got, want, bounds, f"fp32 {what} of subset {s.sid}"))
    m.close()
    if precision == "fp32":
        print(f"full-size PP stage 3 fp32: worst err/bound {qmax:.3f}")
