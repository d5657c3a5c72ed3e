"""The oracle's OpenMP build (the all-core CPU timing) splits the row conditionals over threads;
each row's arithmetic is unchanged, so a sweep gives bit-identical states to the serial build,
and a failing row is reported as the first failing row in both builds."""
import numpy as np
import pytest

import oracle
from paper_1703_00734_gb300 import synth


def _sweeps(openmp, n=3):
    oracle.use_openmp(openmp)
    try:
        d = synth.make_workload(None, N=400, D=230, M=9000, pattern="zipf", K=6, sigma=0.5,
                                tau=4.0, seed=21, s_row=1.2, s_col=1.2)
        K = d["K"]
        p = oracle.plan(d["N"], d["D"], d["row"], d["col"], d["val"], 1, 1)
        s = p.subsets[0]
        prior = oracle.NWPrior(K)
        st = oracle.new_chain(d["X0"][p.row_perm], d["W0"][p.col_perm], K)
        lay = oracle.stage_draw_layout([s], K)
        H = oracle.hyper_block_len(K)
        for t in range(n):
            dr = synth.sweep_draws([(s.n, s.d)], K, prior.nu0, synth.rng_for(4, t))
            oracle.sweep_subset(s, st, K, d["tau"], prior, dr[0:H], dr[H:2 * H],
                                dr[lay[(0, "zx")]:lay[(0, "zx")] + s.n * K],
                                dr[lay[(0, "zw")]:lay[(0, "zw")] + s.d * K])
        return st.X.copy(), st.W.copy(), st.LamX.copy()
    finally:
        oracle.use_openmp(False)


def test_openmp_build_is_bit_identical():
    try:
        oracle.build(openmp=True)
    except Exception as e:            # no OpenMP runtime: nothing to compare
        pytest.skip(f"no OpenMP build: {e}")
    a = _sweeps(False)
    b = _sweeps(True)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_openmp_build_reports_the_first_failing_row():
    try:
        oracle.build(openmp=True)
    except Exception as e:
        pytest.skip(f"no OpenMP build: {e}")
    import ctypes
    K, R = 3, 300
    rng = np.random.default_rng(0)
    ptr = np.zeros(R + 1, np.int64)              # no observations: Lambda_r = prior of row r
    idx = np.zeros(1, np.int32)
    val = np.zeros(1)
    P = np.zeros((1, K))
    mu = rng.standard_normal((R, K))
    Lam = np.tile(np.eye(K), (R, 1, 1))
    for r in (57, 123, 250):                     # not positive definite
        Lam[r] = -np.eye(K)
    z = rng.standard_normal((R, K))
    for openmp in (False, True):
        oracle.use_openmp(openmp)
        try:
            X = np.zeros((R, K))
            bad = ctypes.c_int64(-1)
            st = oracle.lib().orc_update_rows(K, R, ptr.ctypes.data, idx.ctypes.data,
                                              val.ctypes.data, P.ctypes.data, 1.0, None, None, 1,
                                              mu.ctypes.data, Lam.ctypes.data, z.ctypes.data,
                                              X.ctypes.data, ctypes.byref(bad))
        finally:
            oracle.use_openmp(False)
        assert st == oracle.ORC_NOT_PD and bad.value == 57
