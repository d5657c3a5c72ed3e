"""The library's host-side preprocessing (bmf_plan: validation, the Section 5.2 order, the I x J
grid), checked on the CPU against the oracle's planner, which is written independently: the
orders, the cuts and the per-subset entry counts must be identical (integer work, bit-exact),
and invalid inputs must fail with the documented status codes."""
import numpy as np
import pytest

import oracle
from paper_1703_00734_gb300 import synth

bmf = pytest.importorskip("paper_1703_00734_gb300.bmf")


@pytest.fixture(scope="module")
def lib():
    from paper_1703_00734_gb300 import build
    build.build()
    return bmf.load()


@pytest.mark.parametrize("order", ["decreasing", "none"])
@pytest.mark.parametrize("I,J", [(1, 1), (2, 3), (4, 4), (5, 2)])
def test_plan_matches_the_oracle(lib, order, I, J):
    d = synth.make_workload(None, N=400, D=250, M=12000, pattern="zipf", K=4, sigma=0.5,
                            tau=4.0, seed=31 + I * J, s_row=1.2, s_col=1.1)
    got = bmf.plan(d["N"], d["D"], d["row"], d["col"], d["val"], I, J, order=order)
    ref = oracle.plan(d["N"], d["D"], d["row"], d["col"], d["val"], I, J, order=order)
    np.testing.assert_array_equal(got["row_perm"], ref.row_perm)
    np.testing.assert_array_equal(got["col_perm"], ref.col_perm)
    np.testing.assert_array_equal(got["row_bounds"], ref.row_bounds)
    np.testing.assert_array_equal(got["col_bounds"], ref.col_bounds)
    np.testing.assert_array_equal(got["subset_nnz"], [s.nnz for s in ref.subsets])
    assert got["subset_nnz"].sum() == len(d["row"])


def test_plan_with_given_cuts(lib):
    d = synth.make_workload(None, N=300, D=200, M=6000, pattern="uniform", K=3, sigma=0.5,
                            tau=4.0, seed=40)
    rb, cb = [0, 10, 10, 300], [0, 150, 200]                   # an empty row block is allowed
    got = bmf.plan(300, 200, d["row"], d["col"], d["val"], 3, 2, row_bounds=rb, col_bounds=cb)
    ref = oracle.plan(300, 200, d["row"], d["col"], d["val"], 3, 2, row_bounds=rb, col_bounds=cb)
    np.testing.assert_array_equal(got["row_bounds"], rb)
    np.testing.assert_array_equal(got["subset_nnz"], [s.nnz for s in ref.subsets])


def _status(lib, N, D, row, col, val, I=1, J=1, rb=None, order=1):
    row, col, val = (np.ascontiguousarray(row, np.int32), np.ascontiguousarray(col, np.int32),
                     np.ascontiguousarray(val, np.float64))
    rb = None if rb is None else np.ascontiguousarray(rb, np.int64)
    st = lib.bmf_plan(N, D, len(row), row.ctypes.data, col.ctypes.data, val.ctypes.data, order,
                      I, None if rb is None else rb.ctypes.data, J, None, None, None, None, None,
                      None)
    return st, lib.bmf_last_error(None).decode()


def test_plan_rejects_invalid_input(lib):
    ok = ([0, 1, 2], [0, 1, 0], [1.0, 2.0, 3.0])
    assert _status(lib, 3, 2, *ok)[0] == 0
    st, msg = _status(lib, 3, 2, [0, 1, 0], [0, 1, 0], [1.0, 2.0, 3.0])   # duplicate (0, 0)
    assert st == 1 and "duplicate" in msg
    st, msg = _status(lib, 3, 2, [0, 3, 2], [0, 1, 0], [1.0, 2.0, 3.0])   # row out of range
    assert st == 1 and "range" in msg
    st, msg = _status(lib, 3, 2, [0, 1, 2], [0, 1, 0], [1.0, np.nan, 3.0])
    assert st == 4 and "finite" in msg                                     # BMF_E_NONFINITE
    assert _status(lib, 3, 2, *ok, I=4)[0] == 1                            # I > N
    assert _status(lib, 3, 2, *ok, I=2, rb=[0, 3, 2])[0] != 0              # cuts not increasing
    assert _status(lib, 3, 2, *ok, order=7)[0] == 1
