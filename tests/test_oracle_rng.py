"""Pins of the oracle's counter-based draws (the numbers the library's device generator must
reproduce): Philox4x64-10 against numpy's independent implementation and the published
known-answer vectors, and the normal and chi-square transforms against their distributions.
All inputs are fixed, so every statistical check below is deterministic."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x64_10_kat.txt")
stats = pytest.importorskip("scipy.stats")


def test_philox_known_answers():
    n = 0
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        out = oracle.philox4x64(w[:4], w[4:6])
        assert [int(x) for x in out] == w[6:10]
        n += 1
    assert n == 2


def test_philox_matches_numpy_bit_generator():
    # numpy's Philox (4 x 64 bits, 10 rounds) advances its counter before each block, so the
    # first block of a generator started at counter c is the function at c + 1.
    rng = np.random.default_rng(11)
    for _ in range(20):
        ctr = [int(x) for x in rng.integers(1, 2 ** 63, 4)]
        key = [int(x) for x in rng.integers(0, 2 ** 63, 2)]
        start = [ctr[0] - 1] + ctr[1:]
        ref = np.random.Philox(key=key, counter=start).random_raw(4)
        assert [int(x) for x in oracle.philox4x64(ctr, key)] == [int(x) for x in ref]


def _normals(seed=5, t=3, sid=2, K=8, n=25_000):
    _, _, zx, zw = oracle.gen_subset(seed, t, sid, K, float(K), n, 7)
    return zx.ravel(), zw


def test_normal_stream_is_standard_normal():
    z, _ = _normals()
    n = len(z)
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # the cosine and sine of one pair, and the two pairs of one call, are uncorrelated
    for lag in (1, 2, 3, 4):
        r = np.corrcoef(z[:-lag], z[lag:])[0, 1]
        assert abs(r) < 5 / np.sqrt(n), lag
    # both branches are symmetric about zero
    for b in range(4):
        assert abs(z[b::4].mean()) < 5 / np.sqrt(n / 4)


def test_hyper_block_normals_are_standard_normal():
    K = 12
    vals = np.concatenate([oracle.gen_subset(9, t, 0, K, float(K), 3, 4)[0][K:]
                           for t in range(1, 1201)])
    assert stats.kstest(vals, "norm").pvalue > 1e-3


@pytest.mark.parametrize("nu0", [0.7, 3.0, 40.0, 5000.0])
def test_chi_square_stream_has_the_right_law(nu0):
    # K = 1, n = 1: hx[0] ~ chi2(nu0 + 1); nu0 = 0.7 takes the a < 1 boost (dof 1.7)
    dof = nu0 + 1
    c = np.array([oracle.gen_subset(21, t, 1, 1, nu0, 1, 2)[0][0] for t in range(1, 3001)])
    assert stats.kstest(c, stats.chi2(dof).cdf).pvalue > 1e-3
    assert abs(c.mean() - dof) < 5 * np.sqrt(2 * dof / len(c))
    # the W block of the same call uses dof nu0 + d = nu0 + 2
    cw = np.array([oracle.gen_subset(21, t, 1, 1, nu0, 1, 2)[1][0] for t in range(1, 1001)])
    assert stats.kstest(cw, stats.chi2(nu0 + 2).cdf).pvalue > 1e-3


def test_chi_square_dof_per_diagonal_entry():
    # block entry k has dof nu0 + n - k
    K, n = 6, 30
    c = np.array([oracle.gen_subset(4, t, 0, K, float(K), n, 5)[0][:K] for t in range(1, 2001)])
    for k in range(K):
        assert stats.kstest(c[:, k], stats.chi2(K + n - k).cdf).pvalue > 1e-3, k


def test_streams_are_distinct():
    a = oracle.gen_subset(1, 1, 0, 4, 4.0, 50, 50)
    assert not np.allclose(a[2], a[3])                                # X vs W
    assert not np.allclose(a[2], oracle.gen_subset(1, 2, 0, 4, 4.0, 50, 50)[2])   # sweep
    assert not np.allclose(a[2], oracle.gen_subset(1, 1, 1, 4, 4.0, 50, 50)[2])   # subset
    assert not np.allclose(a[2], oracle.gen_subset(2, 1, 0, 4, 4.0, 50, 50)[2])   # seed
    assert not np.allclose(a[0][4:], a[1][4:])                        # hyper normals X vs W
    # a row's draws do not depend on how many rows the subset has
    b = oracle.gen_subset(1, 1, 0, 4, 4.0, 80, 50)
    assert np.array_equal(a[2], b[2][:50])


def test_batch_layout():
    class S:
        def __init__(self, sid, n, d):
            self.sid, self.n, self.d = sid, n, d
    subs = [S(1, 5, 3), S(4, 2, 6)]
    K = 3
    buf = oracle.gen_batch_draws(subs, K, 3.0, 7, 2)
    lay = oracle.stage_draw_layout(subs, K)
    assert len(buf) == lay["total"]
    for s in subs:
        hx, hw, zx, zw = oracle.gen_subset(7, 2, s.sid, K, 3.0, s.n, s.d)
        H = oracle.hyper_block_len(K)
        assert np.array_equal(buf[lay[(s.sid, "hx")]:lay[(s.sid, "hx")] + H], hx)
        assert np.array_equal(buf[lay[(s.sid, "hw")]:lay[(s.sid, "hw")] + H], hw)
        assert np.array_equal(buf[lay[(s.sid, "zx")]:lay[(s.sid, "zx")] + s.n * K], zx.ravel())
        assert np.array_equal(buf[lay[(s.sid, "zw")]:lay[(s.sid, "zw")] + s.d * K], zw.ravel())
