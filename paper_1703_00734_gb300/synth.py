"""Seeded synthetic inputs: observation patterns, planted low-rank values, train/test splits,
initial chain states and the standard-normal / chi-square variates a Gibbs sweep consumes.

This module holds none of the sampler's arithmetic; it only produces random inputs.  Both the
CUDA library (through the tests and the benchmark) and the oracle are fed from it.

Workloads (the paper's data sets are not available; these stand in for them with the shapes
and statistics of the rating matrices the paper uses, Section 5.3):
  * ``planted``  -- uniform random pattern, X, W ~ N(0, 1), y = x^T w + N(0, sigma^2)
                    (the paper's simulated-data recipe, Section 5.3, with other sizes).
  * ``zipf``     -- capped product model: a pair (n, d) is drawn with probability
                    proportional to p_n q_d, p and q Zipf(s) weights over randomly permuted
                    ranks; duplicates are redrawn until exactly M distinct pairs exist, so the
                    heaviest rows and columns saturate (fully observed), as in rating data.
  * ratings      -- y = clip(round(3.5 + x^T w + N(0, sigma^2)), 1, 5) with X, W entries of
                    variance K^{-1/2} (so x^T w has unit variance).
  * ``dense``    -- every cell of Y = X W^T + E observed (X, W, E standard normal), then split
                    by a missingness scenario (Section 5.3, simulated data): ``random``, a
                    uniformly random fraction held out as the test set; ``structured``, cell
                    (n, d) kept for training with probability w_n w_d, where w_n and w_d run in
                    equal steps from 0.9 down to 0.005 over the rows and over the columns (about
                    80% of the cells end up missing, i.e. in the test set).
"""
from __future__ import annotations

import os

import numpy as np


def rng_for(*key) -> np.random.Generator:
    """Independent generator for a tuple of non-negative integers."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(k) for k in key])))


# ---------------------------------------------------------------------------------------
# Observation patterns
# ---------------------------------------------------------------------------------------

def uniform_pairs(N: int, D: int, M: int, rng) -> tuple[np.ndarray, np.ndarray]:
    """M distinct (row, col) pairs uniformly at random."""
    if M > N * D:
        raise ValueError("more pairs than cells")
    keys = rng.choice(N * D, size=M, replace=False) if N * D <= 50_000_000 else None
    if keys is None:
        keys = _distinct_keys(lambda m: rng.integers(0, N, m) * D + rng.integers(0, D, m), M,
                              N * D)
    return (keys // D).astype(np.int32), (keys % D).astype(np.int32)


def _distinct_keys(draw, M, ncells):
    """Draw keys in rounds, keeping the first occurrence of each new key in draw order, until
    exactly M distinct keys exist (membership in a bitset over all cells)."""
    bits = np.zeros((ncells + 63) // 64, np.uint64)
    parts = []
    need = M
    accept = 1.0
    while need > 0:
        m = int(min(max(need / max(accept, 0.02) * 1.05 + 1024, 1024), 4 * M + 1024))
        cand = np.asarray(draw(m), np.int64)

        def fresh(a, b):
            c = cand[a:b]
            word, bit = c >> 6, (c & 63).astype(np.uint64)
            return c[((bits[word] >> bit) & np.uint64(1)) == 0]

        cand = _parallel(fresh, m)
        take = cand[_first_occurrences(cand, ncells)][:need]
        np.bitwise_or.at(bits, take >> 6, np.left_shift(np.uint64(1), (take & 63).astype(np.uint64)))
        accept = max(len(take) / m, 1e-3)
        parts.append(take)
        need -= len(take)
    return np.concatenate(parts) if parts else np.empty(0, np.int64)


def _first_occurrences(keys, ncells, parts=16):
    """Ascending positions of the first occurrence of each distinct key (key ranges are
    deduplicated independently on a thread pool; same result as one np.unique)."""
    if len(keys) <= 1 << 22:
        _, first = np.unique(keys, return_index=True)
        return np.sort(first)
    bucket = keys // -(-ncells // parts)

    def one(b):
        sel = np.flatnonzero(bucket == b)
        _, first = np.unique(keys[sel], return_index=True)
        return sel[first]

    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(min(parts, os.cpu_count() or 1)) as ex:
        pos = np.concatenate(list(ex.map(one, range(parts))))
    return np.sort(pos, kind="stable")


def zipf_weights(n: int, s: float, rng) -> np.ndarray:
    ranks = rng.permutation(n) + 1
    w = ranks.astype(np.float64) ** (-s)
    return w / w.sum()


def _inverse_cdf(cdf, u, guide):
    """Index of the first cdf entry >= u (same result as searchsorted), found from a guide table
    (Chen & Asau 1974): start at the first index of u's bucket and step forward."""
    L, n = len(guide), len(cdf)
    i = np.minimum(guide[np.minimum((u * L).astype(np.int64), L - 1)], n - 1)
    act = np.nonzero(cdf[i] < u)[0]
    while len(act):
        act = act[i[act] < n - 1]
        i[act] += 1
        act = act[cdf[i[act]] < u[act]]
    return i


def _parallel(fn, n, chunk=1 << 22):
    """fn(a, b) over [0, n) in chunks on a thread pool, results concatenated in order (the
    numpy kernels inside release the GIL; the result does not depend on the thread count)."""
    starts = range(0, n, chunk)
    if n <= chunk:
        return fn(0, n)
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(min(16, os.cpu_count() or 1)) as ex:
        return np.concatenate(list(ex.map(lambda a: fn(a, min(a + chunk, n)), starts)))


def zipf_pairs(N: int, D: int, M: int, s_row: float, s_col: float, rng):
    """M distinct pairs from the capped product model (module docstring)."""
    p = np.cumsum(zipf_weights(N, s_row, rng))
    q = np.cumsum(zipf_weights(D, s_col, rng))
    p /= p[-1]
    q /= q[-1]
    gp = np.searchsorted(p, np.arange(16 * N) / (16 * N))
    gq = np.searchsorted(q, np.arange(16 * D) / (16 * D))

    def draw(m):
        u, v = rng.random(m), rng.random(m)
        r = _parallel(lambda a, b: _inverse_cdf(p, u[a:b], gp), m)
        c = _parallel(lambda a, b: _inverse_cdf(q, v[a:b], gq), m)
        return r.astype(np.int64) * D + c

    keys = _distinct_keys(draw, M, N * D)
    return (keys // D).astype(np.int32), (keys % D).astype(np.int32)


# ---------------------------------------------------------------------------------------
# Values
# ---------------------------------------------------------------------------------------

def planted_values(N, D, row, col, K_true, x_sd, w_sd, noise_sd, rng, ratings=False,
                   base=3.5):
    X = rng.standard_normal((N, K_true)) * x_sd
    W = rng.standard_normal((D, K_true)) * w_sd
    y = np.empty(len(row))
    B = 1 << 22
    for a in range(0, len(row), B):
        r, c = row[a:a + B], col[a:a + B]
        y[a:a + B] = np.einsum("ij,ij->i", X[r], W[c])
    y += rng.standard_normal(len(row)) * noise_sd
    if ratings:
        y = np.clip(np.rint(base + y), 1.0, 5.0)
    return y, X, W


def split(nnz: int, test_frac: float, rng):
    """Boolean mask of held-out entries (uniformly at random)."""
    perm = rng.permutation(nnz)
    m = np.zeros(nnz, bool)
    m[perm[: int(round(test_frac * nnz))]] = True
    return m


def structured_missing(N: int, D: int, rng) -> np.ndarray:
    """Test (missing) mask over the N x D cells in row-major order for the structured
    scenario: a cell is kept for training with probability w_n w_d, w_n and w_d equally
    spaced from 0.9 down to 0.005 (Section 5.3)."""
    wn = np.linspace(0.9, 0.005, N)
    wd = np.linspace(0.9, 0.005, D)
    keep = rng.random((N, D)) < wn[:, None] * wd[None, :]
    return ~keep.reshape(-1)


def init_state(n: int, K: int, sd: float, rng) -> np.ndarray:
    return rng.standard_normal((n, K)) * sd


# ---------------------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------------------

WORKLOADS = {
    # name: (N, D, M, pattern, params)
    "planted-1000x500-k10": dict(N=1000, D=500, M=25_000, pattern="uniform", K=10, sigma=0.5,
                                 x_sd=1.0, w_sd=1.0, ratings=False, tau=4.0, seed=0),
    "zipf-69878x10677-10M-k10": dict(N=69_878, D=10_677, M=10_000_000, pattern="zipf",
                                     s_row=1.2, s_col=1.2, K=10, sigma=0.8, ratings=True,
                                     tau=1.5625, seed=1),
    "pp4x4-100000x20000-20M-k16": dict(N=100_000, D=20_000, M=20_000_000, pattern="zipf",
                                       s_row=1.2, s_col=1.2, K=16, sigma=0.5, x_sd=1.0,
                                       w_sd=1.0, ratings=False, tau=4.0, seed=2, I=4, J=4),
    "zipf-480189x17770-100M-k32": dict(N=480_189, D=17_770, M=100_000_000, pattern="zipf",
                                       s_row=1.1, s_col=1.1, K=32, sigma=0.8, ratings=True,
                                       tau=1.5625, seed=3),
    "uniform-200000x50000-50M-k64": dict(N=200_000, D=50_000, M=50_000_000,
                                         pattern="uniform", K=64, sigma=0.3, x_sd=1.0,
                                         w_sd=1.0, ratings=False, tau=1.0 / 0.09, seed=4),
    # the paper's simulated data sets (Section 5.3): 6,040 x 3,706, K = 5, unit noise, 80% of
    # the cells missing at random or in the structured pattern
    "sim-6040x3706-k5": dict(N=6040, D=3706, pattern="dense", K=5, sigma=1.0, x_sd=1.0,
                             w_sd=1.0, ratings=False, tau=1.0, seed=5, missing="random",
                             test_frac=0.8),
    "sim-6040x3706-k5-structured": dict(N=6040, D=3706, pattern="dense", K=5, sigma=1.0,
                                        x_sd=1.0, w_sd=1.0, ratings=False, tau=1.0, seed=6,
                                        missing="structured"),
}


def make_workload(name: str = None, test_frac: float = 0.1, scale: float = 1.0, **over):
    """Build a named workload (optionally shrunk by ``scale``: N and D by scale, M by scale^2;
    N, D or M given in ``over`` are taken as they are).  Returns a dict
    with the train/test COO (original indices), the planted factors and initial states."""
    cfg = dict(WORKLOADS[name]) if name else {}
    sizes = {k: over.pop(k) for k in ("N", "D", "M") if k in over}
    cfg.update(over)
    N = sizes["N"] if "N" in sizes else max(2, int(round(cfg["N"] * scale)))
    D = sizes["D"] if "D" in sizes else max(2, int(round(cfg["D"] * scale)))
    K = cfg["K"]
    seed = cfg.get("seed", 0)
    rng = rng_for(seed, 1)
    if cfg["pattern"] == "dense":
        keys = np.arange(N * D, dtype=np.int64)
        row, col = (keys // D).astype(np.int32), (keys % D).astype(np.int32)
    else:
        M = sizes["M"] if "M" in sizes else max(4, int(round(cfg["M"] * scale * scale)))
        if cfg["pattern"] == "uniform":
            row, col = uniform_pairs(N, D, M, rng)
        else:
            row, col = zipf_pairs(N, D, M, cfg["s_row"], cfg["s_col"], rng)
    if cfg.get("ratings"):
        sd = K ** (-0.25)
        y, Xt, Wt = planted_values(N, D, row, col, K, sd, sd, cfg["sigma"], rng_for(seed, 2),
                                   ratings=True)
    else:
        y, Xt, Wt = planted_values(N, D, row, col, K, cfg.get("x_sd", 1.0), cfg.get("w_sd", 1.0),
                                   cfg["sigma"], rng_for(seed, 2))
    if cfg.get("missing") == "structured":
        test = structured_missing(N, D, rng_for(seed, 3))
    else:
        test = split(len(row), cfg.get("test_frac", test_frac), rng_for(seed, 3))
    tr = ~test
    X0 = init_state(N, K, 0.1, rng_for(seed, 4))
    W0 = init_state(D, K, 0.1, rng_for(seed, 5))
    return dict(name=name, N=N, D=D, K=K, tau=cfg["tau"], sigma=cfg["sigma"],
                I=cfg.get("I", 1), J=cfg.get("J", 1),
                row=row[tr].copy(), col=col[tr].copy(), val=y[tr].copy(),
                test_row=row[test].copy(), test_col=col[test].copy(), test_val=y[test].copy(),
                X_true=Xt, W_true=Wt, X0=X0, W0=W0, seed=seed)


# ---------------------------------------------------------------------------------------
# Draw buffers (layout of the library's public header: per sweep, hyperparameter blocks of
# every subset of the batch, then z for all X rows, then z for all W rows)
# ---------------------------------------------------------------------------------------

def hyper_block(K: int, nu: float, rng) -> np.ndarray:
    """chi-square variates with dof nu - k (k = 0..K-1), K(K-1)/2 normals, K normals."""
    dof = nu - np.arange(K)
    return np.concatenate([rng.chisquare(dof), rng.standard_normal(K * (K - 1) // 2),
                           rng.standard_normal(K)])


def sweep_draws(subset_sizes, K: int, nu0: float, rng) -> np.ndarray:
    """One sweep's draws for a batch; subset_sizes = [(n_rows, n_cols), ...] in id order."""
    parts = []
    for n, d in subset_sizes:
        parts.append(hyper_block(K, nu0 + n, rng))
        parts.append(hyper_block(K, nu0 + d, rng))
    nx = sum(n for n, _ in subset_sizes)
    nw = sum(d for _, d in subset_sizes)
    parts.append(rng.standard_normal(nx * K))
    parts.append(rng.standard_normal(nw * K))
    return np.concatenate(parts)


def draws(subset_sizes, K: int, nu0: float, n_sweeps: int, seed: int, stream: int = 0):
    """n_sweeps consecutive sweeps of draws; sweep t uses generator (seed, stream, t)."""
    return np.concatenate([sweep_draws(subset_sizes, K, nu0, rng_for(seed, 7, stream, t))
                           for t in range(n_sweeps)])
