"""The ORACLE: a plain, slow FP64 CPU restatement of the BPMF Gibbs sweep inside the
posterior-propagation (PP) scheme of Qin et al., "Distributed Bayesian Matrix Factorization
with Limited Communication" (arXiv 1703.00734).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code with the CUDA library and never imports it;
the library never imports this package.

Layout:
  * ``bmf_oracle.c``  -- FP64 numerical core (conditionals, Normal-Wishart draw, moment
    matching and the dominant-mode / mixture summaries, Algorithm 2 aggregation, log-joint
    gradient), compiled with gcc into
    ``oracle/_build/liborc.so`` (single thread: the tests and the CPU baseline) and, on
    request (``use_openmp``), into ``liborc_omp.so`` with the row conditionals split over
    threads (same results; the all-core timing).
  * this module       -- ctypes bindings, the I x J grid planning (Section 3, Fig. 1), the
    per-subset CSR/CSC lists, and the stage orchestration of Algorithm 1 (Section 4.1) with
    the stage-wise hyperparameter rule of Section 5.1.

Readings of points the paper leaves open (each is a documented convention shared with the
library's public header, not shared code):
  * rows/columns are reordered by decreasing number of training observations, ties by
    original index (Section 5.2, "row/column order: decreasing");
  * subset (i, j) has id s = i*J + j (0-based); stage 1 is (0,0), stage 2 has exactly one of
    i, j equal to 0, stage 3 the rest (Eqs. 10-12);
  * a propagated factor starts its chain at the propagated mean, a non-propagated factor at
    the caller's initial state;
  * the draw buffer of one sweep of one stage is [hyper blocks][zX][zW]: one hyperparameter
    block of K(K+3)/2 numbers for X then one for W for every subset of the stage in id order
    (a block for a propagated factor is present but unused), then the standard normals of all
    stacked X rows, then those of all stacked W rows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_SO_OMP = os.path.join(_BUILD, "liborc_omp.so")
_SRC = os.path.join(_HERE, "bmf_oracle.c")
_lib = None
_openmp = False

ORC_OK, ORC_NOT_PD = 0, 1


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the C core with gcc (FP contraction off so results do not depend on the
    host's FMA support); ``openmp`` builds the variant whose row conditionals run on all
    cores."""
    os.makedirs(_BUILD, exist_ok=True)
    so = _SO_OMP if openmp else _SO
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(_SRC):
        tmp = so + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared"]
                              + (["-fopenmp"] if openmp else []) + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, so)
    return so


def use_openmp(on: bool = True) -> int:
    """Switch this process to the OpenMP build (or back); returns the thread count the row
    conditionals use (1 for the serial build).  Results do not change."""
    global _lib, _openmp
    if on != _openmp:
        _lib, _openmp = None, on
    if not on:
        return 1
    build(openmp=True)
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def lib():
    global _lib
    if _lib is None:
        so = build(openmp=_openmp)
        L = ctypes.CDLL(so)
        P = ctypes.c_void_p
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.orc_nw_posterior.argtypes = [i32, i64, P, P, f64, f64, P, P, P, P, P, P, P]
        L.orc_nw_draw.argtypes = [i32, P, f64, P, P, P, P, P, P]
        L.orc_update_rows.argtypes = [i32, i64, P, P, P, P, f64, P, P, i32, P, P, P, P, P]
        L.orc_sweep.argtypes = [i32, i64, i64, P, P, P, P, P, P, f64, P, f64, f64, P,
                                i32, P, P, i32, P, P, P, P, P, P, P, P, P,
                                i32, f64, f64, P, P, P]
        L.orc_noise_update.argtypes = [i32, i64, P, P, P, P, P, i32, f64, f64, P, P]
        L.orc_gen_noise.argtypes = [ctypes.c_uint64, i64, i32, i64, P, P]
        L.orc_moments_accumulate.argtypes = [i32, i64, P, P, P]
        L.orc_moments_accumulate.restype = None
        L.orc_mm_finalize.argtypes = [i32, i64, i64, P, P, P, P, P]
        L.orc_aggregate.argtypes = [i32, i64, i32, P, P, f64, P, P, P, P]
        L.orc_min_eig.argtypes = [i32, P]
        L.orc_min_eig.restype = f64
        L.orc_predict.argtypes = [i32, i64, P, P, P, P, f64, P]
        L.orc_predict.restype = None
        L.orc_logjoint_grad.argtypes = [i32, i64, i64, i64, P, P, P, P, P, f64, P, P, P, P,
                                        P, P, P, P]
        L.orc_logjoint_grad.restype = None
        L.orc_philox4x64.argtypes = [P, P, P]
        L.orc_philox4x64.restype = None
        L.orc_gen_subset.argtypes = [ctypes.c_uint64, i64, i32, i32, f64, i64, i64, P, P, P, P]
        L.orc_lambda_means.argtypes = [i32, i32, P, f64, i32, P]
        L.orc_fit_summaries.argtypes = [i32, i64, i32, P, i32, i32, f64, P, P, P, P, P, P]
        L.orc_mix_choose.argtypes = [i32, i64, i32, P, P, P, P, P, P, P]
        _lib = L
    return _lib


def _p(a):
    """Pointer of a C-contiguous numpy array (None -> NULL)."""
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    pass


def _check(st, what):
    if st != ORC_OK:
        raise OracleError(f"{what}: status {st}")


# ---------------------------------------------------------------------------------------
# Normal-Wishart prior and the hyperparameter step (Section 5.1 and its footnote)
# ---------------------------------------------------------------------------------------

@dataclass
class NWPrior:
    """Normal-Wishart hyperprior (mu0, beta0, nu0, W0).  The paper does not state the
    values; the defaults are the usual BPMF choice mu0 = 0, beta0 = 2, nu0 = K, W0 = I."""
    K: int
    mu0: np.ndarray = None
    beta0: float = 2.0
    nu0: float = None
    W0: np.ndarray = None

    def __post_init__(self):
        if self.mu0 is None:
            self.mu0 = np.zeros(self.K)
        if self.nu0 is None:
            self.nu0 = float(self.K)
        if self.W0 is None:
            self.W0 = np.eye(self.K)
        self.mu0 = _f64(self.mu0)
        self.W0 = _f64(self.W0)


def hyper_block_len(K: int) -> int:
    """chi2[K] + below-diagonal normals K(K-1)/2 + z_mu[K]."""
    return K + K * (K - 1) // 2 + K


def nw_posterior(X, prior: NWPrior):
    X = _f64(X).reshape(-1, prior.K)
    N, K = X.shape
    xbar, Sbar, mus, Wsi = np.zeros(K), np.zeros((K, K)), np.zeros(K), np.zeros((K, K))
    bs, ns = ctypes.c_double(), ctypes.c_double()
    _check(lib().orc_nw_posterior(K, N, _p(X), _p(prior.mu0), prior.beta0, prior.nu0,
                                  _p(prior.W0), _p(xbar), _p(Sbar), _p(mus),
                                  ctypes.byref(bs), ctypes.byref(ns), _p(Wsi)), "nw_posterior")
    return dict(xbar=xbar, Sbar=Sbar, mu_star=mus, beta_star=bs.value, nu_star=ns.value,
                Wstar_inv=Wsi)


def nw_draw(post, hdraw, K):
    nlow = K * (K - 1) // 2
    chi2 = _f64(hdraw[:K]).copy()
    nrm = _f64(hdraw[K:K + nlow]).copy()
    zmu = _f64(hdraw[K + nlow:K + nlow + K]).copy()
    mus = _f64(post["mu_star"])
    wsi = _f64(post["Wstar_inv"])
    mu, Lam = np.zeros(K), np.zeros((K, K))
    _check(lib().orc_nw_draw(K, _p(mus), post["beta_star"], _p(wsi), _p(chi2), _p(nrm),
                             _p(zmu), _p(mu), _p(Lam)), "nw_draw")
    return mu, Lam


def update_rows(ptr, idx, val, P, tau, mu_p, Lam_p, z, per_row_prior=False, tau_partner=None,
                tau_row=None):
    """Draw every row of a CSR block from its Gaussian conditional (see bmf_oracle.c); the
    noise precision of an entry is tau_partner[partner], tau_row[row] or tau."""
    mu_p, Lam_p, z = _f64(mu_p), _f64(Lam_p), _f64(z)
    K = mu_p.shape[-1]
    P = _f64(P).reshape(-1, K)
    ptr = np.ascontiguousarray(ptr, np.int64)
    idx = np.ascontiguousarray(idx, np.int32)
    val = _f64(val)
    R = len(ptr) - 1
    out = np.zeros((R, K))
    bad = ctypes.c_int64(-1)
    tp = None if tau_partner is None else _f64(tau_partner)
    tr = None if tau_row is None else _f64(tau_row)
    st = lib().orc_update_rows(K, R, _p(ptr), _p(idx), _p(val), _p(P), tau, _p(tp), _p(tr),
                               int(per_row_prior), _p(mu_p), _p(Lam_p), _p(z), _p(out),
                               ctypes.byref(bad))
    if st:
        raise OracleError(f"update_rows: row {bad.value} not positive definite")
    return out


@dataclass
class NoiseModel:
    """Sampled noise precision (Section 2.1): mode "global" (one precision per chain) or
    "column" (one per column, tau_d), Gamma(a0, b0) priors (shape, rate), chains starting at
    tau0."""
    mode: str
    a0: float
    b0: float
    tau0: float

    @property
    def code(self):
        return {"fixed": 0, "global": 1, "column": 2}[self.mode]


def noise_update(cptr, cidx, cval, X, W, mode, a0, b0, draw):
    """The noise precisions given the new X, W and their chi-square variates (see
    orc_noise_update); returns tau per column."""
    X, W = _f64(X), _f64(W)
    D, K = W.shape
    tau = np.zeros(D)
    lib().orc_noise_update(K, D, _p(np.ascontiguousarray(cptr, np.int64)),
                           _p(np.ascontiguousarray(cidx, np.int32)), _p(_f64(cval)), _p(X), _p(W),
                           {"global": 1, "column": 2}[mode], float(a0), float(b0), _p(_f64(draw)),
                           _p(tau))
    return tau


def noise_dofs(sub, noise: NoiseModel):
    """Degrees of freedom of a subset's noise variates: 2 a0 + n_d per column, or 2 a0 + the
    subset's entries."""
    counts = np.diff(sub.cptr).astype(np.float64)
    if noise.mode == "column":
        return 2.0 * noise.a0 + counts
    return np.array([2.0 * noise.a0 + counts.sum()])


def mm_finalize(S1, S2, S):
    S1, S2 = _f64(S1), _f64(S2)
    R, K = S1.shape
    mu, Lam = np.zeros((R, K)), np.zeros((R, K, K))
    bad = ctypes.c_int64(-1)
    st = lib().orc_mm_finalize(K, R, int(S), _p(S1), _p(S2), _p(mu), _p(Lam), ctypes.byref(bad))
    if st:
        raise OracleError(f"mm_finalize: row {bad.value} covariance not positive definite")
    return mu, Lam


def aggregate(mu, Lam, eps_rel=1e-6):
    """Algorithm 2 over J submodels: mu [J, R, K], Lam [J, R, K, K]; submodel 0 is the
    propagated one."""
    mu, Lam = _f64(mu), _f64(Lam)
    J, R, K = mu.shape
    mus, Ls = np.zeros((R, K)), np.zeros((R, K, K))
    ncorr, bad = ctypes.c_int64(0), ctypes.c_int64(-1)
    st = lib().orc_aggregate(K, R, J, _p(mu), _p(Lam), eps_rel, _p(mus), _p(Ls),
                             ctypes.byref(ncorr), ctypes.byref(bad))
    if st:
        raise OracleError(f"aggregate: row {bad.value} not positive definite")
    return mus, Ls, ncorr.value


def min_eig(M):
    M = _f64(M)
    return lib().orc_min_eig(M.shape[0], _p(M))


def predict(row, col, Xm, Wm, offset=0.0):
    Xm, Wm = _f64(Xm), _f64(Wm)
    K = Xm.shape[1]
    row = np.ascontiguousarray(row, np.int32)
    col = np.ascontiguousarray(col, np.int32)
    out = np.zeros(len(row))
    lib().orc_predict(K, len(row), _p(row), _p(col), _p(Xm), _p(Wm), float(offset), _p(out))
    return out


def logjoint_grad(row, col, val, X, W, log_a, muX, LamX, muW, LamW):
    X, W = _f64(X), _f64(W)
    muX, LamX, muW, LamW = _f64(muX), _f64(LamX), _f64(muW), _f64(LamW)
    N, K = X.shape
    D = W.shape[0]
    row = np.ascontiguousarray(row, np.int32)
    col = np.ascontiguousarray(col, np.int32)
    val = _f64(val)
    gX, gW = np.zeros_like(X), np.zeros_like(W)
    ga, v = ctypes.c_double(), ctypes.c_double()
    lib().orc_logjoint_grad(K, N, D, len(row), _p(row), _p(col), _p(val), _p(X), _p(W),
                            float(log_a), _p(muX), _p(LamX), _p(muW), _p(LamW), _p(gX), _p(gW),
                            ctypes.byref(ga), ctypes.byref(v))
    return gX, gW, ga.value, v.value


# ---------------------------------------------------------------------------------------
# Grid planning (Section 3: an I x J partition of rows and columns; Section 5.2 ordering)
# ---------------------------------------------------------------------------------------

def density_order(counts):
    """New-to-old permutation sorting by decreasing count, ties by original index."""
    counts = np.asarray(counts, np.int64)
    return np.lexsort((np.arange(len(counts)), -counts)).astype(np.int64)


def equal_bounds(n, parts):
    return np.array([(i * n) // parts for i in range(parts + 1)], np.int64)


def _csr(nrows, r, c, v):
    """CSR of a COO block, entries of a row sorted by column index."""
    o = np.lexsort((c, r))
    r, c, v = r[o], c[o], v[o]
    ptr = np.zeros(nrows + 1, np.int64)
    np.add.at(ptr, r + 1, 1)
    return np.cumsum(ptr), c.astype(np.int32), v.astype(np.float64)


@dataclass
class Subset:
    sid: int
    i: int
    j: int
    stage: int
    r0: int
    r1: int
    c0: int
    c1: int
    rptr: np.ndarray = None
    ridx: np.ndarray = None
    rval: np.ndarray = None
    cptr: np.ndarray = None
    cidx: np.ndarray = None
    cval: np.ndarray = None

    @property
    def n(self):
        return self.r1 - self.r0

    @property
    def d(self):
        return self.c1 - self.c0

    @property
    def nnz(self):
        return int(self.rptr[-1])


@dataclass
class Plan:
    N: int
    D: int
    I: int
    J: int
    row_perm: np.ndarray      # new -> old
    col_perm: np.ndarray
    row_bounds: np.ndarray    # in the new order
    col_bounds: np.ndarray
    offset: float             # training mean, subtracted from the values
    subsets: list = field(default_factory=list)

    def stage_subsets(self, stage):
        return [s for s in self.subsets if s.stage == stage]


def subset_stage(i, j):
    if i == 0 and j == 0:
        return 1
    if i == 0 or j == 0:
        return 2
    return 3


def plan(N, D, row, col, val, I=1, J=1, order="decreasing", row_bounds=None, col_bounds=None,
         center=True):
    """Reorder, split into the I x J grid and build per-subset CSR (rows) and CSC (columns)
    with local indices.  Values are centred by the training mean when ``center``."""
    row = np.asarray(row, np.int64)
    col = np.asarray(col, np.int64)
    val = np.asarray(val, np.float64)
    if order == "decreasing":
        rperm = density_order(np.bincount(row, minlength=N))
        cperm = density_order(np.bincount(col, minlength=D))
    else:
        rperm = np.arange(N, dtype=np.int64)
        cperm = np.arange(D, dtype=np.int64)
    rrank = np.empty(N, np.int64)
    rrank[rperm] = np.arange(N)
    crank = np.empty(D, np.int64)
    crank[cperm] = np.arange(D)
    rb = equal_bounds(N, I) if row_bounds is None else np.asarray(row_bounds, np.int64)
    cb = equal_bounds(D, J) if col_bounds is None else np.asarray(col_bounds, np.int64)
    offset = float(val.sum() / len(val)) if (center and len(val)) else 0.0
    v = val - offset
    nr, nc = rrank[row], crank[col]
    bi = np.searchsorted(rb, nr, side="right") - 1
    bj = np.searchsorted(cb, nc, side="right") - 1
    P = Plan(N, D, I, J, rperm, cperm, rb, cb, offset)
    for i in range(I):
        for j in range(J):
            m = (bi == i) & (bj == j)
            s = Subset(i * J + j, i, j, subset_stage(i, j), int(rb[i]), int(rb[i + 1]),
                       int(cb[j]), int(cb[j + 1]))
            lr, lc, lv = nr[m] - rb[i], nc[m] - cb[j], v[m]
            s.rptr, s.ridx, s.rval = _csr(s.n, lr, lc, lv)
            s.cptr, s.cidx, s.cval = _csr(s.d, lc, lr, lv)
            P.subsets.append(s)
    return P


# ---------------------------------------------------------------------------------------
# Draw buffer layout (shared convention; see the module docstring)
# ---------------------------------------------------------------------------------------

def stage_draw_layout(subsets, K, noise: NoiseModel = None):
    """Offsets of one sweep's draws for a list of subsets processed together; with sampled
    noise, each subset's noise variates follow the z's (one per column, or one)."""
    H = hyper_block_len(K)
    lay = {}
    off = 0
    for s in subsets:
        lay[(s.sid, "hx")] = off
        lay[(s.sid, "hw")] = off + H
        off += 2 * H
    for s in subsets:
        lay[(s.sid, "zx")] = off
        off += s.n * K
    for s in subsets:
        lay[(s.sid, "zw")] = off
        off += s.d * K
    if noise is not None and noise.mode != "fixed":
        for s in subsets:
            lay[(s.sid, "nz")] = off
            off += s.d if noise.mode == "column" else 1
    lay["total"] = off
    return lay


# ---------------------------------------------------------------------------------------
# Counter-based draws (Philox4x64-10, Box-Muller, Marsaglia-Tsang; see bmf_oracle.c)
# ---------------------------------------------------------------------------------------

def philox4x64(ctr, key):
    """The four 64-bit output words of Philox4x64-10 at counter ctr[4], key key[2]."""
    c = np.asarray(ctr, np.uint64)
    k = np.asarray(key, np.uint64)
    out = np.zeros(4, np.uint64)
    lib().orc_philox4x64(_p(c), _p(k), _p(out))
    return out


def gen_subset(seed, t, sid, K, nu0, n, d):
    """Generated draws of sweep t (1-based) of subset sid with n rows, d columns:
    (hyper block X, hyper block W, zX [n, K], zW [d, K])."""
    H = hyper_block_len(K)
    hx, hw = np.zeros(H), np.zeros(H)
    zx, zw = np.zeros((n, K)), np.zeros((d, K))
    _check(lib().orc_gen_subset(int(seed), int(t), int(sid), int(K), float(nu0), int(n), int(d),
                                _p(hx), _p(hw), _p(zx), _p(zw)), "gen_subset")
    return hx, hw, zx, zw


def gen_noise(seed, t, sid, dof):
    """The noise-precision chi-square variates of sweep t of subset sid (orc_gen_noise)."""
    dof = _f64(dof)
    out = np.zeros(len(dof))
    _check(lib().orc_gen_noise(int(seed), int(t), int(sid), len(dof), _p(dof), _p(out)),
           "gen_noise")
    return out


def gen_batch_draws(subsets, K, nu0, seed, t, noise: NoiseModel = None):
    """One sweep's generated draws for subsets processed together, in the shared layout."""
    parts = [gen_subset(seed, t, s.sid, K, nu0, s.n, s.d) for s in subsets]
    tail = []
    if noise is not None and noise.mode != "fixed":
        tail = [gen_noise(seed, t, s.sid, noise_dofs(s, noise)) for s in subsets]
    return np.concatenate([np.concatenate([p[0], p[1]]) for p in parts]
                          + [p[2].ravel() for p in parts] + [p[3].ravel() for p in parts] + tail)


# ---------------------------------------------------------------------------------------
# Per-subset chain state and Algorithm 1
# ---------------------------------------------------------------------------------------

@dataclass
class ChainState:
    X: np.ndarray
    W: np.ndarray
    muX: np.ndarray
    LamX: np.ndarray
    muW: np.ndarray
    LamW: np.ndarray
    prior_x: int = 0            # 1 = per-row propagated prior on X
    prior_w: int = 0
    muX_row: np.ndarray = None
    LamX_row: np.ndarray = None
    muW_row: np.ndarray = None
    LamW_row: np.ndarray = None
    S1X: np.ndarray = None
    S2X: np.ndarray = None
    S1W: np.ndarray = None
    S2W: np.ndarray = None
    n_kept: int = 0
    t: int = 0                   # sweeps done
    samples_X: list = None       # retained samples (kept for the DM / GMM summaries only)
    samples_W: list = None
    mixX: dict = None            # propagated mixture prior (GMM summary): pi, mu, Lam per row
    mixW: dict = None
    tau_col: np.ndarray = None   # sampled noise precision per column (None: the fixed tau)


def new_chain(X0, W0, K):
    X0, W0 = _f64(X0).copy(), _f64(W0).copy()
    N, D = X0.shape[0], W0.shape[0]
    return ChainState(X0, W0, np.zeros(K), np.eye(K), np.zeros(K), np.eye(K),
                      S1X=np.zeros((N, K)), S2X=np.zeros((N, K, K)),
                      S1W=np.zeros((D, K)), S2W=np.zeros((D, K, K)))


def sweep_subset(sub: Subset, st: ChainState, K, tau, prior: NWPrior, hx, hw, zX, zW,
                 noise: NoiseModel = None, noise_draw=None):
    """One Gibbs sweep of one subset (order: Theta_X, Theta_W, X, W, then the sampled noise
    precision when ``noise`` is given)."""
    hyper = np.concatenate([st.muX, st.LamX.ravel(), st.muW, st.LamW.ravel()])
    bad = ctypes.c_int64(-1)
    X, W = st.X, st.W
    hx, hw, zX, zW = _f64(hx).copy(), _f64(hw).copy(), _f64(zX).copy(), _f64(zW).copy()
    nmode = 0 if noise is None else noise.code
    if nmode and st.tau_col is None:
        st.tau_col = np.full(sub.d, float(noise.tau0))
    nd = None if not nmode else _f64(noise_draw).copy()
    st_ = lib().orc_sweep(K, sub.n, sub.d, _p(sub.rptr), _p(sub.ridx), _p(sub.rval),
                          _p(sub.cptr), _p(sub.cidx), _p(sub.cval), float(tau),
                          _p(prior.mu0), prior.beta0, prior.nu0, _p(prior.W0),
                          st.prior_x, _p(st.muX_row), _p(st.LamX_row),
                          st.prior_w, _p(st.muW_row), _p(st.LamW_row),
                          _p(hx), _p(hw), _p(zX), _p(zW),
                          _p(X), _p(W), _p(hyper), nmode,
                          float(noise.a0) if nmode else 0.0, float(noise.b0) if nmode else 0.0,
                          _p(nd), _p(st.tau_col if nmode else None), ctypes.byref(bad))
    if st_:
        raise OracleError(f"sweep of subset {sub.sid}: status {st_}, row {bad.value}")
    KK = K * K
    st.muX, st.LamX = hyper[:K].copy(), hyper[K:K + KK].reshape(K, K).copy()
    st.muW, st.LamW = hyper[K + KK:2 * K + KK].copy(), hyper[2 * K + KK:].reshape(K, K).copy()
    st.t += 1


def keep_sample(t, burnin, thin):
    """Sweep t (1-based count of sweeps done) is retained after burn-in, every thin-th."""
    return t > burnin and (t - burnin - 1) % thin == 0


def accumulate(st: ChainState):
    L = lib()
    K = st.X.shape[1]
    L.orc_moments_accumulate(K, st.X.shape[0], _p(st.X), _p(st.S1X), _p(st.S2X))
    L.orc_moments_accumulate(K, st.W.shape[0], _p(st.W), _p(st.S1W), _p(st.S2W))
    st.n_kept += 1
    if st.samples_X is not None:
        st.samples_X.append(st.X.copy())
        st.samples_W.append(st.W.copy())


# ---------------------------------------------------------------------------------------
# Dominant-mode and mixture summaries (Section 4.1 "PP DM" / "PP GMM", Section 5.1)
# ---------------------------------------------------------------------------------------
SUMMARY_MODES = {"mm": 0, "dm": 1, "gmm": 2}


def lambda_means(x, lam, max_iter=100):
    """lambda-means clustering of the rows of x (S x K) with squared-distance penalty lam;
    returns (cluster of each row, number of clusters)."""
    x = _f64(x)
    S, K = x.shape
    assign = np.zeros(max(S, 1), np.int32)
    n = lib().orc_lambda_means(K, S, _p(x), float(lam), int(max_iter), _p(assign))
    if n < 0:
        raise OracleError("lambda-means: out of memory")
    return assign[:S], n


def fit_summaries(samples, mode, lam=0.0, C=3):
    """Per-row summaries of retained samples [S][R][K] (see orc_fit_summaries):
    pi [R][C], mu [R][C][K], Lam [R][C][K][K], pooled_mu [R][K], pooled_Lam [R][K][K]."""
    samples = _f64(samples)
    S, R, K = samples.shape
    C = 1 if mode in ("mm", "dm") else int(C)
    out = dict(pi=np.zeros((R, C)), mu=np.zeros((R, C, K)), Lam=np.zeros((R, C, K, K)),
               pooled_mu=np.zeros((R, K)), pooled_Lam=np.zeros((R, K, K)))
    bad = ctypes.c_int64(-1)
    st = lib().orc_fit_summaries(K, R, S, _p(samples), SUMMARY_MODES[mode], C, float(lam),
                                 _p(out["pi"]), _p(out["mu"]), _p(out["Lam"]),
                                 _p(out["pooled_mu"]), _p(out["pooled_Lam"]), ctypes.byref(bad))
    _check(st, f"fit_summaries({mode}) row {bad.value}")
    return out


def mix_choose(mix, X):
    """Component of each row's mixture prior with the largest responsibility at X; returns
    (chosen, mu_rows [R][K], Lam_rows [R][K][K])."""
    X = _f64(X)
    R, K = X.shape
    C = mix["pi"].shape[1]
    chosen = np.zeros(max(R, 1), np.int32)
    mu_out, Lam_out = np.zeros((R, K)), np.zeros((R, K, K))
    st = lib().orc_mix_choose(K, R, C, _p(_f64(mix["pi"])), _p(_f64(mix["mu"])),
                              _p(_f64(mix["Lam"])), _p(X), _p(chosen), _p(mu_out), _p(Lam_out))
    _check(st, "mix_choose")
    return chosen[:R], mu_out, Lam_out


def run_stage(plan_: Plan, stage, chains: dict, K, tau, prior, draws_per_sweep, T, burnin=0,
              thin=1, noise: NoiseModel = None):
    """T sweeps of every subset of one stage.  ``draws_per_sweep(t)`` returns the stage's
    draw buffer of sweep t (0-based)."""
    subs = plan_.stage_subsets(stage)
    lay = stage_draw_layout(subs, K, noise)
    sampled = noise is not None and noise.mode != "fixed"
    for t in range(T):
        dr = np.asarray(draws_per_sweep(t), np.float64)
        assert dr.shape == (lay["total"],), (dr.shape, lay["total"])
        H = hyper_block_len(K)
        for s in subs:
            st = chains[s.sid]
            # a propagated mixture prior: each row's component is chosen at its current value
            # (X is unchanged until its own update, W likewise, so choosing both here is the
            # same as choosing right before each factor's draws)
            if st.mixX is not None:
                _, st.muX_row, st.LamX_row = mix_choose(st.mixX, st.X)
            if st.mixW is not None:
                _, st.muW_row, st.LamW_row = mix_choose(st.mixW, st.W)
            nz = None
            if sampled:
                m = s.d if noise.mode == "column" else 1
                nz = dr[lay[(s.sid, "nz")]:lay[(s.sid, "nz")] + m]
            sweep_subset(s, st, K, tau, prior,
                         dr[lay[(s.sid, "hx")]:lay[(s.sid, "hx")] + H],
                         dr[lay[(s.sid, "hw")]:lay[(s.sid, "hw")] + H],
                         dr[lay[(s.sid, "zx")]:lay[(s.sid, "zx")] + s.n * K],
                         dr[lay[(s.sid, "zw")]:lay[(s.sid, "zw")] + s.d * K],
                         noise if sampled else None, nz)
            if keep_sample(st.t, burnin, thin):
                accumulate(st)


def finalize(st: ChainState, summary="mm", lam=0.0, C=3):
    """Per-row (mu, Lambda) of X and of W of one subset: moment matched (summary "mm"), of
    the dominant lambda-means mode ("dm"), or the pooled moments of the fitted mixture ("gmm",
    whose components are returned too, for propagation).  Returns (mx, Lx, mw, Lw) for "mm",
    (mx, Lx, mw, Lw, mixX, mixW) otherwise (mix* None for "dm")."""
    if summary == "mm":
        mx, Lx = mm_finalize(st.S1X, st.S2X, st.n_kept)
        mw, Lw = mm_finalize(st.S1W, st.S2W, st.n_kept)
        return mx, Lx, mw, Lw
    fx = fit_summaries(np.stack(st.samples_X), summary, lam, C)
    fw = fit_summaries(np.stack(st.samples_W), summary, lam, C)
    if summary == "dm":
        return fx["mu"][:, 0], fx["Lam"][:, 0], fw["mu"][:, 0], fw["Lam"][:, 0], None, None
    return (fx["pooled_mu"], fx["pooled_Lam"], fw["pooled_mu"], fw["pooled_Lam"],
            dict(pi=fx["pi"], mu=fx["mu"], Lam=fx["Lam"]),
            dict(pi=fw["pi"], mu=fw["mu"], Lam=fw["Lam"]))


def setup_stage_chains(plan_: Plan, stage, X0, W0, K, finals: dict, summary="mm",
                       propagate=True):
    """Chains of one stage.  X0/W0 are the caller's initial states in the reordered index
    space.  Propagated priors (Algorithm 1):
      stage 2, (i,0): W^(0) from subset (0,0);  (0,j): X^(0) from subset (0,0);
      stage 3, (i,j): X^(i) from subset (i,0), W^(j) from subset (0,j).
    propagate=False: every subset keeps the standard priors and starts at the initial state
    (embarrassingly parallel MCMC, the baseline of Sections 5.4 and 5.6)."""
    J = plan_.J
    chains = {}
    for s in plan_.stage_subsets(stage):
        st = new_chain(X0[s.r0:s.r1], W0[s.c0:s.c1], K)
        if summary != "mm":
            st.samples_X, st.samples_W = [], []
        src_x = src_w = None
        if not propagate:
            pass
        elif stage == 2:
            if s.j == 0:
                src_w = 0                  # subset (0,0)
            else:
                src_x = 0
        elif stage == 3:
            src_x = s.i * J + 0            # subset (i,0)
            src_w = 0 * J + s.j            # subset (0,j)
        if src_x is not None:
            mx, Lx = finals[src_x][0], finals[src_x][1]
            st.prior_x, st.muX_row, st.LamX_row = 1, mx.copy(), Lx.copy()
            st.X = mx.copy()
            if summary == "gmm":
                st.mixX = finals[src_x][4]        # chain starts at the mixture's mean
        if src_w is not None:
            mw, Lw = finals[src_w][2], finals[src_w][3]
            st.prior_w, st.muW_row, st.LamW_row = 1, mw.copy(), Lw.copy()
            st.W = mw.copy()
            if summary == "gmm":
                st.mixW = finals[src_w][5]
        chains[s.sid] = st
    return chains


def aggregate_plan(plan_: Plan, finals: dict, K, eps_rel=1e-6):
    """Eq. 14 / Algorithm 2 for every row block of X and column block of W.
    X^(i): submodel (1) is subset (i,0), the others (i,j), j >= 1.
    W^(j): submodel (1) is subset (0,j), the others (i,j), i >= 1.
    Returns posterior means (in the reordered index space) and the correction count."""
    I, J = plan_.I, plan_.J
    Xm = np.zeros((plan_.N, K))
    Wm = np.zeros((plan_.D, K))
    nc = 0
    for i in range(I):
        sids = [i * J + j for j in range(J)]
        mu = np.stack([finals[s][0] for s in sids])
        Lam = np.stack([finals[s][1] for s in sids])
        m, _, c = aggregate(mu, Lam, eps_rel)
        Xm[plan_.row_bounds[i]:plan_.row_bounds[i + 1]] = m
        nc += c
    for j in range(J):
        sids = [i * J + j for i in range(I)]
        mu = np.stack([finals[s][2] for s in sids])
        Lam = np.stack([finals[s][3] for s in sids])
        m, _, c = aggregate(mu, Lam, eps_rel)
        Wm[plan_.col_bounds[j]:plan_.col_bounds[j + 1]] = m
        nc += c
    return Xm, Wm, nc


def pp_run(plan_: Plan, K, tau, prior, X0, W0, draws_fn, T, burnin, thin, eps_rel=1e-6,
           summary="mm", lam=0.0, C=3, propagate=True):
    """Algorithm 1: stages I, II, III (each stage's subsets in id order), then Algorithm 2.
    ``draws_fn(stage, t)`` gives the stage's draw buffer for sweep t.  X0/W0 are in the
    reordered index space.  ``summary``: the approximation propagated between stages and
    aggregated -- "mm" moment matching, "dm" dominant mode, "gmm" mixture of the C largest
    lambda-means modes (penalty ``lam``), propagated as a mixture prior whose component is
    chosen by responsibility before each draw and aggregated through its pooled moments.
    Returns the aggregated posterior means, the per-subset finals and the chains."""
    finals, all_chains = {}, {}
    for stage in (1, 2, 3):
        subs = plan_.stage_subsets(stage)
        if not subs:
            continue
        chains = setup_stage_chains(plan_, stage, X0, W0, K, finals, summary, propagate)
        run_stage(plan_, stage, chains, K, tau, prior, lambda t: draws_fn(stage, t), T,
                  burnin, thin)
        for sid, st in chains.items():
            finals[sid] = finalize(st, summary, lam, C)
        all_chains.update(chains)
    Xm, Wm, nc = aggregate_plan(plan_, finals, K, eps_rel)
    return dict(Xm=Xm, Wm=Wm, finals=finals, chains=all_chains, n_corrected=nc)


def rmse(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.sqrt(np.mean((a - b) ** 2))) if len(a) else 0.0
