"""Thin ctypes binding of libbmf.so (include/bmf.h): argument marshalling only.  Every step of
the sampler runs in the CUDA library; nothing here computes.  Loading fails loudly when the
library has not been built (``python paper_1703_00734_gb300/build.py``)."""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbmf.so")

BMF_FP64, BMF_FP32, BMF_BF16, BMF_TF32 = 0, 1, 2, 3
PRECISION = {"fp64": BMF_FP64, "fp32": BMF_FP32, "bf16": BMF_BF16, "tf32": BMF_TF32}
ORDER = {"none": 0, "decreasing": 1}
MOMENTS = {"auto": 0, "mean": 1, "full": 2}
SUMMARY = {"mm": 0, "dm": 1, "gmm": 2}
NOISE = {"fixed": 0, "global": 1, "column": 2}
FACTOR_X, FACTOR_W = 0, 1
STATUS = {0: "BMF_OK", 1: "BMF_E_ARG", 2: "BMF_E_SHAPE", 3: "BMF_E_NOT_PD",
          4: "BMF_E_NONFINITE", 5: "BMF_E_TIMEOUT", 6: "BMF_E_OOM", 7: "BMF_E_CUDA",
          8: "BMF_E_STATE"}


class BmfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("precision", ctypes.c_int32), ("tau", ctypes.c_double),
                ("beta0", ctypes.c_double), ("nu0", ctypes.c_double),
                ("mu0", ctypes.POINTER(ctypes.c_double)), ("W0", ctypes.POINTER(ctypes.c_double)),
                ("order", ctypes.c_int32), ("center", ctypes.c_int32), ("burnin", ctypes.c_int32),
                ("thin", ctypes.c_int32), ("seed", ctypes.c_uint64), ("eps_rel", ctypes.c_double),
                ("moments", ctypes.c_int32), ("summary", ctypes.c_int32),
                ("components", ctypes.c_int32), ("lam", ctypes.c_double),
                ("max_samples", ctypes.c_int32), ("independent", ctypes.c_int32),
                ("noise", ctypes.c_int32), ("noise_a0", ctypes.c_double),
                ("noise_b0", ctypes.c_double)]


class Draws(ctypes.Structure):
    _fields_ = [("ptr", ctypes.c_void_p), ("len", ctypes.c_int64), ("on_device", ctypes.c_int32)]


class SweepStats(ctypes.Structure):
    _fields_ = [("rmse_sample", ctypes.c_double), ("rmse_mean", ctypes.c_double),
                ("sweeps", ctypes.c_int64), ("kept", ctypes.c_int64)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 16), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double)]


class Schedule(ctypes.Structure):
    _fields_ = [("chunks_x", ctypes.c_int32), ("chunks_w", ctypes.c_int32),
                ("gram_blocks_per_sm", ctypes.c_int32), ("row_weight", ctypes.c_double),
                ("graph", ctypes.c_int32), ("cond_lanes", ctypes.c_int32)]


def _sched_dict(sc):
    return dict(chunks_x=sc.chunks_x, chunks_w=sc.chunks_w,
                gram_blocks_per_sm=sc.gram_blocks_per_sm, row_weight=sc.row_weight,
                graph=sc.graph, cond_lanes=sc.cond_lanes)


class SubsetInfo(ctypes.Structure):
    _fields_ = [("i", ctypes.c_int32), ("j", ctypes.c_int32), ("stage", ctypes.c_int32),
                ("row0", ctypes.c_int64), ("row1", ctypes.c_int64), ("col0", ctypes.c_int64),
                ("col1", ctypes.c_int64), ("nnz", ctypes.c_int64)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libbmf.so and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(path)
    P, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    st = ctypes.c_int
    L.bmf_init.argtypes = [ctypes.POINTER(P), ctypes.POINTER(Config), i64, i64, i64, P, P, P, i32, P,
                           i32, P, P, P, i64, P, P, P, P]
    L.bmf_init.restype = st
    L.bmf_draws_per_sweep.argtypes = [P, i32, i32]
    L.bmf_draws_per_sweep.restype = i64
    L.bmf_sweep.argtypes = [P, i32, i32, ctypes.POINTER(Draws), ctypes.POINTER(SweepStats)]
    L.bmf_sweep.restype = st
    L.bmf_stage.argtypes = [P, i32, i32, ctypes.POINTER(Draws), ctypes.POINTER(SweepStats)]
    L.bmf_stage.restype = st
    L.bmf_predict.argtypes = [P, i64, P, P, P, P, P]
    L.bmf_predict.restype = st
    L.bmf_test_rmse.argtypes = [P, ctypes.POINTER(f64)]
    L.bmf_test_rmse.restype = st
    L.bmf_restart.argtypes = [P, P, P, ctypes.c_uint64]
    L.bmf_restart.restype = st
    L.bmf_posterior_means.argtypes = [P, P, P, ctypes.POINTER(i64)]
    L.bmf_posterior_means.restype = st
    L.bmf_get_state.argtypes = [P, i32, P, P, P]
    L.bmf_get_state.restype = st
    L.bmf_set_state.argtypes = [P, i32, P, P]
    L.bmf_set_state.restype = st
    L.bmf_get_moments.argtypes = [P, i32, i32, P, P, ctypes.POINTER(i64)]
    L.bmf_get_moments.restype = st
    L.bmf_get_posterior.argtypes = [P, i32, i32, P, P]
    L.bmf_get_posterior.restype = st
    L.bmf_set_prior.argtypes = [P, i32, i32, P, P]
    L.bmf_set_prior.restype = st
    L.bmf_get_noise.argtypes = [P, i32, P]
    L.bmf_get_noise.restype = st
    L.bmf_get_subset_info.argtypes = [P, i32, ctypes.POINTER(SubsetInfo)]
    L.bmf_get_subset_info.restype = st
    L.bmf_get_perm.argtypes = [P, P, P]
    L.bmf_get_perm.restype = st
    L.bmf_profile_enable.argtypes = [P, i32]
    L.bmf_profile_enable.restype = st
    L.bmf_profile_read.argtypes = [P, ctypes.POINTER(KernelTime), i32]
    L.bmf_profile_read.restype = i32
    L.bmf_launch_count.argtypes = [P]
    L.bmf_launch_count.restype = i64
    L.bmf_logjoint_grad.argtypes = [P, i32, P, P, i64, f64, P, P, ctypes.POINTER(f64),
                                    ctypes.POINTER(f64)]
    L.bmf_logjoint_grad.restype = st
    L.bmf_langevin.argtypes = [P, i32, i32, P, P, i64, f64, f64, P, P, ctypes.POINTER(i32),
                               ctypes.POINTER(f64)]
    L.bmf_langevin.restype = st
    L.bmf_aggregate_static.argtypes = [i32, i64, i32, P, P, f64, P, ctypes.POINTER(i64), P]
    L.bmf_aggregate_static.restype = st
    L.bmf_set_monitor.argtypes = [P, i32]
    L.bmf_set_monitor.restype = st
    L.bmf_set_schedule.argtypes = [P, ctypes.POINTER(Schedule)]
    L.bmf_set_schedule.restype = st
    L.bmf_get_schedule.argtypes = [P, ctypes.POINTER(Schedule)]
    L.bmf_get_schedule.restype = st
    L.bmf_autotune.argtypes = [P, i32, i32, i32, ctypes.POINTER(Schedule)]
    L.bmf_autotune.restype = st
    L.bmf_generate_draws.argtypes = [P, i32, i32, i64, i32, P, i32]
    L.bmf_generate_draws.restype = st
    L.bmf_fit_summaries.argtypes = [i32, i64, i32, P, i32, i32, f64, P, P, P, P, P, P, P]
    L.bmf_fit_summaries.restype = st
    L.bmf_plan.argtypes = [i64, i64, i64, P, P, P, i32, i32, P, i32, P, P, P, P, P, P]
    L.bmf_plan.restype = st
    L.bmf_destroy.argtypes = [P]
    L.bmf_destroy.restype = None
    L.bmf_last_error.argtypes = [P]
    L.bmf_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return None if a is None else a.ctypes.data


def aggregate_static(K, R, J, mu_ptr, lam_ptr, out_ptr, eps_rel=1e-6, stream=None):
    """bmf_aggregate_static on device pointers (see include/bmf.h): Eq. 14 / Algorithm 2 over J
    submodels for R rows, allocating nothing.  Returns the number of corrected pairs."""
    L = load()
    nc = ctypes.c_int64()
    st = L.bmf_aggregate_static(int(K), int(R), int(J), mu_ptr, lam_ptr, float(eps_rel), out_ptr,
                                ctypes.byref(nc), ctypes.c_void_p(stream) if stream else None)
    if st:
        raise BmfError(st, L.bmf_last_error(None).decode())
    return nc.value


def fit_summaries(samples, mode, lam, C=3, stream=None):
    """bmf_fit_summaries on a device tensor of samples [S, R, K] (FP64): per-row dominant-mode /
    mixture / all-sample Gaussian fits (include/bmf.h).  Returns a dict of device tensors
    (pi, mu, Lam, pooled_mu, pooled_Lam, assign)."""
    import torch
    L = load()
    S, R, K = samples.shape
    m = SUMMARY[mode] if isinstance(mode, str) else int(mode)
    C = 1 if m != 2 else int(C)
    dev = samples.device
    f64 = dict(dtype=torch.float64, device=dev)
    out = dict(pi=torch.zeros((R, C), **f64), mu=torch.zeros((R, C, K), **f64),
               Lam=torch.zeros((R, C, K, K), **f64), pooled_mu=torch.zeros((R, K), **f64),
               pooled_Lam=torch.zeros((R, K, K), **f64),
               assign=torch.zeros((R, S), dtype=torch.int32, device=dev))
    x = samples.contiguous()
    st = L.bmf_fit_summaries(int(K), int(R), int(S), x.data_ptr(), m, C, float(lam),
                             out["pi"].data_ptr(), out["mu"].data_ptr(), out["Lam"].data_ptr(),
                             out["pooled_mu"].data_ptr(), out["pooled_Lam"].data_ptr(),
                             out["assign"].data_ptr(), ctypes.c_void_p(stream) if stream else None)
    if st:
        raise BmfError(st, L.bmf_last_error(None).decode())
    return out


def plan(N, D, row, col, val, I=1, J=1, order="decreasing", row_bounds=None, col_bounds=None):
    """The library's host-side preprocessing alone (bmf_plan: no GPU needed): row/column
    order, grid cuts and training entries per subset."""
    L = load()
    row, col, val = _arr(row, np.int32), _arr(col, np.int32), _arr(val, np.float64)
    rb = None if row_bounds is None else _arr(row_bounds, np.int64)
    cb = None if col_bounds is None else _arr(col_bounds, np.int64)
    out = dict(row_perm=np.zeros(N, np.int64), col_perm=np.zeros(D, np.int64),
               row_bounds=np.zeros(I + 1, np.int64), col_bounds=np.zeros(J + 1, np.int64),
               subset_nnz=np.zeros(I * J, np.int64))
    s = L.bmf_plan(N, D, len(row), _ptr(row), _ptr(col), _ptr(val), ORDER[order], I, _ptr(rb), J,
                   _ptr(cb), _ptr(out["row_perm"]), _ptr(out["col_perm"]),
                   _ptr(out["row_bounds"]), _ptr(out["col_bounds"]), _ptr(out["subset_nnz"]))
    if s:
        raise BmfError(s, L.bmf_last_error(None).decode())
    return out


class BMF:
    """One context of the library: the training data split into an I x J grid, one Gibbs chain
    per subset.  Indices are 0-based in the original order."""

    def __init__(self, N, D, row, col, val, K, tau, precision="fp64", I=1, J=1, row_bounds=None,
                 col_bounds=None, X0=None, W0=None, test=None, beta0=2.0, nu0=None, mu0=None,
                 W0_prior=None, order="decreasing", center=True, burnin=0, thin=1, seed=0,
                 eps_rel=1e-6, moments="auto", summary="mm", components=3, lam=0.0,
                 max_samples=0, independent=False, noise="fixed", noise_a0=1.0, noise_b0=1.0,
                 stream=None):
        L = load()
        self.L = L
        self.N, self.D, self.K, self.I, self.J = int(N), int(D), int(K), int(I), int(J)
        self._keep = []
        row, col, val = _arr(row, np.int32), _arr(col, np.int32), _arr(val, np.float64)
        X0 = _arr(np.zeros((N, K)) if X0 is None else X0, np.float64)
        W0 = _arr(np.zeros((D, K)) if W0 is None else W0, np.float64)
        if test is not None:
            tr, tc, tv = (_arr(test[0], np.int32), _arr(test[1], np.int32),
                          _arr(test[2], np.float64))
        else:
            tr = tc = tv = None
        mu0a = None if mu0 is None else _arr(mu0, np.float64)
        W0a = None if W0_prior is None else _arr(W0_prior, np.float64)
        rb = None if row_bounds is None else _arr(row_bounds, np.int64)
        cb = None if col_bounds is None else _arr(col_bounds, np.int64)
        dp = ctypes.POINTER(ctypes.c_double)
        cfg = Config(K=K, precision=PRECISION[precision] if isinstance(precision, str) else precision,
                     tau=float(tau), beta0=float(beta0), nu0=float(nu0 if nu0 is not None else K),
                     mu0=mu0a.ctypes.data_as(dp) if mu0a is not None else None,
                     W0=W0a.ctypes.data_as(dp) if W0a is not None else None,
                     order=ORDER[order], center=int(bool(center)), burnin=int(burnin),
                     thin=int(thin), seed=int(seed), eps_rel=float(eps_rel),
                     moments=MOMENTS[moments], summary=SUMMARY[summary],
                     components=int(components), lam=float(lam), max_samples=int(max_samples),
                     independent=int(bool(independent)), noise=NOISE[noise],
                     noise_a0=float(noise_a0), noise_b0=float(noise_b0))
        self.precision = cfg.precision
        h = ctypes.c_void_p()
        st = L.bmf_init(ctypes.byref(h), ctypes.byref(cfg), N, D, len(row), _ptr(row), _ptr(col),
                        _ptr(val), I, _ptr(rb), J, _ptr(cb), _ptr(X0), _ptr(W0),
                        0 if tr is None else len(tr), _ptr(tr), _ptr(tc), _ptr(tv),
                        ctypes.c_void_p(stream) if stream else None)
        if st:
            raise BmfError(st, L.bmf_last_error(None).decode())
        self.h = h

    # -- helpers --------------------------------------------------------------------------
    def _check(self, st):
        if st:
            raise BmfError(st, self.L.bmf_last_error(self.h).decode())

    @staticmethod
    def _draws(draws):
        if draws is None:
            return None, None
        if hasattr(draws, "data_ptr"):          # a torch tensor
            dev = draws.is_cuda
            d = Draws(ptr=draws.data_ptr(), len=draws.numel(), on_device=int(dev))
            return d, draws
        a = _arr(draws, np.float64)
        return Draws(ptr=a.ctypes.data, len=a.size, on_device=0), a

    @staticmethod
    def _stats(s):
        return dict(rmse_sample=s.rmse_sample, rmse_mean=s.rmse_mean, sweeps=s.sweeps, kept=s.kept)

    # -- API -------------------------------------------------------------------------------
    def draws_per_sweep(self, stage=1, subset=-1):
        return int(self.L.bmf_draws_per_sweep(self.h, stage, subset))

    def set_schedule(self, chunks_x=1, chunks_w=1, gram_blocks_per_sm=4, row_weight=0.0,
                     graph=0, cond_lanes=0):
        """Launch schedule (include/bmf.h, bmf_schedule); the sampled values do not depend on it."""
        sc = Schedule(chunks_x=chunks_x, chunks_w=chunks_w, gram_blocks_per_sm=gram_blocks_per_sm,
                      row_weight=float(row_weight), graph=int(graph), cond_lanes=int(cond_lanes))
        self._check(self.L.bmf_set_schedule(self.h, ctypes.byref(sc)))

    def set_monitor(self, on=True):
        """Per-sweep test-RMSE monitor on or off (bmf_set_monitor); sampled values unchanged."""
        self._check(self.L.bmf_set_monitor(self.h, int(bool(on))))

    def get_schedule(self):
        sc = Schedule()
        self._check(self.L.bmf_get_schedule(self.h, ctypes.byref(sc)))
        return _sched_dict(sc)

    def autotune(self, stage=1, subset=-1, sweeps_per_trial=3):
        """Time candidate launch schedules on a batch and install the fastest (the chains are
        restored; no sampled value changes).  Returns the chosen schedule."""
        sc = Schedule()
        self._check(self.L.bmf_autotune(self.h, stage, subset, int(sweeps_per_trial),
                                        ctypes.byref(sc)))
        return _sched_dict(sc)

    def generate_draws(self, t0, n=1, stage=1, subset=-1, out=None):
        """The device generator's draws of sweeps t0 .. t0 + n - 1 of a batch (stage, or one
        subset).  out: a torch tensor (device or host) or a host numpy array of
        n * draws_per_sweep doubles; without it a new host array is returned."""
        per = self.draws_per_sweep(stage, subset)
        if per < 0:    # invalid batch: the library reports it
            self._check(self.L.bmf_generate_draws(self.h, stage, subset, int(t0), int(n), None, 0))
        if out is not None and hasattr(out, "data_ptr"):      # a torch tensor
            assert out.numel() == n * per and out.dtype.itemsize == 8
            self._check(self.L.bmf_generate_draws(self.h, stage, subset, int(t0), int(n),
                                                  out.data_ptr(), int(out.is_cuda)))
            return out
        if out is not None:                                   # a host numpy array
            assert out.dtype == np.float64 and out.size == n * per and out.flags.c_contiguous
            self._check(self.L.bmf_generate_draws(self.h, stage, subset, int(t0), int(n),
                                                  _ptr(out), 0))
            return out
        a = np.zeros(n * per)
        self._check(self.L.bmf_generate_draws(self.h, stage, subset, int(t0), int(n), _ptr(a), 0))
        return a

    def sweep(self, subset=0, n=1, draws=None):
        d, keep = self._draws(draws)
        s = SweepStats()
        self._check(self.L.bmf_sweep(self.h, subset, n, ctypes.byref(d) if d else None,
                                     ctypes.byref(s)))
        del keep
        return self._stats(s)

    def stage(self, stage, n=1, draws=None):
        d, keep = self._draws(draws)
        s = SweepStats()
        self._check(self.L.bmf_stage(self.h, stage, n, ctypes.byref(d) if d else None,
                                     ctypes.byref(s)))
        del keep
        return self._stats(s)

    def predict(self, row, col, y=None):
        row, col = _arr(row, np.int32), _arr(col, np.int32)
        out = np.zeros(len(row))
        ya = None if y is None else _arr(y, np.float64)
        r = ctypes.c_double()
        self._check(self.L.bmf_predict(self.h, len(row), _ptr(row), _ptr(col), _ptr(ya),
                                       _ptr(out), ctypes.byref(r) if ya is not None else None))
        return out, (r.value if ya is not None else None)

    def test_rmse(self):
        """RMSE of the posterior-mean prediction of the held-out entries given at construction
        (aggregated on the device; bmf_test_rmse)."""
        r = ctypes.c_double()
        self._check(self.L.bmf_test_rmse(self.h, ctypes.byref(r)))
        return r.value

    def restart(self, seed, X0=None, W0=None):
        """A new run of Algorithm 1 on the same data (bmf_restart): every chain back to the
        initial state (X0 / W0 in the original order replace the stored one when given)."""
        Xa = None if X0 is None else _arr(X0, np.float64)
        Wa = None if W0 is None else _arr(W0, np.float64)
        self._check(self.L.bmf_restart(self.h, _ptr(Xa), _ptr(Wa), int(seed)))

    def posterior_means(self):
        Xm, Wm = np.zeros((self.N, self.K)), np.zeros((self.D, self.K))
        nc = ctypes.c_int64()
        self._check(self.L.bmf_posterior_means(self.h, _ptr(Xm), _ptr(Wm), ctypes.byref(nc)))
        return Xm, Wm, nc.value

    def get_noise(self, s):
        """Current noise precision of each column of subset s (bmf_get_noise)."""
        _, d = self._dims(s)
        tau = np.zeros(d)
        self._check(self.L.bmf_get_noise(self.h, s, _ptr(tau)))
        return tau

    def subset_info(self, s):
        info = SubsetInfo()
        self._check(self.L.bmf_get_subset_info(self.h, s, ctypes.byref(info)))
        return dict(i=info.i, j=info.j, stage=info.stage, row0=info.row0, row1=info.row1,
                    col0=info.col0, col1=info.col1, nnz=info.nnz)

    def perm(self):
        rp, cp = np.zeros(self.N, np.int64), np.zeros(self.D, np.int64)
        self._check(self.L.bmf_get_perm(self.h, _ptr(rp), _ptr(cp)))
        return rp, cp

    def _dims(self, s):
        i = self.subset_info(s)
        return i["row1"] - i["row0"], i["col1"] - i["col0"]

    def get_state(self, s=0):
        n, d = self._dims(s)
        K = self.K
        X, W = np.zeros((n, K)), np.zeros((d, K))
        hyp = np.zeros(2 * (K + K * K))
        self._check(self.L.bmf_get_state(self.h, s, _ptr(X), _ptr(W), _ptr(hyp)))
        H = K + K * K
        return X, W, dict(muX=hyp[:K].copy(), LamX=hyp[K:H].reshape(K, K).copy(),
                          muW=hyp[H:H + K].copy(), LamW=hyp[H + K:].reshape(K, K).copy())

    def set_state(self, s, X=None, W=None):
        Xa = None if X is None else _arr(X, np.float64)
        Wa = None if W is None else _arr(W, np.float64)
        self._check(self.L.bmf_set_state(self.h, s, _ptr(Xa), _ptr(Wa)))

    def get_moments(self, s, factor):
        n, d = self._dims(s)
        m = n if factor == FACTOR_X else d
        S1, S2 = np.zeros((m, self.K)), np.zeros((m, self.K, self.K))
        kept = ctypes.c_int64()
        self._check(self.L.bmf_get_moments(self.h, s, factor, _ptr(S1), _ptr(S2),
                                           ctypes.byref(kept)))
        return S1, S2, kept.value

    def get_posterior(self, s, factor):
        n, d = self._dims(s)
        m = n if factor == FACTOR_X else d
        mu, Lam = np.zeros((m, self.K)), np.zeros((m, self.K, self.K))
        self._check(self.L.bmf_get_posterior(self.h, s, factor, _ptr(mu), _ptr(Lam)))
        return mu, Lam

    def set_prior(self, s, factor, mu, Lam):
        mu, Lam = _arr(mu, np.float64), _arr(Lam, np.float64)
        self._check(self.L.bmf_set_prior(self.h, s, factor, _ptr(mu), _ptr(Lam)))

    def logjoint_grad(self, s, X_ptr, W_ptr, ld, log_alpha, gX_ptr, gW_ptr):
        """Masked log-joint of subset s at device FP32 factors (see include/bmf.h); gradients
        into gX/gW (device); returns (value, d value / d log alpha)."""
        v, ga = ctypes.c_double(), ctypes.c_double()
        self._check(self.L.bmf_logjoint_grad(self.h, s, X_ptr, W_ptr, int(ld), float(log_alpha),
                                             gX_ptr, gW_ptr, ctypes.byref(ga), ctypes.byref(v)))
        return v.value, ga.value

    def langevin(self, s, n_steps, X_ptr, W_ptr, ld, log_alpha, eps, noise_ptr, uniforms=None):
        """n_steps Langevin moves (MALA when uniforms are given) on device FP32 factors;
        returns (accepted, final log-joint)."""
        u = None if uniforms is None else _arr(uniforms, np.float64)
        acc, v = ctypes.c_int32(), ctypes.c_double()
        self._check(self.L.bmf_langevin(self.h, s, int(n_steps), X_ptr, W_ptr, int(ld),
                                        float(log_alpha), float(eps), noise_ptr, _ptr(u),
                                        ctypes.byref(acc), ctypes.byref(v)))
        return acc.value, v.value

    def profile(self, on=True):
        self._check(self.L.bmf_profile_enable(self.h, int(bool(on))))

    def profile_read(self):
        buf = (KernelTime * 16)()
        n = self.L.bmf_profile_read(self.h, buf, 16)
        return {buf[k].name.decode(): (buf[k].launches, buf[k].total_ms) for k in range(n)}

    def launch_count(self):
        return int(self.L.bmf_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.L.bmf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
