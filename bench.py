#!/usr/bin/env python
"""Benchmark of the BPMF Gibbs sweep inside posterior propagation (Qin et al., arXiv 1703.00734,
Algorithm 1, Eq. 14 / Algorithm 2, Section 5.1) on one GB300.

Default workload pp4x4-100000x20000-20M-k16: a 100,000 x 20,000 Zipf(1.2) matrix with 20M
observations (18M train), Gaussian values of a rank-16 truth plus noise, K = 16, on a 4 x 4 grid
(stage sizes 1 / 6 / 9 subsets of uneven size).  A step is one whole PP run: the three stages of
200 sweeps each (burn-in 100; all subsets of a stage batched into the same launches; FP32
gathers and Gram, FP64 Cholesky/Wishart/moments), moment matching and propagation between
stages, the eigenvalue-corrected aggregation and the prediction of the held-out entries.  The
headline `value` is PP sweeps/s (a PP sweep sweeps every subset chain of the three stages once,
visiting each training entry once per half-sweep, like a plain sweep of the whole matrix), with
the plain FP64 and FP32 samplers on the whole matrix at the same sweep count and the test RMSE
of all three beside it, plus the plain-sweep benchmark of the 69,878 x 10,677 Zipf matrix
(`plain_sweep_zipf`).  `--impl reference` times the FP64 CPU oracle instead.

Other workloads (--workload): zipf-69878x10677-10M-k10 and zipf-480189x17770-100M-k32 run the
plain-sweep benchmark (a step is one Gibbs sweep of the 1 x 1 sampler);
uniform-200000x50000-50M-k64 times the log-joint adjoint, Langevin moves and Gibbs sweeps at
K = 64; sim-6040x3706-k5 and sim-6040x3706-k5-structured run PP on 1x1 ... 30x30 grids in both
row/column orders and report test RMSE and time per partition (the paper's simulated-data
experiment).

Prints ONE JSON line (rank 0).  For --gpus N > 1 (torchrun) every rank runs an independent
replica of the workload (one chain does not shard across GPUs) and value sums them.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "pp4x4-100000x20000-20M-k16"
# arithmetic of the path per --precision: gathers and Gram sums, then the FP64 conditional
DTYPE = {"fp32": "f32+f64", "bf16": "bf16+f64", "tf32": "tf32+f64", "fp64": "f64"}
PLAIN_WORKLOAD = "zipf-69878x10677-10M-k10"
METRIC = "Gibbs sweeps/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 ALU peak: 152 SMs x 2 FP64 FMA/clock x 2 FLOP x 2.07 GHz (unit count and maximum clock
# of this GPU; a dependent-free DFMA loop measured 1.19 TFLOP/s, 1.89 FMA/clock/SM).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def wait_first(self, limit=3.0):
        """Block until the sampler has written its first line (or `limit` seconds)."""
        t_end = time.time() + limit
        while self.proc and self.path and time.time() < t_end:
            if os.path.getsize(self.path) > 0:
                return
            time.sleep(0.02)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------------------
# ranks (torchrun, one process per GPU): replicas of the workload, timed together
# ---------------------------------------------------------------------------------------
def barrier(world):
    if world > 1:
        import torch
        torch.distributed.barrier()


def max_over_ranks(ms, world, device):
    """The slowest rank's time (every rank gets it)."""
    if world == 1:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, max_ms, world):
    """Units all ranks processed per second of the slowest rank's time."""
    return world * units_per_rank / (max_ms / 1e3)


# ---------------------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------------------
def load_workload(name, scale=1.0):
    from paper_1703_00734_gb300 import synth
    t = time.time()
    d = synth.make_workload(name, scale=scale)
    log(f"workload {name}: N={d['N']} D={d['D']} train={len(d['row'])} "
        f"test={len(d['test_row'])} ({time.time() - t:.1f}s)")
    return d


def make_draws(d, K, nu0, n_sweeps, seed, out=None):
    """n_sweeps of draw buffers for the single-subset (1 x 1) sampler."""
    from paper_1703_00734_gb300 import synth
    sizes = [(d["N"], d["D"])]
    return np.concatenate([synth.sweep_draws(sizes, K, nu0, synth.rng_for(seed, 1, t))
                           for t in range(n_sweeps)])


def algorithmic(d, K, prec):
    """Algorithmic work per launch of each kernel class (the cost terms of Section 4.3)."""
    M = len(d["row"])
    b = {"fp64": 8, "fp32": 4, "tf32": 4, "bf16": 2}[prec]
    bval = 8 if prec == "fp64" else 4
    per_obs = 4 + bval + K * b              # index + value + gathered partner row
    nt = K * (K + 1) // 2
    fma_row = nt + K + (K ** 3 - K) // 6 + K * (K - 1)   # assembly, Cholesky, two solves
    return {
        "gram_x": ("hbm", M * per_obs, "GB/s"),
        "gram_w": ("hbm", M * per_obs, "GB/s"),
        "cond_x": ("alu", 2.0 * fma_row * d["N"], "TFLOP/s"),
        "cond_w": ("alu", 2.0 * fma_row * d["D"], "TFLOP/s"),
    }


# ---------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1703_00734_gb300 import bmf

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    d = load_workload(args.workload, args.scale)
    K, tau = d["K"], d["tau"]
    nu0 = float(K)
    test = (d["test_row"], d["test_col"], d["test_val"])
    W, S = args.warmup, args.steps

    def context(prec):
        m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], K, tau, prec, X0=d["X0"],
                    W0=d["W0"], test=test, burnin=args.burnin, seed=rank, stream=stream.cuda_stream)
        if not args.no_tune:
            schedules[prec] = m.autotune(1, -1, 3)   # restores the chain: no value changes
        return m

    schedules = {}

    per = None
    # ---- headline: reduced-precision path, inputs resident ---------------------------
    m = context(args.precision)
    per = m.draws_per_sweep(1)
    host = make_draws(d, K, nu0, W + S, seed=100 + rank)
    assert host.size == per * (W + S)
    dr = torch.from_numpy(host).to(dev)
    # clock samples (nvidia-smi, every 100 ms) from the warm-up through the timed region and
    # 0.3 s of the same (untimed) sweeps after it, so that a short timed region still has
    # samples taken under the same load
    clk = ClockSampler(local_rank).__enter__()
    clk.wait_first()
    m.sweep(0, W, dr[: W * per])
    torch.cuda.synchronize()
    barrier(world)
    n0 = m.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    st = m.sweep(0, S, dr[W * per:(W + S) * per])
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    launches = m.launch_count() - n0
    t_end = time.perf_counter() + 0.3
    while time.perf_counter() < t_end:
        m.sweep(0, S, dr[W * per:(W + S) * per])
    clk.__exit__(None, None, None)
    torch.cuda.synchronize()
    barrier(world)
    ms = max_over_ranks(ms, world, dev)
    rmse_red = st["rmse_mean"]
    # ---- per-kernel timing over the same number of steps (profiling pass) ------------
    # one launch per kernel and half (no row chunks), so that each launch's event time is the
    # kernel's own duration and not shared with an overlapping chunk on another stream
    tuned = m.get_schedule()
    m.set_schedule(1, 1, tuned["gram_blocks_per_sm"], 0.0, 0)
    m.profile(True)
    m.sweep(0, S, dr[W * per:(W + S) * per])
    prof = m.profile_read()
    m.profile(False)
    m.set_schedule(**tuned)
    # ---- e2e: host (pinned) draws copied in every step, stats read back ---------------
    pinned = torch.from_numpy(host[W * per:(W + S) * per].copy()).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(S):
        m.sweep(0, 1, pinned[k * per:(k + 1) * per])
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    m.close()
    del dr
    # ---- plain FP64 GPU sweep, same data and draws ------------------------------------
    fp64 = None
    if not args.no_fp64:
        S64 = min(S, args.fp64_steps)
        m64 = context("fp64")
        dr64 = torch.from_numpy(host[: (W + S64) * per]).to(dev)
        m64.sweep(0, W, dr64[: W * per])
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st64 = m64.sweep(0, S64, dr64[W * per:(W + S64) * per])
        b.record(stream)
        b.synchronize()
        fp64 = {"sweeps_per_s": S64 / (a.elapsed_time(b) / 1e3), "steps": S64,
                "rmse_mean": st64["rmse_mean"]}
        m64.close()
        del dr64
    # RMSE of the reduced-precision chain at the same sweep count as the FP64 chain
    rmse_same = None
    if fp64 is not None:
        mr = context(args.precision)
        drr = torch.from_numpy(host[: (W + fp64["steps"]) * per]).to(dev)
        str_ = mr.sweep(0, W + fp64["steps"], drr)
        rmse_same = str_["rmse_mean"]
        mr.close()
        del drr
    if rank != 0:
        return None
    sweeps_s = whole_job_rate(S, ms, world)
    M = len(d["row"])
    gflops = 2 * M * 2 * K * K * sweeps_s / 1e9
    # roofline of the dominant kernel class
    algo = algorithmic(d, K, args.precision)
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    kernels = {}
    for name, (n, tot) in prof.items():
        if n == 0:
            continue
        avg_ms = tot / n
        ent = {"launches": n, "avg_us": avg_ms * 1e3, "share": None}
        if name in algo:
            bound, work, unit = algo[name]
            ach = work / (avg_ms / 1e3) / (1e9 if unit == "GB/s" else 1e12)
            peak = hbm if unit == "GB/s" else FP64_PEAK_TFLOPS
            ent.update(bound=bound, achieved=ach, peak=peak, unit=unit, frac=ach / peak)
        kernels[name] = ent
    total = sum(v["avg_us"] * v["launches"] for v in kernels.values())
    for v in kernels.values():
        v["share"] = v["avg_us"] * v["launches"] / total if total else None
    dom = max((k for k in kernels if "bound" in kernels[k]),
              key=lambda k: kernels[k]["avg_us"] * kernels[k]["launches"])
    kd = kernels[dom]
    roof = {"kernel": dom, "bound": kd["bound"], "achieved": kd["achieved"], "peak": kd["peak"],
            "unit": kd["unit"], "frac": kd["frac"], "traffic": traffic_for(dom, args.precision, args.workload),
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if kd["unit"] == "GB/s"
            else "derived: 152 SMs x 2 FP64 FMA/clk x 2 x 2.07 GHz"}
    out = {
        "metric": METRIC, "value": sweeps_s, "unit": "sweeps/s", "n_gpus": world, "steps": S,
        "warmup": W, "ms_per_step": ms / S, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[args.precision],
        "data": "synthetic (seeded Zipf(1.2) rating matrix standing in for a MovieLens-shaped "
                "data set; no real data available)",
        "config": {"workload": args.workload,
                   "N": d["N"], "D": d["D"], "train_obs": M, "test_obs": len(d["test_row"]),
                   "K": K, "tau": tau, "precision": args.precision, "grid": "1x1",
                   "l2": "inputs larger than L2 (observation lists 144 MB > 129 MB L2)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "obsK2_gflops": gflops,
        "schedule": schedules,
        "rmse": {"reduced": rmse_red, "reduced_at_fp64_steps": rmse_same,
                 "fp64": fp64["rmse_mean"] if fp64 else None,
                 "abs_diff": abs(rmse_same - fp64["rmse_mean"]) if fp64 else None},
        "fp64_plain": fp64,
        "speedup_vs_fp64_plain": sweeps_s / world / fp64["sweeps_per_s"] if fp64 else None,
        "roofline": roof,
        "kernels": kernels,
        "e2e": {"value": world * S / e2e_s, "unit": "sweeps/s",
                "h2d_bytes_per_step": per * 8, "d2h_bytes_per_step": 8 + 16},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if world == 1 and not args.no_cpu_baseline and args.workload == PLAIN_WORKLOAD:
        out["cpu_baseline"] = cpu_baseline(d, args.cpu_seconds)
        out["cpu_all_cores"] = cpu_all_cores(d, args.cpu_seconds)
    return out


# ---------------------------------------------------------------------------------------
# posterior propagation on an I x J grid: three batched stages, then Algorithm 2
# ---------------------------------------------------------------------------------------
PP_SWEEPS, PP_BURNIN = 200, 100      # per stage (100 retained samples, K + 1 <= 100)
PP_CLASSES = ("gram_x", "cond_x", "gram_w", "cond_w")


def stage_geometry(m, I, J):
    """Per stage: X rows, W rows and training entries of its subsets (every training entry is
    in exactly one subset, so the three stages together visit each once per half-sweep)."""
    g = {1: [0, 0, 0], 2: [0, 0, 0], 3: [0, 0, 0]}
    for sid in range(I * J):
        info = m.subset_info(sid)
        q = g[info["stage"]]
        q[0] += info["row1"] - info["row0"]
        q[1] += info["col1"] - info["col0"]
        q[2] += info["nnz"]
    return g


def pp_algorithmic(geom, K, prec):
    """Algorithmic work per launch of each kernel class in each stage (one launch per class and
    sweep with one row chunk): Gram pass bytes = entries x (index + value + gathered partner
    row); conditional FLOPs = rows x 2 x (assembly + Cholesky + two solves) FMAs."""
    b = {"fp64": 8, "fp32": 4, "tf32": 4, "bf16": 2}[prec]
    bval = 8 if prec == "fp64" else 4
    per_obs = 4 + bval + K * b
    fma_row = K * (K + 1) // 2 + K + (K ** 3 - K) // 6 + K * (K - 1)
    out = {}
    for st, (nx, nw, nnz) in geom.items():
        out[(st, "gram_x")] = ("hbm", nnz * per_obs, "GB/s")
        out[(st, "gram_w")] = ("hbm", nnz * per_obs, "GB/s")
        out[(st, "cond_x")] = ("alu", 2.0 * fma_row * nx, "TFLOP/s")
        out[(st, "cond_w")] = ("alu", 2.0 * fma_row * nw, "TFLOP/s")
    return out


def pp_kernel_table(prof_by_stage, algo, hbm):
    """Per (stage, kernel class): launches, mean launch time and, for the Gram and conditional
    classes, achieved work against the peak.  `stream_time_share` is the class's summed launch
    time over the summed time of all classes: classes on side streams (hyperparameter draws,
    test RMSE, generator) overlap the main stream, so it is not a critical-path share."""
    rows = {}
    total = sum(t for prof in prof_by_stage.values() for (_, t) in prof.values())
    for st, prof in prof_by_stage.items():
        for name, (n, t) in prof.items():
            if n == 0:
                continue
            ent = {"stage": st, "kernel": name, "launches": n, "avg_us": t / n * 1e3,
                   "stream_time_share": t / total if total else None}
            if (st, name) in algo:
                bound, work, unit = algo[(st, name)]
                ach = work / (t / n / 1e3) / (1e9 if unit == "GB/s" else 1e12)
                peak = hbm if unit == "GB/s" else FP64_PEAK_TFLOPS
                ent.update(bound=bound, work_per_launch=work, achieved=ach, peak=peak,
                           unit=unit, frac=ach / peak)
            rows[f"s{st}.{name}"] = ent
    return rows


def run_pp(args, rank, world, local_rank):
    """A step is one whole PP run (Algorithm 1, then Algorithm 2): the three stages of
    PP_SWEEPS sweeps each (burn-in PP_BURNIN; every stage's subsets batched into the same
    launches; the run's draws resident in HBM), moment matching and propagation between stages, the
    eigenvalue-corrected aggregation and the posterior-mean prediction of the held-out entries.
    The context restarts every chain before each step (bmf_restart, a new seed per step).
    value = PP sweeps/s: one PP sweep is one sweep of every subset chain of the three stages,
    which visits every training entry once per half-sweep, as a plain sweep of the whole matrix
    does; the plain FP64 and reduced-precision samplers run the same number of sweeps on the
    whole matrix beside it."""
    import torch
    from paper_1703_00734_gb300 import bmf

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    d = load_workload(args.workload, args.scale)
    K, tau, I, J = d["K"], d["tau"], d["I"], d["J"]
    T, B = args.pp_sweeps, args.pp_burnin
    if T - B < K + 1:
        raise SystemExit(f"--pp-sweeps minus --pp-burnin must keep at least K + 1 = {K + 1} "
                         "samples per chain for moment matching")
    test = (d["test_row"], d["test_col"], d["test_val"])
    M, n_test = len(d["row"]), len(d["test_row"])
    Wu, S = max(1, args.warmup), args.steps
    seed0 = 1000 * (rank + 1)
    t0 = time.perf_counter()
    m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], K, tau, args.precision, I=I, J=J,
                X0=d["X0"], W0=d["W0"], test=test, burnin=B, seed=seed0,
                stream=stream.cuda_stream)
    init_ms = (time.perf_counter() - t0) * 1e3
    # the per-sweep test-RMSE monitor is off: PP predicts once per run, from the aggregated
    # posterior (bmf_test_rmse)
    m.set_monitor(False)
    geom = stage_geometry(m, I, J)
    ev = lambda: torch.cuda.Event(enable_timing=True)

    # first (untimed) run: the schedule tuner on each stage's batch as it opens
    schedules = {}
    for stage in (1, 2, 3):
        m.stage(stage, 0, None)                     # opens the stage (priors installed)
        schedules[stage] = (m.autotune(stage, -1, 3) if not args.no_tune
                            else m.get_schedule())
        m.stage(stage, T, None)
    m.test_rmse()

    # the draws are inputs of a run, resident in HBM when the timed region starts: every step's
    # draws (three stages of T sweeps) come from the device generator with the step's seed,
    # before the clock
    pers = {st: m.draws_per_sweep(st) for st in (1, 2, 3)}
    dbuf = {st: torch.empty(pers[st] * T, dtype=torch.float64, device=dev) for st in (1, 2, 3)}

    def prepare(seed):
        m.restart(seed)
        for st in (1, 2, 3):
            m.generate_draws(1, T, stage=st, out=dbuf[st])
        torch.cuda.synchronize()

    def pp_step(seed, draws=True):
        m.restart(seed)
        for stage in (1, 2, 3):
            m.set_schedule(**schedules[stage])
            m.stage(stage, T, dbuf[stage] if draws else None)
        return m.test_rmse()

    clk = ClockSampler(local_rank).__enter__()
    clk.wait_first()
    for w in range(1, Wu):
        prepare(seed0 + w)
        pp_step(seed0 + w)
    torch.cuda.synchronize()
    barrier(world)
    launches, rmses, run_ms = 0, [], []
    for k in range(S):
        prepare(seed0 + 100 + k)
        barrier(world)
        n0 = m.launch_count()
        a, b = ev(), ev()
        a.record(stream)
        rmses.append(pp_step(seed0 + 100 + k))
        b.record(stream)
        b.synchronize()
        run_ms.append(a.elapsed_time(b))
        launches += m.launch_count() - n0
    clk.__exit__(None, None, None)
    torch.cuda.synchronize()
    barrier(world)
    ms = max_over_ranks(float(np.sum(run_ms)), world, dev)

    # the same runs with the draws made inside the run by the device generator (draws == NULL)
    gen_ms, gen_rmse = [], []
    for k in range(min(S, 3)):
        a, b = ev(), ev()
        a.record(stream)
        gen_rmse.append(pp_step(seed0 + 100 + k, draws=False))
        b.record(stream)
        b.synchronize()
        gen_ms.append(a.elapsed_time(b))

    # per-kernel timing: one more run, untimed, with the library's event tracing on and one
    # launch per kernel class and half (no row chunks, no graph), stage by stage
    prepare(seed0 + 99)
    m.restart(seed0 + 99)
    prof_by_stage = {}
    for stage in (1, 2, 3):
        sc = dict(schedules[stage])
        m.set_schedule(1, 1, sc["gram_blocks_per_sm"], 0.0, 0, sc.get("cond_lanes", 0))
        m.profile(True)
        m.stage(stage, T, dbuf[stage])
        prof_by_stage[stage] = m.profile_read()
        m.profile(False)
    m.test_rmse()
    del dbuf

    # e2e through the C ABI with host buffers: the initial state and every stage's draws copied
    # in from pinned host memory (bmf_restart, bmf_stage), and bmf_predict of the held-out
    # entries given as pinned host arrays, the predictions copied back
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    hX0, hW0 = pin(d["X0"]), pin(d["W0"])
    hr, hc, hv = pin(d["test_row"].astype(np.int32)), pin(d["test_col"].astype(np.int32)), \
        pin(d["test_val"].astype(np.float64))
    hbuf = {st: torch.empty(pers[st] * T, dtype=torch.float64).pin_memory() for st in (1, 2, 3)}
    n_e2e = max(2, S // 4)
    e2e_s, e2e_rmse, e2e_runs = 0.0, [], []
    for k in range(-1, n_e2e):                 # one untimed run first (first use of the buffers)
        m.restart(seed0 + 200 + k)
        for st in (1, 2, 3):
            m.generate_draws(1, T, stage=st, out=hbuf[st])     # host, before the clock
        torch.cuda.synchronize()
        te = time.perf_counter()
        m.restart(seed0 + 200 + k, X0=hX0, W0=hW0)
        for st in (1, 2, 3):
            m.set_schedule(**schedules[st])
            m.stage(st, T, hbuf[st])
        yhat, r = m.predict(hr, hc, hv)
        dt = time.perf_counter() - te
        if k >= 0:
            e2e_s += dt
            e2e_rmse.append(r)
        e2e_runs.append(dt * 1e3)
    h2d = hX0.nbytes + hW0.nbytes + hr.nbytes + hc.nbytes + hv.nbytes + \
        sum(8 * pers[st] * T for st in (1, 2, 3))
    d2h = n_test * 8 + 8
    del hbuf
    m.close()

    # the plain samplers on the whole matrix, same number of sweeps, their draws resident in
    # HBM as for PP (device generator before the clock)
    plain = {}
    for prec in ("fp64", args.precision):
        mp = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], K, tau, prec, X0=d["X0"],
                     W0=d["W0"], test=test, burnin=B, seed=seed0 + 7, stream=stream.cuda_stream)
        mp.set_monitor(False)
        sch = mp.autotune(1, -1, 3) if not args.no_tune else mp.get_schedule()
        mp.sweep(0, 2, None)
        mp.restart(seed0 + 7)
        pbuf = torch.empty(mp.draws_per_sweep(1) * T, dtype=torch.float64, device=dev)
        mp.generate_draws(1, T, stage=1, out=pbuf)
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record(stream)
        mp.restart(seed0 + 7)
        mp.sweep(0, T, pbuf)
        r = mp.test_rmse()
        b.record(stream)
        b.synchronize()
        pms = a.elapsed_time(b)
        plain[prec] = {"sweeps_per_s": T / (pms / 1e3), "ms_per_run": pms, "sweeps": T,
                       "burnin": B, "rmse": r, "schedule": sch}
        del pbuf
        mp.close()
    if rank != 0:
        return None
    sweeps_s = whole_job_rate(S * T, ms, world)
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    algo = pp_algorithmic(geom, K, args.precision)
    kernels = pp_kernel_table(prof_by_stage, algo, hbm)
    dom = max((k for k in kernels if "bound" in kernels[k]),
              key=lambda k: kernels[k]["avg_us"] * kernels[k]["launches"])
    kd = kernels[dom]
    roof = {"kernel": dom, "bound": kd["bound"], "achieved": kd["achieved"], "peak": kd["peak"],
            "unit": kd["unit"], "frac": kd["frac"],
            "traffic": traffic_for(dom, args.precision, args.workload),
            "work_per_launch": kd["work_per_launch"],
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if kd["unit"] == "GB/s"
            else "derived: 152 SMs x 2 FP64 FMA/clk x 2 x 2.07 GHz"}
    rmse_pp = float(np.mean(rmses))
    r64 = plain["fp64"]["rmse"]
    out = {
        "metric": METRIC, "value": sweeps_s, "unit": "sweeps/s", "n_gpus": world, "steps": S,
        "warmup": Wu, "ms_per_step": ms / S, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[args.precision],
        "data": "synthetic (seeded Zipf(1.2) pattern, Gaussian values of a rank-16 truth plus "
                "N(0, 0.5^2) noise; no real data available)",
        "config": {"workload": args.workload, "N": d["N"], "D": d["D"], "train_obs": M,
                   "test_obs": n_test, "K": K, "tau": tau, "grid": f"{I}x{J}",
                   "subsets_per_stage": [sum(1 for s in range(I * J)
                                             if m_stage(s, I, J) == st) for st in (1, 2, 3)],
                   "sweeps_per_stage": T, "burnin": B, "precision": args.precision,
                   "step": "one whole PP run: 3 stages x sweeps_per_stage sweeps (all subsets of "
                           "a stage batched), moment matching, Algorithm 2, held-out prediction",
                   "unit_of_value": "PP sweep = one sweep of every subset chain of the three "
                                    "stages (each training entry visited once per half-sweep)",
                   "draws": "inputs resident in HBM: each step's draws made by the device "
                            "generator (Philox4x64-10) with a new seed before the clock; "
                            "device_generator below times the runs with the draws made inside",
                   "monitor": "per-sweep test-RMSE monitor off (PP and plain); the held-out "
                              "RMSE is computed once per run from the posterior means",
                   "l2": "inputs larger than L2 (observation lists 288 MB > 129 MB L2)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "obsK2_gflops": 2 * M * 2 * K * K * sweeps_s / 1e9,
        "stage_sweeps_per_s": 3 * sweeps_s,
        "run_ms": {"mean": float(np.mean(run_ms)), "min": float(np.min(run_ms)),
                   "max": float(np.max(run_ms))},
        "device_generator": {"sweeps_per_s": T / (float(np.mean(gen_ms)) / 1e3),
                             "ms_per_run": float(np.mean(gen_ms)), "runs": len(gen_ms),
                             "rmse_mean": float(np.mean(gen_rmse))},
        "rmse": {"pp_mean_over_steps": rmse_pp, "pp_min": float(np.min(rmses)),
                 "pp_max": float(np.max(rmses)), "plain_fp64": r64,
                 "plain_reduced": plain[args.precision]["rmse"],
                 "abs_diff_pp_vs_plain_fp64": abs(rmse_pp - r64),
                 "budget": 0.002, "within_budget": abs(rmse_pp - r64) <= 0.002},
        "plain": plain,
        "speedup_vs_plain_fp64": sweeps_s / world / plain["fp64"]["sweeps_per_s"],
        "speedup_note": "PP sweeps/s over plain FP64 sweeps/s at the same sweeps per chain "
                        f"({T}, burn-in {B}); |RMSE difference| beside it",
        "roofline": roof,
        "kernels": kernels,
        "schedule": {f"stage{k}": v for k, v in schedules.items()},
        "e2e": {"value": world * n_e2e * T / e2e_s, "unit": "sweeps/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "rmse_mean": float(np.mean(e2e_rmse)),
                "runs_ms": [round(x, 1) for x in e2e_runs], "untimed_first_run": True,
                "what": "bmf_restart from pinned host X0/W0, 3 x bmf_stage with each stage's "
                        "draws copied from pinned host memory, bmf_predict of the held-out "
                        "entries from pinned host arrays with the predictions read back; host "
                        "wall clock"},
        "init_ms": init_ms,
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_pp(d, args.cpu_seconds, threads=1)
        out["cpu_all_cores"] = cpu_baseline_pp(d, args.cpu_seconds, threads=0)
    return out


def m_stage(sid, I, J):
    i, j = divmod(sid, J)
    return 1 if i == 0 and j == 0 else (2 if i == 0 or j == 0 else 3)


# ---------------------------------------------------------------------------------------
# the adjoint of the masked log-joint, Langevin moves and Gibbs sweeps at K = 64
# ---------------------------------------------------------------------------------------
def run_adjoint(args, rank, world, local_rank):
    import torch
    from paper_1703_00734_gb300 import bmf

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    d = load_workload(args.workload, args.scale)
    K, tau = d["K"], d["tau"]
    N, D, M = d["N"], d["D"], len(d["row"])
    S, Wm = args.steps, args.warmup
    m = bmf.BMF(N, D, d["row"], d["col"], d["val"], K, tau, "fp32", X0=d["X0"], W0=d["W0"],
                test=(d["test_row"], d["test_col"], d["test_val"]), burnin=1, seed=rank,
                stream=stream.cuda_stream)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    # Gibbs sweeps (device generator for the draws)
    m.sweep(0, Wm, None)
    torch.cuda.synchronize()
    a, b = ev(), ev()
    with ClockSampler(local_rank) as clk:
        a.record(stream)
        st = m.sweep(0, S, None)
        b.record(stream)
        b.synchronize()
        gibbs_ms = a.elapsed_time(b) / S
        # the adjoint at the current sample
        X, W, hyp = m.get_state(0)
        ld = (K + 3) // 4 * 4
        dX = torch.zeros((N, ld), dtype=torch.float32, device=dev)
        dW = torch.zeros((D, ld), dtype=torch.float32, device=dev)
        dX[:, :K] = torch.from_numpy(X.astype(np.float32)).to(dev)
        dW[:, :K] = torch.from_numpy(W.astype(np.float32)).to(dev)
        gX, gW = torch.empty_like(dX), torch.empty_like(dW)
        la = float(np.log(tau))
        for _ in range(Wm):
            m.logjoint_grad(0, dX.data_ptr(), dW.data_ptr(), ld, la, gX.data_ptr(), gW.data_ptr())
        torch.cuda.synchronize()
        n0 = m.launch_count()
        a.record(stream)
        for _ in range(S):
            m.logjoint_grad(0, dX.data_ptr(), dW.data_ptr(), ld, la, gX.data_ptr(), gW.data_ptr())
        b.record(stream)
        b.synchronize()
        grad_ms = a.elapsed_time(b) / S
        launches = m.launch_count() - n0
        m.profile(True)
        m.logjoint_grad(0, dX.data_ptr(), dW.data_ptr(), ld, la, gX.data_ptr(), gW.data_ptr())
        prof = m.profile_read()
        m.profile(False)
        # Langevin moves: unadjusted, then Metropolis-adjusted, eps small enough to accept
        L = min(S, 10)
        rng = np.random.default_rng(100 + rank)
        xi = torch.from_numpy(rng.standard_normal(L * (N + D) * K).astype(np.float32)).to(dev)
        eps = 1e-6
        torch.cuda.synchronize()
        a.record(stream)
        m.langevin(0, L, dX.data_ptr(), dW.data_ptr(), ld, la, eps, xi.data_ptr())
        b.record(stream)
        b.synchronize()
        ula_ms = a.elapsed_time(b) / L
        a.record(stream)
        eps_mh = 1e-11     # Metropolis-adjusted moves in (N + D) K dimensions need tiny steps
        acc, _ = m.langevin(0, L, dX.data_ptr(), dW.data_ptr(), ld, la, eps_mh, xi.data_ptr(),
                            uniforms=rng.random(L))
        b.record(stream)
        b.synchronize()
        mala_ms = a.elapsed_time(b) / L
    m.close()
    if rank != 0:
        return None
    # algorithmic bytes of one gradient evaluation: each of the two passes reads every
    # observation's index, value and FP32 partner row (8 + 4K bytes per observation and side)
    per_obs_side = 4 + 4 + 4 * K
    algo = 2 * M * per_obs_side
    items = {k: (n, t) for k, (n, t) in prof.items() if n}
    adj_ms = items.get("adjoint", (1, grad_ms))[1] / max(items.get("adjoint", (1, 0))[0], 1)
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    ach = algo / (grad_ms / 1e3) / 1e9
    return {
        "metric": "log-joint gradient evaluations/s (adjoint, K=64)", "impl": "ours",
        "value": 1e3 / grad_ms, "unit": "grad evals/s", "n_gpus": world, "steps": S,
        "warmup": Wm, "ms_per_step": grad_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "N": N, "D": D, "train_obs": M, "K": K,
                   "l2": "inputs larger than L2"},
        "gibbs": {"sweeps_per_s": 1e3 / gibbs_ms, "ms_per_sweep": gibbs_ms,
                  "rmse_mean": st["rmse_mean"], "precision": "fp32 (split TF32 Gram)"},
        "langevin": {"ula_steps_per_s": 1e3 / ula_ms, "mala_steps_per_s": 1e3 / mala_ms,
                     "mala_accepted": acc, "mala_steps": L, "eps_ula": eps, "eps_mala": eps_mh},
        "roofline": {"kernel": "adjoint (both passes, whole evaluation)", "bound": "hbm",
                     "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                     "traffic": traffic_for("adjoint", "fp32", args.workload),
                     "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)",
                     "note": "algorithmic bytes count every gathered partner row; the partner "
                             "tables stay in L1/L2, so DRAM traffic (ncu) is far below them and "
                             "frac can exceed 1: the item pass is bound by L1 wavefronts"},
        "adjoint_launch_ms": adj_ms, "gpu_launches": launches, "clocks": clk.summary(),
    }


MODES = {"uniform-200000x50000-50M-k64": "adjoint", "sim-6040x3706-k5": "partitions",
         "sim-6040x3706-k5-structured": "partitions"}


# ---------------------------------------------------------------------------------------
# test RMSE and wall-clock time of PP against the partition (Section 5.3, simulated data)
# ---------------------------------------------------------------------------------------
PART_GRIDS = (1, 3, 5, 10, 30)
PART_SWEEPS, PART_BURNIN, PART_THIN = 1200, 800, 2    # the paper's chains (200 samples kept)


PART_DATASETS = 5                                     # independent data sets (Table 3 means)


def run_partitions(args, rank, world, local_rank):
    """One PP run per r x r grid and row/column order on each of PART_DATASETS independent
    simulated data sets (the paper averages five): three stages of 1200 sweeps (burn-in 800,
    thin 2; device generator), then aggregation (Eq. 14, Algorithm 2) and the posterior-mean
    prediction of every held-out cell.  FP64 throughout, as in the paper's runs.  Time per run:
    host clock around the stages plus the prediction call.  Reported per grid and order: the
    mean test RMSE over the data sets (and each one), the mean time."""
    import torch
    from paper_1703_00734_gb300 import bmf, synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    T, B = PART_SWEEPS, PART_BURNIN
    if args.scale < 1.0:                  # shrunk runs (tests, captures): shorter chains
        T, B = 120, 80
    n_sets = args.datasets if args.datasets > 0 else PART_DATASETS
    base_seed = synth.WORKLOADS[args.workload]["seed"]
    runs, launches = [], 0
    with ClockSampler(local_rank) as clk:
        for ds in range(n_sets):
            # data set 0 is the named workload; the others draw X, W, E and the missing cells
            # from independent seeds
            t0 = time.time()
            d = synth.make_workload(args.workload, scale=args.scale,
                                    **({} if ds == 0 else {"seed": base_seed + 1000 * ds}))
            log(f"data set {ds}: N={d['N']} D={d['D']} train={len(d['row'])} "
                f"test={len(d['test_row'])} ({time.time() - t0:.1f}s)")
            K, tau = d["K"], d["tau"]
            for order in ("decreasing", "none"):
                for g in PART_GRIDS:
                    if g > min(d["N"], d["D"]):
                        continue
                    m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], K, tau, "fp64",
                                I=g, J=g, X0=d["X0"], W0=d["W0"], order=order, burnin=B,
                                thin=PART_THIN, seed=rank + 17 * ds, stream=stream.cuda_stream)
                    m.set_monitor(False)
                    torch.cuda.synchronize()
                    n0 = m.launch_count()
                    stage_ms = []
                    t0 = time.perf_counter()
                    for stage in ((1,) if g == 1 else (1, 2, 3)):
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        m.stage(stage, T, None)
                        e1.record(stream)
                        e1.synchronize()
                        stage_ms.append(e0.elapsed_time(e1))
                    _, rmse = m.predict(d["test_row"], d["test_col"], d["test_val"])
                    secs = time.perf_counter() - t0
                    launches += m.launch_count() - n0
                    m.close()
                    runs.append({"dataset": ds, "grid": f"{g}x{g}", "order": order, "rmse": rmse,
                                 "seconds": secs, "stage_ms": stage_ms})
                    log(f"set {ds} {order} {g}x{g}: rmse {rmse:.4f} in {secs:.2f} s")
    if rank != 0:
        return None
    table = []
    for order in ("decreasing", "none"):
        for g in PART_GRIDS:
            rs = [q for q in runs if q["order"] == order and q["grid"] == f"{g}x{g}"]
            if not rs:
                continue
            table.append({"grid": f"{g}x{g}", "order": order,
                          "rmse_mean": float(np.mean([q["rmse"] for q in rs])),
                          "rmse_sd": float(np.std([q["rmse"] for q in rs])),
                          "rmse_by_dataset": [q["rmse"] for q in rs],
                          "seconds_mean": float(np.mean([q["seconds"] for q in rs])),
                          "datasets": len(rs)})
    for r in table:
        base = next(q for q in table if q["order"] == r["order"] and q["grid"] == "1x1")
        r["wts"] = base["seconds_mean"] / r["seconds_mean"]
    head = next((r for r in table if r["grid"] == "10x10" and r["order"] == "decreasing"),
                table[-1])
    return {
        "metric": "test RMSE of PP by partition (simulated data, Section 5.3)", "impl": "ours",
        "value": head["rmse_mean"], "unit": "RMSE", "n_gpus": world, "steps": T, "warmup": 0,
        "ms_per_step": head["seconds_mean"] * 1e3 / (3 * T), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "K": 5, "tau": 1.0, "sweeps_per_stage": T,
                   "burnin": B, "thin": PART_THIN, "datasets": n_sets,
                   "value_run": f"{head['grid']} {head['order']}, mean over {n_sets} data sets"},
        "table": table, "runs": runs, "gpu_launches": launches, "clocks": clk.summary(),
    }


# ---------------------------------------------------------------------------------------
# correlations of the subset posteriors (Section 5.6): PP against independent subsets
# ---------------------------------------------------------------------------------------
CORR_GRIDS = (3, 5, 10)


def align_latent(A, B):
    """B's latent columns permuted and sign-flipped to match A's: greedily pair the columns with
    the largest absolute correlation (the alignment applied to embarrassingly parallel MCMC
    before correlating its subset posteriors, Section 5.6)."""
    K = A.shape[1]
    Az = (A - A.mean(0)) / (A.std(0) + 1e-300)
    Bz = (B - B.mean(0)) / (B.std(0) + 1e-300)
    Cm = Az.T @ Bz / len(A)
    perm, sign = np.zeros(K, int), np.ones(K)
    free_a, free_b = set(range(K)), set(range(K))
    for _ in range(K):
        i, j = max(((i, j) for i in free_a for j in free_b), key=lambda ij: abs(Cm[ij]))
        perm[i], sign[i] = j, 1.0 if Cm[i, j] >= 0 else -1.0
        free_a.discard(i)
        free_b.discard(j)
    return B[:, perm] * sign


def block_correlation(A, B):
    """Pearson correlation of two posterior-mean blocks over all their entries."""
    a, b = A.ravel() - A.mean(), B.ravel() - B.mean()
    return float(a @ b / np.sqrt((a @ a) * (b @ b)))


def subset_correlations(means, I, J):
    """cor(X^(i,0), X^(i,j)) for j >= 1 and cor(W^(0,j), W^(i,j)) for i >= 1 (0-based), raw and
    after aligning the latent dimensions; means[sid] = (X mean block, W mean block)."""
    raw, aligned = [], []
    for i in range(I):
        for j in range(1, J):
            A, B = means[i * J][0], means[i * J + j][0]
            raw.append(block_correlation(A, B))
            aligned.append(block_correlation(A, align_latent(A, B)))
    for j in range(J):
        for i in range(1, I):
            A, B = means[j][1], means[i * J + j][1]
            raw.append(block_correlation(A, B))
            aligned.append(block_correlation(A, align_latent(A, B)))
    stats = lambda v: {"mean": float(np.mean(v)), "min": float(np.min(v)), "max": float(np.max(v)),
                       "pairs": len(v)}
    return {"raw": stats(raw), "aligned": stats(aligned)}


def run_correlations(args, rank, world, local_rank):
    """Section 5.6 on the simulated data: for each grid, PP (Algorithm 1, moment matching) and
    embarrassingly parallel MCMC (every subset with the standard priors, no propagation) on the
    same data, 1200 sweeps per subset chain (burn-in 800, thin 2; device generator); the
    posterior means of every subset's X and W blocks (means of the retained samples), and the
    correlations between blocks estimated in subsets that share rows or columns."""
    import torch
    from paper_1703_00734_gb300 import bmf

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    d = load_workload(args.workload, args.scale)
    K, tau = d["K"], d["tau"]
    T, B = PART_SWEEPS, PART_BURNIN
    if args.scale < 1.0:
        T, B = 120, 80
    out_rows = []
    with ClockSampler(local_rank) as clk:
        for g in CORR_GRIDS:
            if g > min(d["N"], d["D"]):
                continue
            row = {"grid": f"{g}x{g}"}
            for method, indep in (("pp", False), ("independent", True)):
                m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], K, tau, "fp64", I=g,
                            J=g, X0=d["X0"], W0=d["W0"], burnin=B, thin=PART_THIN, seed=rank + 5,
                            independent=indep, moments="full", stream=stream.cuda_stream)
                t0 = time.perf_counter()
                for stage in (1, 2, 3):
                    m.stage(stage, T, None)
                means = {sid: (m.get_posterior(sid, 0)[0], m.get_posterior(sid, 1)[0])
                         for sid in range(g * g)}
                _, rmse = m.predict(d["test_row"], d["test_col"], d["test_val"])
                row[method] = dict(subset_correlations(means, g, g), rmse=rmse,
                                   seconds=time.perf_counter() - t0)
                m.close()
                log(f"{g}x{g} {method}: corr raw {row[method]['raw']['mean']:.3f} aligned "
                    f"{row[method]['aligned']['mean']:.3f} rmse {rmse:.4f}")
            out_rows.append(row)
    if rank != 0:
        return None
    head = next((r for r in out_rows if r["grid"] == "5x5"), out_rows[-1])
    return {
        "metric": "correlation of subset posterior means (Section 5.6)", "impl": "ours",
        "value": head["pp"]["raw"]["mean"], "unit": "Pearson r", "n_gpus": world, "steps": T,
        "warmup": 0, "ms_per_step": head["pp"]["seconds"] * 1e3 / (3 * T),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "K": K,
                                         "sweeps_per_stage": T, "burnin": B, "thin": PART_THIN,
                                         "value_run": f"{head['grid']} PP, raw correlation"},
        "grids": out_rows, "clocks": clk.summary(),
    }


def traffic_for(kernel, prec, workload):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu summary, if one
    matches (null otherwise)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        f = line.split()
        if len(f) >= 4 and not line.startswith("#") and f[0] == kernel and f[1] == prec \
                and f[2] == workload:
            return float(f[3])
    return None


# ---------------------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline / reference arm)
# ---------------------------------------------------------------------------------------
def oracle_sweeps(d, budget_s, max_sweeps, warmup=0):
    import oracle
    K = d["K"]
    p = oracle.plan(d["N"], d["D"], d["row"], d["col"], d["val"], 1, 1)
    s = p.subsets[0]
    prior = oracle.NWPrior(K)
    st = oracle.new_chain(d["X0"][p.row_perm], d["W0"][p.col_perm], K)
    lay = oracle.stage_draw_layout([s], K)
    H = oracle.hyper_block_len(K)

    def one(t):
        """One oracle sweep; returns its time (the draw buffer is made before the clock)."""
        dr = make_draws(d, K, prior.nu0, 1, seed=900 + t)
        t0 = time.perf_counter()
        oracle.sweep_subset(s, st, K, d["tau"], prior, dr[0:H], dr[H:2 * H],
                            dr[lay[(0, "zx")]:lay[(0, "zx")] + s.n * K],
                            dr[lay[(0, "zw")]:lay[(0, "zw")] + s.d * K])
        return time.perf_counter() - t0

    for t in range(warmup):
        one(t)
    done, busy = 0, 0.0
    while done < max_sweeps and (done == 0 or busy < budget_s):
        busy += one(warmup + done)
        done += 1
    return done, busy


def cpu_baseline(d, budget):
    n, secs = oracle_sweeps(d, budget, 1000)
    return {"value": n / secs, "unit": "sweeps/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} full FP64 oracle sweeps of the same workload, single thread "
                      f"({secs:.1f} s, draw generation excluded)"}


def cpu_all_cores(d, budget):
    """The oracle's OpenMP build (row conditionals over all host cores, same results)."""
    import oracle
    try:
        threads = oracle.use_openmp(True)
        n, secs = oracle_sweeps(d, budget, 1000)
    except Exception as e:                       # no OpenMP runtime on this host
        return {"unavailable": f"OpenMP build of the oracle failed: {e}"}
    finally:
        oracle.use_openmp(False)
    return {"value": n / secs, "unit": "sweeps/s", "cores": threads,
            "kind": "oracle, OpenMP over rows",
            "sample": f"{n} full FP64 oracle sweeps of the same workload ({secs:.1f} s, draw "
                      f"generation excluded; hyperparameter step and moments single-threaded)"}


def _reference_line(metric, v, unit, n, secs, config, sample, warmup=0, cores=1,
                    kind="oracle"):
    return {"impl": "reference", "metric": metric, "value": v, "unit": unit, "n_gpus": 1,
            "steps": n, "warmup": warmup, "ms_per_step": secs * 1e3 / n,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config,
            "cpu_baseline": {"value": v, "unit": unit, "cores": cores, "kind": kind,
                             "sample": sample},
            "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


class OraclePP:
    """The oracle's PP sweeps on a grid workload: one PP sweep is one sweep of every subset of
    stage 1, then of stage 2, then of stage 3 (each stage's batch), chains continuing from one
    PP sweep to the next; the propagated factors carry unit Gaussian priors (a sweep's cost does
    not depend on their values).  Draw generation is outside the clock."""

    def __init__(self, d):
        import oracle
        self.d, self.K = d, d["K"]
        self.p = oracle.plan(d["N"], d["D"], d["row"], d["col"], d["val"], d["I"], d["J"])
        self.prior = oracle.NWPrior(self.K)
        K = self.K
        finals = {s.sid: (np.zeros((s.n, K)), np.tile(np.eye(K), (s.n, 1, 1)),
                          np.zeros((s.d, K)), np.tile(np.eye(K), (s.d, 1, 1)))
                  for s in self.p.subsets}
        X0, W0 = d["X0"][self.p.row_perm], d["W0"][self.p.col_perm]
        self.chains = {st: oracle.setup_stage_chains(self.p, st, X0, W0, K, finals)
                       for st in (1, 2, 3)}
        self.t = 0

    def sweep(self):
        """One PP sweep; returns its time in seconds."""
        import oracle
        from paper_1703_00734_gb300 import synth
        secs = 0.0
        for st in (1, 2, 3):
            subs = self.p.stage_subsets(st)
            dr = synth.sweep_draws([(s.n, s.d) for s in subs], self.K, self.prior.nu0,
                                   synth.rng_for(901, st, self.t))
            t0 = time.perf_counter()
            oracle.run_stage(self.p, st, self.chains[st], self.K, self.d["tau"], self.prior,
                             lambda t: dr, 1)
            secs += time.perf_counter() - t0
        self.t += 1
        return secs


def cpu_baseline_pp(d, budget, threads=1):
    """The oracle's PP sweeps/s on the bench workload, time-bounded: single thread (threads=1)
    or its OpenMP build over all host cores (threads=0; bit-identical results)."""
    import oracle
    try:
        used = oracle.use_openmp(threads != 1) if threads != 1 else 1
        o = OraclePP(d)
        n, secs = 0, 0.0
        while n == 0 or secs < budget:
            secs += o.sweep()
            n += 1
    except Exception as e:                       # no OpenMP runtime on this host
        return {"unavailable": f"oracle run failed: {e}"}
    finally:
        if threads != 1:
            oracle.use_openmp(False)
    return {"value": n / secs, "unit": "sweeps/s", "cores": used,
            "kind": "oracle" if threads == 1 else "oracle, OpenMP over rows",
            "sample": f"{n} PP sweeps (one sweep of every subset of the three stages) of the "
                      f"same workload, FP64, {secs:.1f} s, draw generation outside the clock"}


def reference_pp(args, d):
    """The reference arm on the PP workload: the oracle as it stands, its OpenMP build on all
    host cores (row conditionals split over threads, results bit-identical to one thread), on
    the metric of our arm (sweeps/s; each step one PP sweep, a bounded sample of the same
    workload: a whole run of 3 x 200 sweeps would take hours), W untimed and K timed steps."""
    import oracle
    try:
        cores, kind = oracle.use_openmp(True), "oracle, OpenMP over rows"
    except Exception:                            # no OpenMP runtime on this host
        cores, kind = 1, "oracle"
    try:
        o = OraclePP(d)
        for _ in range(args.warmup):
            o.sweep()
        n = max(args.steps, 1)
        secs = sum(o.sweep() for _ in range(n))
    finally:
        oracle.use_openmp(False)
    return _reference_line(METRIC, n / secs, "sweeps/s", n, secs,
                           {"workload": args.workload, "N": d["N"], "D": d["D"],
                            "train_obs": len(d["row"]), "test_obs": len(d["test_row"]),
                            "K": d["K"], "grid": f"{d['I']}x{d['J']}", "precision": "fp64"},
                           f"{n} PP sweeps (one sweep of every subset of the three stages), "
                           f"{cores} threads, {secs:.1f} s, draw generation outside the clock",
                           warmup=args.warmup, cores=cores, kind=kind)


def reference_adjoint(args, d):
    """The oracle's FP64 gradient of the masked log-joint at the initial state, time-bounded."""
    import oracle
    K = d["K"]
    X, W = np.asarray(d["X0"], np.float64), np.asarray(d["W0"], np.float64)
    mu, Lam = np.zeros(K), np.eye(K)
    la = float(np.log(d["tau"]))
    n, secs = 0, 0.0
    while n == 0 or (secs < args.cpu_seconds and n < max(args.steps, 1)):
        t0 = time.perf_counter()
        oracle.logjoint_grad(d["row"], d["col"], d["val"], X, W, la, mu, Lam, mu, Lam)
        secs += time.perf_counter() - t0
        n += 1
    return _reference_line("log-joint gradient evaluations/s (adjoint, K=64)", n / secs,
                           "grad evals/s", n, secs,
                           {"workload": args.workload, "N": d["N"], "D": d["D"],
                            "train_obs": len(d["row"]), "K": K},
                           f"{n} FP64 gradient evaluations of the whole data, single thread")


def run_reference(args, rank):
    if rank != 0:
        return None
    from paper_1703_00734_gb300 import synth as _synth
    mode = MODES.get(args.workload)
    if mode == "partitions":
        return {"impl": "reference", "unavailable": "the metric is the test RMSE after 3 x 1200 "
                "sweeps per grid, which the single-thread oracle does not reach in a bounded run"}
    if _synth.WORKLOADS.get(args.workload, {}).get("I", 1) > 1:
        return reference_pp(args, load_workload(args.workload, args.scale))
    if mode == "adjoint":
        return reference_adjoint(args, load_workload(args.workload, args.scale))
    d = load_workload(args.workload)
    n, secs = oracle_sweeps(d, args.cpu_seconds * 4, max(args.steps, 1),
                            warmup=min(args.warmup, 1))
    v = n / secs
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "sweeps/s", "n_gpus": 1,
            "steps": n, "warmup": min(args.warmup, 1), "ms_per_step": secs * 1e3 / n,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "K": d["K"],
                                            "precision": "fp64", "grid": "1x1"},
            "cpu_baseline": {"value": v, "unit": "sweeps/s", "cores": 1, "kind": "oracle",
                             "sample": f"{n} full sweeps (time-bounded), single thread"},
            "e2e": {"value": v, "unit": "sweeps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "tf32", "fp64"])
    ap.add_argument("--burnin", type=int, default=2)
    ap.add_argument("--pp-sweeps", type=int, default=PP_SWEEPS,
                    help="sweeps per stage of a PP run (grid workloads)")
    ap.add_argument("--pp-burnin", type=int, default=PP_BURNIN)
    ap.add_argument("--fp64-steps", type=int, default=20)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-plain-zipf", action="store_true",
                    help="skip the plain-sweep benchmark added to the default PP line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default launch schedule instead of running the schedule tuner")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--datasets", type=int, default=0,
                    help="simulated-data experiment: independent data sets (0: five)")
    ap.add_argument("--experiment", default="partitions", choices=["partitions", "correlations"],
                    help="simulated data: the partition experiment (Section 5.3) or the "
                         "subset-posterior correlations (Section 5.6)")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink the workload (rows and columns by s, observations by s^2); "
                         "for profiling captures only, not a bench configuration")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    from paper_1703_00734_gb300 import synth as _synth
    pp = _synth.WORKLOADS.get(args.workload, {}).get("I", 1) > 1
    if args.impl == "reference":
        out = run_reference(args, rank)
    else:
        if world > 1:
            import torch
            torch.cuda.set_device(local_rank)
            torch.distributed.init_process_group("nccl")
        if pp:
            out = run_pp(args, rank, world, local_rank)
            if args.workload == WORKLOAD and not args.no_plain_zipf and args.scale == 1.0:
                sub = argparse.Namespace(**vars(args))
                sub.workload = PLAIN_WORKLOAD
                plain = run_ours(sub, rank, world, local_rank)
                if out is not None:
                    out["plain_sweep_zipf"] = plain
        elif MODES.get(args.workload) == "adjoint":
            out = run_adjoint(args, rank, world, local_rank)
        elif MODES.get(args.workload) == "partitions" and args.experiment == "correlations":
            out = run_correlations(args, rank, world, local_rank)
        elif MODES.get(args.workload) == "partitions":
            out = run_partitions(args, rank, world, local_rank)
        else:
            out = run_ours(args, rank, world, local_rank)
        if world > 1:
            barrier(world)
            import torch
            torch.distributed.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
