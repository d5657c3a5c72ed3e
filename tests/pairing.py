"""Test helpers: run the CUDA library (through the C ABI) and the oracle side by side on the
same seeded inputs and draws."""
import numpy as np

import oracle
from paper_1703_00734_gb300 import synth


def parity_tol(cpu, rel=1e-9):
    """Per-row bound of the FP64 mode: |x_gpu - x_cpu|_inf <= rel * (|x_cpu|_inf + 1e-3 rms)."""
    cpu = np.asarray(cpu)
    if cpu.size == 0:
        return np.zeros(0)
    rms = np.sqrt(np.mean(cpu ** 2)) if cpu.size else 0.0
    return rel * (np.abs(cpu).reshape(len(cpu), -1).max(1) + 1e-3 * rms)


def assert_rows_close(gpu, cpu, rel=1e-9, what=""):
    gpu, cpu = np.asarray(gpu), np.asarray(cpu)
    assert gpu.shape == cpu.shape, (what, gpu.shape, cpu.shape)
    if cpu.size == 0:
        return
    err = np.abs(gpu - cpu).reshape(len(cpu), -1).max(1)
    tol = parity_tol(cpu, rel)
    bad = np.nonzero(err > tol)[0]
    assert len(bad) == 0, (f"{what}: {len(bad)} rows over tolerance; worst row {bad[np.argmax(err[bad] / tol[bad])]} "
                           f"err {err[bad].max():.3e} tol {tol[bad].min():.3e}")


class Pair:
    """A library context and the oracle's chains on the same data."""

    def __init__(self, d, K, I=1, J=1, precision="fp64", burnin=0, thin=1, seed=11, center=True,
                 order="decreasing", prior=None, gen=False, propagate=True, **kw):
        """gen: draws from the counter-based generator (the library's device generator with
        draws == NULL, the oracle's own implementation of it), else from synth."""
        from paper_1703_00734_gb300 import bmf
        self.d, self.K, self.seed, self.gen, self.propagate = d, K, seed, gen, propagate
        if not propagate:
            kw["independent"] = True
        if gen:
            kw["seed"] = seed
        self.prior = prior or oracle.NWPrior(K)
        self.burnin, self.thin = burnin, thin
        test = (d["test_row"], d["test_col"], d["test_val"]) if len(d["test_row"]) else None
        self.m = bmf.BMF(d["N"], d["D"], d["row"], d["col"], d["val"], K, d["tau"], precision,
                         I=I, J=J, X0=d["X0"], W0=d["W0"], test=test, burnin=burnin, thin=thin,
                         beta0=self.prior.beta0, nu0=self.prior.nu0, mu0=self.prior.mu0,
                         W0_prior=self.prior.W0, center=center, order=order, **kw)
        self.p = oracle.plan(d["N"], d["D"], d["row"], d["col"], d["val"], I, J,
                             order=order, center=center, row_bounds=kw.get("row_bounds"),
                             col_bounds=kw.get("col_bounds"))
        self.X0 = d["X0"][self.p.row_perm]
        self.W0 = d["W0"][self.p.col_perm]
        self.finals = {}
        self.chains = {}

    def draws(self, stage, t, subsets=None):
        subs = subsets if subsets is not None else self.p.stage_subsets(stage)
        if self.gen:
            return oracle.gen_batch_draws(subs, self.K, self.prior.nu0, self.seed, t + 1)
        return synth.sweep_draws([(s.n, s.d) for s in subs], self.K, self.prior.nu0,
                                 synth.rng_for(self.seed, stage, t))

    def run_stage(self, stage, T, t0=0, gpu=True, cpu=True):
        """T sweeps of a stage on both sides (sweeps t0 .. t0+T-1 of the stage's draws)."""
        subs = self.p.stage_subsets(stage)
        if cpu:
            if t0 == 0:
                self.chains.update(oracle.setup_stage_chains(self.p, stage, self.X0, self.W0,
                                                             self.K, self.finals,
                                                             propagate=self.propagate))
            stage_chains = {s.sid: self.chains[s.sid] for s in subs}
            oracle.run_stage(self.p, stage, stage_chains, self.K, self.d["tau"], self.prior,
                             lambda t: self.draws(stage, t0 + t), T, self.burnin, self.thin)
        stats = None
        if gpu:
            dr = None if self.gen else np.concatenate([self.draws(stage, t0 + t) for t in range(T)])
            stats = self.m.stage(stage, T, dr)
        return stats

    def finish_stage(self, stage):
        for s in self.p.stage_subsets(stage):
            self.finals[s.sid] = oracle.finalize(self.chains[s.sid])

    def compare_subset(self, sid, rel=1e-9, hyper=True):
        X, W, hyp = self.m.get_state(sid)
        st = self.chains[sid]
        assert_rows_close(X, st.X, rel, f"X of subset {sid}")
        assert_rows_close(W, st.W, rel, f"W of subset {sid}")
        if hyper:
            if not st.prior_x:
                assert_rows_close(hyp["LamX"], st.LamX, rel, f"Lambda_X of subset {sid}")
                assert_rows_close(hyp["muX"][None], st.muX[None], rel, f"mu_X of subset {sid}")
            if not st.prior_w:
                assert_rows_close(hyp["LamW"], st.LamW, rel, f"Lambda_W of subset {sid}")
                assert_rows_close(hyp["muW"][None], st.muW[None], rel, f"mu_W of subset {sid}")
