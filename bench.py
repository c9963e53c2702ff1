#!/usr/bin/env python
"""Throughput of the GFCCSD hot path on GB300: converged G(omega) columns per second.

One step = one batch of (omega, p) linear systems of eq. xplin solved by GMRES to
tol through the C ABI, including right-hand sides, left vectors and the G overlaps
(every row of the hot path after the one-time setup of gfcc_create).  The default
workload is the C60-shaped one (o=90 v=450 L=1800, IP, the 30 highest occupied
orbitals, eta 0.005, tol 1e-8): mixed precision (BF16 tensor-core sigma products
inside FP64-accurate iterative refinement), one frequency x 30 orbitals per step.
Beside it the line carries the plain FP64 GPU path on a sample of the same systems
(its columns/s and the mixed path's multiple of it), a check of the mixed G rows
against those FP64 rows, and the CPU oracle's rate.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl gb300|reference]

Under torchrun each rank drives its own GPU with its own context and its own
frequencies (the (omega, p) tasks are independent: weak scaling, no data-path
collective); the timed region is bracketed by barriers and the slowest rank's time
is reported.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2010_04768_gb300.synthetic import workload  # noqa: E402

# ------------------------------------------------------------------------------------------------
# workloads: each step solves `per_step` frequencies x all orbitals of the list
# ------------------------------------------------------------------------------------------------
WORKLOADS = {
    # o=40 v=200 L=800, 40 orbitals nearest the gap, 64 frequencies in [-1.2, 0.5], eta 0.005, tol 1e-8
    "medium-ip-fp64": dict(base="medium", sector="IP", precision="fp64", per_step=1),
    "medium-ip-mixed": dict(base="medium", sector="IP", precision="mixed", per_step=1),
    "medium-ipea-mixed": dict(base="medium", sector="IP+EA", precision="mixed", per_step=1),
    "medium-ip-mixed-4f": dict(base="medium", sector="IP", precision="mixed", per_step=4),
    "medium-ipea-mixed-4f": dict(base="medium", sector="IP+EA", precision="mixed", per_step=4),
    "medium-ipea-fp64": dict(base="medium", sector="IP+EA", precision="fp64", per_step=1),
    # frequency sweeps: each step solves a window of `per_step` consecutive grid frequencies in one call,
    # one frequency per batch, each system started from the initial guess named (GFCC_OPT_GUESS)
    "medium-ipea-mixed-sweep": dict(base="medium", sector="IP+EA", precision="mixed", per_step=8, sweep=True),
    "medium-ipea-mixed-sweep-minres": dict(base="medium", sector="IP+EA", precision="mixed", per_step=8, sweep=True,
                                           guess="minres"),
    "medium-ip-mixed-sweep": dict(base="medium", sector="IP", precision="mixed", per_step=16, sweep=True),
    "medium-ip-mixed-sweep-minres": dict(base="medium", sector="IP", precision="mixed", per_step=16, sweep=True,
                                         guess="minres"),
    "medium-ip-mixed-sweep-learned": dict(base="medium", sector="IP", precision="mixed", per_step=16, sweep=True,
                                          guess="learned"),
    # 16 molecules of uneven size (o ~ U{10..60}, v = 5 o, L = 4 v, 16-96 frequencies in [-1.0, -0.3], 8-32
    # highest occupied orbitals, IP, eta 0.005): each step solves one frequency of every molecule,
    # all molecules at once through gfcc_solve_batch
    "uneven16-ip-mixed": dict(base="uneven16", sector="IP", precision="mixed", per_step=1, uneven=True),
    # C60-shaped: o=90 v=450 L=1800, the 30 highest occupied orbitals, 128 frequencies in [-1.0, -0.3]
    "c60-ip-mixed": dict(base="c60", sector="IP", precision="mixed", per_step=1),
    "c60-ip-fp64": dict(base="c60", sector="IP", precision="fp64", per_step=1),
    # learned initial guesses on the C60-shaped problem (256 frequencies in [-1.0, -0.3]: spacing 0.55
    # eta): each step solves 16 consecutive grid frequencies x 30 orbitals in one call, each system
    # started from the guess named (the learned model needs 8 converged neighbours, so the first
    # frequencies of a window start from zero); the model is trained beforehand on another seed of the
    # same shape
    "c60x256-ip-mixed-sweep": dict(base="c60x256", sector="IP", precision="mixed", per_step=16, sweep=True),
    "c60x256-ip-mixed-sweep-minres": dict(base="c60x256", sector="IP", precision="mixed", per_step=16, sweep=True,
                                          guess="minres"),
    "c60x1024-ip-mixed-sweep": dict(base="c60x1024", sector="IP", precision="mixed", per_step=16, sweep=True),
    "c60x1024-ip-mixed-sweep-minres": dict(base="c60x1024", sector="IP", precision="mixed", per_step=16, sweep=True,
                                           guess="minres"),
    "c60x1024-ip-mixed-sweep-learned": dict(base="c60x1024", sector="IP", precision="mixed", per_step=16, sweep=True,
                                            guess="learned"),
    "c60x256-ip-mixed-sweep-learned": dict(base="c60x256", sector="IP", precision="mixed", per_step=16, sweep=True,
                                           guess="learned"),
    # closed-shell spin-adapted IP (spatial orbitals, FP64), beside the spin-orbital FP64 path on the
    # spin-orbital embedding of the same system
    "medium-closed-shell-ip-fp64": dict(base="medium-closed-shell", sector="IP", precision="fp64", per_step=1),
    "c60-closed-shell-ip-fp64": dict(base="c60-closed-shell", sector="IP", precision="fp64", per_step=1),
    # ground-state CCSD (the step before the Green's function): one step = one T iteration
    "ccsd-medium": dict(ccsd=(40, 200, 800), emulate=True),
    "ccsd-medium-fp64": dict(ccsd=(40, 200, 800), emulate=False),
}
DEFAULT_WORKLOAD = "c60-ip-mixed"
E2E_STEPS = 5        # steps of the end-to-end (host API) measurement: min(steps, E2E_STEPS)
PLAIN_STEP = 1       # plain FP64 leg: the frequency of this timed step (the step's own G rows compared)
ROW_TOL = 1e-6       # mixed vs plain FP64 G rows (relative 2-norm per row)
FREQ_STRIDE = 17   # timed step k takes grid frequency (k * 17) mod n_omega (coprime with 64: covers the grid)
INNER_RESTART = 60   # restart length of the inner GMRES of the mixed-precision refinement (library default)
# DRAM traffic of the tensor-core GEMM launches from ncu captures of the current kernels (profiles/),
# keyed by roofline phase: {"traffic": DRAM bytes per launch, "algorithmic_bytes": bytes one launch
# must move (operands once, output once), "case": the captured shape}.  A phase without a capture of
# its current kernel reports traffic null.
NCU_TRAFFIC = {
    "ring_bf16": {"traffic": 8.094e9, "algorithmic_bytes": 1.476e9,
                  "case": "umma_pair_gemm_kernel at the C60-shaped ring contraction with M = K = 20250, N = 5400 "
                          "(kernel_cases ring-ip-c60-half; profiles/umma_pair_ring_ip_c60half.md): DRAM bytes of one "
                          "launch of that case, not of a bench launch"},
    "ring_emu": {"traffic": 0.710e9, "algorithmic_bytes": 0.332e9,
                 "case": "umma_pair_gemm_kernel on one digit pair at the medium ring shape M = K = 8000, N = 3200 "
                         "(kernel_cases ring-ip-medium-emu; profiles/umma_pair_digit_pairs_ring_ip_medium.md): mean "
                         "of two pair launches, algorithmic bytes 281-383 MB"},
}

FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # SMs x FP64 FMA/clk/SM x 2 flops x max clock


def ip_sigma_flops(o, v):
    """Algorithmic flops of one complex IP sigma product (2 real vectors)."""
    return 2 * (2 * o**3 * v**2 + 0.5 * o**4 * v + 3 * o**2 * v**2 + 4 * o**3 * v + 2 * o**2 * v + 2 * o**2)


def ea_sigma_flops(o, v):
    return 2 * (2 * o**2 * v**3 + 0.5 * o * v**4 + 3 * o * v**3 + 3 * o**2 * v**2)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples: GFCC_CLOCKS_DIR if set, else the temporary directory
        self.path = os.path.join(os.environ.get("GFCC_CLOCKS_DIR") or tempfile.gettempdir(),
                                 f"clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def step_frequency_indices(step, world, rank, per, nw, sweep=False):
    """Grid indices of the frequencies rank `rank` of `world` solves in step `step` (`per` per step on
    a grid of `nw`).  The (omega, p) tasks are independent, so the ranks shard the frequencies and
    share nothing on the data path.  Sweeps: timed step k takes the window of `per` consecutive grid
    frequencies starting at (k world + r) per; single-frequency steps take grid frequency
    ((k world + r) per + j) FREQ_STRIDE mod nw (FREQ_STRIDE coprime with nw, so distinct steps and ranks
    land on distinct frequencies until the grid is used up).  Warm-up steps (negative k) take the top
    end of the grid."""
    if step < 0:
        return [(nw + step * per + j) % nw for j in range(per)]
    base = (step * world + rank) * per
    if sweep:
        return [(base + j) % nw for j in range(per)]
    return [((base + j) * FREQ_STRIDE) % nw for j in range(per)]


def reduce_over_ranks(dist, seconds, columns, device):
    """(slowest rank's time, columns of all ranks): the only collective of a multi-rank run, on the
    timings after the timed region."""
    if dist is None:
        return seconds, columns
    import torch
    t = torch.tensor([seconds, float(columns)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), int(round(float(t[1])))


def sectors_of(spec):
    return ("IP", "EA") if spec["sector"] in ("IP+EA", "BOTH") else (spec["sector"],)


class MediumOracle:
    """The CPU oracle as it stands on the medium workload's IP sector (o=40 v=200 L=800): the
    stand-in for the C60-shaped workload, whose dense oracle intermediates (the ovvv block alone is
    66 GB) do not fit the host.  column(c) solves one (omega, p) IP system with the oracle's GMRES
    (same eta / tol / restart / preconditioner as the workload) and forms its G row; times are
    scaled to the C60-shaped size by the ratio of the IP sigma flops and, when known, of the FP64
    GMRES iteration counts."""

    def __init__(self):
        from oracle.gfcc_ref import GFCCOracle
        self.med = workload("medium")
        pr = self.med.problem()
        t0 = time.perf_counter()
        self.orc = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=self.med.o, sectors=("IP",))
        self.t_setup = time.perf_counter() - t0
        self.omega = self.med.omegas[FREQ_STRIDE % self.med.omegas.size]

    def warm(self):
        """One sigma product (a bounded warm-up of the oracle's code path)."""
        self.orc.ip_apply(self.omega, self.med.eta)(self.orc.ip_rhs(int(self.med.orbitals[0])).astype(complex))

    def column(self, c):
        from oracle.gfcc_ref import gmres
        med, orc = self.med, self.orc
        p = int(med.orbitals[c % med.orbitals.size])
        t0 = time.perf_counter()
        D = (self.omega - 1j * med.eta) + orc.ip_diag()
        x, its, rel, ok = gmres(orc.ip_apply(self.omega, med.eta), orc.ip_rhs(p), med.tol, med.restart, 50, diag=D)
        np.stack([orc.ip_left(int(q)) for q in med.orbitals]) @ x
        return time.perf_counter() - t0, its, bool(ok)

    def extrapolate(self, wl, t_cols, its_cols, its_target=None):
        t_col = float(np.mean(t_cols))
        its_med = float(np.mean(its_cols))
        scale = ip_sigma_flops(wl.o, wl.v) / ip_sigma_flops(self.med.o, self.med.v)
        it_scale = (its_target / its_med) if its_target else 1.0
        t_est = t_col * scale * it_scale
        sample = (f"extrapolated: {len(t_cols)} IP column(s) of the medium workload (o=40 v=200 L=800; omega "
                  f"{self.omega:.4f}, eta {self.med.eta}, tol {self.med.tol}, GMRES({self.med.restart}), diagonal "
                  f"preconditioner) solved by the numpy FP64 oracle, {t_col:.2f} s per column ({its_med:.0f} "
                  f"iterations; oracle setup {self.t_setup:.1f} s excluded like gfcc_create), scaled by the IP "
                  f"sigma flop ratio {scale:.1f} (o={wl.o} v={wl.v} vs o=40 v=200)" +
                  (f" and the iteration ratio {its_target:.1f} / {its_med:.0f} (FP64 GMRES iterations of the "
                   f"C60-shaped systems on the plain FP64 GPU path)" if its_target else
                   " (iteration count taken equal)") +
                  "; the oracle cannot hold the C60-shaped intermediates")
        return {"value": 1.0 / t_est, "unit": "columns/s", "cores": os.cpu_count(), "kind": "oracle",
                "sample": sample, "seconds": t_est}


def cpu_baseline_extrapolated(wl, its_target=None, columns=1):
    """cpu_baseline for the C60-shaped workload: MediumOracle columns scaled to the C60 size."""
    mo = MediumOracle()
    t_cols, its_cols = [], []
    for c in range(columns):
        t, its, ok = mo.column(c)
        t_cols.append(t)
        its_cols.append(its)
    return mo.extrapolate(wl, t_cols, its_cols, its_target)


def cpu_baseline(wl, spec, problem, max_columns=1):
    """The CPU oracle as it stands, on a bounded sample of the same workload: `max_columns` IP columns
    solved by its GMRES (same tolerance, restart and preconditioner); for the EA sector, whose oracle
    sigma product alone takes tens of seconds, one sigma product is timed and an EA column is
    estimated as that time x the GMRES iterations of the sampled IP column(s) (40 without IP)."""
    from oracle.gfcc_ref import GFCCOracle, gmres
    secs = sectors_of(spec)
    t0 = time.perf_counter()
    orc = GFCCOracle(problem.fock, problem.chol, problem.t1, problem.t2, o=wl.o, sectors=secs)
    t_setup = time.perf_counter() - t0
    cols, its_ip, t_ip, t_ea_est, t_sig_ea = 0, 0, 0.0, 0.0, None
    for c in range(max_columns):
        # the frequencies of the timed steps 1, 2, ... (step 0 sits deep in the 2h1p continuum and
        # would take the CPU several minutes per column), first orbital of the list
        om = wl.omegas[((c + 1) * FREQ_STRIDE) % wl.omegas.size]
        p = int(wl.orbitals[0])
        if "IP" in secs:
            t0 = time.perf_counter()
            D = (om - 1j * wl.eta) + orc.ip_diag()
            x, its, rel, ok = gmres(orc.ip_apply(om, wl.eta), orc.ip_rhs(p), wl.tol, wl.restart, 50, diag=D)
            G = np.stack([orc.ip_left(int(q)) for q in wl.orbitals]) @ x
            t_ip += time.perf_counter() - t0
            cols += 1 if ok else 0
            its_ip += its
        if "EA" in secs:
            if t_sig_ea is None:
                y = orc.ea_rhs(p).astype(complex)
                t0 = time.perf_counter()
                orc.ea_apply(om, wl.eta)(y)
                t_sig_ea = time.perf_counter() - t0
            n_it = its_ip / max(1, c + 1) if "IP" in secs else 40
            t_ea_est += t_sig_ea * n_it
            cols += 1
    dt = t_ip + t_ea_est
    sample = (f"{max_columns} (omega, p) column(s) per sector {'+'.join(secs)} of the same workload (omega of timed "
              f"step 1, first orbital), numpy FP64 with the same tol/restart/preconditioner; oracle setup "
              f"{t_setup:.1f} s excluded like gfcc_create")
    if "IP" in secs:
        sample += f"; IP: full GMRES ({its_ip} iterations, {t_ip:.1f} s)"
    if "EA" in secs:
        sample += (f"; EA: one sigma product timed ({t_sig_ea:.1f} s) x the IP iteration count per column "
                   f"(estimated, {t_ea_est:.1f} s)")
    return {"value": cols / dt, "unit": "columns/s", "cores": os.cpu_count(), "kind": "oracle", "sample": sample,
            "seconds": dt}


def train_guess_model(gfcc, spec, wl, seed=1, n_freq=24):
    """Train the learned-guess model on the method's own converged solutions of another problem of
    the same shape (seed `seed`): a zero-guess sweep over n_freq frequencies with the solutions kept,
    3 samples per system, 1500 Adam steps.  The frequencies are spread over the grid, or, on grids
    finer than the broadening (spacing < eta), n_freq consecutive grid frequencies from a quarter of
    the way in, so that the neighbour distances of the training samples are those of a sweep.
    Excluded from the timed region like gfcc_create."""
    from paper_2010_04768_gb300.synthetic import make_problem, mlp_init_params
    t0 = time.perf_counter()
    pr = make_problem(wl.o, wl.v, wl.L, seed=seed)
    g = gfcc.GFCC(pr, sectors=spec["sector"], precision=spec["precision"])
    g.set_option(gfcc.OPT_RESTART, wl.restart)
    g.set_option(gfcc.OPT_KEEP_SOLUTIONS, 1)
    if wl.omegas[1] - wl.omegas[0] < wl.eta:
        q = wl.omegas.size // 4
        om = wl.omegas[q:q + n_freq]
    else:
        om = wl.omegas[np.linspace(0, wl.omegas.size - 1, n_freq).round().astype(int)]
    g.solve(om, wl.eta, wl.orbitals, wl.tol)
    model = gfcc.MLP(mlp_init_params(256, seed), 256, gfcc.MLP_FP32)
    added = model.collect(g, samples_per_system=3, seed=seed)
    g.close()
    loss = model.train(steps=1500, minibatch=256, lr=1e-3, seed=seed)
    ev = model.eval()
    info = {"train_problem_seed": seed, "train_frequencies": int(n_freq), "samples": int(added),
            "final_loss": loss, "eval": {k: float(v) for k, v in ev.items()},
            "seconds": time.perf_counter() - t0}
    return model, info


def run_reference(args, world, rank):
    """--impl reference: the CPU oracle (the baseline of this hot path) on rank 0 only.  Each step
    is a bounded sample of the workload: one (omega, p) column solved by the oracle (for the
    C60-shaped workload: one medium-workload IP column, extrapolated; see MediumOracle); each
    warm-up step is one oracle sigma product."""
    if rank != 0:
        return 0
    spec = WORKLOADS[args.workload]
    if spec.get("uneven"):
        print(json.dumps({"impl": "reference", "unavailable": "the oracle has no multi-molecule batch; run the "
                          "reference arm on a single-molecule workload"}), flush=True)
        return 0
    if spec.get("ccsd"):
        # the oracle's T residual at half the shape, scaled by the o^2 v^4 ratio (the oracle's vvvv
        # block at the full shape alone would be 12.8 GB); each step is one such residual
        from oracle import ccsd_ref
        from paper_2010_04768_gb300.synthetic import make_problem
        o, v, L = spec["ccsd"]
        so, sv, sL = o // 2, v // 2, L // 2
        sp = make_problem(so, sv, sL, seed=0, with_t=False)
        rng = np.random.default_rng(0)
        st1 = 0.01 * rng.standard_normal((so, sv))
        g = 0.02 * rng.standard_normal((so, so, sv, sv))
        st2 = 0.25 * (g - g.transpose(1, 0, 2, 3) - g.transpose(0, 1, 3, 2) + g.transpose(1, 0, 3, 2))
        for _ in range(args.warmup):
            ccsd_ref.t_residuals(sp.fock, sp.chol, st1, st2, so)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ccsd_ref.t_residuals(sp.fock, sp.chol, st1, st2, so)
        ts = (time.perf_counter() - t0) / max(1, args.steps)
        scale = (o / so) ** 2 * (v / sv) ** 4
        val = 1.0 / (ts * scale)
        sample = (f"extrapolated: oracle T residuals at o={so} v={sv} L={sL}, {ts:.2f} s each, scaled by the "
                  f"o^2 v^4 ratio {scale:.0f}")
        print(json.dumps({"impl": "reference", "metric": "CCSD T iterations/sec", "value": val, "unit": "iterations/s",
                          "n_gpus": 0, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * ts * scale,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic",
                          "config": {"workload": f"ground-state CCSD o={o} v={v} L={L} (medium shape)"},
                          "cpu_baseline": {"value": val, "unit": "iterations/s", "cores": os.cpu_count(),
                                           "kind": "oracle", "sample": sample},
                          "e2e": {"value": val, "unit": "iterations/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return 0
    wl = workload(spec["base"])
    if wl.name.startswith("c60") and not wl.closed_shell:
        mo = MediumOracle()
        for _ in range(args.warmup):
            mo.warm()
        t_cols, its_cols = [], []
        for k in range(args.steps):
            t, its, ok = mo.column(k)
            t_cols.append(t)
            its_cols.append(its)
        res = mo.extrapolate(wl, t_cols, its_cols)
        seconds = res["seconds"] * args.steps
    else:
        problem = wl.problem()
        if wl.closed_shell:
            # the closed-shell oracle; each step one column (the frequency of timed step 1)
            cols = [cpu_baseline_closed_shell(wl, problem) for _ in range(max(1, args.steps))]
            seconds = sum(c["seconds"] for c in cols)
            res = dict(cols[0], value=len(cols) / seconds)
        else:
            res = cpu_baseline(wl, spec, problem, max_columns=max(1, args.steps))
            seconds = res["seconds"]
    line = {"metric": "converged G(omega) columns/sec", "value": res["value"], "unit": "columns/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * seconds / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": config_of(spec, wl, 1),
            "cpu_baseline": {k: res[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": res["value"], "unit": "columns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def config_of(spec, wl, world):
    return {"workload": f"{wl.name}: o={wl.o} v={wl.v} L={wl.L}, sector {spec['sector']}, "
                        f"{spec['per_step']} frequency x {wl.orbitals.size} orbitals per step per GPU",
            "o": wl.o, "v": wl.v, "L": wl.L, "sector": spec["sector"], "precision": spec["precision"],
            "eta": wl.eta, "tol": wl.tol, "restart": wl.restart,
            **({"inner_restart": INNER_RESTART} if spec["precision"] == "mixed" else {}), "preconditioner": "diag",
            "columns_per_step": spec["per_step"] * int(wl.orbitals.size) * len(sectors_of(spec)) * world,
            "parallelism": f"{world} independent GPU(s), frequencies sharded", "l2": "inputs larger than L2 "
            "(ring matrix and Krylov basis are each > 129 MB)",
            **({"closed_shell": "spin-adapted IP over spatial orbitals (gfcc_create_rhf); contractions of at least "
                                "1e9 flops as FP64-accurate digit-plane products"} if wl.closed_shell else {})}


def uneven_specs(seed=4, count=16):
    """The molecules of the uneven batch: seeded draws of o, frequency count and orbital count."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        o = int(rng.integers(10, 61))
        nf = int(rng.integers(16, 97))
        no = int(min(o, rng.integers(8, 33)))
        out.append(dict(o=o, v=5 * o, L=20 * o, n_freq=nf, n_orb=no, seed=100 + k))
    return out


def run_uneven(args, spec, world, rank, dist=None):
    """Uneven multi-molecule batch: one context per molecule, every step one frequency of each
    molecule x its orbitals, solved concurrently by gfcc_solve_batch (host API: G read back every
    step; the value is host-timed around the synchronous call)."""
    import torch
    from paper_2010_04768_gb300 import gfcc
    from paper_2010_04768_gb300.synthetic import make_problem
    mols = uneven_specs()
    ctxs, grids, orbs = [], [], []
    t0 = time.perf_counter()
    for m in mols:
        pr = make_problem(m["o"], m["v"], m["L"], seed=m["seed"])
        g = gfcc.GFCC(pr, sectors=spec["sector"], precision=spec["precision"])
        g.set_option(gfcc.OPT_RESTART, 30)
        ctxs.append(g)
        grids.append(np.linspace(-1.0, -0.3, m["n_freq"]))
        orbs.append(np.arange(m["o"] - m["n_orb"], m["o"], dtype=np.int32))
        del pr
    setup_s = time.perf_counter() - t0
    eta, tol = 0.005, 1e-8

    def step(k):
        # rank r, step k: molecule i solves its grid frequency ((k world + r) 7 + i) mod n_freq (warm-up
        # steps, negative k, stay off the timed ones); ranks share nothing on the data path
        kk = k * world + rank if k >= 0 else k
        reqs = [(grids[i][[(kk * 7 + i) % grids[i].size]], eta, orbs[i], tol) for i in range(len(ctxs))]
        Gs, codes = gfcc.solve_batch(ctxs, reqs)
        cols = 0
        for g in ctxs:
            cols += int(np.sum(g.stats()[2] == 0))
        return cols

    for k in range(args.warmup):
        step(-1 - k)
    launches0 = gfcc.launch_count()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    with Clocks(torch.cuda.current_device()) as clk:
        t0 = time.perf_counter()
        cols = sum(step(k) for k in range(args.steps))
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        dt = time.perf_counter() - t0
    launches = gfcc.launch_count() - launches0
    dt, cols = reduce_over_ranks(dist, dt, cols, "cuda")
    line = {
        "metric": "converged G(omega) columns/sec", "value": cols / dt, "unit": "columns/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f64", "data": "synthetic",
        "config": {"workload": "uneven16: 16 molecules, o ~ U{10..60}, v = 5o, L = 4v, one frequency x 8-32 "
                               "orbitals of each per step, IP, mixed precision, gfcc_solve_batch",
                   "molecules": mols, "eta": eta, "tol": tol, "columns_per_step": int(sum(o.size for o in orbs)),
                   "l2": "inputs larger than L2"},
        "e2e": {"value": cols / dt, "unit": "columns/s", "h2d_bytes_per_step": int(sum(8 + 4 * o.size for o in orbs)),
                "d2h_bytes_per_step": int(sum(16 * o.size * o.size for o in orbs)),
                "note": "the step itself is the host API call (host arrays in and out)"},
        "setup_s": setup_s, "gpu_launches": int(launches), "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    for g in ctxs:
        g.close()
    return 0


def run_ccsd(args, spec, world, rank, dist=None):
    """Ground-state CCSD on the device (gfcc_ccsd): warm-up iterations from zero amplitudes, then
    exactly `steps` T iterations (residual, Jacobi step, DIIS) from the warmed-up amplitudes, timed by
    the library around its iteration loop (stream-synchronised).  The e2e figure is the same call
    host-timed (Hamiltonian and amplitudes uploaded, amplitudes read back).  Each rank solves its own
    problem (seed = rank): replicas, no collective.  A full T + Lambda solve of the same problem is
    reported beside it, and the CPU oracle's T residual on a smaller problem, scaled."""
    import torch
    from paper_2010_04768_gb300 import gfcc
    from paper_2010_04768_gb300.synthetic import make_problem
    o, v, L = spec["ccsd"]
    pr = make_problem(o, v, L, seed=rank, with_t=False)
    t1, t2, _, _, info_w, _ = gfcc.ccsd(pr.fock, pr.chol, o, tol=1e-14, max_iter=max(1, args.warmup),
                                        want_lambda=False, emulate=spec["emulate"])
    launches0 = gfcc.launch_count()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    with Clocks(torch.cuda.current_device()) as clk:
        t0 = time.perf_counter()
        torch.cuda.nvtx.range_push("step")   # lets a profiler select the timed iterations
        g1, g2, _, _, info, code = gfcc.ccsd(pr.fock, pr.chol, o, tol=1e-14, max_iter=args.steps, want_lambda=False,
                                             emulate=spec["emulate"], guess=(t1, t2))
        torch.cuda.nvtx.range_pop()
        e2e_s = time.perf_counter() - t0
    launches = gfcc.launch_count() - launches0
    dt, iters = reduce_over_ranks(dist, info["t_seconds"], int(info["t_iters"]), "cuda")
    peaks = measured_peaks()
    flops = info["t_flops_per_iter"]
    achieved = flops * args.steps / info["t_seconds"] / 1e12
    if spec["emulate"]:
        peak, bound = peaks.get("bf16_tflops_sustained", 1727.1), "tensor"
        pnote = ("bf16_tflops_sustained of measured; achieved = the iteration's counted FP64 contraction flops "
                 "(method flops, one product per FP64-accurate contraction) / iteration time")
    else:
        peak, bound = FP64_PEAK_TFLOPS, "alu"
        pnote = "FP64 DFMA peak derived from 152 SMs x 2 FMA/clk x 2070 MHz; achieved = counted flops / time"
    # a full T + Lambda solve of the same problem (not timed as steps; digit-plane contractions only:
    # on the FP64 units a full solve of this shape takes several minutes)
    full, fcode = {}, None
    if spec["emulate"]:
        _, _, _, _, full, fcode = gfcc.ccsd(pr.fock, pr.chol, o, tol=1e-8, max_iter=100, emulate=True)
    line = {
        "metric": "CCSD T iterations/sec", "value": iters / dt, "unit": "iterations/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(1, iters), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16-digit-planes+f64" if spec["emulate"] else "f64",
        "data": "synthetic",
        "config": {"workload": f"ground-state CCSD o={o} v={v} L={L} (medium shape), T iterations from warmed-up "
                               "amplitudes", "emulate": bool(spec["emulate"]), "l2": "inputs larger than L2"},
        "e2e": {"value": args.steps / e2e_s, "unit": "iterations/s",
                "h2d_bytes_per_step": int(8 * (pr.fock.size + pr.chol.size + t1.size + t2.size) / args.steps),
                "d2h_bytes_per_step": int(8 * (t1.size + t2.size) / args.steps),
                "note": "host-timed gfcc_ccsd call: upload, setup of the call, the iterations, read-back"},
        "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None, "note": pnote, "flops_per_iteration": flops},
        "full_solve": ({"code": fcode, "e_corr": full["e_corr"], "t_iters": full["t_iters"],
                        "t_seconds": full["t_seconds"], "lambda_iters": full["lambda_iters"],
                        "lambda_seconds": full["lambda_seconds"], "tol": 1e-8} if full else None),
        "gpu_launches": int(launches), "clocks": clk.summary(), "code": code,
    }
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle's T residual (numpy FP64, all host cores) at o/2, v/2, L/2, scaled by the
        # o^2 v^4 ratio of the dominant ladder term
        from oracle import ccsd_ref
        so, sv, sL = o // 2, v // 2, L // 2
        sp = make_problem(so, sv, sL, seed=0, with_t=False)
        rng = np.random.default_rng(0)
        st1 = 0.01 * rng.standard_normal((so, sv))
        g = 0.02 * rng.standard_normal((so, so, sv, sv))
        st2 = 0.25 * (g - g.transpose(1, 0, 2, 3) - g.transpose(0, 1, 3, 2) + g.transpose(1, 0, 3, 2))
        t0 = time.perf_counter()
        ccsd_ref.t_residuals(sp.fock, sp.chol, st1, st2, so)
        ts = time.perf_counter() - t0
        scale = (o / so) ** 2 * (v / sv) ** 4
        line["cpu_baseline"] = {"value": 1.0 / (ts * scale), "unit": "iterations/s", "cores": os.cpu_count(),
                                "kind": "oracle",
                                "sample": f"extrapolated: one oracle T residual at o={so} v={sv} L={sL} took {ts:.2f} s, "
                                          f"scaled by the o^2 v^4 ratio {scale:.0f}"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain-fp64", action="store_true")
    ap.add_argument("--no-mor", action="store_true")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch
    from paper_2010_04768_gb300 import gfcc
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    spec = WORKLOADS[args.workload]
    if spec.get("uneven"):
        return run_uneven(args, spec, world, rank, dist)
    if spec.get("ccsd"):
        return run_ccsd(args, spec, world, rank, dist)
    wl = workload(spec["base"])
    model = guess_train = None
    if spec.get("guess") == "learned":
        # trained (and its context freed) before the timed context exists: two C60-shaped contexts
        # and their setup temporaries do not fit on the device together
        model, guess_train = train_guess_model(gfcc, spec, wl)
    problem = wl.problem()
    t0 = time.perf_counter()
    ctx = gfcc.GFCC(problem, sectors=spec["sector"], precision=spec["precision"], closed_shell=wl.closed_shell)
    setup_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    ctx.set_stream(stream.cuda_stream)
    ctx.set_option(gfcc.OPT_RESTART, wl.restart)
    ctx.set_option(gfcc.OPT_INNER_RESTART, INNER_RESTART)
    ctx.set_option(gfcc.OPT_PRECOND, gfcc.PRECOND_DIAG)
    nw = wl.omegas.size
    no = int(wl.orbitals.size)
    per = spec["per_step"]
    orb_dev = torch.tensor(wl.orbitals, dtype=torch.int32, device="cuda")
    G_dev = torch.zeros((per, no, no, 2), dtype=torch.float64, device="cuda")
    if spec.get("sweep"):
        ctx.set_option(gfcc.OPT_BATCH, no)
    if spec.get("guess") == "minres":
        ctx.set_option(gfcc.OPT_GUESS, gfcc.GUESS_MINRES)
    elif spec.get("guess") == "learned":
        ctx.set_guess_model(model)
        ctx.set_option(gfcc.OPT_GUESS, gfcc.GUESS_LEARNED)

    def freqs(step):
        return wl.omegas[step_frequency_indices(step, world, rank, per, nw, bool(spec.get("sweep")))]

    iter_log = []

    def device_step(k):
        om = torch.tensor(freqs(k), dtype=torch.float64, device="cuda")
        code = ctx.solve_device(om.data_ptr(), per, wl.eta, orb_dev.data_ptr(), no, wl.tol, G_dev.data_ptr())
        it, rr, st = ctx.stats()
        if k >= 0:
            kind, _, rel0 = ctx.guess_stats()
            outer = ctx.refine_stats()
            iter_log.append((int(it.sum()), it.size, int(np.sum(kind != 0)), float(np.mean(rel0)), int(outer.sum())))
        return int(np.sum(st == 0)), code

    for k in range(args.warmup):
        device_step(-1 - k)
    barrier()
    ctx.profile(True)
    launches0 = gfcc.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    converged = 0
    with Clocks(local) as clk:
        barrier()
        ev0.record(stream)
        for k in range(args.steps):
            torch.cuda.nvtx.range_push("step")   # lets a profiler select the timed steps
            c, _ = device_step(k)
            torch.cuda.nvtx.range_pop()
            converged += c
        ev1.record(stream)
        barrier()
    launches = gfcc.launch_count() - launches0
    dt = ev0.elapsed_time(ev1) / 1e3
    prof = ctx.profile_read()
    ctx.profile(False)
    dt, total_cols = reduce_over_ranks(dist, dt, converged, "cuda")
    value = total_cols / dt

    # end to end through the host C ABI: host omegas / orbitals in pinned memory, G read back every step
    # (the first min(steps, E2E_STEPS) timed steps' frequencies)
    e2e_steps = max(1, min(args.steps, E2E_STEPS))
    om_pin = torch.empty(per, dtype=torch.float64, pin_memory=True)
    orb_pin = torch.tensor(wl.orbitals, dtype=torch.int32).pin_memory()
    G_pin = torch.empty((per, no, no, 2), dtype=torch.float64, pin_memory=True)
    G_e2e = []
    barrier()
    t0 = time.perf_counter()
    e2e_cols = 0
    for k in range(e2e_steps):
        om_pin.numpy()[:] = freqs(k)
        G, code = ctx.solve(om_pin.numpy(), wl.eta, orb_pin.numpy(), wl.tol)
        G_pin.numpy().reshape(-1)[:] = G.view(np.float64).reshape(-1)
        if k <= PLAIN_STEP:
            G_e2e.append(G.copy())
        e2e_cols += int(np.sum(ctx.stats()[2] == 0))
    barrier()
    e2e_dt = time.perf_counter() - t0
    e2e_dt, e2e_cols = reduce_over_ranks(dist, e2e_dt, e2e_cols, "cuda")

    # plain FP64 GPU path on a sample of the same systems (mixed workloads only): the rows of PLAIN_SAMPLE
    # orbitals of the list at the frequency of timed step 0, solved by FP64 GMRES with the FP64 sigma
    # product on the same context (gfcc_solve_block: rows over the sample, columns over the whole list)
    plain = row_check = None
    ks = min(PLAIN_STEP, len(G_e2e) - 1)
    if spec["precision"] == "mixed" and rank == 0 and not args.no_plain_fp64:
        plain, row_check = plain_fp64_leg(gfcc, ctx, wl, freqs(ks)[:1], G_e2e[ks][:1], stream)
    spin_orbital = None
    if wl.closed_shell and rank == 0 and not args.no_plain_fp64:
        spin_orbital = spin_orbital_leg(gfcc, problem, wl, freqs(ks)[:1], G_e2e[ks][:1])
    mor = None
    if (rank == 0 and not args.no_mor and len(sectors_of(spec)) == 1 and not spec.get("sweep")
            and not wl.closed_shell):
        mor = mor_leg(gfcc, ctx, wl, spec, freqs(0)[0], G_e2e[0][0])

    peaks = measured_peaks()
    rf = roofline_entries(prof, spec, peaks, closed_shell=wl.closed_shell)
    dominant = max(rf, key=lambda k: rf[k]["ms_total"]) if rf else None
    # sigma TFLOP/s: algorithmic flops of every complex sigma product (inner BF16, FP64 and the
    # FP64-accurate residuals) at F_IP / F_EA each, over the device time of the sigma products
    sigma_ms, _, sigma_fl = prof["sigma"]
    sigma_tflops = sigma_fl / (sigma_ms / 1e3) / 1e12 if sigma_ms > 0 else None
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    line = {
        "metric": "converged G(omega) columns/sec", "value": value, "unit": "columns/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": ("bf16-digit-planes+f64" if wl.closed_shell else "f64" if spec["precision"] == "fp64" else "bf16+f64"),
        "data": "synthetic", "config": config_of(spec, wl, world),
        "e2e": {"value": e2e_cols / e2e_dt, "unit": "columns/s", "h2d_bytes_per_step": 8 * per + 4 * no,
                "d2h_bytes_per_step": 16 * per * no * no, "steps": e2e_steps,
                "note": f"the first {e2e_steps} timed steps' frequencies through gfcc_solve (host arrays in and out)"},
        "roofline": rf.get(dominant),
        "roofline_other": {k: v for k, v in rf.items() if k != dominant},
        "sigma_tflops": sigma_tflops,
        "phases_ms": {k: round(v[0], 3) for k, v in prof.items()},
        "setup_s": setup_s,
        "iterations_per_column": sum(x[0] for x in iter_log) / max(1, sum(x[1] for x in iter_log)),
        "fp64_residuals_per_column": sum(x[4] for x in iter_log) / max(1, sum(x[1] for x in iter_log)),
        "guess": {"kind": spec.get("guess", "zero"),
                  "guessed_fraction": sum(x[2] for x in iter_log) / max(1, sum(x[1] for x in iter_log)),
                  "mean_initial_relres": float(np.mean([x[3] for x in iter_log])) if iter_log else None,
                  "training": guess_train},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    # device time of the solve calls inside the timed phases (sigma products, Arnoldi, least squares,
    # right-hand sides / left vectors / overlaps, guesses); the rest is launch and host-read gaps
    inside = sum(prof[k][0] for k in ("sigma", "arnoldi", "lsq", "overlap", "guess"))
    if prof["solve"][0] > 0:
        line["solve_time_in_phases"] = {"solve_ms": prof["solve"][0], "phases_ms": inside,
                                        "fraction": inside / prof["solve"][0]}
    if mor is not None:
        line["mor"] = mor
    if spin_orbital is not None:
        line["spin_orbital_fp64"] = spin_orbital
        line["vs_spin_orbital_fp64"] = value / spin_orbital["value"] if spin_orbital["value"] else None
    if plain is not None:
        line["plain_fp64"] = plain
        line["vs_plain_fp64"] = value / plain["value"] if plain["value"] else None
        line["sampled_row_check"] = row_check
    if not args.no_cpu_baseline:
        try:
            if wl.name.startswith("c60") and not wl.closed_shell:
                cb = cpu_baseline_extrapolated(wl, plain["iterations_per_column"] if plain else None)
            elif wl.closed_shell:
                cb = cpu_baseline_closed_shell(wl, problem)
            else:
                cb = cpu_baseline(wl, spec, problem, max_columns=1)
            line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        except Exception as e:  # report, do not hide, a failing baseline
            line["cpu_baseline"] = {"value": None, "error": repr(e)}
    print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def plain_fp64_leg(gfcc, ctx, wl, om, G_mixed, stream):
    """Plain FP64 GPU path (FP64 sigma products, FP64 GMRES, same preconditioner, restart and tol) on
    one row of G, the highest orbital of the list (the HOMO for the valence list), at frequency om
    (a timed step's), on the mixed context's FP64 operators; its columns/s, and the relative 2-norm
    error of the mixed G row (G_mixed[0][row]) against it.  (The FP64 path runs at the rate of the
    FP64 units, about 0.9 s per sigma product of one C60-shaped system, so a sample of one system keeps
    this leg to about a minute at a frequency of average difficulty.)"""
    import torch
    no = int(wl.orbitals.size)
    rows = [no - 1]
    P = wl.orbitals[rows]
    ctx.set_option(gfcc.OPT_PRECISION, gfcc.PREC_FP64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    G64, code = ctx.solve_block(om, wl.eta, P, wl.orbitals, wl.tol)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    it, rr, st = ctx.stats()
    ctx.set_option(gfcc.OPT_PRECISION, gfcc.PREC_MIXED_BF16)
    cols = int(np.sum(st == 0))
    errs = [float(np.linalg.norm(G_mixed[0, r] - G64[0, a]) / np.linalg.norm(G64[0, a])) for a, r in enumerate(rows)]
    plain = {"value": cols / dt, "unit": "columns/s", "columns": cols, "seconds": dt,
             "iterations_per_column": float(np.mean(it)), "max_relres": float(np.max(rr)),
             "sample": f"{len(rows)} (omega, p) IP system(s) of the same workload (omega of timed step {PLAIN_STEP} = "
                       f"{om[0]:.5f}, "
                       f"orbitals {P.tolist()}) with their G rows over all {no} orbitals, solved in one call "
                       f"(gfcc_solve_block) by FP64 GMRES({wl.restart}) with FP64 sigma products (DFMA "
                       f"contractions), same tol / preconditioner, on the same context; host-timed"}
    check = {"rows": P.tolist(), "omega": float(om[0]), "max_rel_err": max(errs), "rel_err": errs, "tol": ROW_TOL,
             "passed": bool(max(errs) <= ROW_TOL and cols == len(rows))}
    return plain, check


def spin_orbital_leg(gfcc, problem, wl, om, G_cs):
    """The same system through the spin-orbital FP64 path: the spin-orbital embedding of the closed-shell
    problem (2o occupied, 2v virtual spin-orbitals), one row of G (the highest orbital of the list, alpha
    spin) at frequency om (a timed step's) by gfcc_solve_block with the columns over the alpha spin-orbitals
    of the list; its columns/s (host-timed, setup excluded) and the relative 2-norm difference of the
    closed-shell G row (G_cs[0][row]) from it."""
    import torch
    from paper_2010_04768_gb300.synthetic import Problem
    o, v = wl.o, wl.v
    n = o + v
    al = np.where(np.arange(n) < o, np.arange(n), 2 * o + (np.arange(n) - o))   # alpha spin-orbital of p
    be = np.where(np.arange(n) < o, o + np.arange(n), 2 * o + v + (np.arange(n) - o))
    F = np.zeros((2 * n, 2 * n))
    F[np.ix_(al, al)] = problem.fock
    F[np.ix_(be, be)] = problem.fock
    Ls = np.zeros((problem.L, 2 * n, 2 * n))
    Ls[:, al[:, None], al[None, :]] = problem.chol
    Ls[:, be[:, None], be[None, :]] = problem.chol
    # spin-orbital amplitudes: T_IJ^AB = d(sI,sA) d(sJ,sB) t_ij^ab - d(sI,sB) d(sJ,sA) t_ij^ba
    so_o, so_v = np.repeat([0, 1], o), np.repeat([0, 1], v)
    io, iv = np.tile(np.arange(o), 2), np.tile(np.arange(v), 2)
    T1 = (so_o[:, None] == so_v[None, :]) * problem.t1[io][:, iv]
    t = problem.t2[io][:, io][:, :, iv][:, :, :, iv]
    d1 = (so_o[:, None, None, None] == so_v[None, None, :, None]) & (so_o[None, :, None, None] == so_v[None, None, None, :])
    d2 = (so_o[:, None, None, None] == so_v[None, None, None, :]) & (so_o[None, :, None, None] == so_v[None, None, :, None])
    T2 = np.ascontiguousarray(d1 * t - d2 * np.swapaxes(t, 2, 3))
    del t, d1, d2
    t0 = time.perf_counter()
    g = gfcc.GFCC(Problem(o=2 * o, v=2 * v, L=problem.L, fock=F, chol=Ls, t1=T1, t2=T2), sectors="IP")
    setup_s = time.perf_counter() - t0
    g.set_option(gfcc.OPT_RESTART, wl.restart)
    g.set_option(gfcc.OPT_PRECOND, gfcc.PRECOND_DIAG)
    no = int(wl.orbitals.size)
    row = no - 1
    cols = al[wl.orbitals].astype(np.int32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Gso, code = g.solve_block(om, wl.eta, cols[row:row + 1], cols, wl.tol)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    it, rr, st = g.stats()
    g.close()
    done = int(np.sum(st == 0))
    err = float(np.linalg.norm(G_cs[0, row] - Gso[0, 0]) / np.linalg.norm(Gso[0, 0]))
    return {"value": done / dt, "unit": "columns/s", "columns": done, "seconds": dt, "setup_s": setup_s,
            "iterations_per_column": float(np.mean(it)), "g_row_rel_diff": err,
            "sample": f"1 (omega, p) IP system (omega {om[0]:.5f}, spatial orbital {int(wl.orbitals[row])} alpha) of "
                      f"the spin-orbital embedding (o={2 * o} v={2 * v} spin-orbitals, FP64 sigma and GMRES({wl.restart}),"
                      f" same tol and preconditioner), its G row over the list's alpha spin-orbitals; host-timed"}


def cpu_baseline_closed_shell(wl, problem):
    """The closed-shell oracle (closed-form spatial equations, numpy FP64) on one column of the workload:
    the first orbital of the list at the frequency of timed step 1, GMRES with the same tol, restart and
    preconditioner; its setup excluded like gfcc_create."""
    from oracle.rhf_ref import RHFClosed
    from oracle.gfcc_ref import gmres
    t0 = time.perf_counter()
    C = RHFClosed(problem.fock, problem.chol, problem.t1, problem.t2, o=wl.o)
    t_setup = time.perf_counter() - t0
    om = wl.omegas[FREQ_STRIDE % wl.omegas.size]
    z = om - 1j * wl.eta
    t0 = time.perf_counter()
    x, its, rel, ok = gmres(lambda y: z * y + C.sigma(y), C.rhs(int(wl.orbitals[0])), wl.tol, wl.restart, 50,
                            diag=z + C.diag())
    np.stack([C.left(int(q)) for q in wl.orbitals]) @ x
    dt = time.perf_counter() - t0
    return {"value": (1 if ok else 0) / dt, "unit": "columns/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"1 closed-shell IP column (omega {om:.5f}, orbital {int(wl.orbitals[0])}): {its} GMRES iterations "
                      f"in {dt:.1f} s; oracle setup {t_setup:.1f} s excluded", "seconds": dt}


MOR_SAMPLES = 3       # model-order reduction leg: frequencies whose solutions span the subspace
MOR_GRID = 1000       # model G evaluated on this many frequencies over the workload's window


def mor_leg(gfcc, ctx, wl, spec, om0, G0):
    """Model-order reduction (eq. model) on the workload: the full systems of MOR_SAMPLES frequencies of
    the grid (its two ends and middle, all orbitals) span the subspace; the model G over MOR_GRID
    frequencies of the window; its accuracy at the sampled frequencies (interpolation) and at the
    frequency of timed step 0 (not sampled) against that step's full solve."""
    import torch
    sector = sectors_of(spec)[0]
    samp = np.array([wl.omegas[0], wl.omegas[wl.omegas.size // 2], wl.omegas[-1]])
    if np.any(np.abs(samp - om0) < 1e-12):
        samp = samp + 0.5 * (wl.omegas[1] - wl.omegas[0])
    mor = gfcc.MOR(ctx, sector)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Gs, code = mor.expand(samp, wl.eta, wl.orbitals, wl.tol)
    torch.cuda.synchronize()
    t_expand = time.perf_counter() - t0
    grid = np.linspace(wl.omegas[0], wl.omegas[-1], MOR_GRID)
    t0 = time.perf_counter()
    Gm = mor.green(grid, wl.eta, wl.orbitals)
    torch.cuda.synchronize()
    t_model = time.perf_counter() - t0
    Gi = mor.green(samp, wl.eta, wl.orbitals)
    G0m = mor.green(np.array([om0]), wl.eta, wl.orbitals)[0]
    m = mor.dim()
    mor.close()
    no = int(wl.orbitals.size)
    return {"subspace_dim": m, "sampled_omegas": samp.tolist(), "expand_s": t_expand, "expand_code": int(code),
            "grid_points": MOR_GRID, "model_s": t_model, "model_columns_per_s": MOR_GRID * no / t_model,
            "interpolation_max_rel_err": float(np.abs(Gi - Gs).max() / np.abs(Gs).max()),
            "unsampled_omega": float(om0),
            "unsampled_max_rel_err": float(np.abs(G0m - G0).max() / np.abs(G0).max()),
            "note": "expand = full solves of the sampled frequencies + Gram-Schmidt + projection (sigma products "
                    "of the basis); model columns = G rows of the grid's (omega, p) from the dense model "
                    "solves; errors relative to max |G|"}


# roofline candidates: (phase, bound, kernel label, peak key); the FP64 ring phase runs on the DFMA
# units, the tensor-core phases against the measured sustained BF16 rate (kernels timed inside a long
# step), the HBM phases against the measured copy bandwidth
def roofline_entries(prof, spec, peaks, closed_shell=False):
    bf16 = peaks.get("bf16_tflops_sustained", 1727.1)
    hbm = peaks.get("hbm_gbs", 6761.6)
    fp64 = spec["precision"] == "fp64"
    cands = [
        ("ring", "tensor", "umma_bf16_gemm_kernel / umma_pair_gemm_kernel on digit planes + combine (the three "
                           "FP64-accurate ring contractions of the closed-shell operator)") if closed_shell else
        ("ring", "alu", "contract_f64_kernel (FP64 ring contraction)"),
        ("vvvv", "alu" if fp64 else "tensor", "contract_f64_kernel (FP64 EA vvvv contraction)" if fp64 else
         "umma_bf16_gemm_kernel (BF16 EA vvvv contraction)"),
        ("ring_bf16", "tensor", "umma_bf16_gemm_kernel (BF16 ring contraction of the inner sigma)"),
        ("bf16_other", "tensor", "umma_bf16_gemm_kernel + reduce_splits_kernel (the other BF16 products of the "
                                 "inner sigma: oooo, three-body, 1h row)"),
        ("ring_emu", "tensor", "umma_bf16_gemm_kernel / umma_emu_kernel + combine_int_kernel + finalize_kernel "
                               "(FP64-accurate ring contraction of the refinement residual from BF16 digit planes)"),
        ("emu_other", "tensor", "umma_emu_kernel / umma_bf16_gemm_kernel + digit slicing (the other FP64-accurate "
                                "products of the residual: oooo / vvvv, three-body, 1h / 1p row)"),
        ("unpack", "hbm", "unpack_ip_kernel / unpack_ea_tile_kernel / digit kernels (packed vectors into the "
                          "contraction layouts)"),
        ("epilogue", "hbm", "epi::ip2_kernel / epi::ea2_kernel (sigma epilogues)"),
        ("arnoldi", "hbm", "cgs_dots_kernel + cgs_update_norm_kernel (+ vscale) of the Arnoldi step"),
    ]
    rf = {}
    for ph, bound, kernel in cands:
        ms, n_l, work = prof[ph]
        if ms <= 0:
            continue
        if bound == "hbm":
            if ph == "unpack":
                continue   # no algorithmic byte count is kept for this phase; its time shows in phases_ms
            ach, peak, unit = work / (ms / 1e3) / 1e9, hbm, "GB/s"
            note = "hbm_gbs of measured; achieved = algorithmic bytes / device time"
        elif bound == "alu":
            ach, peak, unit = work / (ms / 1e3) / 1e12, FP64_PEAK_TFLOPS, "TFLOP/s"
            note = ("FP64 FMA units: 152 SMs x 2 DFMA/clk x 2070 MHz (derived); cuBLAS DGEMM measured 1.10 TFLOP/s "
                    "on this pool")
        else:
            ach, peak, unit = work / (ms / 1e3) / 1e12, bf16, "TFLOP/s"
            note = "bf16_tflops_sustained of measured (kernels timed inside a long step)"
        e = {"bound": bound, "kernel": kernel, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
             "traffic": None, "launches": n_l, "ms_total": ms, "peak_note": note}
        if ph in ("ring_emu", "emu_other") or (ph == "ring" and closed_shell):
            e["peak_note"] += ("; achieved counts the method's work, one FP64 product per FP64-accurate "
                               "contraction (2 M N K), not the digit-pair products that evaluate it")
        if ph == "ring_emu":
            ms_w, _, work_w = prof["ring_emu_work"]
            if ms_w > 0:
                rate = work_w / (ms_w / 1e3) / 1e12
                e["emulation_rate"] = {"achieved": rate, "unit": "TFLOP/s", "frac": rate / bf16,
                                       "pairs_per_product": work_w / work if work > 0 else None,
                                       "note": "BF16 tensor-core work of all digit pairs / device time"}
        tr = NCU_TRAFFIC.get(ph)
        if tr is not None:
            e["traffic"] = tr["traffic"]
            e["traffic_ratio"] = tr["traffic"] / tr["algorithmic_bytes"]
            e["traffic_case"] = tr["case"]
        rf[ph] = e
    return rf


if __name__ == "__main__":
    sys.exit(main())
