#!/usr/bin/env python
"""Benchmark of the radiation-integral hot path on GB300.

Workload (the plain-FP64 ensemble configuration): 1024 positrons, E = 10 GeV, harmonic planar
well (U0 = 20 eV, d_p = 1.92 A), seeded RK4 trajectories with scattering kicks, 20,000 samples
each (100 um); 512 log-spaced photon energies in [1e-4 E, 0.5 E] x 64 x 64 directions; classical
and Baier-Katkov spin-1/2 models. A step is one pass of the whole path (device checks, the
integral kernel, the particle/angle combine and the angle integral) over a batch of particles
in both models. `value` is the chosen form (mixed precision: FP64 phase base and particle sums,
FP32 sincos and amplitudes) in integrand terms/s; the plain FP64 kernel and the FP64-accurate
double-float kernel are timed on the same inputs and reported beside it. The line also carries
the other workloads, each with its own timing: the analytic undulator (4096 samples, 128 hw x
16x16) in every precision, a graph-captured launch over the first 512 electrons of the lognormal
electron batch, and the learned surrogate trained in the run, at its 1 % contract.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "integrand terms/s (ω·n·t) & spectra/s: plain FP64 vs chosen form at stated err"
N_PART, N_SAMP, N_OMEGA, N_SIDE = 1024, 20000, 512, 64
TUNE_PARTICLES = 8
# launch shapes (R, NW, T) of the mixed kernel per model and its sin/cos split (1/split of the
# terms on the FMA pipe, 0: none): the fastest timed on 32-particle launches of this workload
# (R=2 or 4, NW=4 or 8, T=128 or 256, split 0, 4 or 6); --autotune lets the library's autotuner
# choose instead
SHAPES = {0: (2, 8, 256), 2: (2, 8, 256)}
SPLIT = {0: 6, 2: 0}
# per model: FP64 instructions per term of k_fp64 and k_df, and warp instructions per 32 terms of
# k_df, counted by ncu (smsp__inst_executed_pipe_fp64.sum x 32 / terms, smsp__inst_executed.sum)
# on the launch these legs time: one particle of this workload x 512 hw x 64x64 directions, the
# default shapes (k_fp64 R=2 NW=8 T=64, k_df R=2 NW=4 T=64)
FP64_OPS_PER_TERM = {0: 18.53, 2: 20.58}
DF_FP64_OPS_PER_TERM = {0: 1.276, 2: 1.360}
DF_INST_PER_32_TERMS = {0: 134.5, 2: 159.3}
WORKLOAD = ("positron ensemble: 1024 e+ at 10 GeV, harmonic planar well (U0 = 20 eV, d_p = 1.92 A), "
            "RK4 + scattering kicks, 20000 samples over 100 um; 512 log hw in [1e-4 E, 0.5 E] x 64x64 "
            "directions within +-(theta_L + 3/gamma); classical + spin-1/2")
SM_COUNT, SM_MAX_MHZ = 152, 2070.0
SFU_PER_SM_CLK = 16          # special-function unit ops per SM per clock (4 per SM sub-partition)
FMA_PER_SM_CLK = 128         # FP32 FMA lanes per SM
FP64_PER_SM_CLK = 2          # FP64 FMA per SM per clock
ISSUE_PER_SM_CLK = 128       # 4 schedulers x 1 warp instruction (32 lanes) per clock
SPLIT_EXTRA_SLOTS = 18       # FMA-pipe sin/cos (21 slots) in place of prescale + 2 MUFU (3)


def clocks_per_term(mode, R, pe):
    """Lower bound on SM clocks per term of the mixed integral kernel (k_mixed_pp / k_mixed)
    from its two limits: the SFU (2 MUFU per term it serves, 16 per SM per clock) and the issue
    slots (per SFU term: the phase FMUL, the prescale FMUL, 2 MUFU, 4 or 6 FFMA (I_x, I_y and for
    spin-1/2 J, each re and im) and the term's share of the shared-memory loads, one float4 per
    sample shared by R energies; an FMA-pipe sin/cos term takes 18 slots more). With a split
    1/pe, f is the fraction of the 8R terms of an unrolled group whose index is pe - 1 mod pe."""
    nc = 6 if mode == 2 else 4
    loads = 1.0 / R
    f = (sum(1 for i in range(8 * R) if i % pe == pe - 1) / (8 * R)) if pe else 0.0
    sfu = 2.0 * (1.0 - f) / SFU_PER_SM_CLK
    issue = (4 + nc + loads + SPLIT_EXTRA_SLOTS * f) / ISSUE_PER_SM_CLK
    return max(sfu, issue), f


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=32, help="particles per step (mixed form)")
    ap.add_argument("--fp64-batch", type=int, default=1, help="particles per plain-FP64 step")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--df-batch", type=int, default=4, help="particles per double-float step")
    ap.add_argument("--df-steps", type=int, default=3)
    ap.add_argument("--batch-slice", type=int, default=512,
                    help="electrons of the 4096-electron lognormal batch in its graph launch (0: skip)")
    ap.add_argument("--surrogate-train", type=int, default=32768,
                    help="kernel spectra the in-run surrogate trains on (0: skip the surrogate leg)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", action="store_true",
                    help="choose the launch shapes with the library's autotuner instead of SHAPES")
    return ap.parse_args()


# --------------------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        load = [x for x in sm if x > 0.5 * max(sm)]
        return {"sm_mhz": statistics.median(load or sm), "sm_max_mhz": float(rows[0][2]),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit()),
                "samples": len(rows), "reasons": reasons}


# --------------------------------------------------------------------------- helpers
def workload_inputs():
    from paper_1910_10391_gb300 import inputs as I
    return I.workload_positron_ensemble(N_PART, N_SAMP, seed=2, n_omega=N_OMEGA, n_side=N_SIDE)


def terms_of(n_particles, grid):
    return n_particles * N_SAMP * grid.n_omega * grid.n_angles


def cpu_sample_bins(grid, n_dirs, seed=11):
    import numpy as np
    rng = np.random.default_rng(seed)
    dirs = rng.choice(grid.n_angles, size=n_dirs, replace=False)
    bi = np.repeat(np.arange(grid.n_omega), n_dirs)
    bj = np.tile(dirs, grid.n_omega)
    return bi, bj


def run_oracle_sample(tr, grid, n_dirs, modes):
    """Oracle (FP64 CPU, all host cores) on particle 0 at every hw x n_dirs directions."""
    import oracle as O
    bi, bj = cpu_sample_bins(grid, n_dirs)
    one = tr.subset([0])
    one.weight[:] = 1.0
    vals = {}
    t0 = time.perf_counter()
    for m in modes:
        vals[m] = O.spectrum_bins(one, grid, {0: O.CLASSICAL, 2: O.SPIN_HALF}[m], bi, bj)
    dt = time.perf_counter() - t0
    terms = len(modes) * len(bi) * N_SAMP
    return vals, bi, bj, terms, dt, O.max_threads()


# --------------------------------------------------------------------------- other workloads
def time_launches(torch, stream, fn, reps):
    """CUDA-event milliseconds of fn() on `stream`, per repetition, after one warm-up call."""
    fn()
    stream.synchronize()
    out = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        stream.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def undulator_leg(rad, torch, dev, reps=5):
    """The analytic single-trajectory workload (e+ at gamma = 1000, x = a sin(2 pi t / lambda),
    4096 samples over 5 periods; 128 linear hw up to 1.2 x the first harmonic x 16 x 16
    directions within +-2/gamma), classical, in every precision; one plan call per launch."""
    from paper_1910_10391_gb300 import inputs as I
    tr, grid = I.workload_undulator_4096()
    inp = rad.DeviceInputs(tr, grid, device=dev)
    terms = tr.n_total * grid.n_omega * grid.n_angles
    st = torch.cuda.current_stream()
    res, cubes = {}, {}
    for prec, name in ((rad.RAD_FP64, "fp64"), (rad.RAD_FP64_DF, "fp64_df"), (rad.RAD_MIXED, "mixed")):
        p = rad.Plan(inp.n_samples, inp.n_particles, inp.n_omega, inp.n_angles, rad.RAD_CLASSICAL, prec, 1, 0)
        out = torch.empty(inp.n_omega * inp.n_angles, dtype=torch.float64, device=dev)

        def run():
            rc = p.execute(*inp.args(), out, None, None, None)
            if rc:
                raise rad.RadError(rc, "rad_plan_execute")

        ms = time_launches(torch, st, run, reps)
        res[name] = {"ms_per_call": statistics.median(ms), "terms_per_s": terms / (statistics.median(ms) * 1e-3),
                     "shape": p.describe()}
        cubes[name] = out.view(inp.n_omega, inp.n_angles).cpu().numpy()
        p.close()
    return {"workload": "undulator: e+ gamma 1000, a = 0.5 A, lambda = 10 um, 4096 uniform samples over 5 "
                        "periods; 128 linear hw to 1.2 x the first harmonic x 16x16 directions within +-2/gamma; "
                        "classical", "terms_per_call": terms, "forms": res,
            "timing": f"CUDA events around one plan call (checks, kernel, combine), median of {reps}"}, (tr, grid, cubes)


def batch_leg(rad, torch, dev, n, tune_particles=8, tune_budget_ms=15000, seed=11):
    """The lognormal electron batch (20 GeV e-, lengths clip(exp(N(ln 2e4, ln10/3))), 2e3, 2e5),
    BCK spin-1/2 with recoil, 1024 log hw x 32x32 directions): its first n electrons (the
    generator's streams are per particle, so they are exactly the full batch's first n) in one
    autotuned, graph-captured launch."""
    from paper_1910_10391_gb300 import inputs as I
    import numpy as np
    L = I.lognormal_lengths(4096, seed=4)[:n]
    tr = I.channeling(n, 20e9, -1, L, 5e-9, seed=4)
    tr.weight[:] = 1.0 / 4096
    grid = I._ensemble_grid(20e9, 20.0, 1024, 32)
    inp = rad.DeviceInputs(tr, grid, device=dev)
    mode = rad.RAD_SPIN_HALF
    plan = rad.Plan(inp.n_samples, inp.n_particles, inp.n_omega, inp.n_angles, mode, rad.RAD_MIXED, 1, 0)
    sub = rad.DeviceInputs(tr.subset(range(tune_particles)), grid, device=dev)
    tp = rad.Plan(sub.n_samples, sub.n_particles, sub.n_omega, sub.n_angles, mode, rad.RAD_MIXED, 1, 0)
    tmp = torch.empty(sub.n_omega * sub.n_angles, dtype=torch.float64, device=dev)
    t0 = time.perf_counter()
    rc = tp.autotune(*sub.args(), tmp, None, None, None, budget_ms=tune_budget_ms)
    if rc:
        raise rad.RadError(rc, "rad_plan_autotune")
    tune_s = time.perf_counter() - t0
    d = dict(kv.split("=") for kv in tp.describe().split())
    tp.close()
    del sub, tmp
    for rc, what in ((plan.set_prepass(int(d.get("pp", "1"))), "set_prepass"),
                     (plan.set_shape(int(d["R"]), int(d["NW"]), int(d["T"]), 1), "set_shape"),
                     (plan.set_sincos_split(int(d.get("pe", "0"))) if d.get("pp", "1") == "1" else 0, "split")):
        if rc:
            raise rad.RadError(rc, what)
    out = torch.empty(inp.n_omega * inp.n_angles, dtype=torch.float64, device=dev)
    st = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    graph = plan.graph(*inp.args(), out, None, None, None, stream=st)

    def run():
        rc = graph.launch(st)
        if rc:
            raise rad.RadError(rc, "rad_graph_launch")

    ms = time_launches(torch, st, run, 1)[0]
    status = rad.rad_device_status(1)
    if status != rad.RAD_OK:
        raise rad.RadError(status, "device status")
    samples = int(tr.lengths().sum())
    terms = samples * inp.n_omega * inp.n_angles
    rng = np.random.default_rng(seed)
    bi = rng.integers(0, inp.n_omega, 24)
    bj = rng.integers(0, inp.n_angles, 24)
    got = out.view(inp.n_omega, inp.n_angles).cpu().numpy()[bi, bj]
    dm = dict(kv.split("=") for kv in plan.describe().split())
    cpt, _ = clocks_per_term(2, int(dm["R"]), int(dm.get("pe", "0")))
    peak = SM_COUNT * SM_MAX_MHZ * 1e6 / cpt
    graph.close()
    plan.close()
    res = {"workload": f"electron batch slice: the first {n} of 4096 e- at 20 GeV, lognormal lengths 2k-200k "
                       f"(median 20k; here {samples} samples, max {int(L.max())}), harmonic planar well, RK4 + "
                       "scattering kicks; 1024 log hw in [1e-4 E, 0.5 E] x 32x32 directions; spin-1/2 with recoil",
           "particles": n, "samples": samples, "terms": terms, "ms": ms, "terms_per_s": terms / (ms * 1e-3),
           "spectra_per_s": n / (ms * 1e-3), "shape": plan_desc_str(dm), "autotune_s": tune_s,
           "launch": "one CUDA-graph launch of the whole path (checks, pre-pass, persistent kernel, combine), "
                     "CUDA events on its stream, after one warm-up launch",
           "roofline": {"bound": "alu", "pipe": "sfu + issue slots", "achieved": terms / (ms * 1e-3) / 1e12,
                        "peak": peak / 1e12, "unit": "Tterm/s", "frac": terms / (ms * 1e-3) / peak}}
    return res, (tr, grid, bi, bj, got)


def surrogate_leg(n_train):
    """The learned surrogate (3 -> 256 x 3 -> 2048 MLPs, BF16 tensor-core GEMMs with FP32
    accumulation, trained by the library's kernels) at its 1 % contract: a 3-network ensemble
    trained in the run on n_train kernel spectra (24 Lorentz factors over [2e3, 4e4]), calibrated on
    16 validation beams, evaluated on 4 held-out beams of 512 entries (two near each end of the
    Lorentz-factor range) with fallback to the kernel until each beam mean's calibrated estimate is
    at most 1 %; gain = kernel time / surrogate-with-fallback time for the beam means."""
    from paper_1910_10391_gb300 import surrogate as S
    t0 = time.perf_counter()
    cfg = S.Config(n_gamma_train=24, n_models=3, steps=6000, batch=512, fallback_rel=0.01, calib_gamma_bins=2)
    x0, th, g = S.sample_entries(cfg, n_train, seed=5, discrete_gamma=True)
    bins = S.kernel_bins(cfg, x0, th, g)
    vx0, vth, vg, vb = S.sample_beams(cfg, 16, 48, seed=7, divergence=cfg.beam_divergence)
    sur = S.Surrogate(cfg)
    sur.fit(S.raw_inputs(cfg, x0, th, g), bins, S.raw_inputs(cfg, vx0, vth, vg), S.kernel_bins(cfg, vx0, vth, vg), vb)
    del bins
    t_train = time.perf_counter() - t0
    lo, hi = cfg.gamma_lo, cfg.gamma_hi
    hx0, hth, hg, hb = S.sample_beams(cfg, 4, 512, seed=6, divergence=cfg.beam_divergence,
                                      gammas=[lo * 1.02, lo * 1.1, hi / 1.1, hi / 1.02])
    rep = S.evaluate(sur, hx0, hth, hg, hb)
    sur.close()
    return {"workload": f"surrogate: 3-network ensemble trained in this run on {n_train} kernel spectra (the full "
                        "configuration trains on 200 000); 4 held-out beams x 512 entries, 256 hw/E x 8 radial bins, "
                        "spin-1/2, fallback to the kernel until the beam mean's estimate <= 1 %",
            "gain": rep["gain"], "spectra_per_s_kernel": rep["spectra_per_s_kernel"],
            "spectra_per_s_surrogate": rep["spectra_per_s_surrogate"], "fallback_fraction": rep["mean_fallback_fraction"],
            "beams": [{"gamma": e["gamma"], "error": e["error"], "estimate": e["estimate"],
                       "n_fallback": e["n_fallback"]} for e in rep["per_beam"]],
            "error_le_estimate_le_1pct": all(e["error"] <= e["estimate"] <= 0.01 for e in rep["per_beam"]),
            "train_s": t_train}


def plan_desc_str(d):
    return " ".join(f"{k}={v}" for k, v in d.items())


# --------------------------------------------------------------------------- reference arm
def reference_arm(args, rank):
    if rank != 0:
        return
    tr, grid = workload_inputs()
    n_dirs = 64
    for _ in range(args.warmup):
        run_oracle_sample(tr, grid, n_dirs, (0, 2))
    t_all = 0.0
    terms_all = 0
    cores = 1
    for _ in range(args.steps):
        _, _, _, terms, dt, cores = run_oracle_sample(tr, grid, n_dirs, (0, 2))
        t_all += dt
        terms_all += terms
    v = terms_all / t_all
    sample = (f"particle 0 of the workload (20000 samples) x all 512 hw x {n_dirs} seeded directions, "
              "classical + spin-1/2, per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "terms/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": v, "unit": "terms/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "terms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# --------------------------------------------------------------------------- our arm
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank)

    import numpy as np
    import torch
    import paper_1910_10391_gb300 as rad
    from paper_1910_10391_gb300 import shard

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    rad.load()

    tr, grid = workload_inputs()
    B = args.batch
    n_batches = N_PART // B
    # whole ensemble resident in HBM (1.64 GB); each step takes a contiguous batch of particles
    d_samples = torch.from_numpy(tr.samples).to(dev)
    d_gamma = torch.from_numpy(tr.gamma).to(dev)
    d_energy = torch.from_numpy(tr.energy_eV).to(dev)
    d_weight = torch.from_numpy(tr.weight).to(dev)
    d_hw = torch.from_numpy(grid.hbar_omega_eV).to(dev)
    d_tx = torch.from_numpy(grid.theta_x).to(dev)
    d_ty = torch.from_numpy(grid.theta_y).to(dev)
    d_dom = torch.from_numpy(grid.d_omega).to(dev)
    no, na = grid.n_omega, grid.n_angles

    def batch_args(b, nb):
        p0 = b * nb
        offs = torch.arange(nb + 1, dtype=torch.int64, device=dev) * N_SAMP
        return (d_samples[p0 * N_SAMP:(p0 + nb) * N_SAMP].contiguous(), offs, d_gamma[p0:p0 + nb],
                d_energy[p0:p0 + nb], d_weight[p0:p0 + nb], d_hw, d_tx, d_ty, d_dom)

    modes = (rad.RAD_CLASSICAL, rad.RAD_SPIN_HALF)
    cube = {m: torch.empty(no * na, dtype=torch.float64, device=dev) for m in modes}
    spec = {m: torch.zeros(no, dtype=torch.float64, device=dev) for m in modes}

    def make_plans(prec, nb):
        return {m: rad.Plan(nb * N_SAMP, nb, no, na, m, prec, 3, 0) for m in modes}

    plans = make_plans(rad.RAD_MIXED, B)
    tuned = {}
    if args.autotune:
        # tune the launch shape on an 8-particle slice of the same grids (long enough per work item
        # to rank the shapes as the 32-particle launches do), then apply it
        sub = batch_args(0, TUNE_PARTICLES)
        for m in modes:
            tp = rad.Plan(TUNE_PARTICLES * N_SAMP, TUNE_PARTICLES, no, na, m, rad.RAD_MIXED, 3, 0)
            tmp_c = torch.empty(no * na, dtype=torch.float64, device=dev)
            tmp_s = torch.empty(no, dtype=torch.float64, device=dev)
            tp.autotune(*sub, tmp_c, tmp_s, None, None, budget_ms=60000)
            d = dict(kv.split("=") for kv in tp.describe().split())
            tuned[m] = (int(d["R"]), int(d["NW"]), int(d["T"]))
            tp.close()
            plans[m].set_prepass(int(d.get("pp", "1")))
            plans[m].set_shape(*tuned[m], 1)
            if int(d.get("pe", "0")):
                plans[m].set_sincos_split(int(d["pe"]))
    else:
        for m in modes:
            rc = plans[m].set_shape(*SHAPES[m], 1)
            if rc:
                raise rad.RadError(rc, "rad_plan_set_shape")
            if SPLIT[m]:
                rc = plans[m].set_sincos_split(SPLIT[m])
                if rc:
                    raise rad.RadError(rc, "rad_plan_set_sincos_split")
    for m in modes:
        plans[m].set_timing(True)

    l2_flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    pending = set()  # plans whose last launch's kernel time has not been read yet

    def read_kernel_ms(ps, m, kernel_ms):
        if kernel_ms is not None and (id(ps), m) in pending:
            kernel_ms.append((m, ps[m].last_kernel_ms()))
            pending.discard((id(ps), m))

    def step(s, ps, nb, kernel_ms=None):
        p0, _ = shard.step_batch(s, rank, world, nb, N_PART)
        a = batch_args(p0 // nb, nb)
        l2_flush.zero_()
        for m in modes:
            # the plan keeps one pair of events: read the previous step's kernel time of this model
            # just before relaunching it; the other model's kernel of the previous step is still
            # queued then, so the device never idles on the read
            read_kernel_ms(ps, m, kernel_ms)
            rc = ps[m].execute(*a, cube[m], spec[m], None, None, accumulate=0)
            if rc:
                raise rad.RadError(rc, "rad_plan_execute")
            if kernel_ms is not None:
                pending.add((id(ps), m))

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(ps, nb, K, W, collect=None):
        for s in range(W):
            step(s, ps, nb)
        barrier()
        t0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for s in range(K):
            step(W + s, ps, nb, collect)
        e1.record()
        barrier()
        for m in modes:
            read_kernel_ms(ps, m, collect)
        wall = time.perf_counter() - t0
        ms = e0.elapsed_time(e1)
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        if dist is not None:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item()), wall

    # ---- chosen form (mixed precision) ----
    clocks = Clocks(local)
    kms = []
    for s in range(args.warmup):
        step(s, plans, B)
    clocks.start()
    ms_total, wall = timed(plans, B, args.steps, 0, kms)
    clk = clocks.stop()
    ms_step = ms_total / args.steps
    terms_step = len(modes) * terms_of(B, grid)
    value = world * terms_step / (ms_step * 1e-3)
    spectra_s = world * len(modes) * B / (ms_step * 1e-3)
    mixed_desc = {m: plans[m].describe() for m in modes}
    launches_per_step = sum(plans[m].kernel_launches() for m in modes)
    ens = shard.allreduce_sum(spec[modes[0]].clone())  # ensemble sum of the last step's spectra over ranks

    # ---- plain FP64 on the same inputs ----
    fp = make_plans(rad.RAD_FP64, args.fp64_batch)
    for m in modes:
        fp[m].set_timing(True)
    fkms = []
    fms, _ = timed(fp, args.fp64_batch, args.fp64_steps, 1, fkms)
    fms_step = fms / args.fp64_steps
    f_terms = len(modes) * terms_of(args.fp64_batch, grid)
    fp64_value = world * f_terms / (fms_step * 1e-3)

    # ---- FP64-accurate double-float form on the same inputs (same tolerance as plain FP64) ----
    dfp = make_plans(rad.RAD_FP64_DF, args.df_batch)
    for m in modes:
        dfp[m].set_timing(True)
    dkms = []
    dms, _ = timed(dfp, args.df_batch, args.df_steps, 1, dkms)
    dms_step = dms / args.df_steps
    df_terms = len(modes) * terms_of(args.df_batch, grid)
    df_value = world * df_terms / (dms_step * 1e-3)

    # ---- end to end through the host-buffer entry point (pinned memory, copies timed) ----
    nb_e = B
    p0 = (rank * nb_e) % N_PART
    h_samples = torch.from_numpy(tr.samples[p0 * N_SAMP:(p0 + nb_e) * N_SAMP]).pin_memory()
    h_offs = torch.arange(nb_e + 1, dtype=torch.int64).pin_memory()
    h_offs.mul_(N_SAMP)
    h_g = torch.from_numpy(tr.gamma[p0:p0 + nb_e].copy()).pin_memory()
    h_e = torch.from_numpy(tr.energy_eV[p0:p0 + nb_e].copy()).pin_memory()
    h_w = torch.from_numpy(tr.weight[p0:p0 + nb_e].copy()).pin_memory()
    h_grid = [torch.from_numpy(x.copy()).pin_memory() for x in
              (grid.hbar_omega_eV, grid.theta_x, grid.theta_y, grid.d_omega)]
    h_cube = torch.empty(no * na, dtype=torch.float64).pin_memory()
    h_spec = torch.empty(no, dtype=torch.float64).pin_memory()
    h_in = [h_samples, h_offs, h_g, h_e, h_w] + h_grid
    h2d = len(modes) * sum(t.numel() * t.element_size() for t in h_in)
    d2h = len(modes) * (h_cube.numel() + h_spec.numel()) * 8

    def e2e_step():
        for m in modes:
            rc = rad.rad_spectrum_host(*h_in, m, rad.RAD_MIXED, h_cube, h_spec)
            if rc:
                raise rad.RadError(rc, "rad_spectrum_host")

    e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        e2e_step()
    barrier()
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    tt = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    e2e_value = world * terms_step / float(tt.item())

    status = rad.rad_device_status(1)
    if status != rad.RAD_OK:
        raise rad.RadError(status, "device status")

    # ---- the other workloads: the analytic undulator in every form, the electron batch slice ----
    und_line, und_data = undulator_leg(rad, torch, dev)
    bat_line, bat_data = batch_leg(rad, torch, dev, args.batch_slice) if args.batch_slice > 0 else (None, None)
    sur_line = surrogate_leg(args.surrogate_train) if args.surrogate_train > 0 and rank == 0 else None

    # ---- roofline of the dominant kernel (mixed integral kernel) ----
    mk = [ms for (_, ms) in kms]
    kernel_ms_avg = sum(mk) / len(mk)
    terms_launch = terms_of(B, grid)
    # ideal time of the launches from the per-mode pipe bound, against their measured time
    t_meas = 0.0
    t_ideal = 0.0
    sfu_ops_total = 0.0
    bound_by_mode = {}
    for (m, ms) in kms:
        dm = dict(kv.split("=") for kv in mixed_desc[m].split())
        cpt, f = clocks_per_term(m, int(dm["R"]), int(dm.get("pe", "0")))
        t_meas += ms * 1e-3
        t_ideal += terms_launch * cpt / (SM_COUNT * SM_MAX_MHZ * 1e6)
        sfu_ops_total += 2.0 * (1.0 - f) * terms_launch
        bound_by_mode[int(m)] = {"clocks_per_term": cpt, "fma_sincos_fraction": f}
    terms_all = terms_launch * len(kms)
    sfu_ops = sfu_ops_total / t_meas
    sfu_peak = SM_COUNT * SFU_PER_SM_CLK * SM_MAX_MHZ * 1e6
    # DRAM bytes per launch of the integral kernel (k_mixed_pp), scaled from its ncu captures on a
    # small case of the same workload (128 particles x 20000 samples x 64 hw x 256 directions,
    # the benchmark's shapes R=2 NW=8 T=256, 38 particle chunks; the two models' mean: 125.16 MB
    # read = the 48-byte pre-pass records once, 6.10 MB written, of which 4.98 MB are the partial
    # sums): reads grow with the samples a launch processes, writes with the partial sums it stores.
    samples_launch = B * N_SAMP
    desc0 = dict(kv.split("=") for kv in mixed_desc[modes[0]].split())
    chunks = int(desc0["chunks"])
    traffic = (125.16e6 * samples_launch / (128 * N_SAMP)
               + 6.10e6 * (chunks * no * na) / (38 * 64 * 256)) if desc0.get("pp") == "1" else None
    roofline = {"bound": "alu", "pipe": "sfu + issue slots",
                "kernel": "k_mixed_pp" if desc0.get("pp") == "1" else "k_mixed",
                "achieved": terms_all / t_meas / 1e12, "peak": terms_all / t_ideal / 1e12, "unit": "Tterm/s",
                "frac": t_ideal / t_meas,
                "traffic": traffic, "traffic_source": "ncu dram__bytes_read/write.sum of a small case, scaled",
                "terms_per_launch": terms_launch, "kernel_ms_avg": kernel_ms_avg, "per_mode": bound_by_mode,
                "sfu_ops_per_s": sfu_ops, "sfu_frac": sfu_ops / sfu_peak,
                "peak_source": "per mode max(2(1-f)/16 SFU, slots/128 issue) clocks per term x 152 SMs x 2070 MHz "
                               "(unit counts and max clock)"}
    fk = [ms for (_, ms) in fkms]
    f_terms_launch = terms_of(args.fp64_batch, grid)
    fp64_kernel_ms = sum(fk) / len(fk)
    fp64_ops_s = sum(FP64_OPS_PER_TERM[int(m)] * f_terms_launch for (m, _) in fkms) / (sum(fk) * 1e-3)
    fp64_roof = {"kernel": "k_fp64", "kernel_ms_avg": fp64_kernel_ms, "launches": len(fk),
                 "terms_per_s": f_terms_launch / (fp64_kernel_ms * 1e-3),
                 "fp64_ops_per_term": FP64_OPS_PER_TERM,
                 "frac_fp64_pipe": fp64_ops_s / (SM_COUNT * FP64_PER_SM_CLK * SM_MAX_MHZ * 1e6)}
    dk = [ms for (_, ms) in dkms]
    df_kernel_ms = sum(dk) / len(dk)
    df_terms_launch = terms_of(args.df_batch, grid)
    df_fp64_s = sum(DF_FP64_OPS_PER_TERM[int(m)] * df_terms_launch for (m, _) in dkms) / (sum(dk) * 1e-3)
    df_inst_s = sum(DF_INST_PER_32_TERMS[int(m)] * df_terms_launch / 32 for (m, _) in dkms) / (sum(dk) * 1e-3)
    # k_df: one FP64 instruction per term (the phase product; the reduction is integer
    # arithmetic) plus the per-(direction, sample) preparation shared by a block's 256 energies and
    # the conversion of the sums of two tiles into FP64 particle amplitudes; it is bound by the
    # issue slots (4 warp instructions per SM per clock), the FP64 pipe second
    df_roof = {"kernel": "k_df", "kernel_ms_avg": df_kernel_ms, "launches": len(dk),
               "terms_per_s": df_terms_launch / (df_kernel_ms * 1e-3),
               "fp64_ops_per_term": DF_FP64_OPS_PER_TERM, "warp_inst_per_32_terms": DF_INST_PER_32_TERMS,
               "frac_fp64_pipe": df_fp64_s / (SM_COUNT * FP64_PER_SM_CLK * SM_MAX_MHZ * 1e6),
               "frac_issue": df_inst_s / (SM_COUNT * ISSUE_PER_SM_CLK / 32 * SM_MAX_MHZ * 1e6)}

    line = {
        "metric": METRIC, "value": value, "unit": "terms/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "particles_per_step": B, "samples_per_particle": N_SAMP,
                   "n_omega": no, "n_angles": na, "modes": ["classical", "spin_half"], "precision": "mixed",
                   "parallelism": f"replicas x{world} (disjoint particle batches)",
                   "l2": "256 MB buffer written between steps (flush)", "shape": mixed_desc},
        "spectra_per_s": spectra_s,
        "plain_fp64": {"value": fp64_value, "unit": "terms/s", "particles_per_step": args.fp64_batch,
                       "steps": args.fp64_steps, "ms_per_step": fms_step, "spectra_per_s": world * len(modes) * args.fp64_batch /
                       (fms_step * 1e-3), "shape": {m: fp[m].describe() for m in modes}, "kernel": fp64_roof},
        "fp64_df": {"value": df_value, "unit": "terms/s", "particles_per_step": args.df_batch,
                    "steps": args.df_steps, "ms_per_step": dms_step, "spectra_per_s": world * len(modes) * args.df_batch /
                    (dms_step * 1e-3), "shape": {m: dfp[m].describe() for m in modes}, "kernel": df_roof,
                    "tolerance": "as plain FP64: 1e-9 of a bin, floor 1e-6 of the peak"},
        "mixed_over_fp64": value / fp64_value,
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": "terms/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "entry": "rad_spectrum_host (pinned host buffers, copies inside the timed region)"},
        "undulator": und_line,
        "electron_batch": bat_line,
        "surrogate": sur_line,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "wall_s_timed": wall,
    }

    # ---- CPU baseline: the oracle on a bounded sample, and the GPU error on that sample ----
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        n_dirs = 128
        vals, bi, bj, terms, dt, cores = run_oracle_sample(tr, grid, n_dirs, modes)
        one = batch_args(0, 1)
        errs = {}
        for prec, name in ((rad.RAD_MIXED, "mixed"), (rad.RAD_FP64, "fp64"), (rad.RAD_FP64_DF, "fp64_df")):
            for m in modes:
                p1 = rad.Plan(N_SAMP, 1, no, na, m, prec, 1, 0)
                c1 = torch.empty(no * na, dtype=torch.float64, device=dev)
                w1 = torch.ones(1, dtype=torch.float64, device=dev)
                a = list(one)
                a[4] = w1
                rc = p1.execute(*a, c1, None, None, None)
                assert rc == 0
                g = c1.view(no, na).cpu().numpy()[bi, bj]
                r = vals[m]
                peak = np.abs(r).max()
                if prec == rad.RAD_MIXED:
                    sel = r >= 1e-3 * peak
                    rel = np.abs(g[sel] - r[sel]) / r[sel]
                    errs[f"{name}_{'classical' if m == 0 else 'spin_half'}"] = {
                        "max_rel_on_bins_ge_1e-3_peak": float(rel.max()),
                        "median_rel": float(np.median(rel)), "bins": int(sel.sum())}
                else:
                    rel = np.abs(g - r) / np.maximum(np.abs(r), 1e-6 * peak)
                    errs[f"{name}_{'classical' if m == 0 else 'spin_half'}"] = {
                        "max_rel_floor_1e-6_peak": float(rel.max()), "bins": int(r.size)}
                p1.close()
        # the other workloads against the oracle: the undulator's full cube, the batch's sampled bins
        utr, ugrid, ucubes = und_data
        uref = O.spectrum_cube(utr, ugrid, O.CLASSICAL)
        upk = np.abs(uref).max()
        for name, c in ucubes.items():
            if name == "mixed":
                sel = uref >= 1e-3 * upk
                und_line["forms"][name]["max_rel_on_bins_ge_1e-3_peak"] = float(
                    (np.abs(c[sel] - uref[sel]) / uref[sel]).max())
            else:
                und_line["forms"][name]["max_rel_floor_1e-6_peak"] = float(
                    (np.abs(c - uref) / np.maximum(np.abs(uref), 1e-6 * upk)).max())
        if bat_data is not None:
            btr, bgrid, bi2, bj2, bgot = bat_data
            bref = O.spectrum_bins(btr, bgrid, O.SPIN_HALF, bi2, bj2)
            bsel = bref >= 1e-3 * np.abs(bref).max()
            bat_line["err_vs_oracle"] = {"bins": int(bi2.size), "bins_ge_1e-3_peak": int(bsel.sum()),
                                         "max_rel": float((np.abs(bgot[bsel] - bref[bsel]) / bref[bsel]).max())}
        line["cpu_baseline"] = {
            "value": terms / dt, "unit": "terms/s", "cores": cores, "kind": "oracle",
            "sample": f"particle 0 (20000 samples) x 512 hw x {n_dirs} seeded directions x 2 models "
                      f"= {terms:.3e} terms in {dt:.1f} s"}
        line["err_vs_oracle"] = errs
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
