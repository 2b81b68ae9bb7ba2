"""Run one radiation-integral case on the GPU and print its timing (profiling and checks).

  python -m paper_1910_10391_gb300.run_case --workload ensemble --particles 128 --samples 20000 \
      --n-omega 64 --n-side 16 --mode classical --precision mixed --repeat 2

Workloads: `ensemble` (10 GeV e+ planar channeling, fixed length), `batch` (20 GeV e-,
lognormal lengths), `undulator` (the analytic 4096-sample trajectory and its grid).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="ensemble", choices=["ensemble", "batch", "undulator"])
    ap.add_argument("--particles", type=int, default=16)
    ap.add_argument("--samples", type=int, default=20000)
    ap.add_argument("--n-omega", type=int, default=512)
    ap.add_argument("--n-side", type=int, default=64)
    ap.add_argument("--mode", default="classical", choices=["classical", "spin0", "spin_half"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed", "fp64_df"])
    ap.add_argument("--shape", default="", help="R,NW,T,chunk_mult")
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--graph", action="store_true", help="replay a captured CUDA graph")
    ap.add_argument("--autotune-subset", type=int, default=0,
                    help="autotune the launch shape on the first N particles and apply it")
    ap.add_argument("--seed", type=int, default=0, help="generator seed (0: the workload's own)")
    ap.add_argument("--prepass", type=int, default=-1, help="mixed precision: 1 pre-pass kernel, 0 inline")
    ap.add_argument("--split", type=int, default=-1,
                    help="pre-pass kernel: 1/split of the terms take sincos on the FMA pipe (0, 4, 6)")
    a = ap.parse_args(argv)

    import torch

    import paper_1910_10391_gb300 as rad
    from paper_1910_10391_gb300 import inputs as I

    if a.workload == "ensemble":
        tr = I.channeling(a.particles, 10e9, +1, a.samples, 5e-9, seed=a.seed or 2)
        grid = I._ensemble_grid(10e9, 20.0, a.n_omega, a.n_side)
    elif a.workload == "batch":
        L = I.lognormal_lengths(a.particles, seed=a.seed or 4)
        tr = I.channeling(a.particles, 20e9, -1, L, 5e-9, seed=a.seed or 4)
        grid = I._ensemble_grid(20e9, 20.0, a.n_omega, a.n_side)
    else:
        tr, grid = I.workload_undulator_4096()
    inp = rad.DeviceInputs(tr, grid)
    mode, prec = rad.MODES[a.mode], rad.PRECISIONS[a.precision]
    plan = rad.Plan(inp.n_samples, inp.n_particles, inp.n_omega, inp.n_angles, mode, prec, 1, 0)
    tuned = None
    if a.autotune_subset > 0:
        sub = tr.subset(range(min(a.autotune_subset, tr.n_particles)))
        si = rad.DeviceInputs(sub, grid)
        tp = rad.Plan(si.n_samples, si.n_particles, si.n_omega, si.n_angles, mode, prec, 1, 0)
        tmp = torch.empty(si.n_omega * si.n_angles, dtype=torch.float64, device="cuda")
        rc = tp.autotune(*si.args(), tmp, None, None, None, budget_ms=120000)
        if rc:
            raise rad.RadError(rc, "autotune")
        d = dict(kv.split("=") for kv in tp.describe().split())
        tuned = (int(d["R"]), int(d["NW"]), int(d["T"]), 1)
        tp.close()
        del si, tmp
        if prec == rad.RAD_MIXED:
            rc = plan.set_prepass(int(d.get("pp", "1")))
            if rc:
                raise rad.RadError(rc, "set_prepass")
        rc = plan.set_shape(*tuned)
        if rc:
            raise rad.RadError(rc, "set_shape")
        if int(d.get("pe", "0")):
            rc = plan.set_sincos_split(int(d["pe"]))
            if rc:
                raise rad.RadError(rc, "set_sincos_split")
    if a.prepass >= 0:
        rc = plan.set_prepass(a.prepass)
        if rc:
            raise rad.RadError(rc, "set_prepass")
    if a.shape:
        rc = plan.set_shape(*[int(x) for x in a.shape.split(",")])
        if rc:
            raise rad.RadError(rc, "set_shape")
    if a.split >= 0:
        rc = plan.set_sincos_split(a.split)
        if rc:
            raise rad.RadError(rc, "set_sincos_split")
    out = torch.empty(inp.n_omega * inp.n_angles, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    times = []
    with torch.cuda.stream(s):
        g = plan.graph(*inp.args(), out, None, None, None, stream=s) if a.graph else None
        for _ in range(a.repeat):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            rc = g.launch(s) if g else plan.execute(*inp.args(), out, None, None, None, stream=s)
            if rc:
                raise rad.RadError(rc, "execute")
            e1.record(s)
            s.synchronize()
            times.append(e0.elapsed_time(e1))
    st = rad.rad_device_status(1)
    if st:
        raise rad.RadError(st, "device status")
    terms = int(tr.lengths().sum()) * inp.n_omega * inp.n_angles
    best = min(times)
    print(json.dumps({"case": vars(a), "shape": plan.describe(), "terms": terms, "ms": times,
                      "terms_per_s": terms / (best * 1e-3), "spectra_per_s": tr.n_particles / (best * 1e-3),
                      "samples_total": int(tr.lengths().sum()), "checksum": float(out.sum().item())}))
    if g:
        g.close()
    plan.close()


if __name__ == "__main__":
    main()
