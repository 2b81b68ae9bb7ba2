"""Time the GPU trajectory integrator (rad_channeling_trajectories, rad_crystal_trajectories
with --potential doyle-turner, or rad_axial_trajectories with --potential axial) on a channeling
ensemble.

  python -m paper_1910_10391_gb300.run_traj --particles 1024 --samples 20000 --precision fp32

Entry conditions: x0 uniform over the channel, theta_x0 ~ N(0, (0.3 theta_L)^2) (the ensemble
workloads' beam), Si(110) harmonic well with U0 = 20 eV, or the synthetic four-Gaussian
Doyle-Turner fit of the input module (3 neighbouring planes on each side), or that fit on the
strings of the Si <110> axis (the crystal library's lattice, 2 cells on each side; entry uniform
over the transverse cell, both angles ~ N(0, (0.3 psi)^2) with psi = sqrt(2 x 35 eV / E), FP64
only). With --adaptive RTOL the records come from rad_trajectories_adaptive (Dormand-Prince
5(4) sub-steps between outputs --output-dt apart, relative tolerance RTOL, at most 2^10 sub-steps
per output; FP64), and the line adds the mean accepted sub-steps per output. Prints one JSON line
with the CUDA-event time of the integrator (best of --repeat) and samples/s.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import _binding as rad
from . import inputs as I


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--particles", type=int, default=1024)
    ap.add_argument("--samples", type=int, default=20000)
    ap.add_argument("--lognormal", action="store_true", help="lengths of the electron batch (2k..200k)")
    ap.add_argument("--energy", type=float, default=10e9)
    ap.add_argument("--charge", type=int, default=+1, choices=[+1, -1])
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32"])
    ap.add_argument("--physics", default="ms", choices=["none", "ms", "ms+ll+loss", "ms+el+ll+loss"])
    ap.add_argument("--potential", default="harmonic", choices=["harmonic", "doyle-turner", "axial"])
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--adaptive", type=float, default=0.0, help="relative tolerance of the adaptive integrator")
    ap.add_argument("--output-dt", type=float, default=5e-9, help="output interval (m/c)")
    a = ap.parse_args(argv)
    import torch
    n = a.particles
    lens = I.lognormal_lengths(n, 4) if a.lognormal else np.full(n, a.samples, dtype=np.int64)
    off = np.zeros(n + 1, dtype=np.int64)
    off[1:] = np.cumsum(lens)
    rng = np.random.default_rng(a.seed)
    thL = math.sqrt(2.0 * 20.0 / a.energy)
    d = lambda v: torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).cuda()
    x0, th = d(rng.uniform(0.0, I.SI110_DP, n)), d(rng.normal(0.0, 0.3 * thL, n))
    E = d(np.full(n, a.energy))
    doff = torch.from_numpy(off).cuda()
    out = torch.empty((int(off[-1]), rad.RAD_NREC), dtype=torch.float64, device="cuda")
    flags = {"none": 0, "ms": rad.RAD_TRAJ_MS,
             "ms+ll+loss": rad.RAD_TRAJ_MS | rad.RAD_TRAJ_LL | rad.RAD_TRAJ_MS_LOSS,
             "ms+el+ll+loss": rad.RAD_TRAJ_MS | rad.RAD_TRAJ_MS_EL | rad.RAD_TRAJ_LL | rad.RAD_TRAJ_MS_LOSS}[a.physics]
    pot = None
    y0 = thy = None
    if a.potential == "axial":
        lat = rad.crystal_string_lattice(rad.RAD_DIAMOND, 5.431e-10, 110)
        pot = rad.RadAxialPotential.make(I.SYNTH_DT_A, I.SYNTH_DT_B, lat, I.SYNTH_DT_AX, I.SYNTH_DT_BX, I.SYNTH_DT_CX,
                                         I.SI_I_EV, n_cells=2)
        psi = math.sqrt(2.0 * 35.0 / a.energy)
        x0, y0 = d(rng.uniform(0.0, lat.cell_x, n)), d(rng.uniform(0.0, lat.cell_y, n))
        th, thy = d(rng.normal(0.0, 0.3 * psi, n)), d(rng.normal(0.0, 0.3 * psi, n))
        if a.precision == "fp32":
            raise SystemExit("the axial integrator is FP64 only")
    elif a.potential == "doyle-turner":
        pot = rad.RadPlanarPotential.make(I.SYNTH_DT_A, I.SYNTH_DT_B, I.SI_N, I.SYNTH_DT_AX, I.SYNTH_DT_BX,
                                          I.SYNTH_DT_CX, I.SI_I_EV, n_neighbours=3)
    elif flags & rad.RAD_TRAJ_MS_EL:
        raise SystemExit("electron scattering needs --potential doyle-turner")
    if a.precision == "fp32":
        if a.adaptive > 0:
            raise SystemExit("the adaptive integrator is FP64 only")
        flags |= rad.RAD_TRAJ_FP32
    ch = rad.RadChannel(20.0, I.SI110_DP, I.EPS_S_EV, I.SI_X0, I.RHO_THERMAL, I.ME_EV, a.charge, flags)
    st = torch.cuda.current_stream()
    steps = torch.zeros(n, dtype=torch.int64, device="cuda") if a.adaptive > 0 else None  # per particle
    ctl = rad.RadStepControl(a.adaptive, 1e-20, 1e-16, 10, 1 << 40) if a.adaptive > 0 else None
    ms = []
    for r in range(a.repeat + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        if ctl is not None:
            rc = rad.rad_trajectories_adaptive(ch, ctl, doff, E, x0, th, out, a.seed, dt=a.output_dt,
                                               planar=pot if a.potential == "doyle-turner" else None,
                                               axial=pot if a.potential == "axial" else None, y0=y0, thy0=thy,
                                               substeps_out=steps)
        elif pot is None:
            rc = rad.rad_channeling_trajectories(ch, doff, E, x0, th, out, a.output_dt, a.seed)
        elif a.potential == "axial":
            rc = rad.rad_axial_trajectories(ch, pot, doff, E, x0, th, out, a.output_dt, a.seed, y0=y0, thy0=thy)
        else:
            rc = rad.rad_crystal_trajectories(ch, pot, doff, E, x0, th, out, a.output_dt, a.seed)
        e1.record(st)
        if rc:
            raise rad.RadError(rc, "trajectory integrator")
        torch.cuda.synchronize()
        if r:  # the first call is a warm-up
            ms.append(e0.elapsed_time(e1))
    status = rad.rad_device_status(1)
    if status:
        raise rad.RadError(status, "device status")
    best = min(ms)
    extra = {}
    if steps is not None:
        extra = {"adaptive_rtol": a.adaptive, "output_dt": a.output_dt,
                 "substeps_per_output": float(steps.double().sum().item()) / max(int(off[-1]) - n, 1)}
    print(json.dumps({**extra, "particles": n, "samples_total": int(off[-1]), "max_length": int(lens.max()),
                      "precision": a.precision, "physics": a.physics, "potential": a.potential,
                      "charge": a.charge, "ms": ms,
                      "samples_per_s": int(off[-1]) / best * 1e3,
                      "checksum": float(out[:, 1].double().abs().sum().item())}))


if __name__ == "__main__":
    main()
