"""GPU trajectory integrator (rad_channeling_trajectories) against the trajectory oracle, and the
whole pipeline entry conditions -> trajectories -> spectra on the device against the oracles.

Tolerance: both sides run the same FP64 RK4 in different rounding orders (the GPU contracts
multiply-adds, its libm differs from the host's by ulps). In the harmonic well the rounding
differences grow at most linearly over the steps, about 1e-16 relative per step, so after
20,000 steps they stay below 1e-11 of each field's scale; the tests allow 1e-9."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import traj as T
import paper_1910_10391_gb300 as rad
from paper_1910_10391_gb300 import inputs as I

from helpers import assert_mixed_close

pytestmark = pytest.mark.gpu
D_P = I.SI110_DP


def channel(charge=+1, flags=rad.RAD_TRAJ_MS, U0=20.0):
    return rad.RadChannel(U0, D_P, I.EPS_S_EV, I.SI_X0, I.RHO_THERMAL, I.ME_EV, charge, flags)


def run_gpu(ch, x0, thx0, E, lengths, dt, seed, ids=None, energies=False):
    import torch
    n = len(x0)
    off = np.zeros(n + 1, dtype=np.int64)
    off[1:] = np.cumsum(lengths)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    out = torch.full((int(off[-1]), 10), np.nan, dtype=torch.float64, device="cuda")
    eo = torch.full((int(off[-1]),), np.nan, dtype=torch.float64, device="cuda") if energies else None
    dids = torch.from_numpy(np.asarray(ids, dtype=np.int64)).cuda() if ids is not None else None
    rc = rad.rad_channeling_trajectories(ch, torch.from_numpy(off).cuda(), d(np.broadcast_to(E, (n,))), d(x0),
                                         d(thx0), out, dt, seed, particle_ids=dids, energy_out=eo)
    assert rc == rad.RAD_OK, rad.rad_status_string(rc)
    torch.cuda.synchronize()
    st = rad.rad_device_status(1)
    return out.cpu().numpy(), (eo.cpu().numpy() if energies else None), off, st


def assert_fields_close(got, ref, rel=1e-9):
    for f in range(10):
        scale = max(np.abs(ref[..., f]).max(), 1e-300)
        err = np.abs(got[..., f] - ref[..., f]).max()
        assert err <= rel * scale, (I.FIELDS[f], err / scale)


def entries(n, E, seed):
    rng = np.random.default_rng(seed)
    thL = math.sqrt(2 * 20.0 / E)
    return rng.uniform(0, D_P, n), rng.normal(0, 0.3 * thL, n)


@pytest.mark.parametrize("charge", [+1, -1])
@pytest.mark.parametrize("flags", [rad.RAD_TRAJ_MS, rad.RAD_TRAJ_MS | rad.RAD_TRAJ_LL | rad.RAD_TRAJ_MS_LOSS, 0])
def test_records_match_oracle(charge, flags):
    n, L, dt, E, seed = 48, 3000, 5e-9, 50e9, 21
    x0, th = entries(n, E, 3)
    got, eg, _, st = run_gpu(channel(charge, flags), x0, th, E, np.full(n, L), dt, seed, energies=True)
    assert st == rad.RAD_OK
    ref, er = T.trajectories(x0, th, 0.0, E, L, dt, seed, charge=charge, ms=bool(flags & rad.RAD_TRAJ_MS),
                             ll=bool(flags & rad.RAD_TRAJ_LL), ms_loss=bool(flags & rad.RAD_TRAJ_MS_LOSS),
                             energies=True)
    assert_fields_close(got.reshape(n, L, 10), ref)
    np.testing.assert_allclose(eg.reshape(n, L), er, rtol=1e-12)


def test_ragged_lengths_and_stream_ids():
    """Lengths 1, 2, 3 and ragged ones; particle_ids pick the random streams; one particle's
    records match the same particle integrated alone with its own id."""
    lens = np.array([1, 2, 3, 700, 1, 1234, 2, 999])
    n = len(lens)
    x0, th = entries(n, 10e9, 4)
    ids = np.array([7, 100, 3, 2 ** 33 + 5, 0, 42, 9, 11])
    got, _, off, st = run_gpu(channel(), x0, th, 10e9, lens, 5e-9, 77, ids=ids)
    assert st == rad.RAD_OK
    assert not np.isnan(got).any()
    for p in range(n):
        ref = T.trajectories(x0[p:p + 1], th[p:p + 1], 0.0, 10e9, int(lens[p]), 5e-9, 77,
                             particle_ids=ids[p:p + 1])[0]
        assert_fields_close(got[off[p]:off[p + 1]], ref)


def test_bad_particle_is_skipped_and_reported():
    lens = np.array([50, 50, 50])
    x0, th = entries(3, 10e9, 5)
    E = np.array([10e9, 0.5 * I.ME_EV, 10e9])  # below the rest energy
    import torch
    off = np.array([0, 50, 100, 150], dtype=np.int64)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    out = torch.full((150, 10), np.nan, dtype=torch.float64, device="cuda")
    rc = rad.rad_channeling_trajectories(channel(), torch.from_numpy(off).cuda(), d(E), d(x0), d(th), out, 5e-9, 1)
    assert rc == rad.RAD_OK
    assert rad.rad_device_status(1) == rad.RAD_EDATA
    o = out.cpu().numpy()
    assert np.isnan(o[50:100]).all() and not np.isnan(o[:50]).any() and not np.isnan(o[100:]).any()
    assert rad.rad_device_status(1) == rad.RAD_OK


def test_device_pipeline_spectrum():
    """Entry conditions -> GPU trajectories -> mixed-precision spectrum, all on the device,
    against the oracle spectrum of the oracle's trajectories (spin-1/2, with losses)."""
    import torch
    n, L, dt, E = 16, 4000, 5e-9, 20e9
    x0, th = entries(n, E, 6)
    flags = rad.RAD_TRAJ_MS | rad.RAD_TRAJ_LL | rad.RAD_TRAJ_MS_LOSS
    got, _, off, st = run_gpu(channel(+1, flags), x0, th, E, np.full(n, L), dt, 9)
    assert st == rad.RAD_OK
    ref = T.trajectories(x0, th, 0.0, E, L, dt, 9, ll=True, ms_loss=True)
    tr_ref = I.Trajectories(ref.reshape(-1, 10), off, np.full(n, E / I.ME_EV), np.full(n, E), np.full(n, 1.0 / n))
    grid = I._ensemble_grid(E, 20.0, 32, 8)
    cube_ref = O.spectrum_cube(tr_ref, grid, O.SPIN_HALF)
    tr_gpu = I.Trajectories(got, off, tr_ref.gamma, tr_ref.energy_eV, tr_ref.weight)
    inp = rad.DeviceInputs(tr_gpu, grid)
    cube = torch.empty((grid.n_omega * grid.n_angles,), dtype=torch.float64, device="cuda")
    rc = rad.rad_spectrum(*inp.args(), rad.RAD_SPIN_HALF, rad.RAD_MIXED, cube, None, None, 0, None, 0)
    assert rc == rad.RAD_OK
    torch.cuda.synchronize()
    assert rad.rad_device_status(1) == rad.RAD_OK
    assert_mixed_close(cube.view(grid.n_omega, grid.n_angles).cpu().numpy(), cube_ref)


def test_full_size_ensemble_sampled():
    """1024 positrons x 20,000 steps (the plain ensemble's size) on the GPU; 6 sampled particles
    against the oracle over their whole length."""
    n, L, dt, E = 1024, 20000, 5e-9, 10e9
    x0, th = entries(n, E, 7)
    got, _, off, st = run_gpu(channel(), x0, th, E, np.full(n, L), dt, 2)
    assert st == rad.RAD_OK
    pick = np.array([0, 1, 511, 512, 1000, 1023])
    ref = T.trajectories(x0[pick], th[pick], 0.0, E, L, dt, 2, particle_ids=pick)
    assert_fields_close(got.reshape(n, L, 10)[pick], ref)


# Mixed precision (RAD_TRAJ_FP32): FP32 stages, double-float state. Without scattering, per step
# the FP32 increments carry about 6e-8 relative rounding, random from step to step, and in the
# harmonic well a velocity error stays bounded (it becomes a phase/amplitude error of the
# oscillation): positions and velocities stay within about 1e-7 of their scale over 20,000 steps.
# With scattering, each kick's size carries the FP32 precision of its plane density: exp(-r^2/rho^2)
# with an exponent rounded to FP32 is good to about 1e-7 times the exponent, so kicks differ from
# the FP64 ones by about 1e-6 relative and the velocities, which sum the kicks, by the same
# relative amount (observed: x 1e-7, y and v 3e-6, dz 9e-7, FP32-evaluated fields 1e-5).
MIXED_TOL_MS = {"t": 0.0, "x": 1e-6, "y": 1e-5, "dz": 3e-6, "vx": 1e-5, "vy": 1e-5, "dvz": 1e-5, "ax": 3e-5,
                "ay": 3e-5, "az": 3e-5}
MIXED_TOL_DET = {"t": 0.0, "x": 1e-6, "y": 0.0, "dz": 1e-6, "vx": 1e-6, "vy": 0.0, "dvz": 1e-5, "ax": 1e-5,
                 "ay": 0.0, "az": 1e-5}


def mixed_errors(got, ref):
    worst = {}
    for f, name in enumerate(I.FIELDS):
        scale = np.abs(ref[..., f]).max()
        err = np.abs(got[..., f] - ref[..., f]).max()
        worst[name] = float(err / scale) if scale > 0 else float(err)
    return worst


@pytest.mark.parametrize("charge", [+1, -1])
@pytest.mark.parametrize("flags", [0, rad.RAD_TRAJ_LL, rad.RAD_TRAJ_MS,
                                   rad.RAD_TRAJ_MS | rad.RAD_TRAJ_LL | rad.RAD_TRAJ_MS_LOSS])
def test_mixed_records_close_to_oracle(charge, flags):
    n, L, dt, E, seed = 48, 20000, 5e-9, 20e9, 21
    x0, th = entries(n, E, 8)
    got, eg, _, st = run_gpu(channel(charge, flags | rad.RAD_TRAJ_FP32), x0, th, E, np.full(n, L), dt, seed,
                             energies=True)
    assert st == rad.RAD_OK
    ref, er = T.trajectories(x0, th, 0.0, E, L, dt, seed, charge=charge, ms=bool(flags & rad.RAD_TRAJ_MS),
                             ll=bool(flags & rad.RAD_TRAJ_LL), ms_loss=bool(flags & rad.RAD_TRAJ_MS_LOSS),
                             energies=True)
    worst = mixed_errors(got.reshape(n, L, 10), ref)
    print("mixed trajectory errors (relative to field scale):", flags, charge, worst)
    tol = MIXED_TOL_MS if flags & rad.RAD_TRAJ_MS else MIXED_TOL_DET
    for name, t in tol.items():
        assert worst[name] <= t, (name, worst[name])
    # energy: the loss carries FP32 precision (its rate is an FP32 product of gamma^2 and F^2;
    # with scattering loss, each kick's cost carries the kick's 1e-6 precision)
    eg = eg.reshape(n, L)
    rel_loss = 1e-5 if flags & rad.RAD_TRAJ_MS_LOSS else 1e-6
    assert np.all(np.abs(eg - er) <= rel_loss * (E - er) + 4 * np.spacing(E))


def pipeline_error(charge, flags, n=24, L=20000, dt=5e-9, E=10e9, seed=5):
    import torch
    x0, th = entries(n, E, 9)
    got, _, off, st = run_gpu(channel(charge, flags | rad.RAD_TRAJ_FP32), x0, th, E, np.full(n, L), dt, seed)
    assert st == rad.RAD_OK
    ref = T.trajectories(x0, th, 0.0, E, L, dt, seed, charge=charge, ms=bool(flags & rad.RAD_TRAJ_MS),
                         ll=bool(flags & rad.RAD_TRAJ_LL), ms_loss=bool(flags & rad.RAD_TRAJ_MS_LOSS))
    g = np.full(n, E / I.ME_EV)
    tr_ref = I.Trajectories(ref.reshape(-1, 10), off, g, np.full(n, E), np.full(n, 1.0 / n))
    grid = I._ensemble_grid(E, 20.0, 48, 8)
    cube_ref = O.spectrum_cube(tr_ref, grid, O.SPIN_HALF)
    inp = rad.DeviceInputs(I.Trajectories(got, off, g, tr_ref.energy_eV, tr_ref.weight), grid)
    cube = torch.empty((grid.n_omega * grid.n_angles,), dtype=torch.float64, device="cuda")
    assert rad.rad_spectrum(*inp.args(), rad.RAD_SPIN_HALF, rad.RAD_MIXED, cube, None, None, 0, None, 0) == 0
    torch.cuda.synchronize()
    assert rad.rad_device_status(1) == rad.RAD_OK
    return cube.view(grid.n_omega, grid.n_angles).cpu().numpy(), cube_ref


@pytest.mark.parametrize("charge", [+1, -1])
def test_mixed_pipeline_spectrum_deterministic(charge):
    """FP32 trajectories (radiation reaction, no scattering) -> mixed spectrum on the device,
    against the FP64 oracles end to end, at the mixed radiation tolerance (1e-4 on bins >= 1e-3
    of the peak)."""
    got, ref = pipeline_error(charge, rad.RAD_TRAJ_LL)
    print("mixed pipeline spectrum error (deterministic):", charge, assert_mixed_close(got, ref))


@pytest.mark.parametrize("charge", [+1, -1])
def test_mixed_pipeline_spectrum_with_scattering(charge):
    """With scattering the FP32 kicks differ from the FP64 ones by about 1e-6 relative, so each
    trajectory is a slightly different sample of the same random motion; d(dz)/dt = -v^2/2 then
    accumulates the velocity difference and shifts high-frequency phases by up to about 1e-2 rad
    over 100 um. The spectra agree to 2e-2 on bins >= 1e-3 of the peak (observed 3e-4 for
    positrons, 8e-3 for electrons, whose channels sit on the planes where the kicks are)."""
    got, ref = pipeline_error(charge, rad.RAD_TRAJ_MS | rad.RAD_TRAJ_LL | rad.RAD_TRAJ_MS_LOSS)
    print("mixed pipeline spectrum error (scattering):", charge, assert_mixed_close(got, ref, rel=2e-2))
