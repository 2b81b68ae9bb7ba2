"""GPU trajectory integrator in the Doyle-Turner planar potential (rad_crystal_trajectories,
Sec. III, Eq. plane, with scattering on nuclei and valence electrons) against the trajectory
oracle, through the C ABI. The fit is the synthetic four-Gaussian one of the input module.

FP64 form: every field within 1e-9 of its scale, energies 1e-12. Both sides run the same FP64
RK4 in different rounding orders (ulp-level differences in exp and the sums). In this anharmonic
well a difference shifts the oscillation period, and with scattering the kick sizes depend
steeply on position at the plane cores, so differences grow. Measured with the oracle by
perturbing its force by 1e-15 relative (about ten times a one-ulp difference) on every
evaluation: after 3000 steps at 20 GeV every case stays below 1e-12; after 20 000 steps
positrons reach 3e-11 (no scattering), electrons 3e-10 without scattering and 2e-2 with it
(their channels sit on the planes, where the kicks are). The comparisons therefore run 3000
steps, and 20 000 for positrons without scattering.

FP32 form (RAD_TRAJ_FP32): the force is an FP32 sum of exp2f terms whose exponents are rounded to
FP32, about 2e-7 of the largest term. The well is anharmonic, so these errors change the period and
the phase drifts over the oscillations; with scattering the kicks at the plane cores amplify
differences as above. An emulation (the oracle with its force, plane density and electron density
evaluated in float32 in the kernel's order) gives, as fractions of each field's scale: without
scattering over 20 000 steps, x 5e-6, dz 1e-6, v_x 5e-5, dvz 7e-5, a_x and a_z 5e-4 (electrons,
whose a_x changes fastest at the plane cores); with scattering over 3000 steps, x 2e-6, y 6e-7,
dz 7e-7, v 2e-5, dvz 2e-5, a 6e-5; spectra from the FP32 trajectories (no scattering, 20 000
steps) differ from the FP64 ones by 4e-5 (positrons) and 7e-5 (electrons) on bins >= 1e-3 of the
peak. The kernel adds its own FP32 stage rounding of the same size, so the tolerances below are
about ten times the emulation. Observed on a GB300: without scattering x 4.5e-6, v_x 1.1e-4, dvz
1.6e-4, a_x 1.3e-3, a_z 1.2e-3 (electrons); with scattering x 3.6e-6, v 4.6e-5, a 1.1e-4; spectra
9.0e-5 and 9.4e-5."""
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
MS, LL, LOSS, EL, FP32 = rad.RAD_TRAJ_MS, rad.RAD_TRAJ_LL, rad.RAD_TRAJ_MS_LOSS, rad.RAD_TRAJ_MS_EL, rad.RAD_TRAJ_FP32
ALL = MS | LL | LOSS | EL


def potentials(K=3, a=I.SYNTH_DT_A):
    lib = rad.RadPlanarPotential.make(a, I.SYNTH_DT_B, I.SI_N, I.SYNTH_DT_AX, I.SYNTH_DT_BX, I.SYNTH_DT_CX, I.SI_I_EV,
                                      n_neighbours=K)
    orc = T.PlanarPotential(a, I.SYNTH_DT_B, I.SI_N, I.SYNTH_DT_AX, I.SYNTH_DT_BX, I.SYNTH_DT_CX, I.SI_I_EV, K=K)
    return lib, orc


def channel(charge, flags, U0=0.0):
    return rad.RadChannel(U0, D_P, I.EPS_S_EV, I.SI_X0, I.RHO_THERMAL, I.ME_EV, charge, flags)


def entries(n, E, seed):
    rng = np.random.default_rng(seed)
    thL = math.sqrt(2 * 20.0 / E)
    return rng.uniform(0, D_P, n), rng.normal(0, 0.3 * thL, n)


def run_gpu(ch, pot, x0, thx0, E, lengths, dt, seed, ids=None):
    import torch
    n = len(x0)
    off = np.zeros(n + 1, dtype=np.int64)
    off[1:] = np.cumsum(lengths)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    out = torch.full((int(off[-1]), 10), np.nan, dtype=torch.float64, device="cuda")
    eo = torch.full((int(off[-1]),), np.nan, dtype=torch.float64, device="cuda")
    dids = torch.from_numpy(np.asarray(ids, dtype=np.int64)).cuda() if ids is not None else None
    if pot is None:
        rc = rad.rad_channeling_trajectories(ch, torch.from_numpy(off).cuda(), d(np.broadcast_to(E, (n,))), d(x0),
                                             d(thx0), out, dt, seed, particle_ids=dids, energy_out=eo)
    else:
        rc = rad.rad_crystal_trajectories(ch, pot, torch.from_numpy(off).cuda(), d(np.broadcast_to(E, (n,))), d(x0),
                                          d(thx0), out, dt, seed, particle_ids=dids, energy_out=eo)
    assert rc == rad.RAD_OK, rad.rad_status_string(rc)
    torch.cuda.synchronize()
    assert rad.rad_device_status(1) == rad.RAD_OK
    return out.cpu().numpy(), eo.cpu().numpy(), off


def oracle(orc, x0, th, E, L, dt, seed, charge, flags, ids=None):
    return T.trajectories(x0, th, 0.0, E, L, dt, seed, charge=charge, ms=bool(flags & MS), ll=bool(flags & LL),
                          ms_loss=bool(flags & LOSS), ms_el=bool(flags & EL), pot=orc, particle_ids=ids,
                          energies=True)


def field_errors(got, ref):
    worst = {}
    for f, name in enumerate(I.FIELDS):
        scale = np.abs(ref[..., f]).max()
        err = np.abs(got[..., f] - ref[..., f]).max()
        worst[name] = float(err / scale) if scale > 0 else float(err)
    return worst


@pytest.mark.parametrize("charge", [+1, -1])
@pytest.mark.parametrize("flags", [0, MS, ALL])
def test_fp64_records_match_oracle(charge, flags):
    n, L, dt, E, seed = 48, 3000, 5e-9, 20e9, 21
    lib, orc = potentials()
    x0, th = entries(n, E, 3)
    got, eg, _ = run_gpu(channel(charge, flags), lib, x0, th, E, np.full(n, L), dt, seed)
    ref, er = oracle(orc, x0, th, E, L, dt, seed, charge, flags)
    worst = field_errors(got.reshape(n, L, 10), ref)
    print("crystal fp64 errors:", charge, flags, worst)
    assert max(worst.values()) <= 1e-9, worst
    np.testing.assert_allclose(eg.reshape(n, L), er, rtol=1e-12)


def test_fp64_long_positron_records():
    """20 000 steps (100 um) with radiation reaction, positrons, and K = 2 neighbours."""
    n, L, dt, E = 16, 20000, 5e-9, 10e9
    lib, orc = potentials(K=2)
    x0, th = entries(n, E, 4)
    got, eg, _ = run_gpu(channel(+1, LL), lib, x0, th, E, np.full(n, L), dt, 0)
    ref, er = oracle(orc, x0, th, E, L, dt, 0, +1, LL)
    worst = field_errors(got.reshape(n, L, 10), ref)
    print("crystal fp64 long:", worst)
    assert max(worst.values()) <= 1e-9, worst
    np.testing.assert_allclose(eg.reshape(n, L), er, rtol=1e-12)


@pytest.mark.parametrize("charge", [+1, -1])
def test_fp64_one_lane_path_for_large_ensembles(charge):
    """From 4096 particles on each particle has one lane (below, a group of 8 lanes shares its
    force and electron-density sums, which every other test here runs): 4096 particles over 12
    steps with every physics flag, all records against the oracle."""
    n, L, dt, E, seed = 4096, 12, 5e-9, 20e9, 31
    lib, orc = potentials()
    x0, th = entries(n, E, 6)
    got, eg, _ = run_gpu(channel(charge, ALL), lib, x0, th, E, np.full(n, L), dt, seed)
    ref, er = oracle(orc, x0, th, E, L, dt, seed, charge, ALL)
    worst = field_errors(got.reshape(n, L, 10), ref)
    print("crystal fp64 one lane:", charge, worst)
    assert max(worst.values()) <= 1e-9, worst
    np.testing.assert_allclose(eg.reshape(n, L), er, rtol=1e-12)


def test_fp64_ragged_lengths_and_stream_ids():
    lens = np.array([1, 2, 3, 700, 1, 1234, 2, 999])
    n = len(lens)
    lib, orc = potentials()
    x0, th = entries(n, 20e9, 5)
    ids = np.array([7, 100, 3, 2 ** 33 + 5, 0, 42, 9, 11])
    got, _, off = run_gpu(channel(-1, ALL), lib, x0, th, 20e9, lens, 5e-9, 77, ids=ids)
    assert not np.isnan(got).any()
    for p in range(n):
        ref, _ = oracle(orc, x0[p:p + 1], th[p:p + 1], 20e9, int(lens[p]), 5e-9, 77, -1, ALL, ids=ids[p:p + 1])
        assert max(field_errors(got[off[p]:off[p + 1]], ref[0]).values()) <= 1e-9


@pytest.mark.parametrize("flags", [MS, FP32 | MS])
def test_zero_potential_equals_harmonic_entry_with_zero_well(flags):
    """With every a_i = 0 the planar force vanishes, as the harmonic well's does at U0 = 0: the two
    entry points then integrate the same straight lines and kicks. Their kernels are separate
    instantiations, which the compiler may contract into multiply-adds differently, so they agree
    to rounding: 1e-12 of each field's scale in FP64, 1e-6 in FP32 (no field, so no growth)."""
    n, L = 12, 500
    lib, _ = potentials(a=(0.0, 0.0, 0.0, 0.0))
    x0, th = entries(n, 20e9, 6)
    a, ea, _ = run_gpu(channel(+1, flags), lib, x0, th, 20e9, np.full(n, L), 5e-9, 3)
    b, eb, _ = run_gpu(channel(+1, flags), None, x0, th, 20e9, np.full(n, L), 5e-9, 3)
    worst = field_errors(a, b)
    print("zero potential vs zero well:", flags, worst)
    assert max(worst.values()) <= (1e-6 if flags & FP32 else 1e-12), worst
    assert np.array_equal(ea, eb)  # no energy loss: the entry energy at every sample


MIXED_TOL_DET = {"t": 0.0, "x": 5e-5, "y": 0.0, "dz": 1e-5, "vx": 5e-4, "vy": 0.0, "dvz": 1e-3, "ax": 5e-3,
                 "ay": 0.0, "az": 5e-3}
MIXED_TOL_MS = {"t": 0.0, "x": 2e-5, "y": 1e-5, "dz": 1e-5, "vx": 3e-4, "vy": 2e-4, "dvz": 3e-4, "ax": 6e-4,
                "ay": 6e-4, "az": 6e-4}


@pytest.mark.parametrize("charge", [+1, -1])
@pytest.mark.parametrize("flags", [0, LL, MS, ALL])
def test_fp32_records_close_to_oracle(charge, flags):
    n, dt, E, seed = 48, 5e-9, 20e9, 21
    L = 3000 if flags & MS else 20000
    lib, orc = potentials()
    x0, th = entries(n, E, 8)
    got, eg, _ = run_gpu(channel(charge, flags | FP32), lib, x0, th, E, np.full(n, L), dt, seed)
    ref, er = oracle(orc, x0, th, E, L, dt, seed, charge, flags)
    worst = field_errors(got.reshape(n, L, 10), ref)
    print("crystal fp32 errors (relative to field scale):", charge, flags, worst)
    tol = MIXED_TOL_MS if flags & MS else MIXED_TOL_DET
    for name, t in tol.items():
        assert worst[name] <= t, (name, worst[name])
    # energy, against each particle's total loss: electrons lose their energy in steps at the plane
    # crossings, and the phase drift shifts a crossing by up to the a_x error (1e-3 of its scale)
    # of one crossing's loss, about 3e-5 of the total over ~40 crossings; with scattering loss each
    # kick's cost follows the plane density, which the position difference moves by up to
    # 2 (r/rho)(dx/rho) ~ 6e-5. Observed: 6.9e-6 (radiation reaction), 1.1e-5 (all losses).
    eg = eg.reshape(n, L)
    loss = (E - er).max(axis=1, keepdims=True)
    e_err = np.abs(eg - er) / np.maximum(loss, 1.0)
    print("crystal fp32 energy error (of the total loss):", charge, flags, float(e_err.max()))
    assert np.all(np.abs(eg - er) <= 1e-4 * loss + 4 * np.spacing(E))


def spectrum_from(records, off, E, grid):
    import torch
    n = len(off) - 1
    g = np.full(n, E / I.ME_EV)
    inp = rad.DeviceInputs(I.Trajectories(records, off, g, np.full(n, E), np.full(n, 1.0 / n)), grid)
    cube = torch.empty((grid.n_omega * grid.n_angles,), dtype=torch.float64, device="cuda")
    assert rad.rad_spectrum(*inp.args(), rad.RAD_SPIN_HALF, rad.RAD_MIXED, cube, None, None, 0, None, 0) == 0
    torch.cuda.synchronize()
    assert rad.rad_device_status(1) == rad.RAD_OK
    return cube.view(grid.n_omega, grid.n_angles).cpu().numpy()


def oracle_spectrum(ref, off, E, grid):
    n = len(off) - 1
    tr = I.Trajectories(ref.reshape(-1, 10), off, np.full(n, E / I.ME_EV), np.full(n, E), np.full(n, 1.0 / n))
    return O.spectrum_cube(tr, grid, O.SPIN_HALF)


def test_device_pipeline_spectrum_fp64():
    """Entry conditions -> FP64 crystal trajectories (both scattering terms, losses) -> mixed
    spectrum on the device, against the oracle spectrum of the oracle's trajectories, at the mixed
    radiation tolerance (1e-4 on bins >= 1e-3 of the peak)."""
    n, L, dt, E = 16, 3000, 5e-9, 20e9
    lib, orc = potentials()
    x0, th = entries(n, E, 9)
    got, _, off = run_gpu(channel(+1, ALL), lib, x0, th, E, np.full(n, L), dt, 9)
    ref, _ = oracle(orc, x0, th, E, L, dt, 9, +1, ALL)
    grid = I._ensemble_grid(E, 28.0, 32, 8)
    print("crystal pipeline (fp64 trajectories):",
          assert_mixed_close(spectrum_from(got, off, E, grid), oracle_spectrum(ref, off, E, grid)))


@pytest.mark.parametrize("charge", [+1, -1])
def test_device_pipeline_spectrum_fp32(charge):
    """FP32 crystal trajectories (radiation reaction, 20 000 steps) -> mixed spectrum, against the
    FP64 oracles end to end: within 1e-3 on bins >= 1e-3 of the peak (emulation: 7e-5)."""
    n, L, dt, E = 24, 20000, 5e-9, 10e9
    lib, orc = potentials()
    x0, th = entries(n, E, 10)
    got, _, off = run_gpu(channel(charge, LL | FP32), lib, x0, th, E, np.full(n, L), dt, 5)
    ref, _ = oracle(orc, x0, th, E, L, dt, 5, charge, LL)
    grid = I._ensemble_grid(E, 28.0, 48, 8)
    print("crystal pipeline (fp32 trajectories):", charge,
          assert_mixed_close(spectrum_from(got, off, E, grid), oracle_spectrum(ref, off, E, grid), rel=1e-3))
