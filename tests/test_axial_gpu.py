"""GPU trajectory integrator in the axial (string) potential (rad_axial_trajectories, Sec. III,
Eq. string, with the strings' densities of nuclei and valence electrons in the scattering)
against the trajectory oracle, through the C ABI, on string lattices from the crystal library
(Si <110> and W <111>) with the synthetic four-Gaussian fit of the input module.

FP64: every field within 1e-9 of its scale, energies 1e-12. The kernel sums each string's
Gaussians over the cells as a product of two one-dimensional sums; the oracle sums the
two-dimensional grid directly; both are the same FP64 sum in different rounding orders. How far
such differences grow was measured with the oracle by perturbing its force by 1e-15 relative on
every evaluation (Si <110>, 10 GeV, entry angles 0.3 of the critical angle): after 3000 steps
positrons stay below 1e-12 with or without scattering and electrons below 5e-12 without it;
electrons with scattering reach 6e-11 after 2000 steps and 1e-6 after 3000 (their kicks near the
strings depend steeply on position). The comparisons run 3000 steps, 2000 for electrons with
scattering."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import traj as T
import paper_1910_10391_gb300 as rad
from paper_1910_10391_gb300 import inputs as I

from helpers import assert_mixed_close

pytestmark = pytest.mark.gpu
MS, LL, LOSS, EL, FP32 = rad.RAD_TRAJ_MS, rad.RAD_TRAJ_LL, rad.RAD_TRAJ_MS_LOSS, rad.RAD_TRAJ_MS_EL, rad.RAD_TRAJ_FP32
ALL = MS | LL | LOSS | EL


def potentials(structure=rad.RAD_DIAMOND, a=5.431e-10, axis=110, K=2):
    lat = rad.crystal_string_lattice(structure, a, axis)
    n = lat.n_strings
    lib = rad.RadAxialPotential.make(I.SYNTH_DT_A, I.SYNTH_DT_B, lat, I.SYNTH_DT_AX, I.SYNTH_DT_BX, I.SYNTH_DT_CX,
                                     I.SI_I_EV, n_cells=K)
    olat = T.StringLattice(lat.cell_x, lat.cell_y, list(lat.sx[:n]), list(lat.sy[:n]), lat.d)
    orc = T.AxialPotential(I.SYNTH_DT_A, I.SYNTH_DT_B, olat, I.SYNTH_DT_AX, I.SYNTH_DT_BX, I.SYNTH_DT_CX, I.SI_I_EV,
                           K=K)
    return lib, orc


def channel(charge, flags):
    return rad.RadChannel(0.0, 0.0, I.EPS_S_EV, I.SI_X0, I.RHO_THERMAL, I.ME_EV, charge, flags)


def entries(n, E, lat, seed):
    rng = np.random.default_rng(seed)
    psi = math.sqrt(2 * 35.0 / E)  # critical angle of the ~35 eV string potential
    return (rng.uniform(0, lat.cell_x, n), rng.uniform(0, lat.cell_y, n), rng.normal(0, 0.3 * psi, n),
            rng.normal(0, 0.3 * psi, n))


def run_gpu(ch, pot, x0, y0, thx, thy, E, lengths, dt, seed, ids=None):
    import torch
    n = len(x0)
    off = np.zeros(n + 1, dtype=np.int64)
    off[1:] = np.cumsum(lengths)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    out = torch.full((int(off[-1]), 10), np.nan, dtype=torch.float64, device="cuda")
    eo = torch.full((int(off[-1]),), np.nan, dtype=torch.float64, device="cuda")
    dids = torch.from_numpy(np.asarray(ids, dtype=np.int64)).cuda() if ids is not None else None
    rc = rad.rad_axial_trajectories(ch, pot, torch.from_numpy(off).cuda(), d(np.broadcast_to(E, (n,))), d(x0), d(thx),
                                    out, dt, seed, y0=d(y0), thy0=d(thy), particle_ids=dids, energy_out=eo)
    assert rc == rad.RAD_OK, rad.rad_status_string(rc)
    torch.cuda.synchronize()
    assert rad.rad_device_status(1) == rad.RAD_OK
    return out.cpu().numpy(), eo.cpu().numpy(), off


def close(got, ref, rel=1e-9):
    scale = np.maximum(np.abs(ref).max(0), 1e-300)
    err = (np.abs(got - ref).max(0) / scale)
    assert np.all(err <= rel), err
    return err


@pytest.mark.parametrize("charge,flags,L", [(+1, 0, 3000), (-1, 0, 3000), (+1, ALL, 3000), (-1, ALL, 2000),
                                            (+1, MS, 3000)])
def test_axial_si110_fp64_matches_oracle(charge, flags, L):
    lib, orc = potentials()
    E, dt, seed = 10e9, 5e-9, 7
    x0, y0, thx, thy = entries(12, E, orc.lat, seed=3 + charge)
    got, eg, _ = run_gpu(channel(charge, flags), lib, x0, y0, thx, thy, E, [L] * 12, dt, seed)
    ref, er = T.axial_trajectories(x0, y0, thx, thy, E, L, dt, seed, orc, charge=charge, ms=bool(flags & MS),
                                   ms_el=bool(flags & EL), ll=bool(flags & LL), ms_loss=bool(flags & LOSS),
                                   energies=True)
    close(got, ref.reshape(-1, 10))
    np.testing.assert_allclose(eg, er.ravel(), rtol=1e-12)
    # the particles move in both transverse directions
    assert np.abs(ref[..., 5]).max() > 1e-6 and np.abs(ref[..., 8]).max() > 0


def test_axial_w111_ragged_lengths_and_stream_ids():
    """W <111> (BCC) strings, ragged lengths 1 .. 1234 and 64-bit stream ids: each particle's records
    equal the oracle's for the same id."""
    w = rad.crystal_element(rad.RAD_W)
    lib, orc = potentials(rad.RAD_BCC, w.a, 111, K=1)
    E, dt = 20e9, 4e-9
    rng = np.random.default_rng(9)
    lengths = rng.integers(1, 1235, 9)
    lengths[0], lengths[1] = 1, 2
    ids = (np.int64(1) << 40) + np.arange(9, dtype=np.int64) * 977
    x0, y0, thx, thy = entries(9, E, orc.lat, seed=4)
    got, _, off = run_gpu(channel(-1, MS | EL), lib, x0, y0, thx, thy, E, lengths, dt, 11, ids=ids)
    for p in range(9):
        ref = T.axial_trajectories(x0[p:p + 1], y0[p:p + 1], thx[p:p + 1], thy[p:p + 1], E, int(lengths[p]), dt, 11,
                                   orc, charge=-1, ms=True, ms_el=True, particle_ids=ids[p:p + 1])
        close(got[off[p]:off[p + 1]], ref[0])


def test_axial_records_feed_the_radiation_kernels():
    """Spin-1/2 spectra of axial positron trajectories (FP64 records): the mixed kernel against the
    radiation oracle on the same records."""
    import torch
    lib, orc = potentials()
    E, dt = 10e9, 5e-9
    x0, y0, thx, thy = entries(4, E, orc.lat, seed=12)
    got, _, off = run_gpu(channel(+1, MS), lib, x0, y0, thx, thy, E, [4000] * 4, dt, 5)
    g = E / I.ME_EV
    tr = I.Trajectories(got, off, np.full(4, g), np.full(4, E), np.full(4, 0.25))
    grid = I._ensemble_grid(E, 35.0, 48, 6)
    ref = O.spectrum_cube(tr, grid, O.SPIN_HALF)
    inp = rad.DeviceInputs(tr, grid)
    out = torch.empty(inp.n_omega * inp.n_angles, dtype=torch.float64, device="cuda")
    assert rad.rad_spectrum(*inp.args(), rad.RAD_SPIN_HALF, rad.RAD_MIXED, out, None, None, 0, None, 0) == rad.RAD_OK
    assert rad.rad_device_status(1) == rad.RAD_OK
    assert_mixed_close(out.view(inp.n_omega, inp.n_angles).cpu().numpy(), ref)


def test_axial_argument_checks():
    import ctypes
    import torch
    lib, _ = potentials()
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    off = torch.tensor([0, 10], dtype=torch.int64, device="cuda")
    out = torch.empty((10, 10), dtype=torch.float64, device="cuda")
    run = lambda ch, pot: rad.rad_axial_trajectories(ch, pot, off, d([10e9]), d([0.0]), d([0.0]), out, 5e-9, 1)
    assert run(channel(+1, FP32), lib) == rad.RAD_EUNSUPPORTED
    assert run(channel(+1, EL), lib) == rad.RAD_EINVAL          # electron scattering needs MS
    assert run(channel(0, 0), lib) == rad.RAD_EINVAL
    assert run(channel(+1, 0), None) == rad.RAD_EINVAL
    for field, bad in (("n_cells", 0), ("n_cells", 5), ("n_terms", 9)):
        p, _ = potentials()
        setattr(p, field, bad)
        assert run(channel(+1, 0), p) == rad.RAD_EINVAL
    p, _ = potentials()
    p.lattice.d = 0.0
    assert run(channel(+1, 0), p) == rad.RAD_EINVAL
    p, _ = potentials()
    p.lattice.n_strings = 9
    assert run(channel(+1, 0), p) == rad.RAD_EINVAL
    # a particle with a non-finite entry is skipped and reported
    rc = rad.rad_axial_trajectories(channel(+1, 0), lib, off, d([10e9]), d([np.nan]), d([0.0]), out, 5e-9, 1)
    assert rc == rad.RAD_OK
    assert rad.rad_device_status(1) == rad.RAD_EDATA


def test_axial_one_lane_path_for_large_ensembles():
    """From 9216 particles on, each particle has one lane (below, a group of 16 lanes shares its
    force evaluation): 32768 positrons over 12 steps with scattering, every record against the
    oracle."""
    lib, orc = potentials(K=1)
    E, dt = 10e9, 5e-9
    x0, y0, thx, thy = entries(32768, E, orc.lat, seed=21)
    got, _, _ = run_gpu(channel(+1, MS), lib, x0, y0, thx, thy, E, [12] * 32768, dt, 3)
    ref = T.axial_trajectories(x0, y0, thx, thy, E, 12, dt, 3, orc, charge=+1, ms=True)
    close(got, ref.reshape(-1, 10))
