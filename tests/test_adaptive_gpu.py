"""GPU adaptive integrator (rad_trajectories_adaptive: Dormand-Prince 5(4) sub-steps with a lower
bound between caller-set output times, Sec. IV) against the oracle's (oracle.traj.
trajectories_adaptive), through the C ABI: records within 1e-9 of each field's scale, energies
1e-12, and the same number of accepted sub-steps for every particle (the step-size decisions
coincide), on non-uniform output times, in the harmonic well, the planar Doyle-Turner potential
with every physics flag, and the axial potential; the lower bound and the sub-step budget."""
import math

import numpy as np
import pytest

from oracle import traj as T
import paper_1910_10391_gb300 as rad
from paper_1910_10391_gb300 import inputs as I

pytestmark = pytest.mark.gpu
MS, LL, LOSS, EL = rad.RAD_TRAJ_MS, rad.RAD_TRAJ_LL, rad.RAD_TRAJ_MS_LOSS, rad.RAD_TRAJ_MS_EL
ALL = MS | LL | LOSS | EL
E = 10e9


def channel(charge, flags, U0=20.0):
    return rad.RadChannel(U0, I.SI110_DP, I.EPS_S_EV, I.SI_X0, I.RHO_THERMAL, I.ME_EV, charge, flags)


def run_gpu(ch, sc, x0, thx, times, seed, planar=None, axial=None, y0=None, thy=None):
    import torch
    n, L = len(x0), len(times)
    off = torch.arange(n + 1, dtype=torch.int64, device="cuda") * L
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    out = torch.full((n * L, 10), np.nan, dtype=torch.float64, device="cuda")
    eo = torch.full((n * L,), np.nan, dtype=torch.float64, device="cuda")
    cnt = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    rc = rad.rad_trajectories_adaptive(ch, sc, off, d(np.full(n, E)), d(x0), d(thx), out, seed,
                                       times=d(np.tile(times, n)), planar=planar, axial=axial,
                                       y0=None if y0 is None else d(y0), thy0=None if thy is None else d(thy),
                                       energy_out=eo, substeps_out=cnt)
    assert rc == rad.RAD_OK, rad.rad_status_string(rc)
    torch.cuda.synchronize()
    st = rad.rad_device_status(1)
    return st, out.cpu().numpy().reshape(n, L, 10), eo.cpu().numpy().reshape(n, L), cnt.cpu().numpy()


def close(got, ref, rel=1e-9):
    scale = np.maximum(np.abs(ref).max((0, 1)), 1e-300)
    err = np.abs(got - ref).max((0, 1)) / scale
    assert np.all(err <= rel), err


def sc(rtol, max_level=10, max_substeps=1 << 30):
    return rad.RadStepControl(rtol, 1e-20, 1e-16, max_level, max_substeps)


@pytest.mark.parametrize("charge", [+1, -1])
def test_harmonic_well_jittered_times(charge):
    rng = np.random.default_rng(1)
    x0, th = rng.uniform(0, I.SI110_DP, 6), rng.normal(0, 2e-5, 6)
    # output intervals of ~200 nm, a fiftieth of the oscillation period: two to five sub-steps each
    t = I.sample_times("jitter", 121, 120 * 200e-9, seed=3)
    st, got, eg, cnt = run_gpu(channel(charge, 0), sc(1e-10), x0, th, t, 0)
    assert st == rad.RAD_OK
    (ref, er), rc = T.trajectories_adaptive(x0, th, 0.0, E, t, 0, rtol=1e-10, atol_x=1e-20, atol_v=1e-16,
                                            max_level=10, charge=charge, ms=False, energies=True, counts=True)
    close(got, ref)
    np.testing.assert_array_equal(cnt, rc)
    assert cnt.min() > 2 * 120, cnt


@pytest.mark.parametrize("charge", [+1, -1])
def test_planar_potential_all_flags_tile_jump_times(charge):
    pot = rad.RadPlanarPotential.make(I.SYNTH_DT_A, I.SYNTH_DT_B, I.SI_N, I.SYNTH_DT_AX, I.SYNTH_DT_BX, I.SYNTH_DT_CX,
                                      I.SI_I_EV, n_neighbours=3)
    opot = T.PlanarPotential(I.SYNTH_DT_A, I.SYNTH_DT_B, I.SI_N, I.SYNTH_DT_AX, I.SYNTH_DT_BX, I.SYNTH_DT_CX, I.SI_I_EV,
                             K=3)
    rng = np.random.default_rng(2)
    x0, th = rng.uniform(0, I.SI110_DP, 4), rng.normal(0, 2e-5, 4)
    t = I.sample_times("tile_jumps", 301, 300 * 8e-9, tile=32)
    st, got, eg, cnt = run_gpu(channel(charge, ALL, 0.0), sc(1e-9), x0, th, t, 9, planar=pot)
    assert st == rad.RAD_OK
    (ref, er), rc = T.trajectories_adaptive(x0, th, 0.0, E, t, 9, rtol=1e-9, atol_x=1e-20, atol_v=1e-16,
                                            max_level=10, charge=charge, pot=opot, ms=True, ms_el=True, ll=True,
                                            ms_loss=True, energies=True, counts=True)
    close(got, ref)
    np.testing.assert_allclose(eg, er, rtol=1e-12)
    np.testing.assert_array_equal(cnt, rc)


def test_axial_potential_geometric_times():
    lat = rad.crystal_string_lattice(rad.RAD_DIAMOND, 5.431e-10, 110)
    pot = rad.RadAxialPotential.make(I.SYNTH_DT_A, I.SYNTH_DT_B, lat, I.SYNTH_DT_AX, I.SYNTH_DT_BX, I.SYNTH_DT_CX,
                                     I.SI_I_EV, n_cells=2)
    olat = T.StringLattice(lat.cell_x, lat.cell_y, list(lat.sx[:4]), list(lat.sy[:4]), lat.d)
    opot = T.AxialPotential(I.SYNTH_DT_A, I.SYNTH_DT_B, olat, I.SYNTH_DT_AX, I.SYNTH_DT_BX, I.SYNTH_DT_CX, I.SI_I_EV,
                            K=2)
    rng = np.random.default_rng(3)
    x0, y0 = rng.uniform(0, lat.cell_x, 3), rng.uniform(0, lat.cell_y, 3)
    psi = math.sqrt(2 * 35.0 / E)
    thx, thy = rng.normal(0, 0.3 * psi, 3), rng.normal(0, 0.3 * psi, 3)
    t = I.sample_times("geometric", 201, 200 * 8e-9)
    st, got, _, cnt = run_gpu(channel(+1, MS | EL), sc(1e-9), x0, thx, t, 4, axial=pot, y0=y0, thy=thy)
    assert st == rad.RAD_OK
    ref, rc = T.trajectories_adaptive(x0, thx, thy, E, t, 4, rtol=1e-9, atol_x=1e-20, atol_v=1e-16, max_level=10,
                                      y0=y0, axial=opot, ms=True, ms_el=True, counts=True)
    close(got, ref)
    np.testing.assert_array_equal(cnt, rc)


def test_one_lane_paths_for_large_ensembles():
    """From 4096 particles on (planar) and 9216 (axial) each particle has one lane; below, a lane
    group shares its field sums, which the tests above run. A few output intervals of 20 ns
    (several sub-steps each) at those sizes, against the oracle, accepted sub-steps included."""
    rng = np.random.default_rng(12)
    t = I.sample_times("jitter", 5, 4 * 20e-9, seed=5)
    n = 4096
    pot = rad.RadPlanarPotential.make(I.SYNTH_DT_A, I.SYNTH_DT_B, I.SI_N, I.SYNTH_DT_AX, I.SYNTH_DT_BX, I.SYNTH_DT_CX,
                                      I.SI_I_EV, n_neighbours=3)
    opot = T.PlanarPotential(I.SYNTH_DT_A, I.SYNTH_DT_B, I.SI_N, I.SYNTH_DT_AX, I.SYNTH_DT_BX, I.SYNTH_DT_CX, I.SI_I_EV,
                             K=3)
    x0, th = rng.uniform(0, I.SI110_DP, n), rng.normal(0, 2e-5, n)
    st, got, eg, cnt = run_gpu(channel(-1, ALL, 0.0), sc(1e-9), x0, th, t, 6, planar=pot)
    assert st == rad.RAD_OK
    (ref, er), rc = T.trajectories_adaptive(x0, th, 0.0, E, t, 6, rtol=1e-9, atol_x=1e-20, atol_v=1e-16,
                                            max_level=10, charge=-1, pot=opot, ms=True, ms_el=True, ll=True,
                                            ms_loss=True, energies=True, counts=True)
    close(got, ref)
    np.testing.assert_allclose(eg, er, rtol=1e-12)
    np.testing.assert_array_equal(cnt, rc)
    n = 9216
    lat = rad.crystal_string_lattice(rad.RAD_DIAMOND, 5.431e-10, 110)
    apot = rad.RadAxialPotential.make(I.SYNTH_DT_A, I.SYNTH_DT_B, lat, I.SYNTH_DT_AX, I.SYNTH_DT_BX, I.SYNTH_DT_CX,
                                      I.SI_I_EV, n_cells=1)
    olat = T.StringLattice(lat.cell_x, lat.cell_y, list(lat.sx[:4]), list(lat.sy[:4]), lat.d)
    oapot = T.AxialPotential(I.SYNTH_DT_A, I.SYNTH_DT_B, olat, I.SYNTH_DT_AX, I.SYNTH_DT_BX, I.SYNTH_DT_CX, I.SI_I_EV,
                             K=1)
    x0, y0 = rng.uniform(0, lat.cell_x, n), rng.uniform(0, lat.cell_y, n)
    psi = math.sqrt(2 * 35.0 / E)
    thx, thy = rng.normal(0, 0.3 * psi, n), rng.normal(0, 0.3 * psi, n)
    ta = t[:3]
    st, got, _, cnt = run_gpu(channel(+1, MS), sc(1e-9), x0, thx, ta, 7, axial=apot, y0=y0, thy=thy)
    assert st == rad.RAD_OK
    ref, rc = T.trajectories_adaptive(x0, thx, thy, E, ta, 7, rtol=1e-9, atol_x=1e-20, atol_v=1e-16, max_level=10,
                                      y0=y0, axial=oapot, ms=True, counts=True)
    close(got, ref)
    np.testing.assert_array_equal(cnt, rc)


def test_lower_bound_budget_and_argument_checks():
    import torch
    x0, th = np.array([0.3e-10, 0.9e-10]), np.array([1e-5, -1e-5])
    t = np.arange(101) * 20e-9
    # max_level 0: one sub-step per interval whatever the error
    st, got, _, cnt = run_gpu(channel(+1, 0), sc(1e-15, max_level=0), x0, th, t, 0)
    assert st == rad.RAD_OK and np.all(cnt == 100)
    # a budget below what the tolerance needs (400 nm intervals at 1e-12 take over ten sub-steps
    # each): the particle stops and RAD_EDATA is recorded
    st, _, _, cnt = run_gpu(channel(+1, 0), sc(1e-12, max_level=12, max_substeps=150), x0, th, 20 * t, 0)
    assert st == rad.RAD_EDATA and np.all(cnt <= 150)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    off = torch.tensor([0, 10], dtype=torch.int64, device="cuda")
    out = torch.empty((10, 10), dtype=torch.float64, device="cuda")
    run = lambda ch, s, **kw: rad.rad_trajectories_adaptive(ch, s, off, d([E]), d([0.0]), d([0.0]), out, 1,
                                                              dt=kw.pop("dt", 5e-9), **kw)
    assert run(channel(+1, rad.RAD_TRAJ_FP32), sc(1e-9)) == rad.RAD_EUNSUPPORTED
    assert run(channel(+1, 0), None) == rad.RAD_EINVAL
    assert run(channel(+1, 0), sc(0.0)) == rad.RAD_EINVAL
    assert run(channel(+1, 0), sc(1e-9, max_level=17)) == rad.RAD_EINVAL
    assert run(channel(+1, 0), sc(1e-9), dt=0.0) == rad.RAD_EINVAL           # no times and no dt
    lat = rad.crystal_string_lattice(rad.RAD_DIAMOND, 5.431e-10, 110)
    ax = rad.RadAxialPotential.make(I.SYNTH_DT_A, I.SYNTH_DT_B, lat, n_cells=1)
    pl = rad.RadPlanarPotential.make(I.SYNTH_DT_A, I.SYNTH_DT_B, I.SI_N)
    assert run(channel(+1, 0), sc(1e-9), planar=pl, axial=ax) == rad.RAD_EINVAL
    # non-increasing times: the particle is skipped and reported
    rc = rad.rad_trajectories_adaptive(channel(+1, 0), sc(1e-9), off, d([E]), d([0.0]), d([0.0]), out, 1,
                                       times=d(np.r_[np.arange(9) * 1e-8, [0.0]]))
    assert rc == rad.RAD_OK and rad.rad_device_status(1) == rad.RAD_EDATA
