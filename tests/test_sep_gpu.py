"""Parity of the separable mixed kernel (tensor direction grids, rad_plan_set_angle_grid) with the
FP64 oracle, through the C ABI.

The kernel forms e^{i phi} of a 2 x 2 block of directions from three sin/cos pairs and three
complex products (the phase of Sec. II separates in theta_x and theta_y). Tolerance as for every
mixed-precision result: relative error <= 1e-4 on bins >= 1e-3 of the peak.
"""
import numpy as np
import pytest

import oracle as O
import paper_1910_10391_gb300 as rad
from paper_1910_10391_gb300 import inputs as I

from helpers import MODE_ORC, assert_mixed_close

pytestmark = pytest.mark.gpu

SEP_SHAPES = [(1, 4, 256, 1), (1, 4, 128, 1), (1, 8, 128, 1), (1, 4, 128, 3)]


def sep_cube(tr, grid, mode, n_x, shape=None, outputs=("cube",), bin_of_angle=None, n_bins=0,
             expect_status=rad.RAD_OK, fill=np.nan):
    import torch
    inp = rad.DeviceInputs(tr, grid, bin_of_angle=bin_of_angle, n_bins=n_bins)
    want = ("cube" in outputs) * 1 + ("spectrum" in outputs) * 2 + ("bins" in outputs) * 4
    oc = torch.full((inp.n_omega * inp.n_angles,), fill, dtype=torch.float64, device="cuda")
    os_ = torch.full((inp.n_omega,), fill, dtype=torch.float64, device="cuda")
    ob = torch.full((inp.n_omega * max(n_bins, 1),), fill, dtype=torch.float64, device="cuda")
    p = rad.Plan(inp.n_samples, inp.n_particles, inp.n_omega, inp.n_angles, mode, rad.RAD_MIXED, want,
                 n_bins if want & 4 else 0)
    assert p.set_angle_grid(n_x) == rad.RAD_OK
    if shape is not None:
        assert p.set_shape(*shape) == rad.RAD_OK, shape
    assert "sep=1" in p.describe(), p.describe()
    rc = p.execute(*inp.args(), oc if want & 1 else None, os_ if want & 2 else None,
                   inp.boa if want & 4 else None, ob if want & 4 else None)
    assert rc == rad.RAD_OK, rad.rad_status_string(rc)
    torch.cuda.synchronize()
    p.close()
    st = rad.rad_device_status(1)
    assert st == expect_status, rad.rad_status_string(st)
    res = {"cube": oc.view(inp.n_omega, inp.n_angles).cpu().numpy()}
    if want & 2:
        res["spectrum"] = os_.cpu().numpy()
    if want & 4:
        res["bins"] = ob.view(inp.n_omega, n_bins).cpu().numpy()
    return res


@pytest.fixture(scope="module")
def ragged_odd_grid():
    """20 electrons, lognormal lengths in [200, 3000] (ragged tiles), 37 hw x (7 x 5) directions:
    odd grid sides leave partial 2 x 2 blocks on the last column and row."""
    L = I.lognormal_lengths(20, seed=14, median=800, lo=200, hi=3000)
    tr = I.channeling(20, 20e9, -1, L, 5e-9, seed=14)
    g = I._ensemble_grid(20e9, 20.0, 37, 4)
    grid = I.make_grid(g.hbar_omega_eV, 7, 5, 1.2e-4, 0.6e-4)
    return tr, grid


@pytest.mark.parametrize("shape", SEP_SHAPES)
@pytest.mark.parametrize("mode", [rad.RAD_CLASSICAL, rad.RAD_SPIN0, rad.RAD_SPIN_HALF])
def test_sep_every_shape_and_mode(ragged_odd_grid, shape, mode):
    tr, grid = ragged_odd_grid
    ref = O.spectrum_cube(tr, grid, MODE_ORC[mode])
    got = sep_cube(tr, grid, mode, 7, shape=shape)["cube"]
    print(shape, mode, assert_mixed_close(got, ref))


@pytest.mark.parametrize("nx,ny", [(1, 6), (6, 1), (2, 2), (3, 3), (16, 16)])
def test_sep_grid_sides(nx, ny):
    """Single rows and columns (degenerate blocks), exact 2 x 2 and larger grids."""
    tr = I.channeling(4, 10e9, +1, 1500, 5e-9, seed=21)
    g = I._ensemble_grid(10e9, 20.0, 45, 4)
    grid = I.make_grid(g.hbar_omega_eV, nx, ny, 2.0e-4, 1.0e-4)
    ref = O.spectrum_cube(tr, grid, O.SPIN_HALF)
    got = sep_cube(tr, grid, rad.RAD_SPIN_HALF, nx)["cube"]
    assert_mixed_close(got, ref)


def test_sep_single_particle_time_split():
    """One particle: the work is split in time and the pieces' amplitudes combine coherently."""
    tr, grid = I.workload_undulator_4096()
    ref = O.spectrum_cube(tr, grid, O.CLASSICAL)
    for shape in [(1, 4, 256, 1), (1, 8, 128, 4)]:
        got = sep_cube(tr, grid, rad.RAD_CLASSICAL, 16, shape=shape)["cube"]
        assert_mixed_close(got, ref)


def test_sep_off_centre_grid_and_outputs():
    """A grid centred away from the axis (large theta_x + theta_y offsets in the phase pieces),
    with the angle-integrated spectrum and radial bins."""
    tr = I.channeling(6, 10e9, +1, 2500, 5e-9, seed=22)
    g = I._ensemble_grid(10e9, 20.0, 33, 4)
    grid = I.make_grid(g.hbar_omega_eV, 10, 8, 1.5e-4, 1.0e-4, center_x=3e-4, center_y=-2e-4)
    boa = I.radial_bins(grid.theta_x - 3e-4, grid.theta_y + 2e-4, 4, 1.6e-4)
    ref = O.spectrum_cube(tr, grid, O.CLASSICAL)
    ref_spec, ref_bins = O.reduce(ref, grid.d_omega, boa, 4)
    out = sep_cube(tr, grid, rad.RAD_CLASSICAL, 10, outputs=("cube", "spectrum", "bins"), bin_of_angle=boa,
                   n_bins=4)
    assert_mixed_close(out["cube"], ref)
    assert_mixed_close(out["spectrum"], ref_spec)
    assert_mixed_close(out["bins"], ref_bins)


def test_sep_matches_list_kernel_and_is_deterministic(ragged_odd_grid):
    import torch
    from helpers import gpu_cube
    tr, grid = ragged_odd_grid
    a = sep_cube(tr, grid, rad.RAD_SPIN_HALF, 7)["cube"]
    b = sep_cube(tr, grid, rad.RAD_SPIN_HALF, 7)["cube"]
    assert np.array_equal(a, b)
    lst = gpu_cube(tr, grid, rad.RAD_SPIN_HALF, rad.RAD_MIXED)["cube"]
    assert_mixed_close(a, lst, rel=2e-4)
    torch.cuda.synchronize()


def test_sep_rejects_a_grid_that_is_not_a_tensor_product(ragged_odd_grid):
    """A declared grid whose theta_x varies down a column: device check fails, outputs unchanged."""
    tr, grid = ragged_odd_grid
    tx = grid.theta_x.copy()
    tx[7 * 3 + 2] += 1e-9
    bad = I.Grid(grid.hbar_omega_eV, tx, grid.theta_y, grid.d_omega)
    out = sep_cube(tr, bad, rad.RAD_CLASSICAL, 7, expect_status=rad.RAD_EDATA, fill=5.0)
    assert np.all(out["cube"] == 5.0)


def test_set_angle_grid_argument_checks(ragged_odd_grid):
    tr, grid = ragged_odd_grid
    inp = rad.DeviceInputs(tr, grid)
    p64 = rad.Plan(inp.n_samples, inp.n_particles, inp.n_omega, inp.n_angles, 0, rad.RAD_FP64, 1, 0)
    assert p64.set_angle_grid(7) == rad.RAD_EINVAL
    p64.close()
    p = rad.Plan(inp.n_samples, inp.n_particles, inp.n_omega, inp.n_angles, 0, rad.RAD_MIXED, 1, 0)
    assert p.set_angle_grid(6) == rad.RAD_EINVAL      # does not divide 35
    assert p.set_angle_grid(-1) == rad.RAD_EINVAL
    assert "sep=0" in p.describe()
    assert p.set_angle_grid(7) == rad.RAD_OK and "sep=1" in p.describe()
    assert p.set_sincos_split(4) == rad.RAD_EINVAL    # the FMA-pipe split belongs to the list kernel
    assert p.set_shape(2, 8, 256, 1) == rad.RAD_OK and "sep=0" in p.describe()  # a list-kernel shape
    assert p.set_angle_grid(7) == rad.RAD_OK and "sep=1" in p.describe()
    assert p.set_angle_grid(0) == rad.RAD_OK and "sep=0" in p.describe()
    p.close()


def test_host_entry_detects_tensor_grid():
    """rad_spectrum_host finds the tensor grid in its host arrays and runs the separable kernel:
    bitwise equal to a plan with the grid declared."""
    tr = I.channeling(4, 10e9, +1, 1800, 5e-9, seed=23)
    g = I._ensemble_grid(10e9, 20.0, 40, 4)
    grid = I.make_grid(g.hbar_omega_eV, 9, 6, 2.0e-4, 1.0e-4)
    host = np.zeros(40 * 54)
    rc = rad.rad_spectrum_host(tr.samples, tr.offsets, tr.gamma, tr.energy_eV, tr.weight, grid.hbar_omega_eV,
                               grid.theta_x, grid.theta_y, grid.d_omega, rad.RAD_SPIN_HALF, rad.RAD_MIXED, host)
    assert rc == rad.RAD_OK
    dev = sep_cube(tr, grid, rad.RAD_SPIN_HALF, 9)["cube"]
    assert np.array_equal(host.reshape(40, 54), dev)


def test_sep_autotune_keeps_parity(ragged_odd_grid):
    import torch
    tr, grid = ragged_odd_grid
    inp = rad.DeviceInputs(tr, grid)
    plan = rad.Plan(inp.n_samples, inp.n_particles, inp.n_omega, inp.n_angles, 2, 1, 1, 0)
    assert plan.set_angle_grid(7) == rad.RAD_OK
    out = torch.zeros(inp.n_omega * inp.n_angles, dtype=torch.float64, device="cuda")
    assert plan.autotune(*inp.args(), out, None, None, None, budget_ms=3000) == 0
    ref = O.spectrum_cube(tr, grid, O.SPIN_HALF)
    assert_mixed_close(out.view(inp.n_omega, inp.n_angles).cpu().numpy(), ref)
    plan.close()
