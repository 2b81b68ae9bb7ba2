"""Parity of the FP64-accurate double-float form (RAD_FP64_DF) with the FP64 oracle, through the
C ABI, at the FP64 tolerance:
  |S_gpu - S_ref| <= 1e-9 * max(S_ref, 1e-6 * peak) per bin (peak = max of the output).
The phase product w* A_k(n) is FP64 as in RAD_FP64 and is reduced exactly with integer
arithmetic; sin, cos, f and the tile sums run in float pairs with error-free products and sums.
"""
import numpy as np
import pytest

import oracle as O
import paper_1910_10391_gb300 as rad
from paper_1910_10391_gb300 import inputs as I

from helpers import MODE_ORC, assert_fp64_close, gpu_cube

pytestmark = pytest.mark.gpu

DF = rad.RAD_FP64_DF


@pytest.fixture(scope="module")
def undulator():
    return I.workload_undulator_4096()


@pytest.fixture(scope="module")
def ragged_batch():
    """24 electrons, lognormal lengths in [200, 5000], 37 hw x 13 directions."""
    L = I.lognormal_lengths(24, seed=4, median=1000, lo=200, hi=5000)
    tr = I.channeling(24, 20e9, -1, L, 5e-9, seed=4)
    g = I._ensemble_grid(20e9, 20.0, 37, 4)
    tx, ty, dom = I.angle_grid(13, 1, 1.2e-4, 0.3e-4)
    return tr, I.Grid(g.hbar_omega_eV, tx, ty, dom)


def test_df_undulator_full_cube(undulator):
    tr, grid = undulator
    ref = O.spectrum_cube(tr, grid, O.CLASSICAL)
    got = gpu_cube(tr, grid, rad.RAD_CLASSICAL, DF)["cube"]
    print("df undulator max rel", assert_fp64_close(got, ref))


@pytest.mark.parametrize("mode", [rad.RAD_SPIN0, rad.RAD_SPIN_HALF])
def test_df_undulator_quantum_modes(undulator, mode):
    tr, grid = undulator
    tr = I.Trajectories(tr.samples, tr.offsets, tr.gamma, np.array([grid.hbar_omega_eV.max() / 0.6]), tr.weight)
    ref = O.spectrum_cube(tr, grid, MODE_ORC[mode])
    got = gpu_cube(tr, grid, mode, DF)["cube"]
    assert_fp64_close(got, ref)


@pytest.mark.parametrize("mode", [rad.RAD_CLASSICAL, rad.RAD_SPIN_HALF])
def test_df_ensemble(mode):
    tr = I.channeling(8, 10e9, +1, 2000, 5e-9, seed=2)
    grid = I._ensemble_grid(10e9, 20.0, 64, 16)
    ref = O.spectrum_cube(tr, grid, MODE_ORC[mode])
    got = gpu_cube(tr, grid, mode, DF)["cube"]
    print("df ensemble max rel", mode, assert_fp64_close(got, ref))


@pytest.mark.parametrize("shape", [(1, 4, 64, 1), (1, 8, 64, 1), (2, 4, 64, 2), (2, 8, 64, 1), (2, 8, 64, 3)])
def test_df_every_shape(ragged_batch, shape):
    tr, grid = ragged_batch
    ref = O.spectrum_cube(tr, grid, O.SPIN_HALF)
    got = gpu_cube(tr, grid, rad.RAD_SPIN_HALF, DF, shape=shape)["cube"]
    assert_fp64_close(got, ref)


@pytest.mark.parametrize("mode", [rad.RAD_CLASSICAL, rad.RAD_SPIN_HALF])
@pytest.mark.parametrize("shape", [None, (1, 4, 64, 1), (2, 8, 64, 2)])
def test_df_energy_tiles_with_a_ragged_tail(mode, shape):
    """A block takes one direction and NW x 32 x R energies: 300 energies make 256 + 44 (R=2, NW=4,
    the default), 128 + 128 + 44 (R=1, NW=4) or 300 of 512 (R=2, NW=8). Particles of 3, 5, 11 and 16
    time tiles end the tile-sum runs, which are converted into FP64 every two tiles, after odd and
    even counts."""
    L = np.array([130, 257, 700, 1023])
    tr = I.channeling(4, 10e9, +1, L, 5e-9, seed=7)
    grid = I._ensemble_grid(10e9, 20.0, 300, 3)
    ref = O.spectrum_cube(tr, grid, MODE_ORC[mode])
    got = gpu_cube(tr, grid, mode, DF, shape=shape)["cube"]
    assert_fp64_close(got, ref)


@pytest.mark.parametrize("mode", [rad.RAD_CLASSICAL, rad.RAD_SPIN_HALF])
def test_df_one_energy_one_direction(mode):
    """A grid of one photon energy and one direction: one work item per time piece, 255 of the
    block's 256 energies idle."""
    tr = I.channeling(3, 10e9, +1, np.array([300, 64, 1000]), 5e-9, seed=9)
    g = I._ensemble_grid(10e9, 20.0, 8, 4)
    grid = I.Grid(g.hbar_omega_eV[5:6], g.theta_x[6:7], g.theta_y[6:7], g.d_omega[6:7])
    ref = O.spectrum_cube(tr, grid, MODE_ORC[mode])
    assert ref.shape == (1, 1) and ref[0, 0] > 0
    got = gpu_cube(tr, grid, mode, DF)["cube"]
    assert_fp64_close(got, ref)


def test_df_single_particle_time_split(undulator):
    tr, grid = undulator
    ref = O.spectrum_cube(tr, grid, O.CLASSICAL)
    for shape in [(1, 8, 64, 1), (2, 8, 64, 4)]:
        got = gpu_cube(tr, grid, rad.RAD_CLASSICAL, DF, shape=shape)["cube"]
        assert_fp64_close(got, ref)


def test_df_spectrum_bins_and_edges():
    parts = [I.elliptical_undulator(n_samples=n) for n in (2, 64, 65, 128, 129, 3)]
    tr = I.concat(parts)
    hw1 = I.undulator_first_harmonic_eV(2000.0, 0.4e-10, 10e-6)
    grid = I.make_grid(np.array([0.3, 1.0, 1.7]) * hw1, 3, 3, 1e-3)
    boa = I.radial_bins(grid.theta_x, grid.theta_y, 2, 1.5e-3)
    ref = O.spectrum_cube(tr, grid, O.CLASSICAL)
    ref_spec, ref_bins = O.reduce(ref, grid.d_omega, boa, 2)
    out = gpu_cube(tr, grid, rad.RAD_CLASSICAL, DF, outputs=("cube", "spectrum", "bins"), bin_of_angle=boa,
                   n_bins=2)
    assert_fp64_close(out["cube"], ref)
    assert_fp64_close(out["spectrum"], ref_spec)
    assert_fp64_close(out["bins"], ref_bins)
    got = gpu_cube(I.straight_line(), grid, rad.RAD_SPIN_HALF, DF)["cube"]
    assert np.all(got == 0.0)


def test_df_full_grid_particle_of_the_ensemble():
    """Particle 0 of the 10 GeV positron ensemble on the full 512 hw x 64 x 64 grid (the grid the
    benchmark times), every energy x 64 seeded directions, both models."""
    tr, grid = I.workload_positron_ensemble(particles=[0])
    rng = np.random.default_rng(13)
    js = rng.integers(0, grid.n_angles, 64)
    bi = np.repeat(np.arange(grid.n_omega), 64)
    bj = np.tile(js, grid.n_omega)
    for mode, omode in ((rad.RAD_CLASSICAL, O.CLASSICAL), (rad.RAD_SPIN_HALF, O.SPIN_HALF)):
        out = gpu_cube(tr, grid, mode, DF)["cube"]
        ref = O.spectrum_bins(tr, grid, omode, bi, bj).reshape(grid.n_omega, 64)
        print("df full grid max rel", mode, assert_fp64_close(out[:, js], ref))


def test_phases_beyond_2_pow_22_rad():
    """Half-millimetre trajectories seen up to 1 mrad off axis at hw up to 0.45 E: phases w* A
    reach ~1e7 rad, beyond the integer reduction's range (2^22 rad), where the double-float kernel
    takes the FP64 Cody-Waite reduction; it stays within the FP64 tolerance."""
    tr = I.channeling(2, 10e9, +1, 20000, 25e-9, seed=31)
    hw = I.omega_log(16, 1e-3 * 10e9, 0.45 * 10e9)
    grid = I.make_grid(hw, 4, 4, 1.0e-3)
    ref = O.spectrum_cube(tr, grid, O.SPIN_HALF)
    got = gpu_cube(tr, grid, rad.RAD_SPIN_HALF, DF)["cube"]
    print("df large phases max rel", assert_fp64_close(got, ref))
