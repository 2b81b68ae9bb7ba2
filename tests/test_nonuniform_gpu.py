"""GPU parity on non-uniform sample times (Sec. IV: the trajectory solver returns records at
caller-controlled times; the time integral uses trapezoid weights w_k = (t_{k+1} - t_{k-1})/2,
one-sided at the ends).

Every kernel reads the neighbours t_{k-1}, t_{k+1} of a sample across time-tile boundaries (the
halo of the staged tile, or the pre-pass's record of the previous tile). These tests feed
analytic trajectories sampled at jittered, geometric and tile-jump times (steps changing exactly
at the first sample of each time tile, T = 64, 128, 256), with lengths 2, 3, T - 1, T, T + 1 and
a few tiles plus a ragged tail, through all three precisions and the time-split path, and compare
with the FP64 oracle: 1e-9 for RAD_FP64 and RAD_FP64_DF, 1e-4 on bins >= 1e-3 of the peak for
RAD_MIXED. Per-particle spectra check each trajectory on its own.
"""
import numpy as np
import pytest

import oracle as O
import paper_1910_10391_gb300 as rad
from paper_1910_10391_gb300 import inputs as I

from helpers import MODE_ORC, assert_fp64_close, assert_mixed_close, gpu_cube

pytestmark = pytest.mark.gpu

G, LAM = 2000.0, 10e-6
LENGTHS = [2, 3, 63, 64, 65, 127, 128, 129, 255, 256, 257, 700, 1031]


def batch(T, kinds=("jitter", "geometric", "tile_jumps")):
    """Elliptical-undulator particles (motion in both planes) at non-uniform times, one per
    length, the time kinds taking turns; the length of each is 3 periods for 1031 samples."""
    parts = []
    for i, L in enumerate(LENGTHS):
        kind = kinds[i % len(kinds)]
        t = I.sample_times(kind, L, 3 * LAM * L / 1031, seed=100 + i, tile=T)
        parts.append(I.elliptical_undulator(G, lam=LAM, times=t))
    tr = I.concat(parts)
    hw1 = I.undulator_first_harmonic_eV(G, 0.4e-10, LAM)
    grid = I.make_grid(I.omega_linear(48, 2.5 * hw1), 4, 4, 2.0 / G)
    tr.energy_eV = np.full(tr.n_particles, 4.0 * hw1)  # recoil u up to 0.6 in the quantum modes
    return tr, grid


@pytest.fixture(scope="module", params=[64, 128, 256])
def case(request):
    T = request.param
    tr, grid = batch(T)
    refs = {m: O.spectrum_cube(tr, grid, MODE_ORC[m]) for m in (rad.RAD_CLASSICAL, rad.RAD_SPIN_HALF)}
    return T, tr, grid, refs


@pytest.mark.parametrize("mode", [rad.RAD_CLASSICAL, rad.RAD_SPIN_HALF])
def test_fp64_forms_nonuniform(case, mode):
    T, tr, grid, refs = case
    if T == 64:  # the FP64 kernels stage 64-sample tiles
        assert_fp64_close(gpu_cube(tr, grid, mode, rad.RAD_FP64, shape=(2, 8, 64, 1))["cube"], refs[mode])
        assert_fp64_close(gpu_cube(tr, grid, mode, rad.RAD_FP64_DF, shape=(2, 4, 64, 1))["cube"], refs[mode])
    else:
        assert_fp64_close(gpu_cube(tr, grid, mode, rad.RAD_FP64)["cube"], refs[mode])
        assert_fp64_close(gpu_cube(tr, grid, mode, rad.RAD_FP64_DF)["cube"], refs[mode])


@pytest.mark.parametrize("mode", [rad.RAD_CLASSICAL, rad.RAD_SPIN_HALF])
@pytest.mark.parametrize("prepass", [True, False])
def test_mixed_nonuniform(case, mode, prepass):
    T, tr, grid, refs = case
    shapes = {64: (2, 8, 64), 128: (2, 8, 128), 256: (2, 8, 256)}
    if prepass and T == 64:
        pytest.skip("the pre-pass kernel stages 128- or 256-sample tiles")
    got = gpu_cube(tr, grid, mode, rad.RAD_MIXED, shape=shapes[T] + (1,), prepass=prepass)["cube"]
    assert_mixed_close(got, refs[mode])


@pytest.mark.parametrize("precision", [rad.RAD_FP64, rad.RAD_FP64_DF, rad.RAD_MIXED])
def test_per_particle_spectra_nonuniform(precision):
    """Each particle's angle-integrated spectrum, so that a wrong weight in any one short or
    long trajectory shows on its own."""
    import torch
    tr, grid = batch(128)
    inp = rad.DeviceInputs(tr, grid)
    out = torch.full((inp.n_particles, inp.n_omega), np.nan, dtype=torch.float64, device="cuda")
    rc = rad.rad_spectrum_particles(*inp.args(), rad.RAD_SPIN_HALF, precision, out)
    assert rc == rad.RAD_OK, rad.rad_status_string(rc)
    torch.cuda.synchronize()
    assert rad.rad_device_status(1) == rad.RAD_OK
    got = out.cpu().numpy()
    for p in range(tr.n_particles):
        one = tr.subset([p])
        ref, _ = O.reduce(O.spectrum_cube(one, grid, O.SPIN_HALF), grid.d_omega)
        if precision == rad.RAD_MIXED:
            assert_mixed_close(got[p], ref)
        else:
            assert_fp64_close(got[p], ref)


@pytest.mark.parametrize("precision", [rad.RAD_FP64, rad.RAD_FP64_DF, rad.RAD_MIXED])
def test_time_split_single_particle_nonuniform(precision):
    """One long particle split into time pieces (amplitude partials combined coherently): the
    piece boundaries fall inside tiles of a tile-jump time grid."""
    t = I.sample_times("tile_jumps", 3001, 9 * LAM, tile=64)
    tr = I.elliptical_undulator(G, lam=LAM, times=t)
    hw1 = I.undulator_first_harmonic_eV(G, 0.4e-10, LAM)
    grid = I.make_grid(I.omega_linear(40, 2.5 * hw1), 3, 3, 2.0 / G)
    ref = O.spectrum_cube(tr, grid, O.CLASSICAL)
    shape = {rad.RAD_FP64: (2, 8, 64, 4), rad.RAD_FP64_DF: (2, 4, 64, 4), rad.RAD_MIXED: (2, 8, 128, 4)}[precision]
    got = gpu_cube(tr, grid, rad.RAD_CLASSICAL, precision, shape=shape)["cube"]
    if precision == rad.RAD_MIXED:
        assert_mixed_close(got, ref)
    else:
        assert_fp64_close(got, ref)
