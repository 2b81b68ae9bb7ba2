"""Per-particle spectra (rad_spectrum_particles) against the oracle, particle by particle."""
import numpy as np
import pytest

import oracle as O
import paper_1910_10391_gb300 as rad
from paper_1910_10391_gb300 import inputs as I

from helpers import assert_fp64_close, assert_mixed_close

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [rad.RAD_FP64, rad.RAD_MIXED])
def test_per_particle_bins_and_spectra(precision):
    import torch
    tr = I.channeling(5, 10e9, +1, 1500, 5e-9, seed=12)
    tr.weight = np.array([1.0, 0.5, 2.0, 1.0, 0.25])
    grid = I._ensemble_grid(10e9, 20.0, 40, 12)
    boa = I.radial_bins(grid.theta_x, grid.theta_y, 6, np.abs(grid.theta_x).max())
    inp = rad.DeviceInputs(tr, grid, bin_of_angle=boa, n_bins=6)
    spec = torch.empty((5, 40), dtype=torch.float64, device="cuda")
    bins = torch.empty((5, 40, 6), dtype=torch.float64, device="cuda")
    rc = rad.rad_spectrum_particles(*inp.args(), rad.RAD_SPIN_HALF, precision, spec, inp.boa, 6, bins)
    assert rc == rad.RAD_OK
    torch.cuda.synchronize()
    assert rad.rad_device_status(1) == rad.RAD_OK
    close = assert_fp64_close if precision == rad.RAD_FP64 else assert_mixed_close
    for p in range(5):
        one = tr.subset([p])
        cube = O.spectrum_cube(one, grid, O.SPIN_HALF)
        s_ref, b_ref = O.reduce(cube, grid.d_omega, boa, 6)
        close(spec[p].cpu().numpy(), s_ref)
        close(bins[p].cpu().numpy(), b_ref)
