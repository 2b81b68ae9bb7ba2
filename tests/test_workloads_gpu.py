"""Further workloads through the C ABI against the oracle: the paper's strong undulator, and a
batch whose record array exceeds 2^31 doubles (64-bit indexing)."""
import numpy as np
import pytest

import oracle as O
import paper_1910_10391_gb300 as rad
from paper_1910_10391_gb300 import inputs as I

from helpers import assert_fp64_close, assert_mixed_close, gpu_cube, strong_undulator_on_axis

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [rad.RAD_FP64, rad.RAD_MIXED])
def test_strong_undulator(precision):
    """2 GeV e-, 53 mm, 20 periods, 1 T (Sec. IV integral test): 40961 samples, 0-500 eV."""
    tr, grid = I.workload_strong_undulator(samples_per_period=2048, n_omega=96, n_side=4)
    got = gpu_cube(tr, grid, rad.RAD_CLASSICAL, precision)["cube"]
    ref = O.spectrum_cube(tr, grid, O.CLASSICAL)
    (assert_fp64_close if precision == rad.RAD_FP64 else assert_mixed_close)(got, ref)


@pytest.mark.parametrize("precision", [rad.RAD_FP64, rad.RAD_MIXED])
def test_strong_undulator_harmonics_closed_form(precision):
    """On-axis harmonics 1..11 of the strong undulator against the Bessel-series line heights
    (exact for this trajectory up to rounding; even harmonics vanish)."""
    import math
    g = 2.0e9 / I.ME_EV
    K = I.undulator_K(1.0, 0.053)
    tr = I.planar_undulator(g, K, 0.053, 20, 2048)
    hw1 = 2 * g * g * I.HBARC_EV_M * (2 * math.pi / 0.053) / (1 + K * K / 2)
    ns = np.arange(1, 12)
    grid = I.Grid(ns * hw1, np.zeros(1), np.zeros(1), np.ones(1))
    got = gpu_cube(tr, grid, rad.RAD_CLASSICAL, precision)["cube"][:, 0]
    ref = np.array([strong_undulator_on_axis(n, K, g, 20) for n in ns])
    odd = ns % 2 == 1
    np.testing.assert_allclose(got[odd], ref[odd], rtol=1e-9 if precision == rad.RAD_FP64 else 1e-4)
    assert np.all(np.abs(got[~odd]) <= (1e-15 if precision == rad.RAD_FP64 else 1e-7) * ref.max())


def test_record_array_beyond_2_pow_31_doubles():
    """220 particles x 1,000,000 samples = 2.2e8 records (2.2e9 doubles, 17.6 GB) on 3 hw x 4
    directions: sample offsets beyond 2^31 doubles in both precisions, every bin against the
    oracle."""
    import torch
    tr = I.channeling(220, 10e9, +1, 1_000_000, 5e-9, seed=31, ms=False)
    assert tr.samples.size > 2 ** 31
    grid = I.make_grid(np.array([2e7, 3e8, 2e9]), 2, 2, 1e-4)
    ref = O.spectrum_cube(tr, grid, O.CLASSICAL)
    assert_fp64_close(gpu_cube(tr, grid, rad.RAD_CLASSICAL, rad.RAD_FP64)["cube"], ref)
    torch.cuda.empty_cache()
    assert_mixed_close(gpu_cube(tr, grid, rad.RAD_CLASSICAL, rad.RAD_MIXED)["cube"], ref)
    del tr
    torch.cuda.empty_cache()


@pytest.mark.parametrize("precision", [rad.RAD_FP64, rad.RAD_MIXED])
def test_more_particles_than_grid_y(precision):
    """70,001 short particles: the pre-pass and the per-particle reduction stride over the
    65,535-block grid y limit; cube and selected per-particle spectra against the oracle."""
    import torch
    n = 70_001
    tr = I.channeling(n, 10e9, +1, 64, 5e-9, seed=5, ms=False)
    grid = I._ensemble_grid(10e9, 20.0, 8, 2)
    ref = O.spectrum_cube(tr, grid, O.SPIN_HALF)
    close = assert_fp64_close if precision == rad.RAD_FP64 else assert_mixed_close
    close(gpu_cube(tr, grid, rad.RAD_SPIN_HALF, precision)["cube"], ref)
    inp = rad.DeviceInputs(tr, grid)
    spec = torch.empty((n, 8), dtype=torch.float64, device="cuda")
    rc = rad.rad_spectrum_particles(*inp.args(), rad.RAD_SPIN_HALF, precision, spec, None, 0, None)
    assert rc == rad.RAD_OK
    torch.cuda.synchronize()
    assert rad.rad_device_status(1) == rad.RAD_OK
    for p in (0, 65_534, 65_535, 65_536, n - 1):
        s_ref, _ = O.reduce(O.spectrum_cube(tr.subset([p]), grid, O.SPIN_HALF), grid.d_omega)
        close(spec[p].cpu().numpy(), s_ref)


@pytest.mark.parametrize("precision", [rad.RAD_FP64, rad.RAD_MIXED])
def test_sections_with_energy_loss(precision):
    """50 GeV positrons with radiation-reaction drag and scattering loss, cut into sections of
    2000 samples (10 um): every section is an entry with the gamma and E it starts with (BCK
    spin-1/2 with recoil), against the oracle on the same entries."""
    sc = I.channeling_sections(6, 50e9, +1, 6001, 5e-9, seed=8, section_samples=2000)
    assert sc.traj.n_particles == 24
    grid = I._ensemble_grid(50e9, 20.0, 48, 6)
    ref = O.spectrum_cube(sc.traj, grid, O.SPIN_HALF)
    got = gpu_cube(sc.traj, grid, rad.RAD_SPIN_HALF, precision)["cube"]
    (assert_fp64_close if precision == rad.RAD_FP64 else assert_mixed_close)(got, ref)


def test_electron_batch_full_size_sampled():
    """The full electron batch (4096 e-, lognormal 2k-200k samples, 1.1e8 records, 1024 hw x
    32x32, spin-1/2 with recoil) in the measured launch configuration: shape autotuned on a
    16-particle slice, one graph-captured launch. 24 seeded bins over all 4096 particles against
    the oracle at the mixed tolerance."""
    import torch
    tr, grid = I.workload_electron_batch()
    inp = rad.DeviceInputs(tr, grid)
    sub = tr.subset(range(16))
    si = rad.DeviceInputs(sub, grid)
    tp = rad.Plan(si.n_samples, 16, si.n_omega, si.n_angles, rad.RAD_SPIN_HALF, rad.RAD_MIXED, 1, 0)
    tmp = torch.empty(si.n_omega * si.n_angles, dtype=torch.float64, device="cuda")
    assert tp.autotune(*si.args(), tmp, None, None, None, budget_ms=20000) == 0
    d = dict(kv.split("=") for kv in tp.describe().split())
    tp.close()
    plan = rad.Plan(inp.n_samples, inp.n_particles, inp.n_omega, inp.n_angles, rad.RAD_SPIN_HALF, rad.RAD_MIXED,
                    1, 0)
    assert plan.set_shape(int(d["R"]), int(d["NW"]), int(d["T"]), 1) == 0
    out = torch.zeros(inp.n_omega * inp.n_angles, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = plan.graph(*inp.args(), out, None, None, None, stream=s)
        assert g.launch(s) == 0
    s.synchronize()
    assert rad.rad_device_status(1) == rad.RAD_OK
    cube = out.view(inp.n_omega, inp.n_angles).cpu().numpy()
    g.close()
    plan.close()
    del inp
    torch.cuda.empty_cache()
    rng = np.random.default_rng(11)
    # energies where the spectrum is significant plus random ones
    bi = np.r_[rng.integers(0, 400, 16), rng.integers(0, grid.n_omega, 8)]
    bj = rng.integers(0, grid.n_angles, 24)
    ref = O.spectrum_bins(tr, grid, O.SPIN_HALF, bi, bj)
    got = cube[bi, bj]
    peak = cube.max()
    sel = ref >= 1e-3 * peak
    assert sel.sum() >= 8
    rel = np.abs(got[sel] - ref[sel]) / ref[sel]
    print("electron batch full size: sampled bins", int(sel.sum()), "max rel err", rel.max())
    assert rel.max() <= 1e-4, rel.max()
    assert np.all(np.abs(got - ref)[~sel] <= 1e-7 * peak)
