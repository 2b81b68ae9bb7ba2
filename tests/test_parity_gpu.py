"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances:
  FP64:  |S_gpu - S_ref| <= 1e-9 * max(S_ref, 1e-6 * peak)  per bin (peak = max of the output)
  mixed: |S_gpu - S_ref| / S_ref <= 1e-4 on bins with S_ref >= 1e-3 * peak
"""
import math

import numpy as np
import pytest

import oracle as O
import paper_1910_10391_gb300 as rad
from paper_1910_10391_gb300 import inputs as I

from helpers import MODE_ORC, assert_fp64_close, assert_mixed_close, gpu_cube

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def undulator():
    return I.workload_undulator_4096()


@pytest.fixture(scope="module")
def ensemble_small():
    """8 positrons x 2000 samples of the 10 GeV ensemble generator; 64 hw x 16 x 16 directions."""
    tr = I.channeling(8, 10e9, +1, 2000, 5e-9, seed=2)
    grid = I._ensemble_grid(10e9, 20.0, 64, 16)
    return tr, grid


@pytest.fixture(scope="module")
def ragged_batch():
    """24 electrons, lognormal lengths in [200, 5000] (median 1000), 37 hw x 13 directions."""
    L = I.lognormal_lengths(24, seed=4, median=1000, lo=200, hi=5000)
    tr = I.channeling(24, 20e9, -1, L, 5e-9, seed=4)
    g = I._ensemble_grid(20e9, 20.0, 37, 4)
    tx, ty, dom = I.angle_grid(13, 1, 1.2e-4, 0.3e-4)
    grid = I.Grid(g.hbar_omega_eV, tx, ty, dom)
    return tr, grid


def oracle_cube(tr, grid, mode):
    return O.spectrum_cube(tr, grid, MODE_ORC[mode])


# --------------------------------------------------------------------------- FP64
def test_fp64_undulator_full_cube(undulator):
    tr, grid = undulator
    ref = oracle_cube(tr, grid, rad.RAD_CLASSICAL)
    got = gpu_cube(tr, grid, rad.RAD_CLASSICAL, rad.RAD_FP64)["cube"]
    assert_fp64_close(got, ref)


@pytest.mark.parametrize("mode", [rad.RAD_SPIN0, rad.RAD_SPIN_HALF])
def test_fp64_undulator_quantum_modes(undulator, mode):
    tr, grid = undulator
    # particle energy such that hw/E reaches 0.6 on this grid (gamma kept): exercises w* and recoil
    tr = I.Trajectories(tr.samples, tr.offsets, tr.gamma, np.array([grid.hbar_omega_eV.max() / 0.6]),
                        tr.weight)
    ref = oracle_cube(tr, grid, mode)
    got = gpu_cube(tr, grid, mode, rad.RAD_FP64)["cube"]
    assert_fp64_close(got, ref)


@pytest.mark.parametrize("mode", [rad.RAD_CLASSICAL, rad.RAD_SPIN_HALF])
def test_fp64_ensemble(ensemble_small, mode):
    tr, grid = ensemble_small
    ref = oracle_cube(tr, grid, mode)
    got = gpu_cube(tr, grid, mode, rad.RAD_FP64)["cube"]
    assert_fp64_close(got, ref)


def test_fp64_ragged_lognormal(ragged_batch):
    tr, grid = ragged_batch
    ref = oracle_cube(tr, grid, rad.RAD_SPIN_HALF)
    got = gpu_cube(tr, grid, rad.RAD_SPIN_HALF, rad.RAD_FP64)["cube"]
    assert_fp64_close(got, ref)


@pytest.mark.parametrize("shape", [(1, 4, 64, 1), (1, 8, 64, 4), (2, 4, 64, 2), (2, 8, 64, 1),
                                   (4, 4, 64, 1), (4, 8, 64, 3)])
def test_fp64_every_shape(ragged_batch, shape):
    tr, grid = ragged_batch
    ref = oracle_cube(tr, grid, rad.RAD_SPIN0)
    got = gpu_cube(tr, grid, rad.RAD_SPIN0, rad.RAD_FP64, shape=shape)["cube"]
    assert_fp64_close(got, ref)


def test_fp64_single_particle_time_split(undulator):
    """One particle: work is split in time and pieces combine coherently (amplitude partials)."""
    tr, grid = undulator
    ref = oracle_cube(tr, grid, rad.RAD_CLASSICAL)
    for shape in [(1, 4, 64, 1), (2, 8, 64, 4), (4, 8, 64, 2)]:
        got = gpu_cube(tr, grid, rad.RAD_CLASSICAL, rad.RAD_FP64, shape=shape)["cube"]
        assert_fp64_close(got, ref)


# --------------------------------------------------------------------------- mixed
def test_mixed_undulator(undulator):
    tr, grid = undulator
    ref = oracle_cube(tr, grid, rad.RAD_CLASSICAL)
    got = gpu_cube(tr, grid, rad.RAD_CLASSICAL, rad.RAD_MIXED)["cube"]
    assert_mixed_close(got, ref)


@pytest.mark.parametrize("mode", [rad.RAD_CLASSICAL, rad.RAD_SPIN0, rad.RAD_SPIN_HALF])
def test_mixed_ensemble(ensemble_small, mode):
    tr, grid = ensemble_small
    ref = oracle_cube(tr, grid, mode)
    got = gpu_cube(tr, grid, mode, rad.RAD_MIXED)["cube"]
    assert_mixed_close(got, ref)


@pytest.mark.parametrize("shape", [(1, 8, 64, 1), (2, 4, 64, 2), (2, 8, 64, 1), (2, 8, 128, 1),
                                   (4, 4, 64, 4), (4, 8, 64, 1), (4, 8, 128, 2), (2, 4, 256, 1),
                                   (2, 8, 256, 3)])
def test_mixed_every_shape(ragged_batch, shape):
    tr, grid = ragged_batch
    ref = oracle_cube(tr, grid, rad.RAD_SPIN_HALF)
    got = gpu_cube(tr, grid, rad.RAD_SPIN_HALF, rad.RAD_MIXED, shape=shape)["cube"]
    assert_mixed_close(got, ref)


@pytest.mark.parametrize("shape", [(2, 8, 128, 1), (2, 8, 256, 2), (2, 4, 256, 1), (4, 8, 128, 1),
                                   (4, 8, 256, 3)])
@pytest.mark.parametrize("mode", [rad.RAD_CLASSICAL, rad.RAD_SPIN_HALF])
def test_mixed_prepass_every_shape(ragged_batch, shape, mode):
    """The kernel fed by the per-sample pre-pass, on uneven lengths and ragged grids."""
    tr, grid = ragged_batch
    ref = oracle_cube(tr, grid, mode)
    got = gpu_cube(tr, grid, mode, rad.RAD_MIXED, shape=shape, prepass=True)["cube"]
    assert_mixed_close(got, ref)


@pytest.mark.parametrize("shape", [(2, 8, 256, 1), (2, 4, 256, 1), (4, 8, 128, 2)])
@pytest.mark.parametrize("split", [0, 4, 6])
@pytest.mark.parametrize("mode", [rad.RAD_CLASSICAL, rad.RAD_SPIN_HALF])
def test_mixed_sincos_split(ragged_batch, shape, split, mode):
    """Part of the terms' sin/cos on the FMA pipe (Cody-Waite reduction, Taylor polynomials), or
    none (split 0; the classical default takes 1/8): the same tolerance as the SFU path, on uneven
    lengths, ragged grids and every quadrant."""
    tr, grid = ragged_batch
    ref = oracle_cube(tr, grid, mode)
    got = gpu_cube(tr, grid, mode, rad.RAD_MIXED, shape=shape, prepass=True, split=split)["cube"]
    print("split", split, shape, assert_mixed_close(got, ref))


def test_mixed_prepass_time_split_and_inline_agree(undulator):
    """One particle split in time (amplitude partials) through both mixed kernels."""
    tr, grid = undulator
    ref = oracle_cube(tr, grid, rad.RAD_CLASSICAL)
    a = gpu_cube(tr, grid, rad.RAD_CLASSICAL, rad.RAD_MIXED, shape=(2, 8, 128, 4), prepass=True)["cube"]
    b = gpu_cube(tr, grid, rad.RAD_CLASSICAL, rad.RAD_MIXED, shape=(2, 8, 128, 4), prepass=False)["cube"]
    assert_mixed_close(a, ref)
    assert_mixed_close(b, ref)


# --------------------------------------------------------------------------- outputs
@pytest.mark.parametrize("precision", [rad.RAD_FP64, rad.RAD_MIXED])
def test_spectrum_and_radial_bins(ensemble_small, precision):
    tr, grid = ensemble_small
    boa = I.radial_bins(grid.theta_x, grid.theta_y, 5, np.abs(grid.theta_x).max())
    ref_cube = oracle_cube(tr, grid, rad.RAD_CLASSICAL)
    ref_spec, ref_bins = O.reduce(ref_cube, grid.d_omega, boa, 5)
    out = gpu_cube(tr, grid, rad.RAD_CLASSICAL, precision, outputs=("cube", "spectrum", "bins"),
                   bin_of_angle=boa, n_bins=5)
    if precision == rad.RAD_FP64:
        assert_fp64_close(out["spectrum"], ref_spec)
        assert_fp64_close(out["bins"], ref_bins)
    else:
        assert_mixed_close(out["spectrum"], ref_spec)
        assert_mixed_close(out["bins"], ref_bins)
    # spectrum without the cube (scratch-only path)
    out2 = gpu_cube(tr, grid, rad.RAD_CLASSICAL, precision, outputs=("spectrum",))
    assert np.array_equal(out2["spectrum"], out["spectrum"])


def test_accumulate_adds(ensemble_small):
    import torch
    tr, grid = ensemble_small
    inp = rad.DeviceInputs(tr, grid)
    oc = torch.zeros(inp.n_omega * inp.n_angles, dtype=torch.float64, device="cuda")
    assert rad.rad_spectrum(*inp.args(), rad.RAD_CLASSICAL, rad.RAD_FP64, oc, None, None, 0, None, 0) == 0
    first = oc.clone()
    assert rad.rad_spectrum(*inp.args(), rad.RAD_CLASSICAL, rad.RAD_FP64, oc, None, None, 0, None, 1) == 0
    torch.cuda.synchronize()
    assert torch.equal(oc, 2 * first)


# --------------------------------------------------------------------------- edges
def test_edge_cases():
    import torch
    # minimum-length particles (L = 2) next to long ones, tile-boundary lengths T and T+1
    parts = [I.elliptical_undulator(n_samples=n) for n in (2, 64, 65, 128, 129, 3)]
    tr = I.concat(parts)
    hw1 = I.undulator_first_harmonic_eV(2000.0, 0.4e-10, 10e-6)
    grid = I.make_grid(np.array([0.3, 1.0, 1.7]) * hw1, 3, 3, 1e-3)
    for prec in (rad.RAD_FP64, rad.RAD_MIXED, rad.RAD_FP64_DF):
        got = gpu_cube(tr, grid, rad.RAD_CLASSICAL, prec)["cube"]
        ref = oracle_cube(tr, grid, rad.RAD_CLASSICAL)
        (assert_mixed_close if prec == rad.RAD_MIXED else assert_fp64_close)(got, ref)
    empty = I.Trajectories(np.zeros((0, 10)), np.array([0]), np.zeros(0), np.zeros(0), np.zeros(0))
    for prec in (rad.RAD_FP64, rad.RAD_FP64_DF):
        # no particles: zeros
        got = gpu_cube(empty, grid, rad.RAD_CLASSICAL, prec)["cube"]
        assert np.all(got == 0.0)
        # straight line: exactly zero on the GPU too
        got = gpu_cube(I.straight_line(), grid, rad.RAD_SPIN_HALF, prec)["cube"]
        assert np.all(got == 0.0)
    # no photon energies / no directions: valid, nothing to do
    g0 = I.Grid(np.zeros(0), grid.theta_x, grid.theta_y, grid.d_omega)
    inp = rad.DeviceInputs(tr, g0)
    assert rad.rad_spectrum(*inp.args(), 0, 0, None, None, None, 0, None, 0) == rad.RAD_OK
    torch.cuda.synchronize()


def test_device_data_checks_leave_outputs_untouched(ensemble_small):
    import torch
    tr, grid = ensemble_small
    bad = I.Trajectories(tr.samples.copy(), tr.offsets, tr.gamma, tr.energy_eV, tr.weight)
    bad.samples[123, 7] = np.nan
    inp = rad.DeviceInputs(bad, grid)
    oc = torch.full((inp.n_omega * inp.n_angles,), 7.0, dtype=torch.float64, device="cuda")
    assert rad.rad_spectrum(*inp.args(), 0, 0, oc, None, None, 0, None, 0) == rad.RAD_OK
    assert rad.rad_device_status(1) == rad.RAD_EDATA
    assert torch.all(oc == 7.0)
    # hw >= E in a quantum mode
    g2 = I.Grid(np.array([1e9, 2e10]), grid.theta_x, grid.theta_y, grid.d_omega)
    inp = rad.DeviceInputs(tr, g2)
    oc = torch.full((2 * inp.n_angles,), 7.0, dtype=torch.float64, device="cuda")
    assert rad.rad_spectrum(*inp.args(), rad.RAD_SPIN_HALF, 1, oc, None, None, 0, None, 0) == 0
    assert rad.rad_device_status(1) == rad.RAD_EDATA
    assert torch.all(oc == 7.0)
    # the status word clears and later calls run normally
    inp = rad.DeviceInputs(tr, grid)
    assert rad.rad_spectrum(*inp.args(), 0, 0, oc.new_zeros(inp.n_omega * inp.n_angles), None, None, 0,
                            None, 0) == 0
    assert rad.rad_device_status(1) == rad.RAD_OK


def test_host_checks():
    import torch
    tr, grid = I.workload_undulator_4096()
    inp = rad.DeviceInputs(tr, grid)
    misaligned = torch.zeros(inp.samples.numel() + 1, dtype=torch.float64, device="cuda")[1:]
    lib = rad.load()
    import ctypes
    rc = lib.rad_spectrum(ctypes.c_void_p(misaligned.data_ptr()), inp.n_samples,
                          ctypes.c_void_p(inp.offsets.data_ptr()), 1, ctypes.c_void_p(inp.gamma.data_ptr()),
                          ctypes.c_void_p(inp.energy.data_ptr()), None, ctypes.c_void_p(inp.hw.data_ptr()),
                          inp.n_omega, ctypes.c_void_p(inp.tx.data_ptr()), ctypes.c_void_p(inp.ty.data_ptr()),
                          None, inp.n_angles, 0, 0, ctypes.c_void_p(inp.hw.data_ptr()), None, None, 0, None, 0,
                          None)
    assert rc == rad.RAD_EINVAL


# --------------------------------------------------------------------------- properties
@pytest.mark.parametrize("precision", [rad.RAD_FP64, rad.RAD_MIXED, rad.RAD_FP64_DF])
def test_bitwise_deterministic(ragged_batch, precision):
    tr, grid = ragged_batch
    a = gpu_cube(tr, grid, rad.RAD_SPIN_HALF, precision)["cube"]
    b = gpu_cube(tr, grid, rad.RAD_SPIN_HALF, precision)["cube"]
    assert np.array_equal(a, b)


def test_graph_replay_and_host_entry(ensemble_small):
    import torch
    tr, grid = ensemble_small
    inp = rad.DeviceInputs(tr, grid)
    n = inp.n_omega * inp.n_angles
    direct = torch.zeros(n, dtype=torch.float64, device="cuda")
    assert rad.rad_spectrum(*inp.args(), 2, 1, direct, None, None, 0, None, 0) == 0
    plan = rad.Plan(inp.n_samples, inp.n_particles, inp.n_omega, inp.n_angles, 2, 1, 1, 0)
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = plan.graph(*inp.args(), out, None, None, None, stream=s)
        for _ in range(2):
            assert g.launch(s) == 0
    s.synchronize()
    assert torch.equal(out, direct)
    assert plan.kernel_launches() == 4  # validate, pre-pass, integral kernel, combine
    g.close()
    plan.close()
    host = np.zeros(n)
    rc = rad.rad_spectrum_host(tr.samples, tr.offsets, tr.gamma, tr.energy_eV, tr.weight, grid.hbar_omega_eV,
                               grid.theta_x, grid.theta_y, grid.d_omega, 2, 1, host)
    assert rc == 0
    assert np.array_equal(host, direct.cpu().numpy())


@pytest.mark.parametrize("precision", [rad.RAD_MIXED, rad.RAD_FP64_DF])
def test_autotune_keeps_parity(ragged_batch, precision):
    import torch
    tr, grid = ragged_batch
    inp = rad.DeviceInputs(tr, grid)
    plan = rad.Plan(inp.n_samples, inp.n_particles, inp.n_omega, inp.n_angles, 2, precision, 1, 0)
    out = torch.zeros(inp.n_omega * inp.n_angles, dtype=torch.float64, device="cuda")
    assert plan.autotune(*inp.args(), out, None, None, None, budget_ms=3000) == 0
    assert "R=" in plan.describe()
    ref = oracle_cube(tr, grid, rad.RAD_SPIN_HALF)
    check = assert_mixed_close if precision == rad.RAD_MIXED else assert_fp64_close
    check(out.view(inp.n_omega, inp.n_angles).cpu().numpy(), ref)
    plan.close()
