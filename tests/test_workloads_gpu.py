"""Further workloads through the C ABI against the oracle: the paper's strong undulator (forward
spectrum, on-axis harmonics and the angular distribution over 0-500 eV within 5/gamma), and a
batch whose record array exceeds 2^31 doubles (64-bit indexing)."""
import numpy as np
import pytest

import oracle as O
import paper_1910_10391_gb300 as rad
from paper_1910_10391_gb300 import inputs as I

from helpers import (assert_fp64_close, assert_mixed_close, gpu_cube, planar_undulator_exact,
                     strong_undulator_on_axis)

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


@pytest.mark.parametrize("precision", [rad.RAD_FP64, rad.RAD_FP64_DF, rad.RAD_MIXED])
def test_strong_undulator_angular_distribution(precision):
    """Sec. IV's second integral test at full size: 40961 samples, 1000 photon energies over
    0-500 eV, 32 x 32 directions within 5/gamma. The cube against the oracle on 24 seeded
    directions (all energies), and dI/dOmega (the trapezoid over the energies) of those directions
    against the oracle's and, within the quadrature's h^2 error (below 1e-5 at 2048 samples per
    period, pinned on the CPU), against the closed form; the whole map is finite and keeps the
    theta_y -> -theta_y symmetry of motion in the x-z plane (Sec. II integrand with y = 0)."""
    tr, grid = I.workload_strong_undulator_angular()
    g, K = float(tr.gamma[0]), I.undulator_K(1.0, 0.053)
    cube = gpu_cube(tr, grid, rad.RAD_CLASSICAL, precision)["cube"]
    rng = np.random.default_rng(21)
    js = np.sort(rng.choice(grid.n_angles, 24, replace=False))
    sub = I.Grid(grid.hbar_omega_eV, grid.theta_x[js], grid.theta_y[js], grid.d_omega[js])
    ref = O.spectrum_cube(tr, sub, O.CLASSICAL)
    hw = grid.hbar_omega_eV
    # dI/dOmega by the library's reduction over the energies, against numpy's trapezoid of the cube
    import torch
    d_cube = torch.from_numpy(np.ascontiguousarray(cube)).cuda()
    d_hw = torch.from_numpy(hw).cuda()
    d_out = torch.full((grid.n_angles,), np.nan, dtype=torch.float64, device="cuda")
    assert rad.rad_angular_distribution(d_cube, d_hw, d_out) == rad.RAD_OK
    dIdO = d_out.cpu().numpy()
    np.testing.assert_allclose(dIdO, np.trapezoid(cube, hw, axis=0), rtol=1e-13)
    dIdO_ref = np.trapezoid(ref, hw, axis=0)
    exact = O.ALPHA / (4 * np.pi ** 2) * planar_undulator_exact(hw, sub.theta_x, sub.theta_y, g, K, 0.053, 20)
    assert np.all(np.abs(dIdO_ref / np.trapezoid(exact, hw, axis=0) - 1) < 1e-5)
    if precision == rad.RAD_MIXED:
        for c in range(len(js)):
            assert_mixed_close(cube[:, js[c]], ref[:, c])
        np.testing.assert_allclose(dIdO[js], dIdO_ref, rtol=1e-4)
    else:
        for c in range(len(js)):
            assert_fp64_close(cube[:, js[c]], ref[:, c])
        np.testing.assert_allclose(dIdO[js], dIdO_ref, rtol=1e-9)
    assert np.all(np.isfinite(dIdO)) and dIdO.min() > 0
    # the cell-centred grid holds (theta_x, theta_y) and (theta_x, -theta_y) in rows iy and 31 - iy
    m = dIdO.reshape(32, 32)
    assert np.allclose(grid.theta_y.reshape(32, 32), -grid.theta_y.reshape(32, 32)[::-1, :], rtol=0, atol=1e-18)
    np.testing.assert_allclose(m, m[::-1, :], rtol=1e-9 if precision != rad.RAD_MIXED else 1e-4)


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


def test_positron_ensemble_full_size_sampled():
    """The full positron ensemble (1024 e+ x 20 000 samples, 512 hw x 64 x 64, classical and
    spin-1/2) in the benchmark's launch configuration: shape autotuned on a 2-particle batch,
    32-particle batches added into one cube (accumulate). 32 seeded bins per model over all
    1024 particles (24 of them in the emission cone) against the oracle at the mixed tolerance;
    the plain FP64 kernel on particle 0 over every energy x 64 seeded directions at the FP64
    tolerance."""
    import torch
    tr, grid = I.workload_positron_ensemble()
    inp = rad.DeviceInputs(tr, grid)
    no, na, L = inp.n_omega, inp.n_angles, 20000
    rng = np.random.default_rng(12)
    a2 = inp.args()

    def part(p0, n):  # particles p0 .. p0+n-1 of the resident ensemble, as one call's arguments
        w = a2[4]
        return (a2[0][p0 * L:(p0 + n) * L], torch.arange(n + 1, dtype=torch.int64, device="cuda") * L,
                a2[2][p0:p0 + n], a2[3][p0:p0 + n], None if w is None else w[p0:p0 + n]) + tuple(a2[5:])

    for mode, omode in ((rad.RAD_CLASSICAL, O.CLASSICAL), (rad.RAD_SPIN_HALF, O.SPIN_HALF)):
        tp = rad.Plan(2 * L, 2, no, na, mode, rad.RAD_MIXED, 3, 0)
        tmp = torch.empty(no * na, dtype=torch.float64, device="cuda")
        tmps = torch.empty(no, dtype=torch.float64, device="cuda")
        assert tp.autotune(*part(0, 2), tmp, tmps, None, None, budget_ms=4000) == 0
        d = dict(kv.split("=") for kv in tp.describe().split())
        tp.close()
        plan = rad.Plan(32 * L, 32, no, na, mode, rad.RAD_MIXED, 3, 0)
        assert plan.set_prepass(int(d["pp"])) == 0
        assert plan.set_shape(int(d["R"]), int(d["NW"]), int(d["T"]), 1) == 0
        if int(d.get("pe", "0")):
            assert plan.set_sincos_split(int(d["pe"])) == 0
        cube = torch.zeros(no * na, dtype=torch.float64, device="cuda")
        spec = torch.zeros(no, dtype=torch.float64, device="cuda")
        for b in range(32):
            assert plan.execute(*part(32 * b, 32), cube, spec, None, None, accumulate=1) == 0
        torch.cuda.synchronize()
        assert rad.rad_device_status(1) == rad.RAD_OK
        plan.close()
        got_cube = cube.view(no, na).cpu().numpy()
        # sample locations: 24 seeded bins among those above 1e-2 of the peak (the emission cone
        # covers a small part of the grid) and 8 seeded bins anywhere
        big = np.flatnonzero(got_cube.ravel() >= 1e-2 * got_cube.max())
        flat = np.r_[rng.choice(big, 24, replace=False), rng.integers(0, no * na, 8)]
        bi, bj = flat // na, flat % na
        ref = O.spectrum_bins(tr, grid, omode, bi, bj)
        got = got_cube[bi, bj]
        peak = got_cube.max()
        sel = ref >= 1e-3 * peak
        assert sel.sum() >= 12
        rel = np.abs(got[sel] - ref[sel]) / ref[sel]
        print("positron ensemble full size, mode", mode, d, "sampled bins", int(sel.sum()), "max rel err",
              rel.max())
        assert rel.max() <= 1e-4, rel.max()
        assert np.all(np.abs(got - ref)[~sel] <= 1e-7 * peak)
        # spectrum = sum_j cube dOmega (the angle integral of the same launches)
        dom = grid.d_omega
        assert np.allclose(spec.cpu().numpy(), (got_cube * dom[None, :]).sum(1), rtol=1e-12, atol=0)
    # plain FP64: particle 0, full grid, 64 directions x every energy
    one = tr.subset([0])
    ref_j = rng.integers(0, na, 64)
    out = gpu_cube(one, grid, rad.RAD_SPIN_HALF, rad.RAD_FP64)["cube"]
    bi2 = np.repeat(np.arange(no), 64)
    bj2 = np.tile(ref_j, no)
    ref = O.spectrum_bins(one, grid, O.SPIN_HALF, bi2, bj2).reshape(no, 64)
    assert_fp64_close(out[:, ref_j], ref)


def test_angular_distribution_edge_cases():
    """The energy integral of a cube: non-uniform photon energies, a ragged number of directions
    (more than one block of threads), one energy (zero) and no directions; against numpy."""
    import torch
    rng = np.random.default_rng(5)
    for n_omega, n_angles in ((37, 1000), (2, 3), (1, 5), (300, 257)):
        hw = np.sort(rng.uniform(1.0, 500.0, n_omega))
        cube = rng.lognormal(0, 2, (n_omega, n_angles))
        out = torch.full((n_angles,), np.nan, dtype=torch.float64, device="cuda")
        rc = rad.rad_angular_distribution(torch.from_numpy(cube).cuda(), torch.from_numpy(hw).cuda(), out)
        assert rc == rad.RAD_OK
        ref = np.trapezoid(cube, hw, axis=0) if n_omega > 1 else np.zeros(n_angles)
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-13, atol=0)
    empty = torch.empty(0, dtype=torch.float64, device="cuda")
    assert rad.rad_angular_distribution(torch.ones(4, dtype=torch.float64, device="cuda"),
                                        torch.ones(4, dtype=torch.float64, device="cuda"), empty) == rad.RAD_OK
