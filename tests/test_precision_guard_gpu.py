"""RAD_MIXED's error-budget guard (Sec. II phase in the mixed form).

The mixed form computes each term's phase offset from its time tile's middle sample in FP32 and
takes sin/cos on the SFU; both errors grow with the offset. Every RAD_MIXED call bounds the
offsets on the device,
  X = max over particles and samples of w*_max (c_max |t_k - t_ref| + |dz_k - dz_ref|
      + max|theta_x| |x_k - x_ref| + max|theta_y| |y_k - y_ref|),
and records RAD_EPRECISION (outputs untouched) when X exceeds the plan's budget (8192 rad unless
the caller sets another). These tests check:
  * a grid far outside the emission cone with coarse time steps trips the guard in every mixed
    entry (pre-pass kernel, inline kernel, no-allocation entry), while RAD_FP64_DF computes the
    same call to the FP64 tolerance of the oracle;
  * the device's X equals the definition above, computed here on the host: the call passes with
    a budget 0.1 % above it and trips 0.1 % below it, in both kernels and both kinds of model.
"""
import numpy as np
import pytest

import oracle as O
import paper_1910_10391_gb300 as rad
from paper_1910_10391_gb300 import inputs as I

from helpers import MODE_ORC, assert_fp64_close, gpu_cube

pytestmark = pytest.mark.gpu
HBARC = 1.973269804e-7  # eV m


def coarse_wide(n_particles, step, widen, n_omega=64, n_side=4, E=10e9, seed=2):
    """Ensemble particles sampled every `step`-th of their 5 nm steps, on a direction grid
    `widen` times the emission cone's width."""
    tr = I.channeling(n_particles, E, +1, 20000, 5e-9, seed=seed)
    parts = [I.single(tr.samples[tr.offsets[p]:tr.offsets[p + 1]][::step], tr.gamma[p])
             for p in range(tr.n_particles)]
    sub = I.concat(parts)
    sub.energy_eV = tr.energy_eV.copy()
    g = I._ensemble_grid(E, 20.0, n_omega, n_side)
    grid = I.Grid(g.hbar_omega_eV, g.theta_x * widen, g.theta_y * widen, g.d_omega * widen ** 2)
    return sub, grid


def phase_bound(tr, grid, T, quantum):
    """X of the guard for tiles of T samples (whole particles, no time split)."""
    tx, ty = np.abs(grid.theta_x).max(), np.abs(grid.theta_y).max()
    th2h = ((grid.theta_x ** 2 + grid.theta_y ** 2) * 0.5).max()
    hmax = grid.hbar_omega_eV.max()
    X = 0.0
    for p in range(tr.n_particles):
        S = tr.samples[tr.offsets[p]:tr.offsets[p + 1]]
        L = len(S)
        g, E = tr.gamma[p], tr.energy_eV[p]
        wsm = (hmax / HBARC) / ((1.0 - hmax / E) if quantum else 1.0)
        k = np.arange(L)
        k0 = (k // T) * T
        ref = k0 + (np.minimum(L - k0, T) - 1) // 2
        d = S - S[ref]
        B = (1.0 / (2 * g * g) + th2h) * np.abs(d[:, 0]) + np.abs(d[:, 3]) + tx * np.abs(d[:, 1]) + ty * np.abs(d[:, 2])
        X = max(X, wsm * B.max())
    return X


def run_plan(tr, grid, mode, shape, prepass, budget=None, whole=False):
    """(status, cube) of one RAD_MIXED plan call whose cube starts at 7.0; whole: the plan must
    keep particles whole (no time split), as phase_bound assumes."""
    import torch
    inp = rad.DeviceInputs(tr, grid)
    p = rad.Plan(inp.n_samples, inp.n_particles, inp.n_omega, inp.n_angles, mode, rad.RAD_MIXED, 1, 0)
    assert p.set_prepass(prepass) == rad.RAD_OK
    assert p.set_shape(*shape, 1) == rad.RAD_OK
    if whole:
        assert "amp=0" in p.describe(), p.describe()
    if budget is not None:
        assert p.set_phase_budget(budget) == rad.RAD_OK
    out = torch.full((inp.n_omega * inp.n_angles,), 7.0, dtype=torch.float64, device="cuda")
    rc = p.execute(*inp.args(), out, None, None, None)
    assert rc == rad.RAD_OK, rad.rad_status_string(rc)
    torch.cuda.synchronize()
    st = rad.rad_device_status(1)
    p.close()
    return st, out.view(inp.n_omega, inp.n_angles).cpu().numpy()


@pytest.mark.parametrize("mode", [rad.RAD_CLASSICAL, rad.RAD_SPIN_HALF])
def test_out_of_budget_call_is_refused_and_fp64_df_computes_it(mode):
    import torch
    tr, grid = coarse_wide(2, 16, 4.0)
    quantum = mode != rad.RAD_CLASSICAL
    assert phase_bound(tr, grid, 128, quantum) > 4 * 8192  # far outside the budget
    for prepass in (True, False):
        st, cube = run_plan(tr, grid, mode, (2, 8, 128), prepass)
        assert st == rad.RAD_EPRECISION, rad.rad_status_string(st)
        assert np.all(cube == 7.0)
    # the one-call entry point (default plan) reports it too, and so does the no-allocation entry
    inp = rad.DeviceInputs(tr, grid)
    out = torch.full((inp.n_omega * inp.n_angles,), 7.0, dtype=torch.float64, device="cuda")
    rc = rad.rad_spectrum(*inp.args(), mode, rad.RAD_MIXED, out, None, None, 0, None, 0)
    assert rc == rad.RAD_OK
    assert rad.rad_device_status(1) == rad.RAD_EPRECISION
    assert torch.all(out == 7.0)
    rc = rad.rad_spectrum_noalloc(inp.samples, inp.offsets, inp.gamma, inp.energy, inp.weight, inp.hw, inp.tx,
                                  inp.ty, mode, out)
    assert rc == rad.RAD_EPRECISION, rad.rad_status_string(rc)
    assert torch.all(out == 7.0)
    assert "RAD_FP64_DF" in rad.rad_status_string(rad.RAD_EPRECISION)
    # the FP64-accurate form has no such limit
    ref = O.spectrum_cube(tr, grid, MODE_ORC[mode])
    got = gpu_cube(tr, grid, mode, rad.RAD_FP64_DF)["cube"]
    assert_fp64_close(got, ref)
    # a caller that accepts the larger error raises the budget and gets the mixed result
    st, cube = run_plan(tr, grid, mode, (2, 8, 128), True, budget=1e7)
    assert st == rad.RAD_OK
    assert np.all(np.isfinite(cube)) and not np.any(cube == 7.0)


@pytest.mark.parametrize("mode", [rad.RAD_CLASSICAL, rad.RAD_SPIN_HALF])
@pytest.mark.parametrize("prepass,T", [(True, 128), (True, 256), (False, 128)])
def test_device_bound_matches_its_definition(mode, prepass, T):
    """64 particles (whole-particle chunks), with the budget just above and just below the
    host's X: the pre-pass forms X in FP64, the inline kernel in FP32 (rounding far below 0.1 %)."""
    tr, grid = coarse_wide(64, 4, 1.5, n_omega=40, n_side=3, seed=7)
    X = phase_bound(tr, grid, T, mode != rad.RAD_CLASSICAL)
    shape = (2, 8, T)
    st, cube = run_plan(tr, grid, mode, shape, prepass, budget=X * 1.001, whole=True)
    assert st == rad.RAD_OK, rad.rad_status_string(st)
    assert np.all(np.isfinite(cube))
    st, cube = run_plan(tr, grid, mode, shape, prepass, budget=X * 0.999, whole=True)
    assert st == rad.RAD_EPRECISION, rad.rad_status_string(st)
    assert np.all(cube == 7.0)


def test_phase_budget_argument_checks():
    p = rad.Plan(40, 2, 4, 4, rad.RAD_CLASSICAL, rad.RAD_MIXED, 1, 0)
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        assert p.set_phase_budget(bad) == rad.RAD_EINVAL
    assert p.set_phase_budget(100.0) == rad.RAD_OK
    p.close()
    q = rad.Plan(40, 2, 4, 4, rad.RAD_CLASSICAL, rad.RAD_FP64_DF, 1, 0)
    assert q.set_phase_budget(100.0) == rad.RAD_EINVAL
    q.close()
