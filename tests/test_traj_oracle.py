"""Pins of the trajectory oracle (oracle/traj.py) against closed forms, conservation laws,
the paper's energy-loss formulas (Sec. III), the published Philox vectors, and the independently
written input generator."""
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import traj as T
from paper_1910_10391_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")
D_P, U0 = I.SI110_DP, 20.0


def test_philox_known_answers():
    with open(os.path.join(GOLD, "philox4x32_10_kat.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for r in rows:
        v = [int(x, 16) for x in r]
        out = T.philox4x32_10(*[np.uint32(x) for x in v[:6]])
        assert [int(o) for o in out] == v[6:10]


def harmonic_entry(n, E, seed):
    rng = np.random.default_rng(seed)
    thL = math.sqrt(2 * U0 / E)
    # channeled: transverse energy below the well depth
    u = rng.uniform(-0.6, 0.6, n)
    th = rng.uniform(-0.6, 0.6, n) * thL
    return 0.5 * D_P + 0.5 * D_P * u, th


def test_harmonic_closed_form():
    """No scattering, channeled positron: x = x_c + A sin(W t + phi) with W^2 = 8 U0/(E d_p^2),
    and dz = integral of (v_z^2 - beta0^2)/(v_z + beta0) along the closed-form motion."""
    E, n, L, dt = 10e9, 6, 4001, 5e-9
    x0, th0 = harmonic_entry(n, E, 1)
    rec = T.trajectories(x0, th0, 0.0, E, L, dt, seed=0, ms=False)
    W = math.sqrt(8 * U0 / (E * D_P ** 2))
    t = np.arange(L) * dt
    g = E / I.ME_EV
    b0 = 1 - 1 / (2 * g * g)
    for p in range(n):
        a = x0[p] - 0.5 * D_P
        A = math.hypot(a, th0[p] / W)
        ph = math.atan2(a, th0[p] / W)
        x = 0.5 * D_P + A * np.sin(W * t + ph)
        v = A * W * np.cos(W * t + ph)
        np.testing.assert_allclose(rec[p, :, 1], x, rtol=0, atol=1e-9 * D_P)
        np.testing.assert_allclose(rec[p, :, 4], v, rtol=0, atol=1e-9 * A * W)
        np.testing.assert_allclose(rec[p, :, 7], -W * W * (x - 0.5 * D_P), rtol=0, atol=1e-8 * A * W * W)

        def dvz(tt):
            vp = A * W * math.cos(W * tt + ph)
            vz = math.sqrt(1 - 1 / g ** 2 - vp * vp)
            return (-vp * vp - 1 / (4 * g ** 4)) / (vz + b0)
        for k in (1000, 2500, L - 1):
            ref = quad(dvz, 0.0, t[k], limit=400, epsabs=0, epsrel=1e-13)[0]
            assert abs(rec[p, k, 3] - ref) <= 1e-9 * abs(ref)


def test_transverse_energy_is_conserved():
    E, L = 20e9, 3001
    x0, th0 = harmonic_entry(5, E, 2)
    rec = T.trajectories(x0, th0, 0.0, E, L, 5e-9, seed=0, ms=False)
    s = rec[:, :, 1] - 0.5 * D_P
    Et = E * rec[:, :, 4] ** 2 / 2 + U0 * (2 * s / D_P) ** 2
    assert np.abs(Et - Et[:, :1]).max() <= 1e-10 * U0


def test_radiation_reaction_is_larmor_power():
    E0, L, dt = 50e9, 3001, 5e-9
    x0, th0 = harmonic_entry(4, E0, 3)
    rec, Es = T.trajectories(x0, th0, 0.0, E0, L, dt, seed=0, ms=False, ll=True, energies=True)
    F = rec[:, :, 7] * Es
    P = (2 / 3) * T.ALPHA * T.HBARC_EV_M * (Es / I.ME_EV) ** 2 * (F / I.ME_EV) ** 2
    lost = np.concatenate([np.zeros((4, 1)), np.cumsum(0.5 * (P[:, 1:] + P[:, :-1]) * dt, 1)], 1)
    assert lost[:, -1].min() > 100.0
    # trapezoid error of the reference: at most dt^2/12 |P'| at each end (Euler-Maclaurin)
    dP = np.abs(np.diff(P, axis=1)).max() / dt
    np.testing.assert_allclose(E0 - Es, lost, rtol=1e-6, atol=dt * dt / 6 * dP)
    # the record's a_z carries d(gamma)/dt: d(v_z)/dt = (gamma_dot/gamma^3 - v.a)/v_z
    g = Es / I.ME_EV
    gd = -P / I.ME_EV
    vz = np.sqrt(1 - 1 / g ** 2 - rec[:, :, 4] ** 2)
    np.testing.assert_allclose(rec[:, :, 9], (gd / g ** 3 - rec[:, :, 4] * rec[:, :, 7]) / vz, rtol=1e-12, atol=0)


def test_scattering_loss_per_kick():
    x0 = np.linspace(0, D_P, 5, endpoint=False) + 0.01 * D_P
    rec, Es = T.trajectories(x0, np.zeros(5), 0.0, 20e9, 1001, 5e-9, seed=4, U0_eV=0.0, ms_loss=True,
                             energies=True)
    th2 = np.diff(rec[:, :, 4], axis=1) ** 2 + np.diff(rec[:, :, 5], axis=1) ** 2
    g = Es[:, :-1] / I.ME_EV
    expect = I.ME_EV * T.ALPHA / (2 * math.pi) * g ** 3 * th2
    assert np.count_nonzero(expect) > 1000
    np.testing.assert_allclose(Es[:, :-1] - Es[:, 1:], expect, rtol=1e-7, atol=4 * np.spacing(20e9))


def test_scattering_mean_square_angle():
    """Over entry positions uniform in the period the plane density averages to 1, so after a
    length l the mean squared angle is (eps_s/E)^2 l/X0 (Sec. III's variance, summed). At
    100 GeV the particles drift far less than the thermal amplitude rho meanwhile, so they
    sample the density where they entered."""
    n, L, dt, E = 4000, 201, 5e-9, 100e9
    x0 = (np.arange(n) + 0.5) / n * D_P
    rec = T.trajectories(x0, np.zeros(n), 0.0, E, L, dt, seed=11, U0_eV=0.0)
    expect = (10.6e6 / E) ** 2 * ((L - 1) * dt) / 0.0937
    # sum of the squared kicks: 400 squared normals per particle weighted by n(x); the plane
    # density's second moment (about 10.2) sets the spread: 3 sigma = 3 sqrt(10.2 / (200 n))
    kicks = np.diff(rec[:, :, 4], axis=1) ** 2 + np.diff(rec[:, :, 5], axis=1) ** 2
    assert abs(kicks.sum(1).mean() / expect - 1) < 3 * math.sqrt(10.2 / (200 * n))
    # the final angle squared has one degree of freedom per axis: 3 sigma = 3 sqrt(2 * 10.2 / n)
    th2 = rec[:, -1, 4] ** 2 + rec[:, -1, 5] ** 2
    assert abs(th2.mean() / expect - 1) < 3 * math.sqrt(2 * 10.2 / n)
    # kicks are symmetric: mean angle consistent with zero
    assert abs(rec[:, -1, 4].mean()) < 4 * math.sqrt(10.2 * expect / 2 / n)


@pytest.mark.parametrize("charge", [+1, -1])
def test_agrees_with_input_generator(charge):
    """The input generator (written separately, plain C) gives the same records to rounding."""
    n, L = 6, 2500
    tr, ex0, eth = I.channeling(n, 10e9, charge, L, 5e-9, seed=2, return_entry=True)
    rec = T.trajectories(ex0, eth, 0.0, 10e9, L, 5e-9, seed=2, charge=charge)
    a = tr.samples.reshape(n, L, 10)
    for f in range(10):
        scale = np.abs(a[..., f]).max()
        assert np.abs(rec[..., f] - a[..., f]).max() <= 1e-12 * scale, I.FIELDS[f]
    sc = I.channeling_sections(n, 50e9, charge, L, 5e-9, seed=2, section_samples=L, keep_energy=True)
    b = sc.traj.samples.reshape(n, L, 10)  # one section per particle
    rec2, Es = T.trajectories(b[:, 0, 1], b[:, 0, 4], 0.0, 50e9, L, 5e-9, seed=2, charge=charge, ll=True,
                              ms_loss=True, energies=True)
    np.testing.assert_allclose(Es, sc.energy_samples.reshape(n, L), rtol=1e-13)
    for f in range(1, 10):
        scale = np.abs(b[..., f]).max()
        assert np.abs(rec2[..., f] - b[..., f]).max() <= 1e-11 * scale, I.FIELDS[f]
