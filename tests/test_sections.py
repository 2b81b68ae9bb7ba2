"""Energy loss and sections in the trajectory generator (Sec. II sections; Sec. III Landau-Lifshitz
drag and the multiple-scattering loss dE = m alpha/(2 pi) gamma^3 theta^2)."""
import math

import numpy as np
import pytest

from paper_1910_10391_gb300 import inputs as I

ALPHA = 7.2973525693e-3


def per_sample(sc, p):
    """Records of particle p with the duplicated boundary samples dropped: one row per sample."""
    tr = sc.traj
    rows = []
    for j in range(sc.sec_offsets[p], sc.sec_offsets[p + 1]):
        r = tr.samples[tr.offsets[j]:tr.offsets[j + 1]]
        rows.append(r if j == sc.sec_offsets[p] else r[1:])
    return np.concatenate(rows)


def test_section_layout():
    sc = I.channeling_sections(3, 50e9, +1, [2001, 1500, 2], 5e-9, seed=2, section_samples=1000)
    assert list(np.diff(sc.traj.offsets)) == [1000, 1000, 3, 1000, 501, 2]
    assert list(sc.parent) == [0, 0, 0, 1, 1, 2]
    assert list(sc.sec_offsets) == [0, 3, 5, 6]
    np.testing.assert_allclose(sc.traj.weight, 1.0 / 3)
    np.testing.assert_array_equal(sc.traj.gamma, sc.traj.energy_eV / I.ME_EV)
    for p in range(3):
        e = sc.traj.energy_eV[sc.sec_offsets[p]:sc.sec_offsets[p + 1]]
        assert e[0] == 50e9 and np.all(np.diff(e) < 0)


def test_without_losses_matches_plain_generator():
    """ll and ms_loss off: the same trajectories as `channeling`, with t and dz restarting at 0
    in every section."""
    L, S = 3001, 700
    ref = I.channeling(4, 10e9, +1, L, 5e-9, seed=9)
    sc = I.channeling_sections(4, 10e9, +1, L, 5e-9, seed=9, section_samples=S, ll=False, ms_loss=False)
    assert np.all(sc.traj.energy_eV == 10e9)
    for p in range(4):
        a = ref.samples[ref.offsets[p]:ref.offsets[p + 1]]
        for j in range(sc.sec_offsets[p], sc.sec_offsets[p + 1]):
            k0 = (j - sc.sec_offsets[p]) * (S - 1)
            r = sc.traj.samples[sc.traj.offsets[j]:sc.traj.offsets[j + 1]]
            b = a[k0:k0 + len(r)]
            same = [1, 2, 4, 5, 6, 7, 8, 9]  # x, y, vx, vy, dvz, ax, ay, az
            np.testing.assert_array_equal(r[:, same], b[:, same])
            np.testing.assert_array_equal(r[:, 0], b[:, 0] - b[0, 0])
            np.testing.assert_allclose(r[:, 3], b[:, 3] - b[0, 3], rtol=0, atol=1e-10 * np.abs(a[:, 3]).max())


def test_radiation_reaction_is_larmor_power():
    """Drag only (no scattering): the energy lost up to every sample equals the integral of the
    relativistic Larmor power (2/3) alpha hbar c gamma^2 F^2/(m c^2)^2 along the trajectory."""
    E0, L = 50e9, 4001
    sc = I.channeling_sections(6, E0, +1, L, 5e-9, seed=3, section_samples=1000, ms=False, keep_energy=True)
    for p in range(6):
        r = per_sample(sc, p)
        E = sc.energy_samples[sc.sample_offsets[p]:sc.sample_offsets[p + 1]]
        F = r[:, 7] * E                                  # field force, eV/m
        P = (2.0 / 3.0) * ALPHA * I.HBARC_EV_M * (E / I.ME_EV) ** 2 * (F / I.ME_EV) ** 2
        t = np.arange(L) * 5e-9
        lost = np.concatenate([[0.0], np.cumsum(0.5 * (P[1:] + P[:-1]) * np.diff(t))])
        assert lost[-1] > 1e3  # tens of keV to MeV over 20 um at 50 GeV
        np.testing.assert_allclose(E0 - E, lost, rtol=1e-5, atol=1e-9 * E0 * 1e-6)


def test_scattering_energy_loss_per_kick():
    """No field (U0 = 0): velocity changes only by the kicks, and each kick of angle theta costs
    m alpha/(2 pi) gamma^3 theta^2 at the energy it happens at."""
    sc = I.channeling_sections(3, 20e9, -1, 2001, 5e-9, seed=4, section_samples=600, U0_eV=0.0,
                               keep_energy=True)
    for p in range(3):
        r = per_sample(sc, p)
        E = sc.energy_samples[sc.sample_offsets[p]:sc.sample_offsets[p + 1]]
        th2 = np.diff(r[:, 4]) ** 2 + np.diff(r[:, 5]) ** 2
        g = E[:-1] / I.ME_EV
        expect = I.ME_EV * ALPHA / (2 * math.pi) * g ** 3 * th2
        assert np.count_nonzero(expect) > 100  # kicks vanish far from the planes (n(r) -> 0)
        # E is stored in eV near 2e10: its differences carry a few ulp of rounding
        np.testing.assert_allclose(E[:-1] - E[1:], expect, rtol=1e-7, atol=4 * np.spacing(20e9))


def test_formation_length():
    # 2 gamma^2 (E - hw)/(E omega) with hbar c restored: 50 GeV e+ emitting 5 GeV
    lf = I.formation_length_m(50e9, 5e9)
    g = 50e9 / I.ME_EV
    assert lf == pytest.approx(2 * g * g * 0.9 * I.HBARC_EV_M / 5e9, rel=1e-14)
    assert 6e-7 < lf < 7e-7


def test_invalid_sections_rejected():
    with pytest.raises(ValueError):
        I.channeling_sections(2, 10e9, +1, [100, 1], 5e-9, seed=1, section_samples=10)
    with pytest.raises(ValueError):
        I.channeling_sections(2, 10e9, +1, 100, 5e-9, seed=1, section_samples=1)
