"""Seeded input generators: RNG known answers, determinism and physical sanity."""
import math
import os

import numpy as np

from paper_1910_10391_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    with open(os.path.join(GOLD, "philox4x32_10_kat.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = I.philox4x32_10(v[0:4], v[4:6])
        assert list(out) == v[6:10]


def test_channeling_deterministic_and_sane():
    a = I.channeling(8, 10e9, +1, 2000, 5e-9, seed=2)
    b = I.channeling(8, 10e9, +1, 2000, 5e-9, seed=2)
    c = I.channeling(8, 10e9, +1, 2000, 5e-9, seed=3)
    assert np.array_equal(a.samples, b.samples)
    assert not np.array_equal(a.samples, c.samples)
    s = a.samples
    g = 10e9 / I.ME_EV
    beta0 = 1 - 1 / (2 * g * g)
    vp2 = s[:, 4] ** 2 + s[:, 5] ** 2
    vz = beta0 + s[:, 6]
    # |beta| fixed by gamma: vz^2 + vp^2 = 1 - 1/gamma^2
    np.testing.assert_allclose(vz ** 2 + vp2, 1 - 1 / g ** 2, rtol=0, atol=1e-15)
    # channeled positrons stay within a few Lindhard angles
    thL = math.sqrt(2 * 20.0 / 10e9)
    assert np.abs(s[:, 4]).max() < 3 * thL
    # uniform time grid
    t = s[a.offsets[0]:a.offsets[1], 0]
    np.testing.assert_allclose(np.diff(t), 5e-9, rtol=1e-9)


def test_channeling_oscillation_period():
    """Without scattering a channeled positron oscillates with lambda_ch = 2 pi d_p sqrt(E/(8 U0))."""
    tr = I.channeling(1, 10e9, +1, 20000, 5e-9, seed=2, ms=False)
    x = tr.samples[:, 1]
    d = I.SI110_DP
    s = (x - 0.5 * d) - d * np.round((x - 0.5 * d) / d)
    zc = np.nonzero(np.diff(np.sign(s)) != 0)[0]
    period = 2 * np.mean(np.diff(tr.samples[zc, 0]))
    lam = 2 * math.pi * d * math.sqrt(10e9 / (8 * 20.0))
    assert abs(period / lam - 1) < 0.01


def test_lognormal_lengths():
    L = I.lognormal_lengths(4096, seed=4)
    assert L.min() >= 2000 and L.max() <= 200000
    assert abs(np.median(L) / 20000 - 1) < 0.05
    assert np.array_equal(L, I.lognormal_lengths(4096, seed=4))


def test_grids():
    tx, ty, dom = I.angle_grid(4, 2, 1e-3, 2e-3)
    assert tx.shape == (8,) and np.allclose(dom, (0.5e-3) * (2e-3))
    assert np.allclose(tx[:4], [-0.75e-3, -0.25e-3, 0.25e-3, 0.75e-3])
    hw = I.omega_log(512, 1e6, 5e9)
    assert hw[0] == 1e6 and abs(hw[-1] / 5e9 - 1) < 1e-12
