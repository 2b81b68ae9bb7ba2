"""Pins of the oracle's adaptive integrator (Sec. IV: RK45 with step-size control, a lower bound on
the step, and records at caller-controlled times), against what the mathematics fixes:
  * the Dormand-Prince tableau satisfies the order conditions of order 5 (solution weights) and 4
    (embedded weights), and each row of the stage matrix sums to its node;
  * on the harmonic well, whose motion has the closed form x = x_c + A sin(Omega t + phi),
    Omega^2 = 8 U0 / (E d_p^2), fixed steps converge at order 5 (error ratio ~32 per halving) and
    the embedded solution at order 4 (~16);
  * the embedded error estimate |y5 - y4| matches the true error of y4 as the step shrinks;
  * the adaptive integrator meets its tolerance against the closed form at every output time,
    also on jittered output times; halving and doubling happen; the lower bound caps the halving.
test_planted_adaptive_mistakes_are_caught swaps the weight vectors, perturbs a node and drops the
lower bound in the oracle, and checks that a pin fails for each."""
import math

import numpy as np
import pytest

from oracle import traj as T
from paper_1910_10391_gb300 import inputs as I

E, U0, DP = 10e9, 20.0, I.SI110_DP
OMEGA = math.sqrt(8 * U0 / (E * DP * DP))


def closed(t, xc, A, ph):
    return xc + A * np.sin(OMEGA * t + ph), A * OMEGA * np.cos(OMEGA * t + ph)


def f_harm(y):
    """(x, v)' in the harmonic well (positron), E fixed."""
    return np.array([y[1], T.force(np.array([y[0]]), U0, DP, +1)[0] / E])


def check_order_conditions():
    A = np.zeros((7, 7))
    for i, row in enumerate(T.DP_A):
        A[i, :len(row)] = row
    c, b5, b4 = np.array(T.DP_C), np.array(T.DP_B5), np.array(T.DP_B4)
    assert np.allclose(A.sum(1), c, rtol=0, atol=1e-15)
    for b, order in ((b5, 5), (b4, 4)):
        conds = [(b.sum(), 1.0), (b @ c, 1 / 2), (b @ c ** 2, 1 / 3), (b @ (A @ c), 1 / 6)]
        if order >= 4:
            conds += [(b @ c ** 3, 1 / 4), (b @ (c * (A @ c)), 1 / 8), (b @ (A @ c ** 2), 1 / 12),
                      (b @ (A @ (A @ c)), 1 / 24)]
        if order >= 5:
            conds += [(b @ c ** 4, 1 / 5), (b @ (c ** 2 * (A @ c)), 1 / 10), (b @ ((A @ c) ** 2), 1 / 20),
                      (b @ (c * (A @ c ** 2)), 1 / 15), (b @ (A @ c ** 3), 1 / 20),
                      (b @ (c * (A @ (A @ c))), 1 / 30), (b @ (A @ (c * (A @ c))), 1 / 40),
                      (b @ (A @ (A @ c ** 2)), 1 / 60), (b @ (A @ (A @ (A @ c))), 1 / 120)]
        for got, want in conds:
            assert abs(got - want) < 1e-14, (order, got, want)
    # the embedded weights are of order 4 only: one fifth-order condition fails
    assert abs(b4 @ c ** 4 - 1 / 5) > 1e-4


def test_tableau_order_conditions():
    check_order_conditions()


def check_convergence_orders():
    xc, A, ph = 0.5 * DP, 0.3e-10, 0.4
    x0, v0 = closed(0.0, xc, A, ph)
    T_end = 2 * math.pi / OMEGA
    errs5, errs4 = [], []
    for n in (80, 160, 320):
        h = T_end / n
        y = np.array([x0, v0])
        for _ in range(n):
            y5, y4 = T.dp5_step(f_harm, y, h)
            y = y5
        ex = np.array(closed(T_end, xc, A, ph))
        # the velocity after one period (the position error of a whole period partly cancels)
        errs5.append(abs(y[1] - ex[1]) / (A * OMEGA))
        # the embedded solution propagated on its own
        y = np.array([x0, v0])
        for _ in range(n):
            y = T.dp5_step(f_harm, y, h)[1]
        errs4.append(abs(y[0] - ex[0]) / A)
    r5 = [errs5[i] / errs5[i + 1] for i in range(2)]
    r4 = [errs4[i] / errs4[i + 1] for i in range(2)]
    assert all(26 < r < 40 for r in r5), r5
    assert all(13 < r < 20 for r in r4), r4


def test_convergence_orders():
    check_convergence_orders()


def check_error_estimate():
    """One step from the closed form: the embedded estimate |y5 - y4| over the true error of y4."""
    xc, A, ph = 0.5 * DP, 0.3e-10, 1.1
    y = np.array(closed(0.0, xc, A, ph))
    for n in (8, 16, 32):
        h = 2 * math.pi / OMEGA / n
        y5, y4 = T.dp5_step(f_harm, y, h)
        ex = np.array(closed(h, xc, A, ph))
        ratio = abs(y5[0] - y4[0]) / abs(y4[0] - ex[0])
        assert abs(ratio - 1) < 0.15 if n == 32 else 0.5 < ratio < 2, (n, ratio)


def test_error_estimate_matches_the_true_error():
    check_error_estimate()


def check_adaptive_meets_tolerance():
    """Positrons in the harmonic well, no scattering: records at jittered output times over three
    oscillation periods, against the closed form; a coarse grid of output times forces halving."""
    rng = np.random.default_rng(2)
    xc = 0.5 * DP
    A, ph = rng.uniform(0.1e-10, 0.8e-10, 3), rng.uniform(0, 2 * math.pi, 3)
    x0, v0 = closed(0.0, xc, A, ph)
    period = 2 * math.pi / OMEGA
    t = I.sample_times("jitter", 61, 3 * period, seed=4)
    rtol = 1e-9
    rec, steps = T.trajectories_adaptive(x0, v0, 0.0, E, t, 0, rtol=rtol, atol_x=1e-20, atol_v=1e-16, max_level=12,
                                         ms=False, counts=True)
    ex_x, ex_v = closed(t[None, :], xc, A[:, None], ph[:, None])
    assert np.abs(rec[..., 1] - ex_x).max() <= 100 * rtol * A.max()
    assert np.abs(rec[..., 4] - ex_v).max() <= 100 * rtol * (A.max() * OMEGA)
    assert np.all(steps > 4 * 60), steps   # the output interval (a twentieth of a period) was split
    np.testing.assert_array_equal(rec[..., 0], np.broadcast_to(t, rec[..., 0].shape))
    # the lower bound: at most 2^max_level sub-steps per interval, whatever the tolerance
    _, s1 = T.trajectories_adaptive(x0, v0, 0.0, E, t, 0, rtol=1e-15, atol_x=1e-30, atol_v=1e-30, max_level=2,
                                    ms=False, counts=True)
    assert np.all(s1 == 4 * 60), s1
    _, s0 = T.trajectories_adaptive(x0, v0, 0.0, E, t, 0, rtol=1e-15, atol_x=1e-30, atol_v=1e-30, max_level=0,
                                    ms=False, counts=True)
    assert np.all(s0 == 60), s0


def test_adaptive_meets_tolerance_and_respects_the_lower_bound():
    check_adaptive_meets_tolerance()


def test_uniform_times_match_the_fixed_step_integrator():
    """With uniform output times and a tolerance met by one step per interval, the records follow
    the RK4 integrator's (both far more accurate than their difference scale), scattering included:
    the kicks, their random streams and their entry into the accelerations are the same."""
    x0, th = np.array([0.5e-10, 0.2e-10]), np.array([1e-5, -2e-5])
    t = np.arange(2001) * 5e-9
    a = T.trajectories_adaptive(x0, th, 0.0, E, t, 3, rtol=1e-9, atol_x=1e-18, atol_v=1e-14, max_level=8)
    b = T.trajectories(x0, th, 0.0, E, 2001, 5e-9, 3)
    scale = np.maximum(np.abs(b).max((0, 1)), 1e-300)
    assert (np.abs(a - b).max((0, 1)) / scale).max() < 1e-9


ADAPTIVE_CHECKS = (check_order_conditions, check_convergence_orders, check_error_estimate,
                   check_adaptive_meets_tolerance)


def _plants():
    step, interval = T.dp5_step, T.adaptive_interval

    def no_lower_bound(f, y, H, level, max_level, scale_abs, rtol, grow_below=2.0 ** -6):
        return interval(f, y, H, level, max_level + 3, scale_abs, rtol, grow_below)

    return {
        "weights swapped": {"DP_B5": T.DP_B4, "DP_B4": T.DP_B5},
        "node c3 perturbed": {"DP_C": T.DP_C[:2] + (0.31,) + T.DP_C[3:]},
        "a43 typo": {"DP_A": T.DP_A[:3] + ((44.0 / 45.0, -56.0 / 15.0, 32.0 / 8.0),) + T.DP_A[4:]},
        "lower bound ignored": {"adaptive_interval": no_lower_bound},
    }


@pytest.mark.parametrize("plant", list(_plants()))
def test_planted_adaptive_mistakes_are_caught(plant, monkeypatch):
    for name, v in _plants()[plant].items():
        monkeypatch.setattr(T, name, v)
    failed = []
    for check in ADAPTIVE_CHECKS:
        try:
            check()
        except AssertionError:
            failed.append(check.__name__)
            break  # one pin is enough (the others may run long with a broken tableau)
    assert failed, f"no pin caught: {plant}"
