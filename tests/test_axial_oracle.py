"""Pins of the oracle's axial (string) continuum potential (Sec. III, Eq. string) and of the
string densities of nuclei and electrons (Sec. III), each against something other than the
real-space sums themselves:
  * two-dimensional Poisson summation: the sum of the strings' Gaussians over the lattice equals
    its Fourier series with coefficients (2 pi e^2 a0 / d) sum_i a_i exp(-C_i |G|^2 / 4) per string,
    G = 2 pi (m / cell_x, n / cell_y), and the force its derivative;
  * the cell mean of the potential is 2 pi e^2 a0 N sum_i a_i, the same as the planar potential's
    mean for the same atom density (periodic quadrature over the cell);
  * thermal smearing: the potential at amplitude rho is the static one (rho = 0) convolved with the
    two-dimensional thermal density exp(-u^2 / rho^2) / (pi rho^2) (Gauss-Hermite quadrature);
  * normalisation: the cell mean of n/N is 1, and a string holds sum a^X + c^X electrons per atom;
  * the lattice's symmetries (the mirror y -> -y and the inversion about the dumbbell centre of
    a diamond <110> cell) and its periods;
  * dynamics: the transverse energy E v_perp^2 / 2 + q U(x, y) is conserved to RK4 accuracy, whose
    error falls by about 2^4 when dt halves.
test_planted_axial_mistakes_are_caught plants single mistakes in the oracle and checks that a
pin fails for each. Physical constants are typed here independently of the oracle (CODATA 2018).
"""
import math

import numpy as np
import pytest

from oracle import traj as T
from paper_1910_10391_gb300 import inputs as I

E2 = 7.2973525693e-3 * 197.3269804e-9   # e^2 = alpha hbar c, eV m
BOHR = 0.529177210903e-10               # a0, m
A_SI = 5.431e-10                        # Si lattice constant, m
RHO = I.RHO_THERMAL


def lattice_110(a=A_SI):
    """Diamond <110>: cell a (along [001]) x a/sqrt 2 (along [1-10]), dumbbells of strings a/4 apart,
    atoms a/sqrt 2 apart along each string (the geometry is pinned in tests/test_crystal_geometry.py)."""
    h = a / (2 * math.sqrt(2))
    return T.StringLattice(a, 2 * h, [0.0, a / 4, a / 2, 3 * a / 4], [0.0, 0.0, h, h], a / math.sqrt(2))


def pot(K=2, rho_lat=None, **kw):
    args = dict(a=I.SYNTH_DT_A, b=I.SYNTH_DT_B, lattice=rho_lat or lattice_110(), ax=I.SYNTH_DT_AX,
                bx=I.SYNTH_DT_BX, cx=I.SYNTH_DT_CX, I_eV=I.SI_I_EV, K=K)
    args.update(kw)
    return T.AxialPotential(**args)


def fourier(x, y, p, rho, deriv=False, M=110):
    """The lattice sum by its two-dimensional Fourier series (cos terms; the sine terms cancel
    between +G and -G)."""
    lat = p.lat
    C = p.b / (4 * math.pi ** 2) + rho * rho
    area = lat.cell_x * lat.cell_y
    m = np.arange(-M, M + 1)
    Gx, Gy = np.meshgrid(2 * math.pi * m / lat.cell_x, 2 * math.pi * m / lat.cell_y, indexing="ij")
    G2 = Gx * Gx + Gy * Gy
    coef = (2 * math.pi * E2 * BOHR / lat.d) * (p.a[None, None, :] * np.exp(-C[None, None, :] * G2[..., None] / 4)).sum(-1)
    coef = coef / area
    x, y = np.asarray(x, np.float64), np.asarray(y, np.float64)
    out = np.zeros(x.shape + (3,)) if deriv else np.zeros(x.shape)
    for sx, sy in zip(lat.sx, lat.sy):
        ph = Gx[None] * (x[:, None, None] - sx) + Gy[None] * (y[:, None, None] - sy)
        if deriv:
            s = np.sin(ph)
            out[:, 0] += (coef[None] * np.cos(ph)).sum((1, 2))
            out[:, 1] += -(coef[None] * Gx[None] * s).sum((1, 2))
            out[:, 2] += -(coef[None] * Gy[None] * s).sum((1, 2))
        else:
            out += (coef[None] * np.cos(ph)).sum((1, 2))
    return out


def points(n=60, seed=3):
    rng = np.random.default_rng(seed)
    lat = lattice_110()
    return rng.uniform(-lat.cell_x, 2 * lat.cell_x, n), rng.uniform(-lat.cell_y, 2 * lat.cell_y, n)


def test_string_lattice_sum_equals_fourier_series():
    check_string_lattice_sum_equals_fourier_series()


def check_string_lattice_sum_equals_fourier_series():
    p = pot(K=5)
    x, y = points()
    x = np.concatenate([x, p.lat.sx[:2], [1e-14]])
    y = np.concatenate([y, p.lat.sy[:2], [-1e-14]])
    f = fourier(x, y, p, RHO, deriv=True)
    U = T.axial_potential(x, y, p, RHO)
    assert np.abs(U - f[:, 0]).max() <= 1e-11 * np.abs(f[:, 0]).max()
    for q in (+1, -1):
        Fx, Fy = T.axial_force(x, y, p, RHO, q)
        scale = np.abs(f[:, 1:]).max()
        assert np.abs(Fx + q * f[:, 1]).max() <= 1e-11 * scale
        assert np.abs(Fy + q * f[:, 2]).max() <= 1e-11 * scale


def test_cell_mean_equals_the_planar_mean():
    check_cell_mean_equals_the_planar_mean()


def check_cell_mean_equals_the_planar_mean():
    """Periodic trapezoid over one cell (spectrally exact for the smooth periodic sum)."""
    p = pot(K=4)
    lat = p.lat
    n = 96
    gx, gy = np.meshgrid((np.arange(n) + 0.5) / n * lat.cell_x, (np.arange(n) + 0.5) / n * lat.cell_y, indexing="ij")
    mean = T.axial_potential(gx.ravel(), gy.ravel(), p, RHO).mean()
    ref = 2 * math.pi * E2 * BOHR * lat.N * p.a.sum()
    assert abs(mean / ref - 1) < 1e-10
    # the planar potential of the same atom density has the same mean (Sec. III, Eq. plane)
    pp = T.PlanarPotential(I.SYNTH_DT_A, I.SYNTH_DT_B, lat.N, K=6)
    xs = (np.arange(400) + 0.5) / 400 * I.SI110_DP
    assert abs(T.planar_potential(xs, pp, I.SI110_DP, RHO).mean() / ref - 1) < 1e-10


def test_thermal_smearing_is_a_2d_gaussian_convolution():
    check_thermal_smearing_is_a_2d_gaussian_convolution()


def check_thermal_smearing_is_a_2d_gaussian_convolution():
    p = pot(K=3)
    z, w = np.polynomial.hermite.hermgauss(48)
    ux, uy = np.meshgrid(z * RHO, z * RHO, indexing="ij")
    ww = np.outer(w, w) / math.pi
    for x, y in [(0.3e-10, 0.1e-10), (1.0e-10, 0.6e-10), (0.05e-10, 0.0), (2.2e-10, 1.7e-10)]:
        smeared = T.axial_potential(np.array([x]), np.array([y]), p, RHO)[0]
        static = T.axial_potential(x - ux.ravel(), y - uy.ravel(), p, 0.0).reshape(ux.shape)
        assert abs((ww * static).sum() / smeared - 1) < 1e-8, (x, y)


def test_symmetries_and_periods():
    check_symmetries_and_periods()


def check_symmetries_and_periods():
    p = pot(K=3)
    lat = p.lat
    x, y = points(40, seed=5)
    U = T.axial_potential(x, y, p, RHO)
    scale = np.abs(U).max()
    assert np.abs(T.axial_potential(x, -y, p, RHO) - U).max() <= 1e-13 * scale
    c = lat.cell_x / 8  # centre of the dumbbell (0, 0)-(a/4, 0)
    assert np.abs(T.axial_potential(2 * c - x, -y, p, RHO) - U).max() <= 1e-13 * scale
    assert np.abs(T.axial_potential(x + lat.cell_x, y - 2 * lat.cell_y, p, RHO) - U).max() <= 1e-13 * scale
    Fx, Fy = T.axial_force(x, y, p, RHO, +1)
    Fx2, Fy2 = T.axial_force(2 * c - x, -y, p, RHO, +1)
    fs = np.hypot(Fx, Fy).max()
    assert np.abs(Fx + Fx2).max() <= 1e-12 * fs and np.abs(Fy + Fy2).max() <= 1e-12 * fs


def test_nucleus_and_electron_counts():
    check_nucleus_and_electron_counts()


def check_nucleus_and_electron_counts():
    p = pot(K=1)
    lat = p.lat
    n = 160
    gx, gy = np.meshgrid((np.arange(n) + 0.5) / n * lat.cell_x, (np.arange(n) + 0.5) / n * lat.cell_y, indexing="ij")
    nn = T.string_density(gx.ravel(), gy.ravel(), lat, RHO, 1).mean()
    ne = T.axial_electron_density(gx.ravel(), gy.ravel(), p, RHO).mean()
    assert abs(nn - 1) < 1e-10
    assert abs(ne / (lat.N * (sum(I.SYNTH_DT_AX) + I.SYNTH_DT_CX)) - 1) < 1e-10


@pytest.mark.parametrize("charge", [+1, -1])
def test_transverse_energy_is_conserved(charge):
    """E v_perp^2 / 2 + q U(x, y) along scattering-free RK4 trajectories (10 GeV, entry inside the
    cell, angles below the critical angle); the drift falls as dt^4."""
    p = pot(K=2)
    rng = np.random.default_rng(8)
    x0, y0 = rng.uniform(0, p.lat.cell_x, 6), rng.uniform(0, p.lat.cell_y, 6)
    th = rng.normal(0, 4e-5, (2, 6))
    E = 10e9

    def drift(dt, L):
        rec = T.axial_trajectories(x0, y0, th[0], th[1], E, L, dt, 0, p, charge=charge, ms=False)
        et = E * (rec[..., 4] ** 2 + rec[..., 5] ** 2) / 2 + charge * T.axial_potential(rec[..., 1], rec[..., 2], p, RHO)
        return np.abs(et - et[:, :1]).max()

    d1, d2 = drift(4e-9, 1001), drift(2e-9, 2001)
    assert d1 < 1e-6 * 30.0, d1
    assert 8.0 < d1 / d2 < 40.0, (d1, d2)


AXIAL_CHECKS = (check_string_lattice_sum_equals_fourier_series, check_cell_mean_equals_the_planar_mean,
                check_thermal_smearing_is_a_2d_gaussian_convolution, check_symmetries_and_periods,
                check_nucleus_and_electron_counts)


def _plants():
    U, F, nn, ne, so = (T.axial_potential, T.axial_force, T.string_density, T.axial_electron_density,
                        T.string_offsets)

    def with_b(f, factor):
        def g(x, y, p, rho, *c):
            q = T.AxialPotential(p.a, p.b * factor, p.lat, p.ax, p.bx, p.cx, p.I_eV, p.K)
            return f(x, y, q, rho, *c)
        return g

    def shifted(x, y, lat, K):
        dx, dy = so(x, y, lat, K)
        return dx + 0.5 * lat.cell_x, dy

    return {
        "prefactor e^2 a0 / d for 2 e^2 a0 / d": {"axial_potential": lambda *a: 0.5 * U(*a),
                                                  "axial_force": lambda *a: tuple(0.5 * v for v in F(*a))},
        "no rho^2 in C_i": {"axial_potential": lambda x, y, p, rho: U(x, y, p, 0.0),
                            "axial_force": lambda x, y, p, rho, c: F(x, y, p, 0.0, c)},
        "B_i = b / (4 pi)": {"axial_potential": with_b(U, math.pi), "axial_force": with_b(F, math.pi)},
        "a_i / sqrt(C_i) as in the planar form": {
            "axial_potential": lambda x, y, p, rho: U(x, y, T.AxialPotential(
                p.a * np.sqrt(p.b / (4 * math.pi ** 2) + rho * rho), p.b, p.lat, p.ax, p.bx, p.cx, p.I_eV, p.K), rho)},
        "force sign": {"axial_force": lambda *a: tuple(-v for v in F(*a))},
        "force without its factor 2": {"axial_force": lambda *a: tuple(0.5 * v for v in F(*a))},
        "strings shifted by half a cell": {"string_offsets": shifted},
        "nuclear density without pi": {"string_density": lambda *a: math.pi * nn(*a)},
        "electron density prefactor 1/d": {"axial_electron_density": lambda x, y, p, rho: ne(x, y, p, rho) + (
            math.pi - 1) * (ne(x, y, p, rho) - p.cx * p.lat.N * nn(x, y, p.lat, rho, p.K))},
    }


@pytest.mark.parametrize("plant", list(_plants()))
def test_planted_axial_mistakes_are_caught(plant, monkeypatch):
    for name, fn in _plants()[plant].items():
        monkeypatch.setattr(T, name, fn)
    failed = []
    for check in AXIAL_CHECKS:
        try:
            check()
        except AssertionError:
            failed.append(check.__name__)
    assert failed, f"no pin caught: {plant}"
