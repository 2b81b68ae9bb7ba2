"""FP64 CPU oracle for planar-channeling trajectories -- test infrastructure only.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import this module;
the CUDA integrator never calls it and the two share no code.

What it computes (arXiv:1910.10391, Sec. III, with the harmonic stand-in for the planar
continuum potential, whose Doyle-Turner tables the paper does not print):
  * potential energy U(s) = U0 (2 s / d_p)^2, s = distance to the nearest channel centre
    (positrons: centres mid-way between planes at (m + 1/2) d_p; electrons: on the planes);
    transverse force F = -dU/ds = -8 U0 s / d_p^2 (eV/m);
  * ultra-relativistic equation of motion with c = 1, lengths and times in metres:
      dx/dt = v_x, dy/dt = v_y, dv_x/dt = F / E, dv_y/dt = 0,
      d(dz)/dt = v_z - beta0, beta0 := 1 - 1/(2 gamma0^2) with gamma0 the entry value,
      v_z = sqrt(1 - 1/gamma^2 - v_perp^2);
  * radiation reaction (Landau-Lifshitz force, Sec. III; its leading term for a static
    transverse field is a drag along the velocity with the relativistic Larmor power):
      dE/dt = -(2/3) alpha hbar c gamma^2 F^2 / (m c^2)^2;
  * one classical Runge-Kutta (RK4) step of dt on (x, y, v_x, v_y, dz, E) between samples;
  * multiple Coulomb scattering on nuclei (Sec. III; the valence-electron term is added with a
    planar potential, below): after each step,
    independent Gaussian kicks of both transverse angles with variance
      (1/2) (eps_s / E)^2 (dt / X0) n(x)/N,  n(x)/N = d_p/(sqrt(pi) rho) sum over the two
      nearest planes of exp(-r^2/rho^2),
    added to v_perp; the next sample's acceleration carries the kick as delta_v / dt, and
    with scattering loss the kick costs dE = m alpha/(2 pi) gamma^3 theta^2 (Sec. III);
  * normals from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), counter
    (particle low word, step, 1, particle high word), key (seed low, seed high), by
    Box-Muller on two 53-bit uniforms ((top 27 bits of word a) * 2^26 + top 26 of word b
    + 1/2) / 2^53, z0 = r cos(2 pi u2), z1 = r sin(2 pi u2), r = sqrt(-2 ln u1).
Records (the radiation integral's input, Sec. II variables): t = k dt, x, y, dz, v_x, v_y,
dvz = v_z - beta0, a_x = F/E + kick, a_y = kick, a_z = (dgamma/dt / gamma^3 - v_perp.a_perp)/v_z.

With a Doyle-Turner planar potential (`PlanarPotential`, Sec. III, Eq. plane) the harmonic
well is replaced by the thermally averaged continuum potential of the planes at x = m d_p,
  U(x) = 2 sqrt(pi) e^2 a0 N d_p sum_planes sum_i a_i / sqrt(C_i) exp(-r^2 / C_i),
  C_i = b_i / (4 pi^2) + rho^2, r = distance to the plane,
for a unit positive charge (a particle of charge sign q feels q U, force -q dU/dx), summed over
the 2K planes m0-K+1 .. m0+K around the cell m0 = floor(x/d_p) that holds x. The fit
coefficients are the caller's (the paper prints no tables). With scattering on valence electrons
(Sec. III, Eq. elscat) each angle's kick variance gains
  (1/2) dt pi r0^2 / (gamma^2 beta^4) max(ln(2 m_e gamma^2 beta^2 / I) - beta^2, 0) n_el(x),
  n_el(x) = (N d_p / sqrt(pi)) sum_planes sum_i a_i^X / sqrt(C_i^X) exp(-r^2 / C_i^X)
            + c^X N n(x)/N,   C_i^X = b_i^X / (4 pi^2) + rho^2
(the prefactor N d_p / sqrt(pi) is the reading under which a plane holds N d_p (sum a^X + c^X)
electrons per unit area, as the X-ray factors' normalisation requires; the paper prints d_p/pi).

Pinned in tests/test_traj_oracle.py: Philox published vectors, the closed-form harmonic
solution and its dz, transverse-energy conservation, the Larmor integral of the energy loss,
the per-kick scattering loss, kick statistics, and agreement with the input generator. The
planar potential is pinned in tests/test_potential_oracle.py by its Fourier series (Poisson
summation), the thermal smearing as a Gaussian convolution, mirror symmetry, the electron count
per plane, transverse-energy conservation and the small-oscillation frequency. The electron-
scattering rate (Eq. elscat) is pinned there too: by the paper's statement that, with uniform
densities, the electron term is 1/Z of the nuclear one (to the factor 2 it resolves), and by
Rutherford kinematics (rate times (p v)^2 over the Bethe logarithm is the same at every energy).
"""
from __future__ import annotations

import math

import numpy as np

ALPHA = 7.2973525693e-3
HBARC_EV_M = 1.973269804e-7
E2_EV_M = ALPHA * HBARC_EV_M      # e^2 (Gaussian units) in eV m
A0_M = 5.29177210903e-11          # Bohr radius, m
R0_M = 2.8179403262e-15           # classical electron radius, m
ME_EV = 0.51099895e6              # electron rest energy, eV (target electrons)

_M0, _M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
_W0, _W1 = np.uint32(0x9E3779B9), np.uint32(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds on uint32 arrays (broadcast): each round multiplies words 0 and 2
    by the two round constants (64-bit products split into high and low halves), mixes with
    words 1 and 3 and the key, then bumps the key by the two Weyl constants."""
    c = [np.asarray(x, dtype=np.uint32) for x in (c0, c1, c2, c3)]
    k = [np.asarray(k0, dtype=np.uint32), np.asarray(k1, dtype=np.uint32)]
    for r in range(10):
        p0 = c[0].astype(np.uint64) * _M0
        p1 = c[2].astype(np.uint64) * _M1
        hi0, lo0 = (p0 >> np.uint64(32)).astype(np.uint32), (p0 & _MASK).astype(np.uint32)
        hi1, lo1 = (p1 >> np.uint64(32)).astype(np.uint32), (p1 & _MASK).astype(np.uint32)
        c = [hi1 ^ c[1] ^ k[0], lo1, hi0 ^ c[3] ^ k[1], lo0]
        if r < 9:  # key bump modulo 2^32
            k = [((k[0].astype(np.uint64) + np.uint64(_W0)) & _MASK).astype(np.uint32),
                 ((k[1].astype(np.uint64) + np.uint64(_W1)) & _MASK).astype(np.uint32)]
    return c


def _u53(a, b):
    m = ((a >> np.uint32(5)).astype(np.uint64) << np.uint64(26)) | (b >> np.uint32(6)).astype(np.uint64)
    return (m.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def kick_normals(seed: int, particles, step: int):
    """(z0, z1) standard normals of the scattering kick after `step` for each particle index."""
    p = np.asarray(particles, dtype=np.uint64)
    r = philox4x32_10(p & _MASK, np.full(p.shape, step & 0xFFFFFFFF, np.uint32), np.full(p.shape, 1, np.uint32),
                      p >> np.uint64(32), np.uint32(seed & 0xFFFFFFFF), np.uint32((seed >> 32) & 0xFFFFFFFF))
    u1, u2 = _u53(r[0], r[1]), _u53(r[2], r[3])
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * math.pi * u2
    return rad * np.cos(ang), rad * np.sin(ang)


def force(x, U0_eV, d_p, charge):
    """Transverse force F (eV/m) of the harmonic planar well."""
    centre = 0.5 * d_p if charge > 0 else 0.0
    u = (x - centre) / d_p
    s = (u - np.floor(u + 0.5)) * d_p
    return -8.0 * U0_eV * s / (d_p * d_p)


class PlanarPotential:
    """Doyle-Turner fit of one plane (Sec. III): electron-scattering terms a [m], b [m^2] of the
    potential; X-ray terms ax [electrons], bx [m^2] and cx of the electron density; atom density
    N [m^-3]; mean ionisation energy I_eV; K neighbouring planes on each side of the cell."""

    def __init__(self, a, b, N, ax=(), bx=(), cx=0.0, I_eV=0.0, K=3):
        self.a, self.b = np.asarray(a, np.float64), np.asarray(b, np.float64)
        self.ax, self.bx = np.asarray(ax, np.float64), np.asarray(bx, np.float64)
        self.N, self.cx, self.I_eV, self.K = float(N), float(cx), float(I_eV), int(K)


def _plane_distances(x, d_p, K):
    """r[..., j] = x - (m0 + j) d_p for j = -K+1 .. K, m0 = floor(x / d_p)."""
    x = np.asarray(x, dtype=np.float64)
    m0 = np.floor(x / d_p)
    j = np.arange(-K + 1, K + 1, dtype=np.float64)
    return x[..., None] - (m0[..., None] + j) * d_p


def planar_potential(x, pot, d_p, rho):
    """U(x) in eV for a unit positive charge: Eq. plane summed over the 2K nearest planes."""
    C = pot.b / (4.0 * math.pi ** 2) + rho * rho
    r2 = _plane_distances(x, d_p, pot.K)[..., None] ** 2
    P = 2.0 * math.sqrt(math.pi) * E2_EV_M * A0_M * pot.N * d_p
    return P * (pot.a / np.sqrt(C) * np.exp(-r2 / C)).sum((-1, -2))


def planar_force(x, pot, d_p, rho, charge):
    """Transverse force -charge dU/dx (eV/m) of the planar potential."""
    C = pot.b / (4.0 * math.pi ** 2) + rho * rho
    r = _plane_distances(x, d_p, pot.K)[..., None]
    P = 2.0 * math.sqrt(math.pi) * E2_EV_M * A0_M * pot.N * d_p
    # d/dr of exp(-r^2/C) is -(2 r / C) exp(-r^2/C)
    return charge * P * (pot.a / np.sqrt(C) * (2.0 * r / C) * np.exp(-r * r / C)).sum((-1, -2))


def electron_density(x, pot, d_p, rho):
    """n_el(x) in m^-3: the X-ray Gaussians of the 2K nearest planes plus c^X times the nuclear
    density (Sec. III)."""
    CX = pot.bx / (4.0 * math.pi ** 2) + rho * rho
    r2 = _plane_distances(x, d_p, pot.K)[..., None] ** 2
    valence = pot.N * d_p / math.sqrt(math.pi) * (pot.ax / np.sqrt(CX) * np.exp(-r2 / CX)).sum((-1, -2))
    return valence + pot.cx * pot.N * plane_density(x, d_p, rho)


def electron_scattering_rate(gamma, n_el, I_eV):
    """Mean squared scattering angle per unit length on electrons, Sec. III Eq. elscat (with the
    paper's factor 2 removed), clamped at 0 where the logarithm's bracket would be negative."""
    gamma = np.asarray(gamma, dtype=np.float64)
    b2 = 1.0 - 1.0 / (gamma * gamma)
    bracket = np.maximum(np.log(2.0 * ME_EV * gamma * gamma * b2 / I_eV) - b2, 0.0)
    return math.pi * R0_M ** 2 / (gamma * gamma * b2 * b2) * bracket * n_el


def plane_density(x, d_p, rho):
    """n(x)/N: Gaussian plane density (thermal amplitude rho) summed over the two nearest planes."""
    m = np.floor(x / d_p)
    r1, r2 = x - m * d_p, (m + 1.0) * d_p - x
    return d_p / (math.sqrt(math.pi) * rho) * (np.exp(-(r1 * r1) / (rho * rho)) + np.exp(-(r2 * r2) / (rho * rho)))


def trajectories(x0, thx0, thy0, E0_eV, n_samples: int, dt: float, seed: int, *, charge=+1,
                 U0_eV=20.0, d_p=1.92e-10, eps_s_eV=10.6e6, X0=0.0937, rho=0.075e-10, ms=True,
                 ll=False, ms_loss=False, mass_eV=0.51099895e6, particle_ids=None, energies=False,
                 pot=None, ms_el=False):
    """Records [n][n_samples][10] of n particles with entry (x0, thx0, thy0) and energy E0
    (scalar or per particle); particle_ids index the random streams (default 0..n-1).
    With energies=True also returns the energy at every sample [n][n_samples]. A PlanarPotential
    `pot` replaces the harmonic well (U0_eV unused); ms_el adds scattering on valence electrons
    to the kicks (needs pot and ms)."""
    if ms_el and (pot is None or not ms):
        raise ValueError("electron scattering needs a planar potential and ms")

    def field(x):
        return force(x, U0_eV, d_p, charge) if pot is None else planar_force(x, pot, d_p, rho, charge)

    x0 = np.asarray(x0, dtype=np.float64)
    n = x0.shape[0]
    pid = np.arange(n, dtype=np.uint64) if particle_ids is None else np.asarray(particle_ids, dtype=np.uint64)
    E0 = np.broadcast_to(np.asarray(E0_eV, dtype=np.float64), (n,)).copy()
    g0 = E0 / mass_eV
    beta0 = 1.0 - 1.0 / (2.0 * g0 * g0)
    s = np.stack([x0, np.zeros(n), np.asarray(thx0, np.float64), np.broadcast_to(np.asarray(thy0, np.float64), (n,)),
                  np.zeros(n), E0], 1)

    def dvz_of(g, vp2, vz):
        # v_z - beta0 without cancellation: (v_z^2 - beta0^2)/(v_z + beta0) with
        # v_z^2 - beta0^2 = (1/gamma0^2 - 1/gamma^2) - v_perp^2 - 1/(4 gamma0^4)
        d_inv = ((g - g0) * (g + g0)) / ((g * g) * (g0 * g0))
        return (d_inv - vp2 - 1.0 / (4.0 * g0 ** 4)) / (vz + beta0)

    def gamma_dot(F, E):
        g = E / mass_eV
        return -(2.0 / 3.0) * ALPHA * HBARC_EV_M * g * g * (F / mass_eV) ** 2 / mass_eV

    def deriv(st):
        g = st[:, 5] / mass_eV
        vp2 = st[:, 2] ** 2 + st[:, 3] ** 2
        vz = np.sqrt(1.0 - 1.0 / (g * g) - vp2)
        F = field(st[:, 0])
        d = np.empty_like(st)
        d[:, 0] = st[:, 2]
        d[:, 1] = st[:, 3]
        d[:, 2] = F / st[:, 5]
        d[:, 3] = 0.0
        d[:, 4] = dvz_of(g, vp2, vz)
        d[:, 5] = gamma_dot(F, st[:, 5]) * mass_eV if ll else 0.0
        return d

    out = np.empty((n, n_samples, 10))
    Es = np.empty((n, n_samples))
    kick = np.zeros((n, 2))
    for k in range(n_samples):
        g = s[:, 5] / mass_eV
        vp2 = s[:, 2] ** 2 + s[:, 3] ** 2
        vz = np.sqrt(1.0 - 1.0 / (g * g) - vp2)
        F = field(s[:, 0])
        ax = F / s[:, 5] + kick[:, 0]
        ay = kick[:, 1]
        gd = gamma_dot(F, s[:, 5]) if ll else np.zeros(n)
        rec = out[:, k]
        rec[:, 0] = k * dt
        rec[:, 1] = s[:, 0]
        rec[:, 2] = s[:, 1]
        rec[:, 3] = s[:, 4]
        rec[:, 4] = s[:, 2]
        rec[:, 5] = s[:, 3]
        rec[:, 6] = dvz_of(g, vp2, vz)
        rec[:, 7] = ax
        rec[:, 8] = ay
        rec[:, 9] = (gd / g ** 3 - (s[:, 2] * ax + s[:, 3] * ay)) / vz
        Es[:, k] = s[:, 5]
        kick[:] = 0.0
        if k == n_samples - 1:
            break
        k1 = deriv(s)
        k2 = deriv(s + 0.5 * dt * k1)
        k3 = deriv(s + 0.5 * dt * k2)
        k4 = deriv(s + dt * k3)
        s = s + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        if ms:
            E = s[:, 5]
            var = 0.5 * (eps_s_eV / E) ** 2 * (dt / X0) * plane_density(s[:, 0], d_p, rho)
            if ms_el:
                var = var + 0.5 * dt * electron_scattering_rate(
                    E / mass_eV, electron_density(s[:, 0], pot, d_p, rho), pot.I_eV)
            z0, z1 = kick_normals(seed, pid, k)
            dthx, dthy = np.sqrt(var) * z0, np.sqrt(var) * z1
            kick[:, 0], kick[:, 1] = dthx / dt, dthy / dt
            s[:, 2] += dthx
            s[:, 3] += dthy
            if ms_loss:
                gk = E / mass_eV
                s[:, 5] = E - mass_eV * ALPHA / (2.0 * math.pi) * gk ** 3 * (dthx * dthx + dthy * dthy)
    return (out, Es) if energies else out


# --------------------------------------------------------------------------------------------
# Axial (string) continuum potential, Sec. III Eq. string
# --------------------------------------------------------------------------------------------
class StringLattice:
    """Strings of atoms along the axis, seen in the transverse plane: a rectangular cell
    (cell_x, cell_y) [m] repeated over the plane, holding strings at (sx[k], sy[k]); d [m] is the
    mean distance between atoms along a string. The atom density is N = n_strings / (d cell_x cell_y)."""

    def __init__(self, cell_x, cell_y, sx, sy, d):
        self.cell_x, self.cell_y, self.d = float(cell_x), float(cell_y), float(d)
        self.sx, self.sy = np.asarray(sx, np.float64), np.asarray(sy, np.float64)

    @property
    def N(self):
        return self.sx.size / (self.d * self.cell_x * self.cell_y)


class AxialPotential:
    """Doyle-Turner fit of one atom (Sec. III): potential terms a [m], b [m^2]; X-ray terms
    ax [electrons], bx [m^2], cx; mean ionisation energy I_eV; the string lattice; K cells summed on
    each side of the particle's cell in both transverse directions."""

    def __init__(self, a, b, lattice, ax=(), bx=(), cx=0.0, I_eV=0.0, K=2):
        self.a, self.b = np.asarray(a, np.float64), np.asarray(b, np.float64)
        self.ax, self.bx = np.asarray(ax, np.float64), np.asarray(bx, np.float64)
        self.lat, self.cx, self.I_eV, self.K = lattice, float(cx), float(I_eV), int(K)


def string_offsets(x, y, lat, K):
    """(dx, dy) [..., n] from every string of the (2K+1)^2 cells around the particle's cell
    (cx, cy) = (floor(x / cell_x), floor(y / cell_y)) to the point (x, y)."""
    x, y = np.asarray(x, np.float64), np.asarray(y, np.float64)
    cx, cy = np.floor(x / lat.cell_x), np.floor(y / lat.cell_y)
    i = np.arange(-K, K + 1, dtype=np.float64)
    ox = ((cx[..., None] + i) * lat.cell_x)[..., :, None, None] + lat.sx[None, None, :]   # [.., i, 1, k]
    oy = ((cy[..., None] + i) * lat.cell_y)[..., None, :, None] + lat.sy[None, None, :]   # [.., 1, j, k]
    dx = x[..., None, None, None] - ox
    dy = y[..., None, None, None] - oy
    dx, dy = np.broadcast_arrays(dx, dy)
    return dx.reshape(dx.shape[:-3] + (-1,)), dy.reshape(dy.shape[:-3] + (-1,))


def axial_potential(x, y, pot, rho):
    """U(x, y) in eV for a unit positive charge: Eq. string summed over the strings of the
    (2K+1)^2 cells around the particle, U_s(r) = (2 e^2 a0 / d) sum_i a_i / C_i exp(-r^2 / C_i),
    C_i = b_i / (4 pi^2) + rho^2."""
    C = pot.b / (4.0 * math.pi ** 2) + rho * rho
    dx, dy = string_offsets(x, y, pot.lat, pot.K)
    r2 = (dx * dx + dy * dy)[..., None]
    return (2.0 * E2_EV_M * A0_M / pot.lat.d * (pot.a / C) * np.exp(-r2 / C)).sum((-1, -2))


def axial_force(x, y, pot, rho, charge):
    """(F_x, F_y) = -charge grad U in eV/m; d/dr exp(-r^2/C) = -(2 r / C) exp(-r^2/C)."""
    C = pot.b / (4.0 * math.pi ** 2) + rho * rho
    dx, dy = string_offsets(x, y, pot.lat, pot.K)
    e = (2.0 * E2_EV_M * A0_M / pot.lat.d * (pot.a / C) * (2.0 / C)
         * np.exp(-((dx * dx + dy * dy)[..., None]) / C)).sum(-1)
    return charge * (dx * e).sum(-1), charge * (dy * e).sum(-1)


def string_density(x, y, lat, rho, K):
    """n(x, y)/N: the nuclear densities of the strings (Sec. III), each
    n_s(r) = exp(-r^2 / rho^2) / (pi rho^2 d), summed over the (2K+1)^2 cells, over the mean N."""
    dx, dy = string_offsets(x, y, lat, K)
    return np.exp(-(dx * dx + dy * dy) / (rho * rho)).sum(-1) / (math.pi * rho * rho * lat.d * lat.N)


def axial_electron_density(x, y, pot, rho):
    """n_el(x, y) in m^-3 (Sec. III): (1/(pi d)) sum_i a_i^X / C_i^X exp(-r^2 / C_i^X) per string
    plus c^X times the nuclear density, C_i^X = b_i^X / (4 pi^2) + rho^2."""
    CX = pot.bx / (4.0 * math.pi ** 2) + rho * rho
    dx, dy = string_offsets(x, y, pot.lat, pot.K)
    r2 = (dx * dx + dy * dy)[..., None]
    val = ((pot.ax / CX) * np.exp(-r2 / CX)).sum((-1, -2)) / (math.pi * pot.lat.d)
    return val + pot.cx * pot.lat.N * string_density(x, y, pot.lat, rho, pot.K)


def axial_trajectories(x0, y0, thx0, thy0, E0_eV, n_samples: int, dt: float, seed: int, pot, *, charge=+1,
                       eps_s_eV=10.6e6, X0=0.0937, rho=0.075e-10, ms=True, ms_el=False, ll=False,
                       ms_loss=False, mass_eV=0.51099895e6, particle_ids=None, energies=False):
    """Records [n][n_samples][10] of n particles entering at (x0, y0) with angles (thx0, thy0) in
    the axial potential `pot` (AxialPotential): the equations, RK4 steps, kicks and records of
    `trajectories`, with the two-dimensional force -charge grad U(x, y) and the string densities."""
    x0 = np.asarray(x0, dtype=np.float64)
    n = x0.shape[0]
    pid = np.arange(n, dtype=np.uint64) if particle_ids is None else np.asarray(particle_ids, dtype=np.uint64)
    E0 = np.broadcast_to(np.asarray(E0_eV, dtype=np.float64), (n,)).copy()
    g0 = E0 / mass_eV
    beta0 = 1.0 - 1.0 / (2.0 * g0 * g0)
    bc = lambda v: np.broadcast_to(np.asarray(v, np.float64), (n,)).copy()
    s = np.stack([x0, bc(y0), bc(thx0), bc(thy0), np.zeros(n), E0], 1)

    def dvz_of(g, vp2, vz):
        d_inv = ((g - g0) * (g + g0)) / ((g * g) * (g0 * g0))
        return (d_inv - vp2 - 1.0 / (4.0 * g0 ** 4)) / (vz + beta0)

    def gamma_dot(F2, E):
        g = E / mass_eV
        return -(2.0 / 3.0) * ALPHA * HBARC_EV_M * g * g * F2 / mass_eV ** 3

    def deriv(st):
        g = st[:, 5] / mass_eV
        vp2 = st[:, 2] ** 2 + st[:, 3] ** 2
        vz = np.sqrt(1.0 - 1.0 / (g * g) - vp2)
        Fx, Fy = axial_force(st[:, 0], st[:, 1], pot, rho, charge)
        d = np.empty_like(st)
        d[:, 0] = st[:, 2]
        d[:, 1] = st[:, 3]
        d[:, 2] = Fx / st[:, 5]
        d[:, 3] = Fy / st[:, 5]
        d[:, 4] = dvz_of(g, vp2, vz)
        d[:, 5] = gamma_dot(Fx * Fx + Fy * Fy, st[:, 5]) * mass_eV if ll else 0.0
        return d

    out = np.empty((n, n_samples, 10))
    Es = np.empty((n, n_samples))
    kick = np.zeros((n, 2))
    for k in range(n_samples):
        g = s[:, 5] / mass_eV
        vp2 = s[:, 2] ** 2 + s[:, 3] ** 2
        vz = np.sqrt(1.0 - 1.0 / (g * g) - vp2)
        Fx, Fy = axial_force(s[:, 0], s[:, 1], pot, rho, charge)
        ax = Fx / s[:, 5] + kick[:, 0]
        ay = Fy / s[:, 5] + kick[:, 1]
        gd = gamma_dot(Fx * Fx + Fy * Fy, s[:, 5]) if ll else np.zeros(n)
        rec = out[:, k]
        rec[:, 0] = k * dt
        rec[:, 1] = s[:, 0]
        rec[:, 2] = s[:, 1]
        rec[:, 3] = s[:, 4]
        rec[:, 4] = s[:, 2]
        rec[:, 5] = s[:, 3]
        rec[:, 6] = dvz_of(g, vp2, vz)
        rec[:, 7] = ax
        rec[:, 8] = ay
        rec[:, 9] = (gd / g ** 3 - (s[:, 2] * ax + s[:, 3] * ay)) / vz
        Es[:, k] = s[:, 5]
        kick[:] = 0.0
        if k == n_samples - 1:
            break
        k1 = deriv(s)
        k2 = deriv(s + 0.5 * dt * k1)
        k3 = deriv(s + 0.5 * dt * k2)
        k4 = deriv(s + dt * k3)
        s = s + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        if ms:
            E = s[:, 5]
            var = 0.5 * (eps_s_eV / E) ** 2 * (dt / X0) * string_density(s[:, 0], s[:, 1], pot.lat, rho, pot.K)
            if ms_el:
                var = var + 0.5 * dt * electron_scattering_rate(
                    E / mass_eV, axial_electron_density(s[:, 0], s[:, 1], pot, rho), pot.I_eV)
            z0, z1 = kick_normals(seed, pid, k)
            dthx, dthy = np.sqrt(var) * z0, np.sqrt(var) * z1
            kick[:, 0], kick[:, 1] = dthx / dt, dthy / dt
            s[:, 2] += dthx
            s[:, 3] += dthy
            if ms_loss:
                gk = E / mass_eV
                s[:, 5] = E - mass_eV * ALPHA / (2.0 * math.pi) * gk ** 3 * (dthx * dthx + dthy * dthy)
    return (out, Es) if energies else out


# --------------------------------------------------------------------------------------------
# Adaptive steps between caller-set output times (Sec. IV: an RK45 solver with step-size control
# and a lower bound on the step, which returns the trajectory at the times the caller asks for)
# --------------------------------------------------------------------------------------------
# Dormand-Prince 5(4) pair (J. R. Dormand, P. J. Prince, J. Comput. Appl. Math. 6 (1980) 19): nodes,
# stage coefficients, the fifth-order weights (the solution) and the embedded fourth-order weights.
DP_C = (0.0, 1.0 / 5.0, 3.0 / 10.0, 4.0 / 5.0, 8.0 / 9.0, 1.0, 1.0)
DP_A = ((),
        (1.0 / 5.0,),
        (3.0 / 40.0, 9.0 / 40.0),
        (44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0),
        (19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0),
        (9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0),
        (35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0))
DP_B5 = (35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0, 0.0)
DP_B4 = (5179.0 / 57600.0, 0.0, 7571.0 / 16695.0, 393.0 / 640.0, -92097.0 / 339200.0, 187.0 / 2100.0, 1.0 / 40.0)


def dp5_step(f, y, h):
    """One Dormand-Prince step of the autonomous system y' = f(y): (fifth-order, fourth-order)."""
    k = []
    for i in range(7):
        yi = y.copy()
        for j, a in enumerate(DP_A[i]):
            yi = yi + h * a * k[j]
        k.append(f(yi))
    y5, y4 = y.copy(), y.copy()
    for i in range(7):
        y5 = y5 + h * DP_B5[i] * k[i]
        y4 = y4 + h * DP_B4[i] * k[i]
    return y5, y4


def step_error(y, y5, y4, scale_abs, rtol):
    """RMS over the state's components of (y5 - y4) / (atol_i + rtol max(|y_i|, |y5_i|))."""
    sc = scale_abs + rtol * np.maximum(np.abs(y), np.abs(y5))
    return float(np.sqrt(np.mean(((y5 - y4) / sc) ** 2)))


def adaptive_interval(f, y, H, level, max_level, scale_abs, rtol, grow_below=2.0 ** -6):
    """Integrate over one output interval H with sub-steps H / 2^m: a step whose error exceeds 1 is
    repeated at half the size (m + 1) unless m is the lower bound max_level, where it is kept; after
    an accepted step with error below grow_below the size doubles (m - 1) when the position is a
    multiple of the doubled step. The position is an integer count of H / 2^max_level, so the
    interval ends exactly at H. Returns (y, level, accepted sub-steps)."""
    unit = 2 ** max_level
    pos, m, n = 0, level, 0
    while pos < unit:
        h = H / (2 ** m)
        y5, y4 = dp5_step(f, y, h)
        err = step_error(y, y5, y4, scale_abs, rtol)
        if err > 1.0 and m < max_level:
            m += 1
            continue
        y = y5
        pos += 2 ** (max_level - m)
        n += 1
        if err < grow_below and m > 0 and pos % (2 ** (max_level - m + 1)) == 0:
            m -= 1
    return y, m, n


def trajectories_adaptive(x0, thx0, thy0, E0_eV, times, seed: int, *, rtol, atol_x, atol_v, max_level, y0=0.0,
                          charge=+1, U0_eV=20.0, d_p=1.92e-10, eps_s_eV=10.6e6, X0=0.0937, rho=0.075e-10, ms=True,
                          ll=False, ms_loss=False, mass_eV=0.51099895e6, particle_ids=None, energies=False, pot=None,
                          axial=None, ms_el=False, counts=False):
    """Records [n][len(times)][10] as `trajectories` (harmonic well, planar potential `pot` or axial
    potential `axial`), with the RK4 step replaced by adaptive Dormand-Prince steps over each output
    interval (adaptive_interval; the level carries over from one interval to the next, starting at
    0) and records at the caller's `times` (increasing, one array for all particles). The kick after
    interval k enters the next record's acceleration as delta_v / w, w = (t_{k+2} - t_k)/2, or the
    last interval's length for the last record (dt for uniform times). With counts=True also
    returns the accepted sub-steps per particle."""
    times = np.asarray(times, dtype=np.float64)
    L = times.shape[0]
    x0 = np.atleast_1d(np.asarray(x0, dtype=np.float64))
    n = x0.shape[0]
    bc = lambda v: np.broadcast_to(np.asarray(v, np.float64), (n,)).copy()
    pid = np.arange(n, dtype=np.uint64) if particle_ids is None else np.asarray(particle_ids, dtype=np.uint64)
    E0 = bc(E0_eV)

    def field(x, y):
        if axial is not None:
            return axial_force(x, y, axial, rho, charge)
        if pot is not None:
            return planar_force(x, pot, d_p, rho, charge), np.zeros_like(x)
        return force(x, U0_eV, d_p, charge), np.zeros_like(x)

    def nuclear(x, y):
        return string_density(x, y, axial.lat, rho, axial.K) if axial is not None else plane_density(x, d_p, rho)

    def electrons(x, y):
        return axial_electron_density(x, y, axial, rho) if axial is not None else electron_density(x, pot, d_p, rho)

    out = np.empty((n, L, 10))
    Es = np.empty((n, L))
    steps = np.zeros(n, dtype=np.int64)
    scale_abs = np.array([atol_x, atol_x, atol_v, atol_v, atol_x, 0.0])
    for p in range(n):
        g0 = E0[p] / mass_eV
        beta0 = 1.0 - 1.0 / (2.0 * g0 * g0)

        def dvz_of(g, vp2, vz):
            d_inv = ((g - g0) * (g + g0)) / ((g * g) * (g0 * g0))
            return (d_inv - vp2 - 1.0 / (4.0 * g0 ** 4)) / (vz + beta0)

        def f(st):
            g = st[5] / mass_eV
            vp2 = st[2] ** 2 + st[3] ** 2
            vz = math.sqrt(1.0 - 1.0 / (g * g) - vp2)
            Fx, Fy = field(np.array([st[0]]), np.array([st[1]]))
            Fx, Fy = float(Fx[0]), float(Fy[0])
            gd = -(2.0 / 3.0) * ALPHA * HBARC_EV_M * g * g * (Fx * Fx + Fy * Fy) / mass_eV ** 3 if ll else 0.0
            return np.array([st[2], st[3], Fx / st[5], Fy / st[5], dvz_of(g, vp2, vz), gd * mass_eV])

        s = np.array([x0[p], bc(y0)[p], bc(thx0)[p], bc(thy0)[p], 0.0, E0[p]])
        kick = np.zeros(2)
        level = 0
        for k in range(L):
            g = s[5] / mass_eV
            vp2 = s[2] ** 2 + s[3] ** 2
            vz = math.sqrt(1.0 - 1.0 / (g * g) - vp2)
            Fx, Fy = field(np.array([s[0]]), np.array([s[1]]))
            Fx, Fy = float(Fx[0]), float(Fy[0])
            ax, ay = Fx / s[5] + kick[0], Fy / s[5] + kick[1]
            gd = -(2.0 / 3.0) * ALPHA * HBARC_EV_M * g * g * (Fx * Fx + Fy * Fy) / mass_eV ** 3 if ll else 0.0
            out[p, k] = (times[k], s[0], s[1], s[4], s[2], s[3], dvz_of(g, vp2, vz), ax, ay,
                         (gd / g ** 3 - (s[2] * ax + s[3] * ay)) / vz)
            Es[p, k] = s[5]
            kick[:] = 0.0
            if k == L - 1:
                break
            s, level, nst = adaptive_interval(f, s, times[k + 1] - times[k], level, max_level, scale_abs, rtol)
            steps[p] += nst
            if ms:
                E = s[5]
                var = 0.5 * (eps_s_eV / E) ** 2 * ((times[k + 1] - times[k]) / X0) * float(
                    nuclear(np.array([s[0]]), np.array([s[1]]))[0])
                if ms_el:
                    var += 0.5 * (times[k + 1] - times[k]) * float(electron_scattering_rate(
                        E / mass_eV, electrons(np.array([s[0]]), np.array([s[1]])), (axial or pot).I_eV)[0])
                z0, z1 = kick_normals(seed, pid[p:p + 1], k)
                dthx, dthy = math.sqrt(var) * float(z0[0]), math.sqrt(var) * float(z1[0])
                w = 0.5 * (times[k + 2] - times[k]) if k + 2 < L else times[k + 1] - times[k]
                kick[0], kick[1] = dthx / w, dthy / w
                s[2] += dthx
                s[3] += dthy
                if ms_loss:
                    gk = E / mass_eV
                    s[5] = E - mass_eV * ALPHA / (2.0 * math.pi) * gk ** 3 * (dthx * dthx + dthy * dthy)
    res = (out, Es) if energies else out
    return (res, steps) if counts else res
