"""Seeded synthetic inputs for the radiation integral: trajectories and grids.

This module creates inputs only. It holds none of the radiation arithmetic
(no phase, no integrand, no spectrum), so the FP64 oracle and the CUDA path can
both consume its output without sharing any of the method's code.

Trajectory record layout (one per time sample, float64, 10 fields, 80 bytes):
    t, x, y, dz, vx, vy, dvz, ax, ay, az
in the small-angle variables of Sec. II (c = 1, lengths and times in metres):
dz = z - beta0 t, dvz = v_z - beta0 with beta0 := 1 - 1/(2 gamma^2), and
(ax, ay, az) = d(beta)/dt. Particles are concatenated; particle p owns records
offsets[p] .. offsets[p+1]-1.

Physical constants (CODATA 2018) used to express workloads in eV and metres.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

HBARC_EV_M = 1.973269804e-7        # hbar*c in eV*m
ME_EV = 0.51099895000e6            # electron rest energy, eV
NREC = 10
FIELDS = ("t", "x", "y", "dz", "vx", "vy", "dvz", "ax", "ay", "az")

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_trajgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C generator in place (gcc, OpenMP, no FMA contraction)."""
    src = os.path.join(_HERE, "trajgen.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", "-fno-fast-math", src, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d, i64, u64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int
            P = ctypes.c_void_p
            lib.tg_channeling.argtypes = [d, d, i32, d, d, d, d, d, d, i32, d, u64, i64, P, P, P, P]
            lib.tg_channeling.restype = i32
            lib.tg_channeling_given.argtypes = [P, d, i32, d, d, d, d, d, i32, d, u64, i64, P, P, P, P]
            lib.tg_channeling_given.restype = i32
            lib.tg_channeling_loss.argtypes = [d, d, i32, d, d, d, d, d, d, i32, i32, i32, d, u64, i64, P,
                                               i64, P, P, P, P, P, P, P, P]
            lib.tg_channeling_loss.restype = i32
            lib.tg_section_count.argtypes = [i64, i64]
            lib.tg_section_count.restype = i64
            lib.tg_lognormal_lengths.argtypes = [u64, i64, d, d, i64, i64, P]
            lib.tg_lognormal_lengths.restype = i32
            lib.tg_philox4x32_10.argtypes = [P, P, P]
            lib.tg_philox4x32_10.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    """Raw Philox4x32-10 block (exposed so tests can check the published vectors)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().tg_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


# --------------------------------------------------------------------------- #
# Containers
# --------------------------------------------------------------------------- #
@dataclasses.dataclass
class Trajectories:
    """Concatenated trajectories plus per-particle scalars (all float64/int64)."""
    samples: np.ndarray       # [n_total, 10]
    offsets: np.ndarray       # [n_particles + 1] int64
    gamma: np.ndarray         # [n_particles]
    energy_eV: np.ndarray     # [n_particles]
    weight: np.ndarray        # [n_particles]

    @property
    def n_particles(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def n_total(self) -> int:
        return int(self.samples.shape[0])

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)

    def subset(self, idx) -> "Trajectories":
        idx = np.asarray(idx, dtype=np.int64)
        parts = [self.samples[self.offsets[p]:self.offsets[p + 1]] for p in idx]
        lens = np.array([len(x) for x in parts], dtype=np.int64)
        off = np.zeros(len(idx) + 1, dtype=np.int64)
        off[1:] = np.cumsum(lens)
        smp = np.ascontiguousarray(np.concatenate(parts, axis=0)) if parts else np.zeros((0, NREC))
        return Trajectories(smp, off, self.gamma[idx].copy(), self.energy_eV[idx].copy(),
                            self.weight[idx].copy())


@dataclasses.dataclass
class Grid:
    """Photon-energy grid and direction grid (cell-centred, dOmega = dtheta_x dtheta_y)."""
    hbar_omega_eV: np.ndarray  # [n_omega]
    theta_x: np.ndarray        # [n_angles]
    theta_y: np.ndarray        # [n_angles]
    d_omega: np.ndarray        # [n_angles]
    nx: int = 0
    ny: int = 0

    @property
    def n_omega(self) -> int:
        return int(self.hbar_omega_eV.shape[0])

    @property
    def n_angles(self) -> int:
        return int(self.theta_x.shape[0])


def single(samples: np.ndarray, gamma: float, mass_eV: float = ME_EV, weight: float = 1.0) -> Trajectories:
    samples = np.ascontiguousarray(samples, dtype=np.float64)
    return Trajectories(samples, np.array([0, samples.shape[0]], dtype=np.int64),
                        np.array([gamma]), np.array([gamma * mass_eV]), np.array([weight]))


def concat(trajs) -> Trajectories:
    trajs = list(trajs)
    lens = np.concatenate([t.lengths() for t in trajs]) if trajs else np.zeros(0, np.int64)
    off = np.zeros(len(lens) + 1, dtype=np.int64)
    off[1:] = np.cumsum(lens)
    return Trajectories(np.ascontiguousarray(np.concatenate([t.samples for t in trajs], axis=0)),
                        off, np.concatenate([t.gamma for t in trajs]),
                        np.concatenate([t.energy_eV for t in trajs]),
                        np.concatenate([t.weight for t in trajs]))


# --------------------------------------------------------------------------- #
# Grids
# --------------------------------------------------------------------------- #
def angle_grid(nx: int, ny: int, half_x: float, half_y: float | None = None,
               center_x: float = 0.0, center_y: float = 0.0) -> tuple:
    """Cell-centred rectangular grid; index j = iy*nx + ix (x fastest)."""
    half_y = half_x if half_y is None else half_y
    dx, dy = 2.0 * half_x / nx, 2.0 * half_y / ny
    tx = center_x - half_x + (np.arange(nx) + 0.5) * dx
    ty = center_y - half_y + (np.arange(ny) + 0.5) * dy
    TX, TY = np.meshgrid(tx, ty, indexing="xy")
    return (np.ascontiguousarray(TX.ravel()), np.ascontiguousarray(TY.ravel()),
            np.full(nx * ny, dx * dy))


def omega_linear(n: int, hw_max: float) -> np.ndarray:
    """hbar*omega_i = (i+1)/n * hw_max, i = 0..n-1 (excludes 0)."""
    return (np.arange(1, n + 1, dtype=np.float64) / n) * hw_max


def omega_log(n: int, lo: float, hi: float) -> np.ndarray:
    return lo * (hi / lo) ** (np.arange(n, dtype=np.float64) / max(n - 1, 1))


def make_grid(hw: np.ndarray, nx: int, ny: int, half_x: float, half_y: float | None = None,
              **kw) -> Grid:
    tx, ty, dom = angle_grid(nx, ny, half_x, half_y, **kw)
    return Grid(np.ascontiguousarray(hw, dtype=np.float64), tx, ty, dom, nx, ny)


def radial_bins(theta_x: np.ndarray, theta_y: np.ndarray, n_bins: int, theta_max: float) -> np.ndarray:
    """bin_of_angle[j] in [0, n_bins) by polar angle, or -1 beyond theta_max."""
    th = np.hypot(theta_x, theta_y)
    b = np.floor(th / theta_max * n_bins).astype(np.int64)
    b[(b >= n_bins) | (th >= theta_max)] = -1
    return b.astype(np.int32)


# --------------------------------------------------------------------------- #
# Analytic trajectories
# --------------------------------------------------------------------------- #
def sample_times(kind: str, n: int, length: float, seed: int = 0, tile: int = 64) -> np.ndarray:
    """n increasing sample times from 0 to `length`:
      uniform     equal steps;
      jitter      steps of relative size 1 + 0.8 (u - 1/2), u uniform (seeded);
      geometric   steps growing geometrically, the last 8 times the first;
      tile_jumps  steps of 1 and 3 alternating every `tile` steps, so that the spacing changes at
                  every multiple of `tile` (the first sample of each time tile);
      smooth      t = length (s + 0.6 sin(2 pi s) / (2 pi)) at uniform s (a smooth monotone map)."""
    if n < 2:
        raise ValueError("need at least 2 samples")
    m = n - 1
    if kind == "uniform":
        return np.linspace(0.0, length, n)
    if kind == "smooth":
        s = np.linspace(0.0, 1.0, n)
        return length * (s + 0.6 * np.sin(2.0 * math.pi * s) / (2.0 * math.pi))
    if kind == "jitter":
        inc = 1.0 + 0.8 * (np.random.default_rng(seed).random(m) - 0.5)
    elif kind == "geometric":
        inc = 8.0 ** (np.arange(m) / max(m - 1, 1))
    elif kind == "tile_jumps":
        inc = np.where((np.arange(m) // tile) % 2 == 0, 1.0, 3.0)
    else:
        raise ValueError(kind)
    t = np.concatenate([[0.0], np.cumsum(inc)])
    return t * (length / t[-1])


def weak_undulator(gamma=1000.0, a=0.5e-10, lam=10e-6, n_periods=5, n_samples=4096,
                   mass_eV=ME_EV, times=None) -> Trajectories:
    """Planar harmonic motion x = a sin(k t), uniform samples over n_periods (or the given
    increasing `times`, which then set n_samples).

    Longitudinal variables to leading order: dvz = -vx^2/2, az = -vx*ax,
    dz = -(a k)^2/4 (t + sin(2kt)/(2k)).
    """
    k = 2.0 * math.pi / lam
    t = np.linspace(0.0, n_periods * lam, n_samples) if times is None else np.asarray(times, np.float64)
    n_samples = t.shape[0]
    s = np.zeros((n_samples, NREC))
    s[:, 0] = t
    s[:, 1] = a * np.sin(k * t)
    s[:, 4] = a * k * np.cos(k * t)
    s[:, 7] = -a * k * k * np.sin(k * t)
    s[:, 6] = -0.5 * s[:, 4] ** 2
    s[:, 9] = -s[:, 4] * s[:, 7]
    s[:, 3] = -0.25 * (a * k) ** 2 * (t + np.sin(2.0 * k * t) / (2.0 * k))
    return single(s, gamma, mass_eV)


def undulator_first_harmonic_eV(gamma, a, lam, theta=0.0):
    k = 2.0 * math.pi / lam
    K = gamma * a * k
    return 2.0 * gamma ** 2 * HBARC_EV_M * k / (1.0 + 0.5 * K * K + (gamma * theta) ** 2)


def circular_arc(gamma, rho, half_angle, n_samples, mass_eV=ME_EV) -> Trajectories:
    """Exact circular motion in the x-z plane, velocity angle alpha(t) = beta t / rho,
    t in [-T, T] with beta T / rho = half_angle; the tangent at t = 0 is the z axis."""
    beta = math.sqrt(1.0 - 1.0 / gamma ** 2)
    beta0 = 1.0 - 1.0 / (2.0 * gamma ** 2)
    # beta - beta0 = (beta^2 - beta0^2)/(beta + beta0) = -1/(4 gamma^4)/(beta + beta0)
    bmb0 = -1.0 / (4.0 * gamma ** 4) / (beta + beta0)
    T = half_angle * rho / beta
    t = np.linspace(-T, T, n_samples)
    al = beta * t / rho
    s = np.zeros((n_samples, NREC))
    s[:, 0] = t
    s[:, 1] = 2.0 * rho * np.sin(0.5 * al) ** 2
    s[:, 4] = beta * np.sin(al)
    # dvz = beta cos(al) - beta0, written without cancellation
    s[:, 6] = bmb0 - 2.0 * beta * np.sin(0.5 * al) ** 2
    # dz = rho sin(al) - beta0 t = beta t (sin(al)/al - 1) + (beta - beta0) t
    with np.errstate(invalid="ignore", divide="ignore"):
        sinc_m1 = np.where(np.abs(al) > 1e-4, np.sin(al) / al - 1.0,
                           -al ** 2 / 6.0 + al ** 4 / 120.0)
    s[:, 3] = beta * t * sinc_m1 + bmb0 * t
    s[:, 7] = beta ** 2 / rho * np.cos(al)
    s[:, 9] = -beta ** 2 / rho * np.sin(al)
    return single(s, gamma, mass_eV)


def straight_line(gamma=1000.0, theta_x=1e-4, theta_y=-2e-4, length=1e-5, n_samples=1024,
                  mass_eV=ME_EV) -> Trajectories:
    """Uniform motion (zero acceleration) in a tilted direction."""
    beta0 = 1.0 - 1.0 / (2.0 * gamma ** 2)
    vp2 = theta_x ** 2 + theta_y ** 2
    vz = math.sqrt(1.0 - 1.0 / gamma ** 2 - vp2)
    dvz = -(vp2 + 1.0 / (4.0 * gamma ** 4)) / (vz + beta0)
    t = np.linspace(0.0, length, n_samples)
    s = np.zeros((n_samples, NREC))
    s[:, 0] = t
    s[:, 1] = theta_x * t
    s[:, 2] = theta_y * t
    s[:, 3] = dvz * t
    s[:, 4] = theta_x
    s[:, 5] = theta_y
    s[:, 6] = dvz
    return single(s, gamma, mass_eV)


# --------------------------------------------------------------------------- #
# Channeling ensembles (C generator)
# --------------------------------------------------------------------------- #
SI110_DP = 1.92e-10        # Si (110) interplanar distance, m
SI_X0 = 0.0937             # Si radiation length, m
EPS_S_EV = 10.6e6          # MS energy constant of Sec. III
RHO_THERMAL = 0.075e-10    # thermal vibration amplitude used for n(r), m (not given in the paper)
SI_N = 4.994e28            # Si atom density, m^-3 (8 atoms per cubic cell of 5.431 A)
SI_I_EV = 173.0            # mean ionisation energy of Si, eV

# A synthetic four-Gaussian planar fit with the form and scale of a Doyle-Turner fit (Sec. III):
# the paper prints no coefficient tables, so these values are made up for tests and benchmarks
# and are not any crystal's. Potential terms a [m], b [m^2]; X-ray terms ax [electrons],
# bx [m^2], cx, with sum(ax) + cx = 14 electrons per atom.
SYNTH_DT_A = (2.0e-10, 2.0e-10, 1.0e-10, 0.3e-10)
SYNTH_DT_B = (40e-20, 10e-20, 2e-20, 0.4e-20)
SYNTH_DT_AX = (5.0, 3.0, 2.5, 1.5)
SYNTH_DT_BX = (30e-20, 8e-20, 1.5e-20, 0.3e-20)
SYNTH_DT_CX = 2.0


def channeling(n_particles: int, E_eV: float, charge: int, lengths, dt: float, seed: int,
               U0_eV: float = 20.0, d_p: float = SI110_DP, sigma_theta_frac: float = 0.3,
               ms: bool = True, mass_eV: float = ME_EV, return_entry: bool = False):
    """Planar-channeling ensemble in a harmonic well (positrons charge=+1, electrons -1)."""
    lens = np.broadcast_to(np.asarray(lengths, dtype=np.int64), (n_particles,)).copy()
    off = np.zeros(n_particles + 1, dtype=np.int64)
    off[1:] = np.cumsum(lens)
    out = np.empty((int(off[-1]), NREC), dtype=np.float64)
    theta_L = math.sqrt(2.0 * U0_eV / E_eV)
    ex0 = np.empty(n_particles)
    eth = np.empty(n_particles)
    rc = _load().tg_channeling(E_eV, mass_eV, int(charge), U0_eV, d_p, sigma_theta_frac * theta_L,
                               EPS_S_EV, SI_X0, RHO_THERMAL, int(bool(ms)), dt, int(seed),
                               n_particles, _ptr(off), _ptr(out), _ptr(ex0), _ptr(eth))
    if rc != 0:
        raise RuntimeError("tg_channeling failed")
    g = E_eV / mass_eV
    tr = Trajectories(out, off, np.full(n_particles, g), np.full(n_particles, E_eV),
                      np.full(n_particles, 1.0 / max(n_particles, 1)))
    if return_entry:
        return tr, ex0, eth
    return tr


def channeling_given(x0, thx0, gammas, n_samples: int, dt: float, charge: int = 1,
                     U0_eV: float = 20.0, d_p: float = SI110_DP, ms: bool = False, seed: int = 0,
                     mass_eV: float = ME_EV) -> Trajectories:
    """Trajectories for given entry conditions (absolute x0, angle) and Lorentz factors."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    thx0 = np.ascontiguousarray(thx0, dtype=np.float64)
    E = np.ascontiguousarray(np.asarray(gammas, dtype=np.float64) * mass_eV)
    n = x0.shape[0]
    off = np.arange(n + 1, dtype=np.int64) * int(n_samples)
    out = np.empty((n * int(n_samples), NREC), dtype=np.float64)
    rc = _load().tg_channeling_given(_ptr(E), mass_eV, int(charge), U0_eV, d_p, EPS_S_EV, SI_X0,
                                     RHO_THERMAL, int(bool(ms)), dt, int(seed), n, _ptr(off),
                                     _ptr(x0), _ptr(thx0), _ptr(out))
    if rc != 0:
        raise RuntimeError("tg_channeling_given failed")
    return Trajectories(out, off, E / mass_eV, E, np.full(n, 1.0 / max(n, 1)))


@dataclasses.dataclass
class Sectioned:
    """Sections of an ensemble with energy loss: each section is one entry of `traj` (its own
    gamma and E, weight of its particle); parent[j] is the particle of section j."""
    traj: Trajectories
    parent: np.ndarray          # [n_sections] int64
    sec_offsets: np.ndarray     # [n_particles + 1] first section of each particle
    energy_samples: np.ndarray | None = None   # [sum L] energy at every sample (optional)
    sample_offsets: np.ndarray | None = None   # [n_particles + 1]


def formation_length_m(E_eV: float, hw_eV: float, mass_eV: float = ME_EV) -> float:
    """Coherence (formation) length of emitting hw from energy E, 2 gamma^2 (E - hw) / (E omega)
    in metres (hbar c restored): a section must be longer than this at the photon energies of
    interest (Sec. II)."""
    g = E_eV / mass_eV
    return 2.0 * g * g * (E_eV - hw_eV) / E_eV * HBARC_EV_M / hw_eV


def channeling_sections(n_particles: int, E_eV: float, charge: int, lengths, dt: float, seed: int,
                        section_samples: int, ll: bool = True, ms_loss: bool = True, ms: bool = True,
                        U0_eV: float = 20.0, d_p: float = SI110_DP, sigma_theta_frac: float = 0.3,
                        mass_eV: float = ME_EV, keep_energy: bool = False) -> Sectioned:
    """Planar-channeling ensemble (entries as `channeling` with the same seed) integrated with
    radiation-reaction drag (Landau-Lifshitz, leading term) and the multiple-scattering energy
    loss of Sec. III, cut into sections of `section_samples` samples that share boundary
    samples; each section enters the radiation integral with the energy it starts with."""
    lens = np.broadcast_to(np.asarray(lengths, dtype=np.int64), (n_particles,)).copy()
    S = int(section_samples)
    if S < 2 or np.any(lens < 2):
        raise ValueError("sections need >= 2 samples and particles >= 2 samples")
    nsec = (lens - 2) // (S - 1) + 1
    rec_off = np.zeros(n_particles + 1, dtype=np.int64)
    rec_off[1:] = np.cumsum(lens + nsec - 1)
    sec_off = np.zeros(n_particles + 1, dtype=np.int64)
    sec_off[1:] = np.cumsum(nsec)
    samp_off = np.zeros(n_particles + 1, dtype=np.int64)
    samp_off[1:] = np.cumsum(lens)
    out = np.empty((int(rec_off[-1]), NREC), dtype=np.float64)
    secE = np.empty(int(sec_off[-1]), dtype=np.float64)
    eS = np.empty(int(samp_off[-1]), dtype=np.float64) if keep_energy else None
    theta_L = math.sqrt(2.0 * U0_eV / E_eV)
    rc = _load().tg_channeling_loss(E_eV, mass_eV, int(charge), U0_eV, d_p, sigma_theta_frac * theta_L,
                                    EPS_S_EV, SI_X0, RHO_THERMAL, int(bool(ms)), int(bool(ll)),
                                    int(bool(ms_loss)), dt, int(seed), n_particles, _ptr(lens), S,
                                    _ptr(rec_off), _ptr(sec_off), _ptr(samp_off), _ptr(out), _ptr(secE),
                                    _ptr(eS) if eS is not None else None, None, None)
    if rc != 0:
        raise RuntimeError("tg_channeling_loss failed")
    # section record ranges: particle p's sections are consecutive; all but the last have S records
    ns = int(sec_off[-1])
    parent = np.repeat(np.arange(n_particles, dtype=np.int64), nsec)
    first = sec_off[parent]
    j_in = np.arange(ns, dtype=np.int64) - first
    start = rec_off[parent] + j_in * S
    last = j_in == nsec[parent] - 1
    slen = np.where(last, (lens[parent] + nsec[parent] - 1) - j_in * S, S)
    off = np.zeros(ns + 1, dtype=np.int64)
    off[1:] = start + slen
    off[:-1] = start
    w = np.full(ns, 1.0 / max(n_particles, 1))
    tr = Trajectories(out, off, secE / mass_eV, secE, w)
    return Sectioned(tr, parent, sec_off, eS, samp_off if keep_energy else None)


def lognormal_lengths(n: int, seed: int, median: float = 20000.0, sigma: float = math.log(10) / 3,
                      lo: int = 2000, hi: int = 200000) -> np.ndarray:
    out = np.empty(n, dtype=np.int64)
    _load().tg_lognormal_lengths(int(seed), n, median, sigma, lo, hi, _ptr(out))
    return out


def planar_undulator(gamma: float, K: float, lam_u: float, n_periods: int, samples_per_period: int,
                     mass_eV: float = ME_EV) -> Trajectories:
    """Planar undulator of deflection parameter K (field B0 sin(2 pi z / lam_u) along y).

    vx = (K/gamma) cos(k t), x = K/(gamma k) sin(k t), k = 2 pi / lam_u, t over whole periods;
    longitudinal variables to leading order in vx: dvz = -vx^2/2, az = -vx ax,
    dz = -(K/gamma)^2/4 (t + sin(2kt)/(2k)).
    """
    k = 2.0 * math.pi / lam_u
    n = n_periods * samples_per_period + 1
    t = np.linspace(0.0, n_periods * lam_u, n)
    amp = K / gamma
    s = np.zeros((n, NREC))
    s[:, 0] = t
    s[:, 1] = amp / k * np.sin(k * t)
    s[:, 4] = amp * np.cos(k * t)
    s[:, 7] = -amp * k * np.sin(k * t)
    s[:, 6] = -0.5 * s[:, 4] ** 2
    s[:, 9] = -s[:, 4] * s[:, 7]
    s[:, 3] = -0.25 * amp ** 2 * (t + np.sin(2.0 * k * t) / (2.0 * k))
    return single(s, gamma, mass_eV)


def undulator_K(B0_T: float, lam_u: float) -> float:
    """K = e B0 lam_u / (2 pi m c) = B0 * lam_u * c / (2 pi * m c^2 / e)."""
    c = 299792458.0
    return B0_T * lam_u * c / (2.0 * math.pi * ME_EV)


def elliptical_undulator(gamma=2000.0, a=0.4e-10, b=0.25e-10, phase=0.7, lam=10e-6, n_periods=3,
                         n_samples=3073, mass_eV=ME_EV, times=None) -> Trajectories:
    """x = a sin(kt), y = b sin(kt + phase): motion in both transverse planes, uniform samples
    over n_periods (or the given increasing `times`, which then set n_samples).

    dvz = -(vx^2 + vy^2)/2, az = -(vx ax + vy ay), dz the exact integral of dvz from t = 0.
    """
    k = 2.0 * math.pi / lam
    t = np.linspace(0.0, n_periods * lam, n_samples) if times is None else np.asarray(times, np.float64)
    n_samples = t.shape[0]
    s = np.zeros((n_samples, NREC))
    s[:, 0] = t
    s[:, 1] = a * np.sin(k * t)
    s[:, 2] = b * np.sin(k * t + phase)
    s[:, 4] = a * k * np.cos(k * t)
    s[:, 5] = b * k * np.cos(k * t + phase)
    s[:, 7] = -a * k * k * np.sin(k * t)
    s[:, 8] = -b * k * k * np.sin(k * t + phase)
    s[:, 6] = -0.5 * (s[:, 4] ** 2 + s[:, 5] ** 2)
    s[:, 9] = -(s[:, 4] * s[:, 7] + s[:, 5] * s[:, 8])
    s[:, 3] = (-0.25 * (a * k) ** 2 * (t + np.sin(2.0 * k * t) / (2.0 * k))
               - 0.25 * (b * k) ** 2 * (t + (np.sin(2.0 * (k * t + phase)) - np.sin(2.0 * phase))
                                        / (2.0 * k)))
    return single(s, gamma, mass_eV)


# --------------------------------------------------------------------------- #
# Named workloads (synthetic stand-ins with the paper's scales: GeV e+-, Si(110)
# d_p = 1.92 A, ~0.1 mm crystals; the crystal potential is a harmonic well)
# --------------------------------------------------------------------------- #
def workload_undulator_4096():
    """Analytic e+ trajectory, gamma = 1000, x = a sin(2 pi t / lambda), a = 0.5 A, lambda = 10 um,
    4096 uniform samples over 5 periods; 128 linear hw up to 1.2 x first-harmonic edge; 16 x 16
    cell-centred directions within +-2/gamma."""
    g, a, lam = 1000.0, 0.5e-10, 10e-6
    tr = weak_undulator(g, a, lam, 5, 4096)
    hw1 = undulator_first_harmonic_eV(g, a, lam)
    grid = make_grid(omega_linear(128, 1.2 * hw1), 16, 16, 2.0 / g)
    return tr, grid


def _ensemble_grid(E_eV, U0_eV, n_omega, n_side, mass_eV=ME_EV):
    g = E_eV / mass_eV
    thL = math.sqrt(2.0 * U0_eV / E_eV)
    half = thL + 3.0 / g
    return make_grid(omega_log(n_omega, 1e-4 * E_eV, 0.5 * E_eV), n_side, n_side, half)


def workload_positron_ensemble(n_particles=1024, n_samples=20000, seed=2, n_omega=512, n_side=64,
                               particles=None):
    """e+ 10 GeV in a harmonic planar well (U0 = 20 eV, d_p = 1.92 A), x0 ~ U[0, d_p),
    theta_x0 ~ N(0, (0.3 theta_L)^2), RK4 dt = 5 nm with scattering kicks; 512 log-spaced hw in
    [1e-4 E, 0.5 E]; 64 x 64 directions within +-(theta_L + 3/gamma).
    `particles` selects a subset (indices) after generation with the full-ensemble seed."""
    E = 10e9
    tr = channeling(n_particles, E, +1, n_samples, 5e-9, seed)
    if particles is not None:
        tr = tr.subset(particles)
        tr.weight = np.full(tr.n_particles, 1.0 / n_particles)
    return tr, _ensemble_grid(E, 20.0, n_omega, n_side)


def workload_electron_batch(n_particles=4096, seed=4, n_omega=1024, n_side=32, median=20000.0,
                            lo=2000, hi=200000, particles=None):
    """e- 20 GeV, same well centred on the planes, lognormal lengths clip(exp(N(ln median,
    ln(10)/3)), lo, hi); 1024 log-spaced hw in [1e-4 E, 0.5 E]; 32 x 32 directions."""
    E = 20e9
    L = lognormal_lengths(n_particles, seed, median=median, lo=lo, hi=hi)
    tr = channeling(n_particles, E, -1, L, 5e-9, seed)
    if particles is not None:
        tr = tr.subset(particles)
        tr.weight = np.full(tr.n_particles, 1.0 / n_particles)
    return tr, _ensemble_grid(E, 20.0, n_omega, n_side)


def workload_strong_undulator_angular(samples_per_period: int = 2048, n_omega: int = 1000, n_side: int = 32):
    """The paper's second integral test (Sec. IV): the same 2 GeV undulator, dI/dOmega over the
    photon energies 0-500 eV in a window of half-width 5/gamma: n_omega linear photon energies
    (500/n_omega ... 500 eV; the trapezoid over them is the energy integral) and n_side x n_side
    cell-centred directions within +-5/gamma."""
    return workload_strong_undulator(samples_per_period, n_omega, n_side, 5.0)


def workload_strong_undulator(samples_per_period: int = 2048, n_omega: int = 256, n_side: int = 8,
                              half_angle_gammas: float = 0.5):
    """The paper's integral test (Sec. IV): 2 GeV electron, planar undulator with 53 mm period,
    20 periods, B0 = 1 T (K = 4.95); photon energies 0-500 eV (linear grid from 2 eV) and a small
    direction grid around the axis (+-half_angle_gammas/gamma)."""
    g = 2.0e9 / ME_EV
    K = undulator_K(1.0, 0.053)
    tr = planar_undulator(g, K, 0.053, 20, samples_per_period)
    grid = make_grid(omega_linear(n_omega, 500.0), n_side, n_side, half_angle_gammas / g)
    return tr, grid
