"""FP64 CPU oracle for the radiation integral -- test infrastructure only.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this package. The CUDA product path never calls it; the two share no code.

This is a thin ctypes wrapper around ``oracle.c`` (plain C, FP64, Neumaier sums,
libm sin/cos). See that file's header for the equations it follows (Sec. II of
arXiv:1910.10391: Eq. 1, Eq. 2, the expanded f/g/phase, the Lindhard substitution
and the BCK spin-1/2 formula) and for the readings taken where the paper is silent.

Parity status: every function here is pinned by tests in tests/test_oracle_pins.py
(straight-line zero, weak-undulator dipole closed form and harmonic positions,
Jackson synchrotron, Larmor energy, integration-by-parts identities for I and J,
unexpanded Lienard-Wiechert brute force, quadrature order, symmetry, additivity).

Submodules: ``traj`` (trajectories of Sec. III: harmonic well or Doyle-Turner planar
potential, scattering on nuclei and electrons, radiation reaction; pinned in
tests/test_traj_oracle.py and tests/test_potential_oracle.py, the electron-scattering rate
included) and ``mlp`` (the surrogate network in FP64 numpy,
pinned by finite differences in tests/test_mlp_reference.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

CLASSICAL, SPIN0, SPIN_HALF = 0, 1, 2
HBARC_EV_M = 1.973269804e-7
ALPHA = 7.2973525693e-3

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """gcc -O2 -fopenmp -ffp-contract=off (no fused multiply-add, IEEE order)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-fno-fast-math", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P, i64, i32, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
            lib.orc_amplitudes.argtypes = [P, i64, d, d, d, d, P]
            lib.orc_amplitudes.restype = i32
            lib.orc_spectrum_bins.argtypes = [P, P, i64, P, P, P, P, i64, P, P, i64, i32, P, P, i64,
                                              P, P, i32]
            lib.orc_spectrum_bins.restype = i32
            lib.orc_spectrum_cube.argtypes = [P, P, i64, P, P, P, P, i64, P, P, i64, i32, P, P, i32]
            lib.orc_spectrum_cube.restype = i32
            lib.orc_reduce.argtypes = [P, i64, i64, P, P, i32, P, P]
            lib.orc_reduce.restype = i32
            lib.orc_set_plant.argtypes = [i32]
            lib.orc_set_plant.restype = None
            lib.orc_max_threads.argtypes = []
            lib.orc_max_threads.restype = i32
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def max_threads() -> int:
    return int(_load().orc_max_threads())


def set_plant(which: int) -> None:
    """Plant a deliberate mistake in the oracle (tests of the pins only); 0 clears it."""
    _load().orc_set_plant(int(which))


def amplitudes(samples, gamma: float, omega_star: float, nx: float, ny: float) -> np.ndarray:
    """[Re Ix, Im Ix, Re Iy, Im Iy, Re Iz, Im Iz, Re J, Im J, sum w|f|, sum w|j|] of one particle."""
    s = _f64(samples)
    out = np.zeros(10)
    rc = _load().orc_amplitudes(_p(s), s.shape[0], float(gamma), float(omega_star), float(nx),
                                float(ny), _p(out))
    if rc:
        raise ValueError("orc_amplitudes: invalid input")
    return out


def _traj_args(tr):
    w = None if tr.weight is None else _f64(tr.weight)
    return (_f64(tr.samples), _i64(tr.offsets), tr.n_particles, _f64(tr.gamma), _f64(tr.energy_eV), w)


def spectrum_bins(tr, grid, mode: int, bin_omega, bin_angle, want_cond: bool = False,
                  n_threads: int = 0):
    s, off, npart, g, e, w = _traj_args(tr)
    hw, tx, ty = _f64(grid.hbar_omega_eV), _f64(grid.theta_x), _f64(grid.theta_y)
    bi, bj = _i64(bin_omega), _i64(bin_angle)
    out = np.zeros(bi.shape[0])
    cond = np.zeros(bi.shape[0]) if want_cond else None
    rc = _load().orc_spectrum_bins(_p(s), _p(off), npart, _p(g), _p(e), _p(w), _p(hw), hw.shape[0],
                                   _p(tx), _p(ty), tx.shape[0], int(mode), _p(bi), _p(bj),
                                   bi.shape[0], _p(out), _p(cond), int(n_threads))
    if rc:
        raise ValueError("orc_spectrum_bins: invalid input")
    return (out, cond) if want_cond else out


def spectrum_cube(tr, grid, mode: int, want_cond: bool = False, n_threads: int = 0):
    """Cube [n_omega, n_angles] of alpha/(4 pi^2) sum_p weight_p S_p."""
    s, off, npart, g, e, w = _traj_args(tr)
    hw, tx, ty = _f64(grid.hbar_omega_eV), _f64(grid.theta_x), _f64(grid.theta_y)
    out = np.zeros((hw.shape[0], tx.shape[0]))
    cond = np.zeros_like(out) if want_cond else None
    rc = _load().orc_spectrum_cube(_p(s), _p(off), npart, _p(g), _p(e), _p(w), _p(hw), hw.shape[0],
                                   _p(tx), _p(ty), tx.shape[0], int(mode), _p(out), _p(cond),
                                   int(n_threads))
    if rc:
        raise ValueError("orc_spectrum_cube: invalid input")
    return (out, cond) if want_cond else out


def reduce(cube, d_omega, bin_of_angle=None, n_rbins: int = 0):
    """(spectrum [n_omega], bins [n_omega, n_rbins] or None) from a cube."""
    c = _f64(cube)
    n_omega, n_angles = c.shape
    dom = _f64(d_omega)
    spec = np.zeros(n_omega)
    bins = None
    boa = None
    if bin_of_angle is not None and n_rbins > 0:
        boa = np.ascontiguousarray(bin_of_angle, dtype=np.int32)
        bins = np.zeros((n_omega, n_rbins))
    rc = _load().orc_reduce(_p(c), n_omega, n_angles, _p(dom), _p(boa), int(n_rbins), _p(spec),
                            _p(bins))
    if rc:
        raise ValueError("orc_reduce: invalid input")
    return spec, bins
