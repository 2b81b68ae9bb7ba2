"""ctypes binding of librad.so (include/rad.h). Argument marshalling only.

The functions named ``rad_*`` mirror the C entry points one to one and take torch
tensors (device tensors for the device entry points, host arrays for
``rad_spectrum_host``). Sizes are taken from the tensors' shapes. Every step of the
computation runs in the CUDA library; if it cannot be built or loaded, ``load()``
raises and nothing falls back to the CPU.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librad.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "rad.h")

RAD_OK, RAD_EINVAL, RAD_ENOMEM, RAD_ECUDA, RAD_ETIMEOUT, RAD_EUNSUPPORTED, RAD_EDATA, RAD_ETOOBIG, RAD_EPRECISION = range(9)
RAD_CLASSICAL, RAD_SPIN0, RAD_SPIN_HALF = 0, 1, 2
RAD_FP64, RAD_MIXED, RAD_FP64_DF = 0, 1, 2
RAD_NREC = 10
RAD_PER_PARTICLE = 8  # rad_plan_create `want` bit: per-particle spectrum/bins
RAD_TRAJ_MS, RAD_TRAJ_LL, RAD_TRAJ_MS_LOSS, RAD_TRAJ_FP32, RAD_TRAJ_MS_EL = 1, 2, 4, 8, 16


class RadChannel(ctypes.Structure):
    """rad_channel: harmonic planar well and scattering model of the trajectory integrator."""
    _fields_ = [("U0_eV", ctypes.c_double), ("d_p", ctypes.c_double), ("eps_s_eV", ctypes.c_double),
                ("X0", ctypes.c_double), ("rho", ctypes.c_double), ("mass_eV", ctypes.c_double),
                ("charge_sign", ctypes.c_int), ("flags", ctypes.c_int)]


class RadPlanarPotential(ctypes.Structure):
    """rad_planar_potential: Doyle-Turner planar fit (potential and X-ray terms) of the crystal."""
    _fields_ = [("n_terms", ctypes.c_int), ("n_neighbours", ctypes.c_int), ("N", ctypes.c_double),
                ("a", ctypes.c_double * 8), ("b", ctypes.c_double * 8), ("ax", ctypes.c_double * 8),
                ("bx", ctypes.c_double * 8), ("cx", ctypes.c_double), ("I_eV", ctypes.c_double)]

    @classmethod
    def make(cls, a, b, N, ax=(), bx=(), cx=0.0, I_eV=0.0, n_neighbours=3):
        if len(a) != len(b) or (len(ax) and len(ax) != len(a)) or len(ax) != len(bx) or not 1 <= len(a) <= 8:
            raise ValueError("a, b (and ax, bx) must have the same length, 1..8")
        pad = lambda v: (ctypes.c_double * 8)(*(list(map(float, v)) + [0.0] * (8 - len(v))))
        return cls(len(a), int(n_neighbours), float(N), pad(a), pad(b), pad(ax), pad(bx), float(cx), float(I_eV))
RAD_DIAMOND, RAD_BCC = 0, 1
RAD_SI, RAD_C, RAD_GE, RAD_W = 0, 1, 2, 3


class RadElement(ctypes.Structure):
    """rad_element: structure, lattice constant, Z, mean ionisation energy, radiation length."""
    _fields_ = [("structure", ctypes.c_int), ("a", ctypes.c_double), ("Z", ctypes.c_int), ("I_eV", ctypes.c_double),
                ("X0", ctypes.c_double)]


class RadStringLattice(ctypes.Structure):
    """rad_string_lattice: rectangular transverse cell, string positions, atom spacing along a string."""
    _fields_ = [("n_strings", ctypes.c_int), ("cell_x", ctypes.c_double), ("cell_y", ctypes.c_double),
                ("sx", ctypes.c_double * 8), ("sy", ctypes.c_double * 8), ("d", ctypes.c_double)]

    @classmethod
    def make(cls, cell_x, cell_y, sx, sy, d):
        if len(sx) != len(sy) or not 1 <= len(sx) <= 8:
            raise ValueError("sx, sy must have the same length, 1..8")
        pad = lambda v: (ctypes.c_double * 8)(*(list(map(float, v)) + [0.0] * (8 - len(v))))
        return cls(len(sx), float(cell_x), float(cell_y), pad(sx), pad(sy), float(d))


class RadPlaneStack(ctypes.Structure):
    """rad_plane_stack: planes per period along the normal, their offsets and areal densities."""
    _fields_ = [("n_planes", ctypes.c_int), ("period", ctypes.c_double), ("offset", ctypes.c_double * 4),
                ("areal", ctypes.c_double * 4)]


class RadAxialPotential(ctypes.Structure):
    """rad_axial_potential: Doyle-Turner fit of the atoms and the string lattice of the axis."""
    _fields_ = [("n_terms", ctypes.c_int), ("n_cells", ctypes.c_int), ("a", ctypes.c_double * 8),
                ("b", ctypes.c_double * 8), ("ax", ctypes.c_double * 8), ("bx", ctypes.c_double * 8),
                ("cx", ctypes.c_double), ("I_eV", ctypes.c_double), ("lattice", RadStringLattice)]

    @classmethod
    def make(cls, a, b, lattice, ax=(), bx=(), cx=0.0, I_eV=0.0, n_cells=2):
        if len(a) != len(b) or (len(ax) and len(ax) != len(a)) or len(ax) != len(bx) or not 1 <= len(a) <= 8:
            raise ValueError("a, b (and ax, bx) must have the same length, 1..8")
        pad = lambda v: (ctypes.c_double * 8)(*(list(map(float, v)) + [0.0] * (8 - len(v))))
        return cls(len(a), int(n_cells), pad(a), pad(b), pad(ax), pad(bx), float(cx), float(I_eV), lattice)


class RadStepControl(ctypes.Structure):
    """rad_step_control: tolerances, lower bound (max_level) and sub-step budget of the adaptive integrator."""
    _fields_ = [("rtol", ctypes.c_double), ("atol_x", ctypes.c_double), ("atol_v", ctypes.c_double),
                ("max_level", ctypes.c_int), ("max_substeps", ctypes.c_int64)]


MODES = {"classical": RAD_CLASSICAL, "spin0": RAD_SPIN0, "spin_half": RAD_SPIN_HALF}
PRECISIONS = {"fp64": RAD_FP64, "mixed": RAD_MIXED, "fp64_df": RAD_FP64_DF}

_lock = threading.Lock()
_lib = None


class RadError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = "?"
        try:
            msg = load().rad_status_string(status).decode()
        except Exception:  # pragma: no cover
            pass
        super().__init__(f"{where}: status {status} ({msg})")


def header_symbols() -> list:
    """Names of the functions declared in include/rad.h."""
    with open(HEADER) as f:
        txt = f.read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rad_[a-z0-9_]+)\s*\(", txt)))


def load(build_if_missing: bool = True):
    """Load librad.so (building it in place with nvcc when missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _build
        if build_if_missing and _build.needs_build():
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} (run paper_1910_10391_gb300.build)")
        lib = ctypes.CDLL(LIB_PATH)
        P, i64, i32, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
        spec_args = [P, i64, P, i64, P, P, P, P, i64, P, P, P, i64, c_int, c_int, P, P, P, i32, P, c_int, P]
        lib.rad_spectrum.argtypes = spec_args
        lib.rad_spectrum.restype = c_int
        lib.rad_spectrum_host.argtypes = spec_args
        lib.rad_spectrum_host.restype = c_int
        lib.rad_spectrum_noalloc.argtypes = [P, i64, P, i64, P, P, P, P, i64, P, P, i64, c_int, P, P]
        lib.rad_spectrum_noalloc.restype = c_int
        lib.rad_spectrum_particles.argtypes = [P, i64, P, i64, P, P, P, P, i64, P, P, P, i64, c_int, c_int, P, P,
                                               i32, P, P]
        lib.rad_spectrum_particles.restype = c_int
        u64, f32 = ctypes.c_uint64, ctypes.c_float
        lib.rad_channeling_trajectories.argtypes = [ctypes.POINTER(RadChannel), i64, P, i64, P, P, P, P, P,
                                                    ctypes.c_double, u64, P, P, P]
        lib.rad_channeling_trajectories.restype = c_int
        lib.rad_crystal_trajectories.argtypes = [ctypes.POINTER(RadChannel), ctypes.POINTER(RadPlanarPotential), i64,
                                                 P, i64, P, P, P, P, P, ctypes.c_double, u64, P, P, P]
        lib.rad_crystal_trajectories.restype = c_int
        lib.rad_axial_trajectories.argtypes = [ctypes.POINTER(RadChannel), ctypes.POINTER(RadAxialPotential), i64,
                                               P, i64, P, P, P, P, P, P, ctypes.c_double, u64, P, P, P]
        lib.rad_axial_trajectories.restype = c_int
        lib.rad_trajectories_adaptive.argtypes = [ctypes.POINTER(RadChannel), ctypes.POINTER(RadPlanarPotential),
                                                  ctypes.POINTER(RadAxialPotential), ctypes.POINTER(RadStepControl),
                                                  i64, P, i64, P, P, P, P, P, P, P, ctypes.c_double, u64, P, P, P, P]
        lib.rad_trajectories_adaptive.restype = c_int
        lib.rad_angular_distribution.argtypes = [P, P, i64, i64, P, P]
        lib.rad_angular_distribution.restype = c_int
        lib.rad_crystal_element.argtypes = [c_int, ctypes.POINTER(RadElement)]
        lib.rad_crystal_element.restype = c_int
        lib.rad_crystal_string_lattice.argtypes = [c_int, ctypes.c_double, c_int, ctypes.POINTER(RadStringLattice)]
        lib.rad_crystal_string_lattice.restype = c_int
        lib.rad_crystal_plane_stack.argtypes = [c_int, ctypes.c_double, c_int, ctypes.POINTER(RadPlaneStack)]
        lib.rad_crystal_plane_stack.restype = c_int
        lib.rad_mlp_create.argtypes = [c_int, c_int, c_int, c_int, i64, u64, ctypes.POINTER(P)]
        lib.rad_mlp_create.restype = c_int
        lib.rad_mlp_destroy.argtypes = [P]
        lib.rad_mlp_destroy.restype = c_int
        lib.rad_mlp_num_params.argtypes = [P]
        lib.rad_mlp_num_params.restype = i64
        lib.rad_mlp_forward.argtypes = [P, P, i64, P, P]
        lib.rad_mlp_forward.restype = c_int
        lib.rad_mlp_backward.argtypes = [P, P, P, P, i64, P, P]
        lib.rad_mlp_backward.restype = c_int
        lib.rad_mlp_adamw.argtypes = [P, f32, f32, f32, f32, f32, P]
        lib.rad_mlp_adamw.restype = c_int
        lib.rad_mlp_train_step.argtypes = [P, P, P, P, i64, f32, f32, P, P]
        lib.rad_mlp_train_step.restype = c_int
        lib.rad_mlp_get.argtypes = [P, c_int, P]
        lib.rad_mlp_get.restype = c_int
        lib.rad_mlp_set_params.argtypes = [P, P]
        lib.rad_mlp_set_params.restype = c_int
        lib.rad_mlp_ensemble_estimate.argtypes = [P, c_int, i64, c_int, P, P, P]
        lib.rad_mlp_ensemble_estimate.restype = c_int
        lib.rad_log_targets.argtypes = [P, i64, ctypes.c_double, P, P]
        lib.rad_log_targets.restype = c_int
        lib.rad_column_stats.argtypes = [P, i64, c_int, P, P, P]
        lib.rad_column_stats.restype = c_int
        lib.rad_standardize.argtypes = [P, i64, c_int, P, P, c_int, P]
        lib.rad_standardize.restype = c_int
        lib.rad_plan_create.argtypes = [i64, i64, i64, i64, c_int, c_int, c_int, i32, ctypes.POINTER(P)]
        lib.rad_plan_create.restype = c_int
        exec_args = [P, P, P, P, P, P, P, P, P, P, P, P, P, P, c_int, P]
        lib.rad_plan_execute.argtypes = exec_args
        lib.rad_plan_execute.restype = c_int
        lib.rad_plan_autotune.argtypes = exec_args[:14] + [c_int, P]
        lib.rad_plan_autotune.restype = c_int
        lib.rad_plan_set_shape.argtypes = [P, c_int, c_int, c_int, c_int]
        lib.rad_plan_set_shape.restype = c_int
        lib.rad_plan_set_prepass.argtypes = [P, c_int]
        lib.rad_plan_set_prepass.restype = c_int
        lib.rad_plan_set_sincos_split.argtypes = [P, c_int]
        lib.rad_plan_set_sincos_split.restype = c_int
        lib.rad_plan_set_phase_budget.argtypes = [P, ctypes.c_double]
        lib.rad_plan_set_phase_budget.restype = c_int
        lib.rad_plan_describe.argtypes = [P, ctypes.c_char_p, c_int]
        lib.rad_plan_describe.restype = c_int
        lib.rad_plan_set_timing.argtypes = [P, c_int]
        lib.rad_plan_set_timing.restype = c_int
        lib.rad_plan_last_kernel_ms.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
        lib.rad_plan_last_kernel_ms.restype = c_int
        lib.rad_plan_kernel_launches.argtypes = [P]
        lib.rad_plan_kernel_launches.restype = c_int
        lib.rad_plan_destroy.argtypes = [P]
        lib.rad_plan_destroy.restype = c_int
        lib.rad_graph_create.argtypes = exec_args + [ctypes.POINTER(P)]
        lib.rad_graph_create.restype = c_int
        lib.rad_graph_launch.argtypes = [P, P]
        lib.rad_graph_launch.restype = c_int
        lib.rad_graph_destroy.argtypes = [P]
        lib.rad_graph_destroy.restype = c_int
        lib.rad_device_status.argtypes = [c_int]
        lib.rad_device_status.restype = c_int
        lib.rad_selftest_bounded_wait.argtypes = [P]
        lib.rad_selftest_bounded_wait.restype = c_int
        lib.rad_status_string.argtypes = [c_int]
        lib.rad_status_string.restype = ctypes.c_char_p
        lib.rad_version.argtypes = []
        lib.rad_version.restype = ctypes.c_char_p
        lib.rad_release.argtypes = []
        lib.rad_release.restype = None
        _lib = lib
        return lib


# --------------------------------------------------------------------------- #
# marshalling helpers
# --------------------------------------------------------------------------- #
def _dev_ptr(t, dtype=None, name="tensor"):
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name}: must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(a, dtype=None, name="array"):
    if a is None:
        return None
    import torch
    if isinstance(a, torch.Tensor):
        if a.is_cuda:
            raise ValueError(f"{name}: must be a host tensor")
        if dtype is not None and a.dtype != dtype:
            raise TypeError(f"{name}: expected {dtype}, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError(f"{name}: must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    import numpy as np
    if not (isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"]):
        raise TypeError(f"{name}: expected a contiguous numpy array or host tensor")
    return ctypes.c_void_p(a.ctypes.data)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _numel(t):
    return 0 if t is None else int(t.numel())


# --------------------------------------------------------------------------- #
# entry points
# --------------------------------------------------------------------------- #
def rad_spectrum(samples, offsets, gamma, energy_eV, weight, hbar_omega_eV, theta_x, theta_y, d_omega,
                 mode, precision, out_cube=None, out_spectrum=None, bin_of_angle=None, n_bins=0,
                 out_bins=None, accumulate=0, stream=None) -> int:
    import torch
    lib = load()
    f64, i64 = torch.float64, torch.int64
    return lib.rad_spectrum(
        _dev_ptr(samples, f64, "samples"), _numel(samples) // RAD_NREC, _dev_ptr(offsets, i64, "offsets"),
        _numel(offsets) - 1, _dev_ptr(gamma, f64, "gamma"), _dev_ptr(energy_eV, f64, "energy_eV"),
        _dev_ptr(weight, f64, "weight"), _dev_ptr(hbar_omega_eV, f64, "hbar_omega_eV"),
        _numel(hbar_omega_eV), _dev_ptr(theta_x, f64, "theta_x"), _dev_ptr(theta_y, f64, "theta_y"),
        _dev_ptr(d_omega, f64, "d_omega"), _numel(theta_x), int(mode), int(precision),
        _dev_ptr(out_cube, f64, "out_cube"), _dev_ptr(out_spectrum, f64, "out_spectrum"),
        _dev_ptr(bin_of_angle, torch.int32, "bin_of_angle"), int(n_bins), _dev_ptr(out_bins, f64, "out_bins"),
        int(accumulate), _stream(stream))


def rad_spectrum_host(samples, offsets, gamma, energy_eV, weight, hbar_omega_eV, theta_x, theta_y, d_omega,
                      mode, precision, out_cube=None, out_spectrum=None, bin_of_angle=None, n_bins=0,
                      out_bins=None, accumulate=0, stream=None) -> int:
    import torch
    lib = load()
    f64, i64 = torch.float64, torch.int64
    n = lambda a: 0 if a is None else int(a.numel() if isinstance(a, torch.Tensor) else a.size)
    return lib.rad_spectrum_host(
        _host_ptr(samples, f64, "samples"), n(samples) // RAD_NREC, _host_ptr(offsets, i64, "offsets"),
        n(offsets) - 1, _host_ptr(gamma, f64, "gamma"), _host_ptr(energy_eV, f64, "energy_eV"),
        _host_ptr(weight, f64, "weight"), _host_ptr(hbar_omega_eV, f64, "hbar_omega_eV"), n(hbar_omega_eV),
        _host_ptr(theta_x, f64, "theta_x"), _host_ptr(theta_y, f64, "theta_y"), _host_ptr(d_omega, f64, "d_omega"),
        n(theta_x), int(mode), int(precision), _host_ptr(out_cube, f64, "out_cube"),
        _host_ptr(out_spectrum, f64, "out_spectrum"), _host_ptr(bin_of_angle, torch.int32, "bin_of_angle"),
        int(n_bins), _host_ptr(out_bins, f64, "out_bins"), int(accumulate), _stream(stream))


def rad_spectrum_noalloc(samples, offsets, gamma, energy_eV, weight, hbar_omega_eV, theta_x, theta_y, mode,
                         out_cube, stream=None) -> int:
    """Mixed-precision cube with the library's fixed scratch (no device allocation); synchronous."""
    import torch
    lib = load()
    f64 = torch.float64
    return lib.rad_spectrum_noalloc(
        _dev_ptr(samples, f64, "samples"), _numel(samples) // RAD_NREC, _dev_ptr(offsets, torch.int64, "offsets"),
        _numel(offsets) - 1, _dev_ptr(gamma, f64, "gamma"), _dev_ptr(energy_eV, f64, "energy_eV"),
        _dev_ptr(weight, f64, "weight"), _dev_ptr(hbar_omega_eV, f64, "hbar_omega_eV"), _numel(hbar_omega_eV),
        _dev_ptr(theta_x, f64, "theta_x"), _dev_ptr(theta_y, f64, "theta_y"), _numel(theta_x), int(mode),
        _dev_ptr(out_cube, f64, "out_cube"), _stream(stream))


def rad_spectrum_particles(samples, offsets, gamma, energy_eV, weight, hbar_omega_eV, theta_x, theta_y, d_omega,
                           mode, precision, out_spectrum=None, bin_of_angle=None, n_bins=0, out_bins=None,
                           stream=None) -> int:
    import torch
    lib = load()
    f64 = torch.float64
    return lib.rad_spectrum_particles(
        _dev_ptr(samples, f64, "samples"), _numel(samples) // RAD_NREC, _dev_ptr(offsets, torch.int64, "offsets"),
        _numel(offsets) - 1, _dev_ptr(gamma, f64, "gamma"), _dev_ptr(energy_eV, f64, "energy_eV"),
        _dev_ptr(weight, f64, "weight"), _dev_ptr(hbar_omega_eV, f64, "hbar_omega_eV"), _numel(hbar_omega_eV),
        _dev_ptr(theta_x, f64, "theta_x"), _dev_ptr(theta_y, f64, "theta_y"), _dev_ptr(d_omega, f64, "d_omega"),
        _numel(theta_x), int(mode), int(precision), _dev_ptr(out_spectrum, f64, "out_spectrum"),
        _dev_ptr(bin_of_angle, torch.int32, "bin_of_angle"), int(n_bins), _dev_ptr(out_bins, f64, "out_bins"),
        _stream(stream))


def rad_channeling_trajectories(channel, offsets, energy_eV, x0, thx0, out, dt, seed, thy0=None,
                                particle_ids=None, energy_out=None, stream=None) -> int:
    """Records of every particle into `out` [n_samples_total][10] (device tensors throughout)."""
    import torch
    f64 = torch.float64
    return load().rad_channeling_trajectories(
        ctypes.byref(channel), _numel(offsets) - 1, _dev_ptr(offsets, torch.int64, "offsets"), _numel(out) // RAD_NREC,
        _dev_ptr(energy_eV, f64, "energy_eV"), _dev_ptr(x0, f64, "x0"), _dev_ptr(thx0, f64, "thx0"),
        _dev_ptr(thy0, f64, "thy0"), _dev_ptr(particle_ids, torch.int64, "particle_ids"), float(dt), int(seed),
        _dev_ptr(out, f64, "out"), _dev_ptr(energy_out, f64, "energy_out"), _stream(stream))


def rad_crystal_trajectories(channel, potential, offsets, energy_eV, x0, thx0, out, dt, seed, thy0=None,
                             particle_ids=None, energy_out=None, stream=None) -> int:
    """rad_channeling_trajectories in the Doyle-Turner planar potential `potential`
    (RadPlanarPotential, or None to see the library reject it)."""
    import torch
    f64 = torch.float64
    return load().rad_crystal_trajectories(
        ctypes.byref(channel), ctypes.byref(potential) if potential is not None else None, _numel(offsets) - 1,
        _dev_ptr(offsets, torch.int64, "offsets"), _numel(out) // RAD_NREC, _dev_ptr(energy_eV, f64, "energy_eV"),
        _dev_ptr(x0, f64, "x0"), _dev_ptr(thx0, f64, "thx0"), _dev_ptr(thy0, f64, "thy0"),
        _dev_ptr(particle_ids, torch.int64, "particle_ids"), float(dt), int(seed), _dev_ptr(out, f64, "out"),
        _dev_ptr(energy_out, f64, "energy_out"), _stream(stream))


def rad_axial_trajectories(channel, potential, offsets, energy_eV, x0, thx0, out, dt, seed, y0=None, thy0=None,
                           particle_ids=None, energy_out=None, stream=None) -> int:
    """Trajectories in the axial (string) potential `potential` (RadAxialPotential)."""
    import torch
    f64 = torch.float64
    return load().rad_axial_trajectories(
        ctypes.byref(channel), ctypes.byref(potential) if potential is not None else None, _numel(offsets) - 1,
        _dev_ptr(offsets, torch.int64, "offsets"), _numel(out) // RAD_NREC, _dev_ptr(energy_eV, f64, "energy_eV"),
        _dev_ptr(x0, f64, "x0"), _dev_ptr(y0, f64, "y0"), _dev_ptr(thx0, f64, "thx0"), _dev_ptr(thy0, f64, "thy0"),
        _dev_ptr(particle_ids, torch.int64, "particle_ids"), float(dt), int(seed), _dev_ptr(out, f64, "out"),
        _dev_ptr(energy_out, f64, "energy_out"), _stream(stream))


def rad_trajectories_adaptive(channel, step_control, offsets, energy_eV, x0, thx0, out, seed, times=None, dt=0.0,
                              planar=None, axial=None, y0=None, thy0=None, particle_ids=None, energy_out=None,
                              substeps_out=None, stream=None) -> int:
    """Trajectories with adaptive Dormand-Prince steps between output times (`times`, device, per
    record; or uniform k dt) in the harmonic well, the planar potential `planar` or the axial
    potential `axial`."""
    import torch
    f64 = torch.float64
    return load().rad_trajectories_adaptive(
        ctypes.byref(channel), ctypes.byref(planar) if planar is not None else None,
        ctypes.byref(axial) if axial is not None else None, ctypes.byref(step_control) if step_control else None,
        _numel(offsets) - 1, _dev_ptr(offsets, torch.int64, "offsets"), _numel(out) // RAD_NREC,
        _dev_ptr(energy_eV, f64, "energy_eV"), _dev_ptr(x0, f64, "x0"), _dev_ptr(y0, f64, "y0"),
        _dev_ptr(thx0, f64, "thx0"), _dev_ptr(thy0, f64, "thy0"), _dev_ptr(particle_ids, torch.int64, "particle_ids"),
        _dev_ptr(times, f64, "times"), float(dt), int(seed), _dev_ptr(out, f64, "out"),
        _dev_ptr(energy_out, f64, "energy_out"), _dev_ptr(substeps_out, torch.int64, "substeps_out"), _stream(stream))


def rad_angular_distribution(cube, hbar_omega_eV, out, stream=None) -> int:
    """dI/dOmega: the trapezoid over the photon energies of a cube [n_omega][n_angles]."""
    import torch
    f64 = torch.float64
    n_omega = _numel(hbar_omega_eV)
    return load().rad_angular_distribution(_dev_ptr(cube, f64, "cube"), _dev_ptr(hbar_omega_eV, f64, "hbar_omega_eV"),
                                           n_omega, _numel(out), _dev_ptr(out, f64, "out"), _stream(stream))


def crystal_element(element) -> RadElement:
    out = RadElement()
    rc = load().rad_crystal_element(int(element), ctypes.byref(out))
    if rc:
        raise RadError(rc, "rad_crystal_element")
    return out


def crystal_string_lattice(structure, a, axis) -> RadStringLattice:
    out = RadStringLattice()
    rc = load().rad_crystal_string_lattice(int(structure), float(a), int(axis), ctypes.byref(out))
    if rc:
        raise RadError(rc, "rad_crystal_string_lattice")
    return out


def crystal_plane_stack(structure, a, plane) -> RadPlaneStack:
    out = RadPlaneStack()
    rc = load().rad_crystal_plane_stack(int(structure), float(a), int(plane), ctypes.byref(out))
    if rc:
        raise RadError(rc, "rad_crystal_plane_stack")
    return out


class MLP:
    """rad_mlp_* handle: x (n_in) -> depth x [Linear(width) -> GELU] -> Linear(n_out)."""

    def __init__(self, n_in=3, width=256, depth=3, n_out=2048, max_batch=1024, seed=0):
        h = ctypes.c_void_p()
        rc = load().rad_mlp_create(int(n_in), int(width), int(depth), int(n_out), int(max_batch), int(seed),
                                   ctypes.byref(h))
        if rc:
            raise RadError(rc, "rad_mlp_create")
        self._h, self.n_in, self.width, self.depth, self.n_out, self.max_batch = h, n_in, width, depth, n_out, max_batch

    @property
    def num_params(self) -> int:
        return int(load().rad_mlp_num_params(self._h))

    def forward(self, x, y=None, stream=None):
        import torch
        if y is None:
            y = torch.empty((x.shape[0], self.n_out), dtype=torch.float32, device=x.device)
        rc = load().rad_mlp_forward(self._h, _dev_ptr(x, torch.float32, "x"), int(x.shape[0]),
                                    _dev_ptr(y, torch.float32, "y"), _stream(stream))
        if rc:
            raise RadError(rc, "rad_mlp_forward")
        return y

    def backward(self, x, t, loss=None, mask=None, stream=None):
        import torch
        rc = load().rad_mlp_backward(self._h, _dev_ptr(x, torch.float32, "x"), _dev_ptr(t, torch.float32, "t"),
                                     _dev_ptr(mask, torch.float32, "mask"), int(x.shape[0]),
                                     _dev_ptr(loss, torch.float32, "loss"), _stream(stream))
        if rc:
            raise RadError(rc, "rad_mlp_backward")

    def adamw(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, stream=None):
        rc = load().rad_mlp_adamw(self._h, float(lr), float(beta1), float(beta2), float(eps), float(weight_decay),
                                  _stream(stream))
        if rc:
            raise RadError(rc, "rad_mlp_adamw")

    def train_step(self, x, t, lr, weight_decay=0.0, loss=None, mask=None, stream=None):
        import torch
        rc = load().rad_mlp_train_step(self._h, _dev_ptr(x, torch.float32, "x"), _dev_ptr(t, torch.float32, "t"),
                                       _dev_ptr(mask, torch.float32, "mask"), int(x.shape[0]), float(lr),
                                       float(weight_decay), _dev_ptr(loss, torch.float32, "loss"), _stream(stream))
        if rc:
            raise RadError(rc, "rad_mlp_train_step")

    def get(self, what=0):
        import numpy as np
        out = np.empty(self.num_params, dtype=np.float32)
        rc = load().rad_mlp_get(self._h, int(what), out.ctypes.data_as(ctypes.c_void_p))
        if rc:
            raise RadError(rc, "rad_mlp_get")
        return out

    def set_params(self, params):
        import numpy as np
        a = np.ascontiguousarray(params, dtype=np.float32)
        rc = load().rad_mlp_set_params(self._h, a.ctypes.data_as(ctypes.c_void_p))
        if rc:
            raise RadError(rc, "rad_mlp_set_params")

    def close(self):
        if getattr(self, "_h", None):
            load().rad_mlp_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


def rad_mlp_ensemble_estimate(preds, mean, err, stream=None):
    import torch
    K, B, O = preds.shape
    rc = load().rad_mlp_ensemble_estimate(_dev_ptr(preds, torch.float32, "preds"), int(K), int(B), int(O),
                                          _dev_ptr(mean, torch.float32, "mean"), _dev_ptr(err, torch.float32, "err"),
                                          _stream(stream))
    if rc:
        raise RadError(rc, "rad_mlp_ensemble_estimate")


def rad_log_targets(values, floor_value, out, stream=None):
    import torch
    rc = load().rad_log_targets(_dev_ptr(values, torch.float64, "values"), int(values.numel()), float(floor_value),
                                _dev_ptr(out, torch.float32, "out"), _stream(stream))
    if rc:
        raise RadError(rc, "rad_log_targets")


def rad_column_stats(y, mean, stdv, stream=None):
    import torch
    rc = load().rad_column_stats(_dev_ptr(y, torch.float32, "y"), int(y.shape[0]), int(y.shape[1]),
                                 _dev_ptr(mean, torch.float32, "mean"), _dev_ptr(stdv, torch.float32, "std"),
                                 _stream(stream))
    if rc:
        raise RadError(rc, "rad_column_stats")


def rad_standardize(y, mean, stdv, inverse=False, stream=None):
    import torch
    rc = load().rad_standardize(_dev_ptr(y, torch.float32, "y"), int(y.shape[0]), int(y.shape[1]),
                                _dev_ptr(mean, torch.float32, "mean"), _dev_ptr(stdv, torch.float32, "std"),
                                int(bool(inverse)), _stream(stream))
    if rc:
        raise RadError(rc, "rad_standardize")


def rad_selftest_bounded_wait(stream=None) -> int:
    return load().rad_selftest_bounded_wait(_stream(stream))


def rad_device_status(reset: int = 1) -> int:
    return load().rad_device_status(int(reset))


def rad_status_string(status: int) -> str:
    return load().rad_status_string(int(status)).decode()


def rad_version() -> str:
    return load().rad_version().decode()


def rad_release() -> None:
    load().rad_release()


class Plan:
    """rad_plan_* bound to one shape; execute / autotune / set_shape / graph."""

    def __init__(self, n_samples_total, n_particles, n_omega, n_angles, mode, precision, want=1, n_bins=0):
        lib = load()
        h = ctypes.c_void_p()
        rc = lib.rad_plan_create(int(n_samples_total), int(n_particles), int(n_omega), int(n_angles),
                                 int(mode), int(precision), int(want), int(n_bins), ctypes.byref(h))
        if rc:
            raise RadError(rc, "rad_plan_create")
        self._h = h
        self.n_bins = n_bins

    def _args(self, samples, offsets, gamma, energy_eV, weight, hw, tx, ty, d_omega, out_cube, out_spectrum,
              bin_of_angle, out_bins):
        import torch
        f64 = torch.float64
        return [self._h, _dev_ptr(samples, f64, "samples"), _dev_ptr(offsets, torch.int64, "offsets"),
                _dev_ptr(gamma, f64, "gamma"), _dev_ptr(energy_eV, f64, "energy_eV"),
                _dev_ptr(weight, f64, "weight"), _dev_ptr(hw, f64, "hw"), _dev_ptr(tx, f64, "theta_x"),
                _dev_ptr(ty, f64, "theta_y"), _dev_ptr(d_omega, f64, "d_omega"),
                _dev_ptr(out_cube, f64, "out_cube"), _dev_ptr(out_spectrum, f64, "out_spectrum"),
                _dev_ptr(bin_of_angle, torch.int32, "bin_of_angle"), _dev_ptr(out_bins, f64, "out_bins")]

    def execute(self, *args, accumulate=0, stream=None) -> int:
        return load().rad_plan_execute(*self._args(*args), int(accumulate), _stream(stream))

    def autotune(self, *args, budget_ms=2000, stream=None) -> int:
        return load().rad_plan_autotune(*self._args(*args), int(budget_ms), _stream(stream))

    def set_shape(self, R, NW, T, chunk_mult=1) -> int:
        return load().rad_plan_set_shape(self._h, int(R), int(NW), int(T), int(chunk_mult))

    def set_prepass(self, enable=True) -> int:
        return load().rad_plan_set_prepass(self._h, int(bool(enable)))

    def set_sincos_split(self, every=4) -> int:
        return load().rad_plan_set_sincos_split(self._h, int(every))

    def set_phase_budget(self, radians) -> int:
        return load().rad_plan_set_phase_budget(self._h, float(radians))

    def describe(self) -> str:
        buf = ctypes.create_string_buffer(512)
        load().rad_plan_describe(self._h, buf, 512)
        return buf.value.decode()

    def set_timing(self, enable=True) -> int:
        return load().rad_plan_set_timing(self._h, int(bool(enable)))

    def last_kernel_ms(self) -> float:
        v = ctypes.c_double()
        rc = load().rad_plan_last_kernel_ms(self._h, ctypes.byref(v))
        if rc:
            raise RadError(rc, "rad_plan_last_kernel_ms")
        return v.value

    def kernel_launches(self) -> int:
        return load().rad_plan_kernel_launches(self._h)

    def graph(self, *args, accumulate=0, stream=None) -> "Graph":
        g = ctypes.c_void_p()
        rc = load().rad_graph_create(*self._args(*args), int(accumulate), _stream(stream), ctypes.byref(g))
        if rc:
            raise RadError(rc, "rad_graph_create")
        return Graph(g, self)

    def close(self):
        if getattr(self, "_h", None):
            load().rad_plan_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


class Graph:
    def __init__(self, h, plan):
        self._h = h
        self._plan = plan  # keeps the plan alive

    def launch(self, stream=None) -> int:
        return load().rad_graph_launch(self._h, _stream(stream))

    def close(self):
        if getattr(self, "_h", None):
            load().rad_graph_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------- #
# convenience layer over the same entry points
# --------------------------------------------------------------------------- #
class DeviceInputs:
    """Trajectories and grid as device tensors (from the inputs module's containers)."""

    def __init__(self, traj, grid, device="cuda", bin_of_angle=None, n_bins=0):
        import torch
        dev = torch.device(device)
        t = lambda a, dt=torch.float64: torch.as_tensor(a, dtype=dt).contiguous().to(dev)
        self.samples = t(traj.samples)
        self.offsets = t(traj.offsets, torch.int64)
        self.gamma = t(traj.gamma)
        self.energy = t(traj.energy_eV)
        self.weight = None if traj.weight is None else t(traj.weight)
        self.hw = t(grid.hbar_omega_eV)
        self.tx = t(grid.theta_x)
        self.ty = t(grid.theta_y)
        self.dom = t(grid.d_omega)
        self.boa = None if bin_of_angle is None else t(bin_of_angle, torch.int32)
        self.n_bins = int(n_bins)
        self.n_omega = int(self.hw.numel())
        self.n_angles = int(self.tx.numel())
        self.n_particles = int(self.offsets.numel() - 1)
        self.n_samples = int(self.samples.numel() // RAD_NREC)

    def args(self):
        return (self.samples, self.offsets, self.gamma, self.energy, self.weight, self.hw, self.tx, self.ty,
                self.dom)


def spectrum(inp: DeviceInputs, mode, precision, cube=True, spec=False, bins=False, stream=None):
    """Allocate outputs and run rad_spectrum; returns dict of device tensors (raises RadError)."""
    import torch
    dev = inp.samples.device if inp.samples.numel() else inp.hw.device
    out = {}
    oc = torch.empty(inp.n_omega * inp.n_angles, dtype=torch.float64, device=dev) if cube else None
    os_ = torch.empty(inp.n_omega, dtype=torch.float64, device=dev) if spec else None
    ob = torch.empty(inp.n_omega * max(inp.n_bins, 1), dtype=torch.float64, device=dev) if bins else None
    rc = rad_spectrum(*inp.args(), MODES.get(mode, mode), PRECISIONS.get(precision, precision), oc, os_,
                      inp.boa if bins else None, inp.n_bins if bins else 0, ob, 0, stream)
    if rc:
        raise RadError(rc, "rad_spectrum")
    if cube:
        out["cube"] = oc.view(inp.n_omega, inp.n_angles)
    if spec:
        out["spectrum"] = os_
    if bins:
        out["bins"] = ob.view(inp.n_omega, inp.n_bins)
    return out
