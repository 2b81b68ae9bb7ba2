"""GB300-native (sm_103a) library for the radiation integral of arXiv:1910.10391.

The compute path is the CUDA library ``librad.so`` (C ABI in include/rad.h),
reached through the thin ctypes binding in ``_binding``; ``inputs`` creates
seeded synthetic trajectories and grids. Importing this package does not load
CUDA; the first call of an ``rad_*`` function loads (and if needed builds) the
library, and raises if it cannot.
"""
from ._binding import (  # noqa: F401
    MODES, PRECISIONS, RAD_CLASSICAL, RAD_ECUDA, RAD_EDATA, RAD_EINVAL, RAD_ENOMEM, RAD_ETIMEOUT,
    RAD_EPRECISION, RAD_ETOOBIG, RAD_EUNSUPPORTED, RAD_FP64, RAD_FP64_DF, RAD_MIXED, RAD_NREC, RAD_OK, RAD_PER_PARTICLE, RAD_SPIN0, RAD_SPIN_HALF, RAD_TRAJ_FP32,
    RAD_TRAJ_LL, RAD_TRAJ_MS, RAD_TRAJ_MS_EL, RAD_TRAJ_MS_LOSS, DeviceInputs, Graph, MLP, Plan, RadChannel, RadError,
    RadPlanarPotential, RadAxialPotential, RadStringLattice, RadPlaneStack, RadElement, RAD_DIAMOND, RAD_BCC, RAD_SI,
    RAD_C, RAD_GE, RAD_W, RadStepControl, rad_trajectories_adaptive, rad_angular_distribution, rad_axial_trajectories, crystal_element, crystal_string_lattice, crystal_plane_stack,
    header_symbols, load, rad_channeling_trajectories, rad_crystal_trajectories, rad_column_stats, rad_device_status, rad_log_targets,
    rad_mlp_ensemble_estimate, rad_release, rad_selftest_bounded_wait, rad_spectrum, rad_spectrum_host,
    rad_spectrum_noalloc, rad_spectrum_particles, rad_standardize, rad_status_string, rad_version, spectrum)
