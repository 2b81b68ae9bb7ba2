"""The C-ABI library loads and exports every entry point include/rad.h declares.

No compute call runs here (there is no GPU in this suite); only host-side argument
checks that return before any CUDA work is enqueued.
"""
import ctypes

import pytest

import paper_1910_10391_gb300 as rad


@pytest.fixture(scope="module")
def lib():
    return rad.load()


def test_exports_every_declared_symbol(lib):
    names = rad.header_symbols()
    assert "rad_spectrum" in names and "rad_plan_create" in names and len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    for code in range(7):
        s = rad.rad_status_string(code)
        assert isinstance(s, str) and s
    assert "sm_103a" in rad.rad_version()


def test_invalid_shapes_rejected_before_device_work(lib):
    h = ctypes.c_void_p()
    assert lib.rad_plan_create(-1, 0, 1, 1, 0, 0, 1, 0, ctypes.byref(h)) == rad.RAD_EINVAL
    assert lib.rad_plan_create(0, 0, 1, 1, 7, 0, 1, 0, ctypes.byref(h)) == rad.RAD_EINVAL   # mode
    assert lib.rad_plan_create(0, 0, 1, 1, 0, 9, 1, 0, ctypes.byref(h)) == rad.RAD_EINVAL   # precision
    assert lib.rad_plan_create(0, 0, 1, 1, 0, 0, 4, 0, ctypes.byref(h)) == rad.RAD_EINVAL   # bins need n_bins
    assert lib.rad_plan_create(3, 2, 1, 1, 0, 0, 1, 0, ctypes.byref(h)) == rad.RAD_EINVAL   # < 2 samples each
    assert lib.rad_plan_create(0, 0, 1, 1, 0, 0, 1, 0, None) == rad.RAD_EINVAL
    assert lib.rad_plan_execute(None, *([None] * 13), 0, None) == rad.RAD_EINVAL
    assert lib.rad_graph_launch(None, None) == rad.RAD_EINVAL
    assert lib.rad_plan_set_shape(None, 2, 8, 64, 1) == rad.RAD_EINVAL
    rc = lib.rad_spectrum(None, 0, None, 0, None, None, None, None, 1, None, None, None, 1, 5, 0,
                          None, None, None, 0, None, 0, None)
    assert rc == rad.RAD_EINVAL


def test_trajectory_argument_checks(lib):
    """rad_channeling_trajectories rejects bad host arguments before any device work."""
    ch = rad.RadChannel(20.0, 1.92e-10, 10.6e6, 0.0937, 0.075e-10, 0.51099895e6, 1, rad.RAD_TRAJ_MS)
    P = ctypes.c_void_p(16)  # never dereferenced: every call below fails its host checks
    args = lambda c, n, dt: (c, n, P, 10, P, P, P, None, None, dt, 1, P, None, None)
    assert lib.rad_channeling_trajectories(*args(None, 1, 5e-9)) == rad.RAD_EINVAL
    assert lib.rad_channeling_trajectories(*args(ctypes.byref(ch), -1, 5e-9)) == rad.RAD_EINVAL
    assert lib.rad_channeling_trajectories(*args(ctypes.byref(ch), 1, 0.0)) == rad.RAD_EINVAL
    assert lib.rad_channeling_trajectories(*args(ctypes.byref(ch), 0, 5e-9)) == rad.RAD_OK
    for bad in (dict(flags=16), dict(charge_sign=0), dict(d_p=0.0), dict(mass_eV=-1.0), dict(U0_eV=-1.0),
                dict(rho=0.0), dict(X0=0.0)):
        c2 = rad.RadChannel(20.0, 1.92e-10, 10.6e6, 0.0937, 0.075e-10, 0.51099895e6, 1, rad.RAD_TRAJ_MS)
        for k, v in bad.items():
            setattr(c2, k, v)
        assert lib.rad_channeling_trajectories(*args(ctypes.byref(c2), 1, 5e-9)) == rad.RAD_EINVAL, bad
    r = lib.rad_channeling_trajectories(ctypes.byref(ch), 1, None, 10, P, P, P, None, None, 5e-9, 1, P, None, None)
    assert r == rad.RAD_EINVAL  # null offsets


def test_crystal_trajectory_argument_checks(lib):
    """rad_crystal_trajectories rejects a missing or malformed planar potential, and electron
    scattering without nuclear scattering, before any device work."""
    from paper_1910_10391_gb300 import inputs as I
    flags = rad.RAD_TRAJ_MS | rad.RAD_TRAJ_MS_EL
    ch = rad.RadChannel(0.0, I.SI110_DP, I.EPS_S_EV, I.SI_X0, I.RHO_THERMAL, I.ME_EV, 1, flags)
    good = dict(a=I.SYNTH_DT_A, b=I.SYNTH_DT_B, N=I.SI_N, ax=I.SYNTH_DT_AX, bx=I.SYNTH_DT_BX, cx=I.SYNTH_DT_CX,
                I_eV=I.SI_I_EV)
    pot = rad.RadPlanarPotential.make(**good)
    P = ctypes.c_void_p(16)  # never dereferenced
    call = lambda c, p, n=1: lib.rad_crystal_trajectories(c, p, n, P, 10, P, P, P, None, None, 5e-9, 1, P, None,
                                                          None)
    assert call(ctypes.byref(ch), ctypes.byref(pot), 0) == rad.RAD_OK
    assert call(ctypes.byref(ch), None) == rad.RAD_EINVAL
    assert call(None, ctypes.byref(pot)) == rad.RAD_EINVAL
    for field, v in (("n_terms", 0), ("n_terms", 9), ("n_neighbours", 0), ("n_neighbours", 9), ("N", 0.0),
                     ("I_eV", 0.0), ("cx", float("nan"))):
        p2 = rad.RadPlanarPotential.make(**good)
        setattr(p2, field, v)
        assert call(ctypes.byref(ch), ctypes.byref(p2), 0) == rad.RAD_EINVAL, field
    for arr, v in (("a", float("inf")), ("b", -1.0), ("bx", -1.0), ("ax", float("nan"))):
        p2 = rad.RadPlanarPotential.make(**good)
        getattr(p2, arr)[1] = v
        assert call(ctypes.byref(ch), ctypes.byref(p2), 0) == rad.RAD_EINVAL, arr
    # a fit whose force coefficients overflow FP32 (rho = 0 and a tiny b_i: C_i ~ 1e-40 m^2) is
    # refused in the FP32 form and accepted in FP64, where they are finite
    c0 = rad.RadChannel(0.0, I.SI110_DP, I.EPS_S_EV, I.SI_X0, 0.0, I.ME_EV, 1, 0)
    tiny = rad.RadPlanarPotential.make((1e-10,), (1e-40 * 4 * 3.141592653589793 ** 2,), I.SI_N)
    assert call(ctypes.byref(c0), ctypes.byref(tiny), 0) == rad.RAD_OK
    c0.flags = rad.RAD_TRAJ_FP32
    assert call(ctypes.byref(c0), ctypes.byref(tiny), 0) == rad.RAD_EINVAL
    # C_i = b/(4 pi^2) + rho^2 must be positive: b = 0 is fine while rho > 0
    p2 = rad.RadPlanarPotential.make(**good)
    p2.b[0] = 0.0
    assert call(ctypes.byref(ch), ctypes.byref(p2), 0) == rad.RAD_OK
    # electron scattering needs nuclear scattering; the harmonic entry point does not know the flag
    c2 = rad.RadChannel(0.0, I.SI110_DP, I.EPS_S_EV, I.SI_X0, I.RHO_THERMAL, I.ME_EV, 1, rad.RAD_TRAJ_MS_EL)
    assert call(ctypes.byref(c2), ctypes.byref(pot), 0) == rad.RAD_EINVAL
    assert lib.rad_channeling_trajectories(ctypes.byref(ch), 0, P, 10, P, P, P, None, None, 5e-9, 1, P, None,
                                           None) == rad.RAD_EINVAL
    # without electron scattering the X-ray terms and I are not needed
    c3 = rad.RadChannel(0.0, I.SI110_DP, I.EPS_S_EV, I.SI_X0, I.RHO_THERMAL, I.ME_EV, -1, rad.RAD_TRAJ_MS)
    p3 = rad.RadPlanarPotential.make(I.SYNTH_DT_A, I.SYNTH_DT_B, I.SI_N)
    assert call(ctypes.byref(c3), ctypes.byref(p3), 0) == rad.RAD_OK
    with pytest.raises(ValueError):
        rad.RadPlanarPotential.make((1.0, 2.0), (1.0,), 1.0)


def _declared_parameter_counts():
    """Number of parameters of every function declared in include/rad.h (comments stripped)."""
    import re
    with open(rad._binding.HEADER) as f:
        txt = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
    txt = re.sub(r"//[^\n]*", "", txt)
    counts = {}
    for m in re.finditer(r"\b(rad_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", txt):
        params = m.group(2).strip()
        counts[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return counts


def test_binding_argument_lists_match_the_header(lib):
    """Every declared function the binding gives argument types to takes as many arguments in
    the binding as the header declares (ctypes would otherwise marshal them silently wrong)."""
    counts = _declared_parameter_counts()
    assert len(counts) == len(rad.header_symbols())
    typed = 0
    for name, n in counts.items():
        f = getattr(lib, name)
        if f.argtypes is not None:
            typed += 1
            assert len(f.argtypes) == n, (name, len(f.argtypes), n)
    assert typed >= 30


def test_binding_return_types_match_the_header(lib):
    """int -> c_int, int64_t -> c_int64, const char * -> c_char_p, void -> None."""
    import re
    with open(rad._binding.HEADER) as f:
        txt = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
    kinds = {"int": ctypes.c_int, "int64_t": ctypes.c_int64, "const char *": ctypes.c_char_p, "void": None}
    seen = 0
    for m in re.finditer(r"^\s*(int64_t|int|const char \*|void)\s*(rad_[a-z0-9_]+)\s*\(", txt, flags=re.M):
        ret, name = m.group(1), m.group(2)
        assert getattr(lib, name).restype == kinds[ret], (name, ret, getattr(lib, name).restype)
        seen += 1
    assert seen == len(rad.header_symbols())


def test_noalloc_rejects_oversize_shapes_without_overflow(lib):
    """rad_spectrum_noalloc compares n_omega * n_angles with its fixed scratch without forming a
    product that could overflow: 2^32 x 2^32 (whose int64 product wraps to 0) and other
    oversize shapes return RAD_ETOOBIG before any device work."""
    P = ctypes.c_void_p(256)  # never dereferenced: every call below fails its host checks
    for n_omega, n_angles in ((1 << 32, 1 << 32), (1 << 62, 4), (3, 1 << 62), (4194273, 1), (2048, 4096)):
        rc = lib.rad_spectrum_noalloc(P, 4, P, 2, P, P, None, P, n_omega, P, P, n_angles, 0, P, None)
        assert rc == rad.RAD_ETOOBIG, (n_omega, n_angles, rc)
    assert lib.rad_spectrum_noalloc(P, 4, P, 2, P, P, None, P, -1, P, P, 4, 0, P, None) == rad.RAD_EINVAL
    assert lib.rad_spectrum_noalloc(P, 4, P, 2, P, P, None, P, 4, P, P, 4, 7, P, None) == rad.RAD_EINVAL
