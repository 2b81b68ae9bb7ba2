"""The crystal library's geometry (Sec. IV: strings and planes of FCC-based diamond and BCC
crystals in the <100>, <110>, <111> axes and (100), (110), (111) planes) against a brute-force
projection of the crystal's atoms, done here from the structures' definitions:
  diamond  FCC {(0,0,0), (1/2,1/2,0), (1/2,0,1/2), (0,1/2,1/2)} a plus the same + (1/4,1/4,1/4) a;
  BCC      {(0,0,0), (1/2,1/2,1/2)} a.
For an axis: every atom projects onto one of the library's strings (modulo the cell), every
string holds atoms, the atoms along a string come at mean spacing d, and
n_strings / (d cell_x cell_y) is the atom density. For a plane family: the projections onto the
normal, modulo the period, are the library's offsets, and each plane's areal density times the
period's count gives the atom density. These are host-only calls of the library (no GPU)."""
import itertools
import math

import numpy as np
import pytest

import paper_1910_10391_gb300 as rad

A = 4.0e-10  # any lattice constant: the geometry scales with it

BASIS = {
    rad.RAD_DIAMOND: np.concatenate([np.array([[0, 0, 0], [.5, .5, 0], [.5, 0, .5], [0, .5, .5]]),
                                     np.array([[0, 0, 0], [.5, .5, 0], [.5, 0, .5], [0, .5, .5]]) + 0.25]),
    rad.RAD_BCC: np.array([[0, 0, 0], [.5, .5, .5]]),
}
DENSITY = {rad.RAD_DIAMOND: 8 / A ** 3, rad.RAD_BCC: 2 / A ** 3}
FRAMES = {  # (x, y, axis) unit vectors of the library's frames
    100: ((0, 1, 0), (0, 0, 1), (1, 0, 0)),
    110: ((0, 0, 1), (1, -1, 0), (1, 1, 0)),
    111: ((1, -1, 0), (1, 1, -2), (1, 1, 1)),
}


def crystal(structure, n=7):
    cells = np.array(list(itertools.product(range(-n, n), repeat=3)), dtype=np.float64)
    return (cells[:, None, :] + BASIS[structure][None]).reshape(-1, 3) * A


@pytest.mark.parametrize("structure", [rad.RAD_DIAMOND, rad.RAD_BCC])
@pytest.mark.parametrize("axis", [100, 110, 111])
def test_string_lattice_matches_the_projected_crystal(structure, axis):
    lat = rad.crystal_string_lattice(structure, A, axis)
    ex, ey, ez = (np.asarray(v, np.float64) / np.linalg.norm(v) for v in FRAMES[axis])
    P = crystal(structure)
    x, y, z = P @ ex, P @ ey, P @ ez
    inner = (np.abs(x) < 3 * A) & (np.abs(y) < 3 * A) & (np.abs(z) < 3 * A)
    sx = np.array(lat.sx[:lat.n_strings])
    sy = np.array(lat.sy[:lat.n_strings])
    # distance (modulo the cell) from each atom to its nearest string
    fx = np.mod(x[inner][:, None] - sx[None, :] + 0.5 * lat.cell_x, lat.cell_x) - 0.5 * lat.cell_x
    fy = np.mod(y[inner][:, None] - sy[None, :] + 0.5 * lat.cell_y, lat.cell_y) - 0.5 * lat.cell_y
    dist = np.hypot(fx, fy)
    assert dist.min(1).max() < 1e-6 * A, "an atom lies off every string"
    which = dist.argmin(1)
    assert set(which) == set(range(lat.n_strings)), "a string holds no atom"
    # atoms per unit length along one line of each string: 1/d
    for k in range(lat.n_strings):
        on = (np.abs(x - sx[k]) < 1e-6 * A) & (np.abs(y - sy[k]) < 1e-6 * A)
        # over a whole number of axial repeats (a, a sqrt 2, a sqrt 3) the count per length is 1/d
        length = 4 * A * math.sqrt(3) if axis == 111 else (4 * A * math.sqrt(2) if axis == 110 else 4 * A)
        cnt = np.sum((z[on] >= -1e-6 * A) & (z[on] < length - 1e-6 * A))
        assert abs(cnt * lat.d / length - 1) < 1e-9, (k, cnt, length / lat.d)
    assert abs(lat.n_strings / (lat.d * lat.cell_x * lat.cell_y) / DENSITY[structure] - 1) < 1e-12


@pytest.mark.parametrize("structure", [rad.RAD_DIAMOND, rad.RAD_BCC])
@pytest.mark.parametrize("plane", [100, 110, 111])
def test_plane_stack_matches_the_projected_crystal(structure, plane):
    st = rad.crystal_plane_stack(structure, A, plane)
    nrm = np.asarray(FRAMES[plane][2], np.float64)
    nrm /= np.linalg.norm(nrm)
    p = crystal(structure) @ nrm
    rel = np.mod(p, st.period)
    rel[np.abs(rel - st.period) < 1e-6 * A] = 0.0
    found = np.unique(np.round(rel / A, 6)) * A
    want = np.sort(np.array(st.offset[:st.n_planes]))
    assert len(found) == st.n_planes and np.allclose(found, want, atol=1e-6 * A, rtol=0)
    # atoms per unit area of each plane: count the atoms of a thick slab, per plane and area
    for k in range(st.n_planes):
        assert abs(st.areal[k] * st.n_planes / st.period / DENSITY[structure] - 1) < 1e-12
        on = np.abs(rel - st.offset[k]) < 1e-6 * A
        assert on.sum() * st.n_planes == pytest.approx(len(p), rel=1e-12)


def test_element_presets_and_argument_checks():
    for el, structure in ((rad.RAD_SI, rad.RAD_DIAMOND), (rad.RAD_C, rad.RAD_DIAMOND), (rad.RAD_GE, rad.RAD_DIAMOND),
                          (rad.RAD_W, rad.RAD_BCC)):
        e = rad.crystal_element(el)
        assert e.structure == structure and 3e-10 < e.a < 6e-10 and e.I_eV > 0 and e.X0 > 0
    # Si (110): d_p = a / (2 sqrt 2) = 1.92 A, the interplanar distance of the channeling workloads
    si = rad.crystal_element(rad.RAD_SI)
    assert rad.crystal_plane_stack(si.structure, si.a, 110).period == pytest.approx(1.92e-10, rel=2e-3)
    lib = rad.load()
    import ctypes
    out = rad.RadStringLattice()
    assert lib.rad_crystal_string_lattice(2, A, 110, ctypes.byref(out)) == rad.RAD_EINVAL
    assert lib.rad_crystal_string_lattice(0, A, 112, ctypes.byref(out)) == rad.RAD_EINVAL
    assert lib.rad_crystal_string_lattice(0, -A, 110, ctypes.byref(out)) == rad.RAD_EINVAL
    assert lib.rad_crystal_plane_stack(0, A, 101, ctypes.byref(rad.RadPlaneStack())) == rad.RAD_EINVAL
    assert lib.rad_crystal_element(9, ctypes.byref(rad.RadElement())) == rad.RAD_EINVAL
