// Crystal geometry of the trajectory integrators (Sec. IV): where the strings of an axis and the
// planes of a plane family of a cubic crystal lie, and element presets. Host code only.
//
// Structures, in units of the cubic lattice constant a:
//   diamond  the FCC lattice {(0,0,0), (1/2,1/2,0), (1/2,0,1/2), (0,1/2,1/2)} plus the same
//            shifted by (1/4,1/4,1/4): 8 atoms per cubic cell (Si, C, Ge);
//   BCC      {(0,0,0), (1/2,1/2,1/2)}: 2 atoms per cubic cell (W).
// Strings: atoms projected along the axis onto the transverse plane, reduced to the smallest
// rectangular cell of the projected pattern; d is the cell's axial repeat length divided by the
// atoms each string holds in it. Planes: atoms projected onto the normal, reduced to the
// smallest repeat length. The tables below are these projections worked out by hand; every
// entry satisfies n_strings / (d cell_x cell_y) = atoms per volume (8/a^3, 2/a^3) and
// sum(areal) / period = atoms per volume.
#include <math.h>

#include "../../include/rad.h"

namespace {

struct Lat {
  int n;
  double cx, cy;  // cell in units of a
  double sx[4], sy[4];
  double d;
};

const double kS2 = 1.41421356237309504880;  // sqrt 2
const double kS3 = 1.73205080756887729353;  // sqrt 3
const double kS6 = 2.44948974278317809820;  // sqrt 6

// diamond: <100> square cell a/2, strings at the corner and the centre-quarter, atoms a apart;
// <110> cell a x a/sqrt 2 with two dumbbells of strings a/4 apart, atoms a/sqrt 2 apart;
// <111> the FCC strings (the basis atom lies on the same [111] line), a triangular lattice of
// spacing a/sqrt 6 in a rectangular cell a/sqrt 2 x a/sqrt 6, two atoms per a sqrt 3.
const Lat kDiamond[3] = {
    {2, 0.5, 0.5, {0.0, 0.25}, {0.0, 0.25}, 1.0},
    {4, 1.0, 1.0 / kS2, {0.0, 0.25, 0.5, 0.75}, {0.0, 0.0, 0.5 / kS2, 0.5 / kS2}, 1.0 / kS2},
    {2, 1.0 / kS2, 1.0 / kS6, {0.0, 0.5 / kS2}, {0.0, 0.5 / kS6}, 0.5 * kS3},
};
// BCC: <100> cell a x a with the body-centre string, atoms a apart; <110> one string per
// a/2 x a/sqrt 2 cell, atoms a sqrt 2 apart; <111> a triangular lattice of spacing a sqrt(2/3),
// atoms a sqrt 3 / 2 apart.
const Lat kBcc[3] = {
    {2, 1.0, 1.0, {0.0, 0.5}, {0.0, 0.5}, 1.0},
    {1, 0.5, 1.0 / kS2, {0.0}, {0.0}, kS2},
    {2, kS2, kS2 / kS3, {0.0, 1.0 / kS2}, {0.0, 1.0 / kS6}, 0.5 * kS3},
};

struct Stack {
  int n;
  double period;       // units of a
  double offset[2];    // units of a
  double areal[2];     // units of 1/a^2
};

// diamond (100): a/4 apart, 2/a^2 each; (110): a/(2 sqrt 2) apart, 2 sqrt 2 / a^2; (111): pairs,
// a period of a/sqrt 3 holding planes at 0 and a sqrt 3 / 4, 4/(sqrt 3 a^2) each.
const Stack kDiamondPlanes[3] = {
    {1, 0.25, {0.0, 0.0}, {2.0, 0.0}},
    {1, 0.5 / kS2, {0.0, 0.0}, {2.0 * kS2, 0.0}},
    {2, 1.0 / kS3, {0.0, 0.25 * kS3}, {4.0 / kS3, 4.0 / kS3}},
};
// BCC (100): a/2 apart, 1/a^2; (110): a/sqrt 2 apart, sqrt 2 / a^2; (111): a/(2 sqrt 3) apart,
// 1/(sqrt 3 a^2).
const Stack kBccPlanes[3] = {
    {1, 0.5, {0.0, 0.0}, {1.0, 0.0}},
    {1, 1.0 / kS2, {0.0, 0.0}, {kS2, 0.0}},
    {1, 0.5 / kS3, {0.0, 0.0}, {1.0 / kS3, 0.0}},
};

int index_of(int hkl) { return hkl == 100 ? 0 : hkl == 110 ? 1 : hkl == 111 ? 2 : -1; }

}  // namespace

extern "C" int rad_crystal_element(int element, rad_element *out) {
  if (!out) return RAD_EINVAL;
  // lattice constants at room temperature; I and X0 as tabulated for the solids
  switch (element) {
    case RAD_SI: *out = rad_element{RAD_DIAMOND, 5.431e-10, 14, 173.0, 0.0937}; return RAD_OK;
    case RAD_C: *out = rad_element{RAD_DIAMOND, 3.567e-10, 6, 81.0, 0.1213}; return RAD_OK;
    case RAD_GE: *out = rad_element{RAD_DIAMOND, 5.658e-10, 32, 350.0, 0.02301}; return RAD_OK;
    case RAD_W: *out = rad_element{RAD_BCC, 3.165e-10, 74, 727.0, 0.003504}; return RAD_OK;
    default: return RAD_EINVAL;
  }
}

extern "C" int rad_crystal_string_lattice(int structure, double a, int axis, rad_string_lattice *out) {
  const int k = index_of(axis);
  if (!out || k < 0 || !(a > 0.0) || !isfinite(a) || (structure != RAD_DIAMOND && structure != RAD_BCC))
    return RAD_EINVAL;
  const Lat &L = structure == RAD_DIAMOND ? kDiamond[k] : kBcc[k];
  rad_string_lattice r{};
  r.n_strings = L.n;
  r.cell_x = L.cx * a;
  r.cell_y = L.cy * a;
  for (int i = 0; i < L.n; ++i) {
    r.sx[i] = L.sx[i] * a;
    r.sy[i] = L.sy[i] * a;
  }
  r.d = L.d * a;
  *out = r;
  return RAD_OK;
}

extern "C" int rad_crystal_plane_stack(int structure, double a, int plane, rad_plane_stack *out) {
  const int k = index_of(plane);
  if (!out || k < 0 || !(a > 0.0) || !isfinite(a) || (structure != RAD_DIAMOND && structure != RAD_BCC))
    return RAD_EINVAL;
  const Stack &S = structure == RAD_DIAMOND ? kDiamondPlanes[k] : kBccPlanes[k];
  rad_plane_stack r{};
  r.n_planes = S.n;
  r.period = S.period * a;
  for (int i = 0; i < S.n; ++i) {
    r.offset[i] = S.offset[i] * a;
    r.areal[i] = S.areal[i] / (a * a);
  }
  *out = r;
  return RAD_OK;
}
