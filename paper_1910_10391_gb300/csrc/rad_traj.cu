// Planar-channeling trajectories on the GPU (Sec. III): one thread integrates one particle
// with classical RK4 steps and writes the records the radiation kernels consume (Sec. II
// variables), so an ensemble goes from entry conditions to spectra without leaving HBM.
//
// Model (harmonic stand-in for the planar continuum potential, c = 1, metres, eV):
//   U(s) = U0 (2 s / d_p)^2, s = distance to the nearest channel centre (positrons: mid-way
//   between planes; electrons: on the planes); F = -8 U0 s / d_p^2;
//   dx/dt = v_x, dy/dt = v_y, dv_x/dt = F / E, dv_y/dt = 0, d(dz)/dt = v_z - beta0,
//   beta0 := 1 - 1/(2 gamma0^2) (entry energy), v_z = sqrt(1 - 1/gamma^2 - v_perp^2);
//   optional radiation-reaction drag (leading Landau-Lifshitz term for a static transverse
//   field): dE/dt = -(2/3) alpha hbar c gamma^2 F^2 / m^2;
//   optional multiple scattering on nuclei after every step: Gaussian kicks of both angles
//   with variance (1/2)(eps_s/E)^2 (dt/X0) n(x)/N, n(x)/N the Gaussian plane density of the
//   two nearest planes; the next sample's acceleration carries the kick as delta_v/dt; with
//   scattering loss each kick costs m alpha/(2 pi) gamma^3 theta^2.
// Doyle-Turner form (rad_crystal_trajectories): the harmonic well is replaced by the thermally
// averaged continuum potential of the planes at x = m d_p (Sec. III, Eq. plane), summed over the
// 2K planes around the particle's cell: F = sum_planes sum_i fk_i r exp(-r^2 / C_i) (in FP64 by a
// geometric walk outward from the nearest plane, three exponentials per term) with
// fk_i = 2 q (2 sqrt(pi) e^2 a0 N d_p) a_i / C_i^(3/2), C_i = b_i/(4 pi^2) + rho^2; with electron
// scattering the kick variance gains (1/2) dt pi r0^2 / (gamma^2 beta^4) [ln(2 m_e gamma^2
// beta^2 / I) - beta^2]_+ n_el(x) (Sec. III), n_el from the X-ray Gaussians of the same planes
// plus c^X times the nuclear density.
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with counter
// (particle low, step, 1, particle high) and key (seed low, seed high); two 53-bit uniforms
// per block and Box-Muller normals.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "rad_internal.cuh"

namespace rad {
namespace {

struct Chan {
  double U0, d_p, eps_s, X0, rho, mass, centre, inv_d, force_k, dens_pref, inv_rho2, var_k, loss_k, ll_k;
  int ms, ll, ms_loss;
};

constexpr int kMaxTerms = 8;
constexpr double kR0 = 2.8179403262e-15;  // classical electron radius, m (CODATA 2018)
constexpr double kMe = 0.51099895e6;      // electron rest energy, eV (target electrons)
constexpr double kA0 = 5.29177210903e-11; // Bohr radius, m (CODATA 2018)

// Doyle-Turner planar potential, FP64 form. Force terms fk[i] r exp(-r^2 ck[i]); electron-
// density terms ek[i] exp(-r^2 eck[i]) and ecx n(x)/N, all pre-multiplied by (1/2) dt pi r0^2.
struct Planar {
  int nt, K, el;
  double fk[kMaxTerms], ck[kMaxTerms], q[kMaxTerms], ek[kMaxTerms], eck[kMaxTerms];
  double ecx, lk;  // q = exp(-2 ck d_p^2); lk = 2 m_e / I
};

// ---------------- Philox4x32-10 ----------------
__device__ __forceinline__ void philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
  const uint64_t m = (static_cast<uint64_t>(a >> 5) << 26) | static_cast<uint64_t>(b >> 6);
  return (static_cast<double>(m) + 0.5) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ void kick_normals(uint64_t seed, uint64_t pid, uint64_t step, double &z0, double &z1) {
  uint32_t c[4] = {static_cast<uint32_t>(pid), static_cast<uint32_t>(step), 1u, static_cast<uint32_t>(pid >> 32)};
  philox(c, static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
  const double u1 = u53(c[0], c[1]), u2 = u53(c[2], c[3]);
  const double r = sqrt(-2.0 * log(u1));
  double s, co;
  sincospi(2.0 * u2, &s, &co);
  z0 = r * co;
  z1 = r * s;
}

// ---------------- field ----------------
__device__ __forceinline__ double force(const Chan &C, double x) {
  const double u = (x - C.centre) * C.inv_d;
  const double s = (u - floor(u + 0.5)) * C.d_p;
  return C.force_k * s;  // -8 U0 s / d_p^2
}

__device__ __forceinline__ double plane_density(const Chan &C, double x) {
  const double m = floor(x * C.inv_d);
  const double r1 = x - m * C.d_p, r2 = (m + 1.0) * C.d_p - x;
  return C.dens_pref * (exp(-(r1 * r1) * C.inv_rho2) + exp(-(r2 * r2) * C.inv_rho2));
}

// The 2K planes of the particle's cell (xi = x - floor(x/d_p) d_p in [0, d_p); plane j at distance
// xi - j d_p, j = 1-K .. K), walked outward from the nearest one, at distance r (|r| <= d_p/2).
// Along the planes each Gaussian is geometric in its ratios: with E_m = exp(-k (r - m d)^2),
// E_{m+1}/E_m = exp(k (2 (r - m d) d - d^2)) and successive ratios differ by the factor
// q = exp(-2 k d^2). So a term costs three exponentials (the nearest plane and the first ratio
// each way, all <= 1) and products, instead of one exponential per plane. The ratios' large
// arguments only touch terms already below exp(-k d^2/4) of the nearest one.
__device__ __forceinline__ double planar_force(const Chan &C, const Planar &P, double x) {
  const double d = C.d_p;
  const double xi = x - floor(x * C.inv_d) * d;
  const bool low = xi < 0.5 * d;
  const double r = low ? xi : xi - d;
  const int n_up = low ? P.K : P.K - 1;  // planes at r - m d, m = 1 .. n_up
  const int n_dn = low ? P.K - 1 : P.K;  // planes at r + m d, m = 1 .. n_dn
  double F = 0.0;
  for (int i = 0; i < P.nt; ++i) {
    const double k = P.ck[i], q = P.q[i];
    const double E0 = exp(-(r * r) * k);
    double s = r * E0;
    double E = E0, rho = exp(k * (2.0 * r * d - d * d)), rm = r;
    for (int m = 0; m < n_up; ++m) {
      E *= rho;
      rho *= q;
      rm -= d;
      s += rm * E;
    }
    E = E0;
    rho = exp(-k * (2.0 * r * d + d * d));
    rm = r;
    for (int m = 0; m < n_dn; ++m) {
      E *= rho;
      rho *= q;
      rm += d;
      s += rm * E;
    }
    F += P.fk[i] * s;
  }
  return F;
}

// (1/2) dt pi r0^2 n_el(x): the X-ray Gaussians of the 2K planes plus c^X N n(x)/N
__device__ __forceinline__ double electron_density_scaled(const Chan &C, const Planar &P, double x, double n_nuc) {
  const double xi = x - floor(x * C.inv_d) * C.d_p;
  double n = P.ecx * n_nuc;
  for (int j = 1 - P.K; j <= P.K; ++j) {
    const double r = xi - j * C.d_p, r2 = r * r;
    for (int i = 0; i < P.nt; ++i) n += P.ek[i] * exp(-r2 * P.eck[i]);
  }
  return n;
}

template <bool DT>
__device__ __forceinline__ double field(const Chan &C, const Planar &P, double x) {
  if constexpr (DT) return planar_force(C, P, x);
  else return force(C, x);
}

// v_z - beta0 without cancellation: ((1/g0^2 - 1/g^2) - vp2 - 1/(4 g0^4)) / (v_z + beta0)
__device__ __forceinline__ double dvz_of(double g, double g0, double q0, double beta0, double vp2, double &vz) {
  vz = sqrt(1.0 - 1.0 / (g * g) - vp2);
  const double d_inv = ((g - g0) * (g + g0)) / ((g * g) * (g0 * g0));
  return (d_inv - vp2 - q0) / (vz + beta0);
}

struct State {
  double x, y, vx, vy, dz, E;
};

template <bool DT>
__device__ __forceinline__ State deriv(const Chan &C, const Planar &P, double g0, double q0, double beta0,
                                       const State &s) {
  const double g = s.E / C.mass;
  const double vp2 = s.vx * s.vx + s.vy * s.vy;
  double vz;
  const double dvz = dvz_of(g, g0, q0, beta0, vp2, vz);
  const double F = field<DT>(C, P, s.x);
  State d;
  d.x = s.vx;
  d.y = s.vy;
  d.vx = F / s.E;
  d.vy = 0.0;
  d.dz = dvz;
  d.E = C.ll ? C.ll_k * (g * g) * (F * F) : 0.0;
  return d;
}

__device__ __forceinline__ State axpy(const State &s, double h, const State &d) {
  return State{s.x + h * d.x, s.y + h * d.y, s.vx + h * d.vx, s.vy + h * d.vy, s.dz + h * d.dz, s.E + h * d.E};
}

template <bool DT>
__global__ void k_channel(const Chan C, const Planar P, int64_t n_particles, const int64_t *__restrict__ offsets,
                          int64_t n_total, const double *__restrict__ energy, const double *__restrict__ x0,
                          const double *__restrict__ thx0, const double *__restrict__ thy0,
                          const int64_t *__restrict__ ids, double dt, uint64_t seed, double *__restrict__ out,
                          double *__restrict__ e_out, int *dev_status) {
  for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < n_particles;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t off = offsets[p], L = offsets[p + 1] - off;
    const double E0 = energy[p];
    if (off < 0 || L < 1 || off + L > n_total || !(E0 > C.mass) || !isfinite(E0) || !isfinite(x0[p]) ||
        !isfinite(thx0[p]) || (thy0 && !isfinite(thy0[p]))) {
      atomicCAS(dev_status, 0, RAD_EDATA);
      continue;
    }
    const uint64_t pid = ids ? static_cast<uint64_t>(ids[p]) : static_cast<uint64_t>(p);
    const double g0 = E0 / C.mass;
    const double beta0 = 1.0 - 1.0 / (2.0 * g0 * g0);
    const double q0 = 1.0 / (4.0 * (g0 * g0) * (g0 * g0));
    State s{x0[p], 0.0, thx0[p], thy0 ? thy0[p] : 0.0, 0.0, E0};
    double kx = 0.0, ky = 0.0;
    double *rec = out + off * kRec;
    for (int64_t k = 0; k < L; ++k, rec += kRec) {
      // record k
      const double g = s.E / C.mass;
      const double vp2 = s.vx * s.vx + s.vy * s.vy;
      double vz;
      const double dvz = dvz_of(g, g0, q0, beta0, vp2, vz);
      const double F = field<DT>(C, P, s.x);
      const double ax = F / s.E + kx, ay = ky;
      const double gdot = C.ll ? C.ll_k * (g * g) * (F * F) / C.mass : 0.0;
      rec[F_T] = static_cast<double>(k) * dt;
      rec[F_X] = s.x;
      rec[F_Y] = s.y;
      rec[F_DZ] = s.dz;
      rec[F_VX] = s.vx;
      rec[F_VY] = s.vy;
      rec[F_DVZ] = dvz;
      rec[F_AX] = ax;
      rec[F_AY] = ay;
      rec[F_AZ] = (gdot / (g * g * g) - (s.vx * ax + s.vy * ay)) / vz;
      if (e_out) e_out[off + k] = s.E;
      kx = ky = 0.0;
      if (k == L - 1) break;
      // RK4 step
      const State k1 = deriv<DT>(C, P, g0, q0, beta0, s);
      const State k2 = deriv<DT>(C, P, g0, q0, beta0, axpy(s, 0.5 * dt, k1));
      const State k3 = deriv<DT>(C, P, g0, q0, beta0, axpy(s, 0.5 * dt, k2));
      const State k4 = deriv<DT>(C, P, g0, q0, beta0, axpy(s, dt, k3));
      const double h6 = dt / 6.0;
      s.x += h6 * (k1.x + 2.0 * k2.x + 2.0 * k3.x + k4.x);
      s.y += h6 * (k1.y + 2.0 * k2.y + 2.0 * k3.y + k4.y);
      s.vx += h6 * (k1.vx + 2.0 * k2.vx + 2.0 * k3.vx + k4.vx);
      s.vy += h6 * (k1.vy + 2.0 * k2.vy + 2.0 * k3.vy + k4.vy);
      s.dz += h6 * (k1.dz + 2.0 * k2.dz + 2.0 * k3.dz + k4.dz);
      s.E += h6 * (k1.E + 2.0 * k2.E + 2.0 * k3.E + k4.E);
      if (C.ms) {
        const double E = s.E;
        const double n_nuc = plane_density(C, s.x);
        double var = C.var_k / (E * E) * n_nuc;
        if (DT && P.el) {
          const double g = E / C.mass, b2 = 1.0 - 1.0 / (g * g);
          const double br = fmax(log(P.lk * (g * g) * b2) - b2, 0.0);
          var += electron_density_scaled(C, P, s.x, n_nuc) * (br / ((g * g) * (b2 * b2)));
        }
        double z0, z1;
        kick_normals(seed, pid, static_cast<uint64_t>(k), z0, z1);
        const double sd = sqrt(var);
        const double dthx = sd * z0, dthy = sd * z1;
        kx = dthx / dt;
        ky = dthy / dt;
        s.vx += dthx;
        s.vy += dthy;
        if (C.ms_loss) {
          const double gk = E / C.mass;
          s.E = E - C.loss_k * (gk * gk * gk) * (dthx * dthx + dthy * dthy);
        }
      }
    }
  }
}

// ------------------------------------------------------------------------------------
// Axial channeling (rad_axial_trajectories): strings of atoms along the axis (Sec. III, Eq.
// string), FP64. The strings of the (2K+1)^2 cells around the particle's cell are summed; each
// string's Gaussian exp(-(dx^2 + dy^2)/C) separates into exp(-dx^2/C) exp(-dy^2/C), and the
// cells of one basis string form a product grid, so the double sum over the cells is a product
// of two sums of 2K+1 terms, each walked outward from the nearest image with three exponentials:
// 6 per basis string and term instead of (2K+1)^2.
// ------------------------------------------------------------------------------------
struct Axial {
  int nt, nb, K, el;
  double Lx, Ly;
  double sx[8], sy[8];
  double fk[kMaxTerms];  // q (2 e^2 a0 / d) (a_i / C_i) (2 / C_i)
  double ck[kMaxTerms];  // 1 / C_i
  double qx[kMaxTerms], qy[kMaxTerms];    // exp(-2 L^2 / C_i) along x and y
  double eqx[kMaxTerms], eqy[kMaxTerms];  // the same for the electron terms (1 / CX_i)
  double rqx, rqy;                         // the same for the nuclear density (1 / rho^2)
  double dens_k;         // 1 / (pi rho^2 N d): n(x, y)/N per unit Gaussian
  double inv_rho2;
  double ek[kMaxTerms], eck[kMaxTerms];  // (1/2) dt pi r0^2 ax_i / (pi d CX_i), 1 / CX_i
  double ecx, lk;                        // (1/2) dt pi r0^2 cx N; 2 m_e / I
};

// sums over the 2K+1 images u_i = u0 - i L (i = -K .. K) of one coordinate: s1 = sum u e^{-u^2 k},
// s0 = sum e^{-u^2 k}, with |u0| < L. Walked outward from the nearest image r = u0 - i0 L
// (|r| <= L/2), as in the planar form: the Gaussian of the next image is the current one times a
// ratio, and successive ratios differ by the factor q = exp(-2 k L^2), so one axis costs three
// exponentials (the nearest image and the first ratio each way, all <= 1) instead of 2K+1.
__device__ __forceinline__ void axis_sums(double u0, double L, int K, double k, double q, double &s1, double &s0) {
  const int i0 = u0 > 0.5 * L ? 1 : (u0 < -0.5 * L ? -1 : 0);
  const double r = u0 - static_cast<double>(i0) * L;
  const double E0 = exp(-(r * r) * k);
  s1 = r * E0;
  s0 = E0;
  double E = E0, rho = exp(k * (2.0 * r * L - L * L)), u = r;
  for (int m = 0; m < K - i0; ++m) {  // images i0 + 1 .. K at r - m L
    E *= rho;
    rho *= q;
    u -= L;
    s1 += u * E;
    s0 += E;
  }
  E = E0;
  rho = exp(-k * (2.0 * r * L + L * L));
  u = r;
  for (int m = 0; m < K + i0; ++m) {  // images i0 - 1 .. -K at r + m L
    E *= rho;
    rho *= q;
    u += L;
    s1 += u * E;
    s0 += E;
  }
}

__device__ __forceinline__ void axial_force(const Axial &A, double x, double y, double &Fx, double &Fy) {
  const double cx = floor(x / A.Lx), cy = floor(y / A.Ly);
  Fx = 0.0;
  Fy = 0.0;
  for (int b = 0; b < A.nb; ++b) {
    // offsets from the strings of the particle's own cell; the images follow at -i L
    const double ux = x - (cx * A.Lx + A.sx[b]);
    const double uy = y - (cy * A.Ly + A.sy[b]);
    for (int t = 0; t < A.nt; ++t) {
      double sx1, sx0, sy1, sy0;
      axis_sums(ux, A.Lx, A.K, A.ck[t], A.qx[t], sx1, sx0);
      axis_sums(uy, A.Ly, A.K, A.ck[t], A.qy[t], sy1, sy0);
      Fx += A.fk[t] * (sx1 * sy0);
      Fy += A.fk[t] * (sx0 * sy1);
    }
  }
}

// n(x, y)/N and, with electron scattering, (1/2) dt pi r0^2 n_el(x, y)
__device__ __forceinline__ void axial_densities(const Axial &A, double x, double y, double &n_nuc, double &n_el) {
  const double cx = floor(x / A.Lx), cy = floor(y / A.Ly);
  double nn = 0.0, ne = 0.0;
  for (int b = 0; b < A.nb; ++b) {
    const double ux = x - (cx * A.Lx + A.sx[b]);
    const double uy = y - (cy * A.Ly + A.sy[b]);
    double s1, sx0, sy0;
    axis_sums(ux, A.Lx, A.K, A.inv_rho2, A.rqx, s1, sx0);
    axis_sums(uy, A.Ly, A.K, A.inv_rho2, A.rqy, s1, sy0);
    nn += sx0 * sy0;
    if (A.el) {
      for (int t = 0; t < A.nt; ++t) {
        axis_sums(ux, A.Lx, A.K, A.eck[t], A.eqx[t], s1, sx0);
        axis_sums(uy, A.Ly, A.K, A.eck[t], A.eqy[t], s1, sy0);
        ne += A.ek[t] * (sx0 * sy0);
      }
    }
  }
  n_nuc = A.dens_k * nn;
  n_el = ne + A.ecx * n_nuc;
}

__device__ __forceinline__ State deriv_axial(const Chan &C, const Axial &A, double g0, double q0, double beta0,
                                             const State &s) {
  const double g = s.E / C.mass;
  const double vp2 = s.vx * s.vx + s.vy * s.vy;
  double vz;
  const double dvz = dvz_of(g, g0, q0, beta0, vp2, vz);
  double Fx, Fy;
  axial_force(A, s.x, s.y, Fx, Fy);
  State d;
  d.x = s.vx;
  d.y = s.vy;
  d.vx = Fx / s.E;
  d.vy = Fy / s.E;
  d.dz = dvz;
  d.E = C.ll ? C.ll_k * (g * g) * (Fx * Fx + Fy * Fy) : 0.0;
  return d;
}

// Small ensembles: one particle per group of kGroup lanes. The lanes share the force evaluation
// (each takes some of the (basis string, term) pairs, the partial forces are summed by a butterfly
// of shuffles within the group) and keep identical copies of the state, so a step's exponentials
// run kGroup-wide instead of on one lane; 1024 particles then fill 16384 lanes instead of 1024.
// The groups of a warp may diverge (different lengths): every shuffle names its own group's lanes.
constexpr int kGroup = 16;
// below this many particles the lane-group kernel runs (16 lanes each); above, one lane each. One
// lane per particle keeps the FP64 pipe busy from about one warp per SM sub-partition on; the
// groups repeat the state update in every lane, so they pay only while the one-lane kernel has
// fewer warps than that (measured on 2048-step Si <110> ensembles: 4096 particles 0.55 s against
// 1.01 s, 8192 0.94 s against 1.02 s, 16384 1.85 s against 1.11 s)
constexpr int64_t kGroupBelow = 9216;

// the sum over the group, identical in every lane (the butterfly adds in a different order in
// each lane, so the group's first lane's sum is broadcast: the lanes' states stay bit-identical)
__device__ __forceinline__ double group_sum(double v, unsigned mask) {
#pragma unroll
  for (int o = kGroup / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, kGroup);
  return __shfl_sync(mask, v, 0, kGroup);
}

__device__ __forceinline__ void axial_force_group(const Axial &A, double x, double y, int gl, unsigned mask,
                                                  double &Fx, double &Fy) {
  const double cx = floor(x / A.Lx), cy = floor(y / A.Ly);
  double fx = 0.0, fy = 0.0;
  for (int q = gl; q < A.nb * A.nt; q += kGroup) {
    const int b = q / A.nt, t = q - b * A.nt;
    const double ux = x - (cx * A.Lx + A.sx[b]);
    const double uy = y - (cy * A.Ly + A.sy[b]);
    double sx1, sx0, sy1, sy0;
    axis_sums(ux, A.Lx, A.K, A.ck[t], A.qx[t], sx1, sx0);
    axis_sums(uy, A.Ly, A.K, A.ck[t], A.qy[t], sy1, sy0);
    fx += A.fk[t] * (sx1 * sy0);
    fy += A.fk[t] * (sx0 * sy1);
  }
  Fx = group_sum(fx, mask);
  Fy = group_sum(fy, mask);
}

__device__ __forceinline__ void axial_densities_group(const Axial &A, double x, double y, int gl, unsigned mask,
                                                      double &n_nuc, double &n_el) {
  const double cx = floor(x / A.Lx), cy = floor(y / A.Ly);
  double nn = 0.0, ne = 0.0, s1, sx0, sy0;
  for (int b = gl; b < A.nb; b += kGroup) {
    axis_sums(x - (cx * A.Lx + A.sx[b]), A.Lx, A.K, A.inv_rho2, A.rqx, s1, sx0);
    axis_sums(y - (cy * A.Ly + A.sy[b]), A.Ly, A.K, A.inv_rho2, A.rqy, s1, sy0);
    nn += sx0 * sy0;
  }
  if (A.el) {
    for (int q = gl; q < A.nb * A.nt; q += kGroup) {
      const int b = q / A.nt, t = q - b * A.nt;
      axis_sums(x - (cx * A.Lx + A.sx[b]), A.Lx, A.K, A.eck[t], A.eqx[t], s1, sx0);
      axis_sums(y - (cy * A.Ly + A.sy[b]), A.Ly, A.K, A.eck[t], A.eqy[t], s1, sy0);
      ne += A.ek[t] * (sx0 * sy0);
    }
  }
  n_nuc = A.dens_k * group_sum(nn, mask);
  n_el = (A.el ? group_sum(ne, mask) : 0.0) + A.ecx * n_nuc;
}

__device__ __forceinline__ State deriv_axial_group(const Chan &C, const Axial &A, double g0, double q0, double beta0,
                                                   const State &s, int gl, unsigned mask) {
  const double g = s.E / C.mass;
  const double vp2 = s.vx * s.vx + s.vy * s.vy;
  double vz;
  const double dvz = dvz_of(g, g0, q0, beta0, vp2, vz);
  double Fx, Fy;
  axial_force_group(A, s.x, s.y, gl, mask, Fx, Fy);
  State d;
  d.x = s.vx;
  d.y = s.vy;
  d.vx = Fx / s.E;
  d.vy = Fy / s.E;
  d.dz = dvz;
  d.E = C.ll ? C.ll_k * (g * g) * (Fx * Fx + Fy * Fy) : 0.0;
  return d;
}

__global__ void k_axial_group(const Chan C, const Axial A, int64_t n_particles, const int64_t *__restrict__ offsets,
                              int64_t n_total, const double *__restrict__ energy, const double *__restrict__ x0,
                              const double *__restrict__ y0, const double *__restrict__ thx0,
                              const double *__restrict__ thy0, const int64_t *__restrict__ ids, double dt,
                              uint64_t seed, double *__restrict__ out, double *__restrict__ e_out, int *dev_status) {
  const int gl = threadIdx.x & (kGroup - 1);
  const unsigned mask = 0xFFFFu << (threadIdx.x & 16);
  const int64_t groups = static_cast<int64_t>(gridDim.x) * (blockDim.x / kGroup);
  for (int64_t p = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / kGroup; p < n_particles;
       p += groups) {
    const int64_t off = offsets[p], L = offsets[p + 1] - off;
    const double E0 = energy[p];
    if (off < 0 || L < 1 || off + L > n_total || !(E0 > C.mass) || !isfinite(E0) || !isfinite(x0[p]) ||
        (y0 && !isfinite(y0[p])) || !isfinite(thx0[p]) || (thy0 && !isfinite(thy0[p]))) {
      if (gl == 0) atomicCAS(dev_status, 0, RAD_EDATA);
      continue;
    }
    const uint64_t pid = ids ? static_cast<uint64_t>(ids[p]) : static_cast<uint64_t>(p);
    const double g0 = E0 / C.mass;
    const double beta0 = 1.0 - 1.0 / (2.0 * g0 * g0);
    const double q0 = 1.0 / (4.0 * (g0 * g0) * (g0 * g0));
    State s{x0[p], y0 ? y0[p] : 0.0, thx0[p], thy0 ? thy0[p] : 0.0, 0.0, E0};
    double kx = 0.0, ky = 0.0;
    double *rec = out + off * kRec;
    for (int64_t k = 0; k < L; ++k, rec += kRec) {
      const double g = s.E / C.mass;
      const double vp2 = s.vx * s.vx + s.vy * s.vy;
      double vz;
      const double dvz = dvz_of(g, g0, q0, beta0, vp2, vz);
      double Fx, Fy;
      axial_force_group(A, s.x, s.y, gl, mask, Fx, Fy);
      const double ax = Fx / s.E + kx, ay = Fy / s.E + ky;
      const double gdot = C.ll ? C.ll_k * (g * g) * (Fx * Fx + Fy * Fy) / C.mass : 0.0;
      // every lane holds the record; lane f writes field f
      double v = 0.0;
      switch (gl) {
        case F_T: v = static_cast<double>(k) * dt; break;
        case F_X: v = s.x; break;
        case F_Y: v = s.y; break;
        case F_DZ: v = s.dz; break;
        case F_VX: v = s.vx; break;
        case F_VY: v = s.vy; break;
        case F_DVZ: v = dvz; break;
        case F_AX: v = ax; break;
        case F_AY: v = ay; break;
        case F_AZ: v = (gdot / (g * g * g) - (s.vx * ax + s.vy * ay)) / vz; break;
        default: break;
      }
      if (gl < kRec) rec[gl] = v;
      if (e_out && gl == 0) e_out[off + k] = s.E;
      kx = ky = 0.0;
      if (k == L - 1) break;
      const State k1 = deriv_axial_group(C, A, g0, q0, beta0, s, gl, mask);
      const State k2 = deriv_axial_group(C, A, g0, q0, beta0, axpy(s, 0.5 * dt, k1), gl, mask);
      const State k3 = deriv_axial_group(C, A, g0, q0, beta0, axpy(s, 0.5 * dt, k2), gl, mask);
      const State k4 = deriv_axial_group(C, A, g0, q0, beta0, axpy(s, dt, k3), gl, mask);
      const double h6 = dt / 6.0;
      s.x += h6 * (k1.x + 2.0 * k2.x + 2.0 * k3.x + k4.x);
      s.y += h6 * (k1.y + 2.0 * k2.y + 2.0 * k3.y + k4.y);
      s.vx += h6 * (k1.vx + 2.0 * k2.vx + 2.0 * k3.vx + k4.vx);
      s.vy += h6 * (k1.vy + 2.0 * k2.vy + 2.0 * k3.vy + k4.vy);
      s.dz += h6 * (k1.dz + 2.0 * k2.dz + 2.0 * k3.dz + k4.dz);
      s.E += h6 * (k1.E + 2.0 * k2.E + 2.0 * k3.E + k4.E);
      if (C.ms) {
        const double E = s.E;
        double n_nuc, n_el;
        axial_densities_group(A, s.x, s.y, gl, mask, n_nuc, n_el);
        double var = C.var_k / (E * E) * n_nuc;
        if (A.el) {
          const double ge = E / C.mass, b2 = 1.0 - 1.0 / (ge * ge);
          const double br = fmax(log(A.lk * (ge * ge) * b2) - b2, 0.0);
          var += n_el * (br / ((ge * ge) * (b2 * b2)));
        }
        double z0, z1;
        kick_normals(seed, pid, static_cast<uint64_t>(k), z0, z1);
        const double sd = sqrt(var);
        const double dthx = sd * z0, dthy = sd * z1;
        kx = dthx / dt;
        ky = dthy / dt;
        s.vx += dthx;
        s.vy += dthy;
        if (C.ms_loss) {
          const double gk = E / C.mass;
          s.E = E - C.loss_k * (gk * gk * gk) * (dthx * dthx + dthy * dthy);
        }
      }
    }
  }
}

// Small ensembles in the Doyle-Turner planar potential: one particle per group of kPGroup lanes, as
// k_axial_group. The force's 2 nt walks (each term's planes above and below the particle, see
// planar_force) are spread over the lanes (one each for the usual 4 terms), and so are the
// electron density's (plane, term) pairs; the group's first lane draws the scattering kick and
// broadcasts it.
constexpr int kPGroup = 8;
static_assert(kRec == 10 && F_AX == 7 && F_AY == 8 && F_AZ == 9 && kPGroup == 8,
              "k_channel_group writes record field f from lane f, fields 8 and 9 from lanes 0 and 1");
// below this many particles the planar lane-group kernel runs
constexpr int64_t kPGroupBelow = 4096;

__device__ __forceinline__ double pgroup_sum(double v, unsigned mask) {
#pragma unroll
  for (int o = kPGroup / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, kPGroup);
  return __shfl_sync(mask, v, 0, kPGroup);
}
__device__ __forceinline__ double planar_force_group(const Chan &C, const Planar &P, double x, int gl,
                                                     unsigned mask) {
  const double d = C.d_p;
  const double xi = x - floor(x * C.inv_d) * d;
  const bool low = xi < 0.5 * d;
  const double r = low ? xi : xi - d;
  double F = 0.0;
  for (int c = gl; c < 2 * P.nt; c += kPGroup) {
    const int i = c >> 1;
    const bool up = (c & 1) == 0;  // planes at r - m d (up) or r + m d (down), m = 1 .. n
    const int n = up ? (low ? P.K : P.K - 1) : (low ? P.K - 1 : P.K);
    const double k = P.ck[i], q = P.q[i];
    const double E0 = exp(-(r * r) * k);
    double s = up ? r * E0 : 0.0;  // the nearest plane counted once, by the upward walk
    double E = E0, rm = r;
    double rho = up ? exp(k * (2.0 * r * d - d * d)) : exp(-k * (2.0 * r * d + d * d));
    const double step = up ? -d : d;
    for (int m = 0; m < n; ++m) {
      E *= rho;
      rho *= q;
      rm += step;
      s += rm * E;
    }
    F += P.fk[i] * s;
  }
  return pgroup_sum(F, mask);
}

// the X-ray Gaussians' part of electron_density_scaled (without the c^X n(x)/N term)
__device__ __forceinline__ double electron_density_group(const Chan &C, const Planar &P, double x, int gl,
                                                         unsigned mask) {
  const double xi = x - floor(x * C.inv_d) * C.d_p;
  double n = 0.0;
  for (int q = gl; q < 2 * P.K * P.nt; q += kPGroup) {
    const int jj = q / P.nt, i = q - jj * P.nt;
    const double r = xi - (jj + 1 - P.K) * C.d_p, r2 = r * r;
    n += P.ek[i] * exp(-r2 * P.eck[i]);
  }
  return pgroup_sum(n, mask);
}

__device__ __forceinline__ State deriv_planar_group(const Chan &C, const Planar &P, double g0, double q0,
                                                    double beta0, const State &s, int gl, unsigned mask) {
  const double g = s.E / C.mass;
  const double vp2 = s.vx * s.vx + s.vy * s.vy;
  double vz;
  const double dvz = dvz_of(g, g0, q0, beta0, vp2, vz);
  const double F = planar_force_group(C, P, s.x, gl, mask);
  State d;
  d.x = s.vx;
  d.y = s.vy;
  d.vx = F / s.E;
  d.vy = 0.0;
  d.dz = dvz;
  d.E = C.ll ? C.ll_k * (g * g) * (F * F) : 0.0;
  return d;
}

__global__ void k_channel_group(const Chan C, const Planar P, int64_t n_particles, const int64_t *__restrict__ offsets,
                                int64_t n_total, const double *__restrict__ energy, const double *__restrict__ x0,
                                const double *__restrict__ thx0, const double *__restrict__ thy0,
                                const int64_t *__restrict__ ids, double dt, uint64_t seed, double *__restrict__ out,
                                double *__restrict__ e_out, int *dev_status) {
  const int gl = threadIdx.x & (kPGroup - 1);
  const unsigned mask = 0xFFu << (threadIdx.x & 24);
  const int64_t groups = static_cast<int64_t>(gridDim.x) * (blockDim.x / kPGroup);
  for (int64_t p = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / kPGroup; p < n_particles;
       p += groups) {
    const int64_t off = offsets[p], L = offsets[p + 1] - off;
    const double E0 = energy[p];
    if (off < 0 || L < 1 || off + L > n_total || !(E0 > C.mass) || !isfinite(E0) || !isfinite(x0[p]) ||
        !isfinite(thx0[p]) || (thy0 && !isfinite(thy0[p]))) {
      if (gl == 0) atomicCAS(dev_status, 0, RAD_EDATA);
      continue;
    }
    const uint64_t pid = ids ? static_cast<uint64_t>(ids[p]) : static_cast<uint64_t>(p);
    const double g0 = E0 / C.mass;
    const double beta0 = 1.0 - 1.0 / (2.0 * g0 * g0);
    const double q0 = 1.0 / (4.0 * (g0 * g0) * (g0 * g0));
    State s{x0[p], 0.0, thx0[p], thy0 ? thy0[p] : 0.0, 0.0, E0};
    double kx = 0.0, ky = 0.0;
    double *rec = out + off * kRec;
    for (int64_t k = 0; k < L; ++k, rec += kRec) {
      const double g = s.E / C.mass;
      const double vp2 = s.vx * s.vx + s.vy * s.vy;
      double vz;
      const double dvz = dvz_of(g, g0, q0, beta0, vp2, vz);
      const double F = planar_force_group(C, P, s.x, gl, mask);
      const double ax = F / s.E + kx, ay = ky;
      const double gdot = C.ll ? C.ll_k * (g * g) * (F * F) / C.mass : 0.0;
      // every lane holds the record; lane f writes field f, lanes 0 and 1 also fields 8 and 9
      const double az = (gdot / (g * g * g) - (s.vx * ax + s.vy * ay)) / vz;
      double v = 0.0;
      switch (gl) {
        case F_T: v = static_cast<double>(k) * dt; break;
        case F_X: v = s.x; break;
        case F_Y: v = s.y; break;
        case F_DZ: v = s.dz; break;
        case F_VX: v = s.vx; break;
        case F_VY: v = s.vy; break;
        case F_DVZ: v = dvz; break;
        default: v = ax; break;  // F_AX = 7, the last lane of the group
      }
      rec[gl] = v;
      if (gl < kRec - kPGroup) rec[gl + kPGroup] = gl == 0 ? ay : az;  // F_AY = 8, F_AZ = 9
      if (e_out && gl == 0) e_out[off + k] = s.E;
      kx = ky = 0.0;
      if (k == L - 1) break;
      const State k1 = deriv_planar_group(C, P, g0, q0, beta0, s, gl, mask);
      const State k2 = deriv_planar_group(C, P, g0, q0, beta0, axpy(s, 0.5 * dt, k1), gl, mask);
      const State k3 = deriv_planar_group(C, P, g0, q0, beta0, axpy(s, 0.5 * dt, k2), gl, mask);
      const State k4 = deriv_planar_group(C, P, g0, q0, beta0, axpy(s, dt, k3), gl, mask);
      const double h6 = dt / 6.0;
      s.x += h6 * (k1.x + 2.0 * k2.x + 2.0 * k3.x + k4.x);
      s.y += h6 * (k1.y + 2.0 * k2.y + 2.0 * k3.y + k4.y);
      s.vx += h6 * (k1.vx + 2.0 * k2.vx + 2.0 * k3.vx + k4.vx);
      s.vy += h6 * (k1.vy + 2.0 * k2.vy + 2.0 * k3.vy + k4.vy);
      s.dz += h6 * (k1.dz + 2.0 * k2.dz + 2.0 * k3.dz + k4.dz);
      s.E += h6 * (k1.E + 2.0 * k2.E + 2.0 * k3.E + k4.E);
      if (C.ms) {
        const double E = s.E;
        const double ne = P.el ? electron_density_group(C, P, s.x, gl, mask) : 0.0;
        double dthx = 0.0, dthy = 0.0;
        if (gl == 0) {  // the kick, drawn once per group
          const double n_nuc = plane_density(C, s.x);
          double var = C.var_k / (E * E) * n_nuc;
          if (P.el) {
            const double ge = E / C.mass, b2 = 1.0 - 1.0 / (ge * ge);
            const double br = fmax(log(P.lk * (ge * ge) * b2) - b2, 0.0);
            var += (P.ecx * n_nuc + ne) * (br / ((ge * ge) * (b2 * b2)));
          }
          double z0, z1;
          kick_normals(seed, pid, static_cast<uint64_t>(k), z0, z1);
          const double sd = sqrt(var);
          dthx = sd * z0;
          dthy = sd * z1;
        }
        dthx = __shfl_sync(mask, dthx, 0, kPGroup);
        dthy = __shfl_sync(mask, dthy, 0, kPGroup);
        kx = dthx / dt;
        ky = dthy / dt;
        s.vx += dthx;
        s.vy += dthy;
        if (C.ms_loss) {
          const double gk = E / C.mass;
          s.E = E - C.loss_k * (gk * gk * gk) * (dthx * dthx + dthy * dthy);
        }
      }
    }
  }
}

__global__ void k_axial(const Chan C, const Axial A, int64_t n_particles, const int64_t *__restrict__ offsets,
                        int64_t n_total, const double *__restrict__ energy, const double *__restrict__ x0,
                        const double *__restrict__ y0, const double *__restrict__ thx0,
                        const double *__restrict__ thy0, const int64_t *__restrict__ ids, double dt, uint64_t seed,
                        double *__restrict__ out, double *__restrict__ e_out, int *dev_status) {
  for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < n_particles;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t off = offsets[p], L = offsets[p + 1] - off;
    const double E0 = energy[p];
    if (off < 0 || L < 1 || off + L > n_total || !(E0 > C.mass) || !isfinite(E0) || !isfinite(x0[p]) ||
        (y0 && !isfinite(y0[p])) || !isfinite(thx0[p]) || (thy0 && !isfinite(thy0[p]))) {
      atomicCAS(dev_status, 0, RAD_EDATA);
      continue;
    }
    const uint64_t pid = ids ? static_cast<uint64_t>(ids[p]) : static_cast<uint64_t>(p);
    const double g0 = E0 / C.mass;
    const double beta0 = 1.0 - 1.0 / (2.0 * g0 * g0);
    const double q0 = 1.0 / (4.0 * (g0 * g0) * (g0 * g0));
    State s{x0[p], y0 ? y0[p] : 0.0, thx0[p], thy0 ? thy0[p] : 0.0, 0.0, E0};
    double kx = 0.0, ky = 0.0;
    double *rec = out + off * kRec;
    for (int64_t k = 0; k < L; ++k, rec += kRec) {
      const double g = s.E / C.mass;
      const double vp2 = s.vx * s.vx + s.vy * s.vy;
      double vz;
      const double dvz = dvz_of(g, g0, q0, beta0, vp2, vz);
      double Fx, Fy;
      axial_force(A, s.x, s.y, Fx, Fy);
      const double ax = Fx / s.E + kx, ay = Fy / s.E + ky;
      const double gdot = C.ll ? C.ll_k * (g * g) * (Fx * Fx + Fy * Fy) / C.mass : 0.0;
      rec[F_T] = static_cast<double>(k) * dt;
      rec[F_X] = s.x;
      rec[F_Y] = s.y;
      rec[F_DZ] = s.dz;
      rec[F_VX] = s.vx;
      rec[F_VY] = s.vy;
      rec[F_DVZ] = dvz;
      rec[F_AX] = ax;
      rec[F_AY] = ay;
      rec[F_AZ] = (gdot / (g * g * g) - (s.vx * ax + s.vy * ay)) / vz;
      if (e_out) e_out[off + k] = s.E;
      kx = ky = 0.0;
      if (k == L - 1) break;
      const State k1 = deriv_axial(C, A, g0, q0, beta0, s);
      const State k2 = deriv_axial(C, A, g0, q0, beta0, axpy(s, 0.5 * dt, k1));
      const State k3 = deriv_axial(C, A, g0, q0, beta0, axpy(s, 0.5 * dt, k2));
      const State k4 = deriv_axial(C, A, g0, q0, beta0, axpy(s, dt, k3));
      const double h6 = dt / 6.0;
      s.x += h6 * (k1.x + 2.0 * k2.x + 2.0 * k3.x + k4.x);
      s.y += h6 * (k1.y + 2.0 * k2.y + 2.0 * k3.y + k4.y);
      s.vx += h6 * (k1.vx + 2.0 * k2.vx + 2.0 * k3.vx + k4.vx);
      s.vy += h6 * (k1.vy + 2.0 * k2.vy + 2.0 * k3.vy + k4.vy);
      s.dz += h6 * (k1.dz + 2.0 * k2.dz + 2.0 * k3.dz + k4.dz);
      s.E += h6 * (k1.E + 2.0 * k2.E + 2.0 * k3.E + k4.E);
      if (C.ms) {
        const double E = s.E;
        double n_nuc, n_el;
        axial_densities(A, s.x, s.y, n_nuc, n_el);
        double var = C.var_k / (E * E) * n_nuc;
        if (A.el) {
          const double ge = E / C.mass, b2 = 1.0 - 1.0 / (ge * ge);
          const double br = fmax(log(A.lk * (ge * ge) * b2) - b2, 0.0);
          var += n_el * (br / ((ge * ge) * (b2 * b2)));
        }
        double z0, z1;
        kick_normals(seed, pid, static_cast<uint64_t>(k), z0, z1);
        const double sd = sqrt(var);
        const double dthx = sd * z0, dthy = sd * z1;
        kx = dthx / dt;
        ky = dthy / dt;
        s.vx += dthx;
        s.vy += dthy;
        if (C.ms_loss) {
          const double gk = E / C.mass;
          s.E = E - C.loss_k * (gk * gk * gk) * (dthx * dthx + dthy * dthy);
        }
      }
    }
  }
}

// ------------------------------------------------------------------------------------
// Adaptive steps between caller-set output times (rad_trajectories_adaptive; Sec. IV: an RK45
// solver with step-size control and a lower bound on the step). Each output interval H is
// integrated with Dormand-Prince 5(4) sub-steps H / 2^m (J. R. Dormand, P. J. Prince, J. Comput.
// Appl. Math. 6 (1980) 19): a sub-step whose embedded error estimate exceeds 1 is repeated at half
// the size unless m is the lower bound max_level, where it is kept; after an accepted sub-step with
// error below 2^-6 the size doubles when the position is a multiple of the doubled size. The
// position is an integer count of H / 2^max_level, so each interval ends exactly at its output
// time, and the level carries over to the next interval. Error: RMS over (x, y, v_x, v_y, dz, E)
// of (y5 - y4) / (atol_i + rtol max(|y_i|, |y5_i|)), atol = (atol_x, atol_x, atol_v, atol_v,
// atol_x, 0). Field kinds: 0 harmonic well, 1 Doyle-Turner planes, 2 axial strings.
// ------------------------------------------------------------------------------------
struct StepCtl {
  double rtol, atol_x, atol_v;
  int max_level;
  int64_t max_substeps;
};

// KIND 0 harmonic, 1 planar (Doyle-Turner), 2 axial; G: one particle per lane group (kPGroup lanes
// for the planar field, kGroup for the axial one; gl the lane within the group, mask the group's
// lanes), as k_channel_group and k_axial_group
template <int KIND, bool G>
__device__ __forceinline__ void field2(const Chan &C, const Planar &P, const Axial &A, double x, double y, double &Fx,
                                       double &Fy, int gl, unsigned mask) {
  if constexpr (KIND == 2) {
    if constexpr (G) axial_force_group(A, x, y, gl, mask, Fx, Fy);
    else axial_force(A, x, y, Fx, Fy);
  } else {
    if constexpr (G && KIND == 1) Fx = planar_force_group(C, P, x, gl, mask);
    else Fx = field<KIND == 1>(C, P, x);
    Fy = 0.0;
  }
}

template <int KIND, bool G>
__device__ __forceinline__ State deriv2(const Chan &C, const Planar &P, const Axial &A, double g0, double q0,
                                        double beta0, const State &s, int gl, unsigned mask) {
  const double g = s.E / C.mass;
  const double vp2 = s.vx * s.vx + s.vy * s.vy;
  double vz;
  const double dvz = dvz_of(g, g0, q0, beta0, vp2, vz);
  double Fx, Fy;
  field2<KIND, G>(C, P, A, s.x, s.y, Fx, Fy, gl, mask);
  State d;
  d.x = s.vx;
  d.y = s.vy;
  d.vx = Fx / s.E;
  d.vy = Fy / s.E;
  d.dz = dvz;
  d.E = C.ll ? C.ll_k * (g * g) * (Fx * Fx + Fy * Fy) : 0.0;
  return d;
}

__device__ __forceinline__ void acc(State &y, double c, const State &k) {
  y.x += c * k.x;
  y.y += c * k.y;
  y.vx += c * k.vx;
  y.vy += c * k.vy;
  y.dz += c * k.dz;
  y.E += c * k.E;
}

__device__ __forceinline__ double err_term(double e, double y, double y5, double atol, double rtol) {
  const double sc = atol + rtol * fmax(fabs(y), fabs(y5));
  const double r = e / sc;
  return r * r;
}

// one Dormand-Prince step: y5 (the solution) and the error estimate's RMS
template <int KIND, bool G>
__device__ __forceinline__ double dp5(const Chan &C, const Planar &P, const Axial &A, double g0, double q0,
                                      double beta0, const StepCtl &S, const State &y, double h, State &y5, int gl,
                                      unsigned mask) {
  constexpr double a21 = 1.0 / 5.0;
  constexpr double a31 = 3.0 / 40.0, a32 = 9.0 / 40.0;
  constexpr double a41 = 44.0 / 45.0, a42 = -56.0 / 15.0, a43 = 32.0 / 9.0;
  constexpr double a51 = 19372.0 / 6561.0, a52 = -25360.0 / 2187.0, a53 = 64448.0 / 6561.0, a54 = -212.0 / 729.0;
  constexpr double a61 = 9017.0 / 3168.0, a62 = -355.0 / 33.0, a63 = 46732.0 / 5247.0, a64 = 49.0 / 176.0,
                   a65 = -5103.0 / 18656.0;
  constexpr double b1 = 35.0 / 384.0, b3 = 500.0 / 1113.0, b4 = 125.0 / 192.0, b5 = -2187.0 / 6784.0,
                   b6 = 11.0 / 84.0;
  // embedded (fourth-order) weights
  constexpr double e1 = 5179.0 / 57600.0, e3 = 7571.0 / 16695.0, e4 = 393.0 / 640.0, e5 = -92097.0 / 339200.0,
                   e6 = 187.0 / 2100.0, e7 = 1.0 / 40.0;
  const State k1 = deriv2<KIND, G>(C, P, A, g0, q0, beta0, y, gl, mask);
  State t = y;
  acc(t, h * a21, k1);
  const State k2 = deriv2<KIND, G>(C, P, A, g0, q0, beta0, t, gl, mask);
  t = y;
  acc(t, h * a31, k1);
  acc(t, h * a32, k2);
  const State k3 = deriv2<KIND, G>(C, P, A, g0, q0, beta0, t, gl, mask);
  t = y;
  acc(t, h * a41, k1);
  acc(t, h * a42, k2);
  acc(t, h * a43, k3);
  const State k4 = deriv2<KIND, G>(C, P, A, g0, q0, beta0, t, gl, mask);
  t = y;
  acc(t, h * a51, k1);
  acc(t, h * a52, k2);
  acc(t, h * a53, k3);
  acc(t, h * a54, k4);
  const State k5 = deriv2<KIND, G>(C, P, A, g0, q0, beta0, t, gl, mask);
  t = y;
  acc(t, h * a61, k1);
  acc(t, h * a62, k2);
  acc(t, h * a63, k3);
  acc(t, h * a64, k4);
  acc(t, h * a65, k5);
  const State k6 = deriv2<KIND, G>(C, P, A, g0, q0, beta0, t, gl, mask);
  y5 = y;
  acc(y5, h * b1, k1);
  acc(y5, h * b3, k3);
  acc(y5, h * b4, k4);
  acc(y5, h * b5, k5);
  acc(y5, h * b6, k6);
  const State k7 = deriv2<KIND, G>(C, P, A, g0, q0, beta0, y5, gl, mask);
  State y4 = y;
  acc(y4, h * e1, k1);
  acc(y4, h * e3, k3);
  acc(y4, h * e4, k4);
  acc(y4, h * e5, k5);
  acc(y4, h * e6, k6);
  acc(y4, h * e7, k7);
  double s2 = err_term(y5.x - y4.x, y.x, y5.x, S.atol_x, S.rtol);
  s2 += err_term(y5.y - y4.y, y.y, y5.y, S.atol_x, S.rtol);
  s2 += err_term(y5.vx - y4.vx, y.vx, y5.vx, S.atol_v, S.rtol);
  s2 += err_term(y5.vy - y4.vy, y.vy, y5.vy, S.atol_v, S.rtol);
  s2 += err_term(y5.dz - y4.dz, y.dz, y5.dz, S.atol_x, S.rtol);
  s2 += err_term(y5.E - y4.E, y.E, y5.E, 0.0, S.rtol);
  return sqrt(s2 / 6.0);
}

template <int KIND, bool G>
__global__ void k_adaptive(const Chan C, const Planar P, const Axial A, const StepCtl S, int64_t n_particles,
                           const int64_t *__restrict__ offsets, int64_t n_total, const double *__restrict__ energy,
                           const double *__restrict__ x0, const double *__restrict__ y0,
                           const double *__restrict__ thx0, const double *__restrict__ thy0,
                           const int64_t *__restrict__ ids, const double *__restrict__ times, double dt, uint64_t seed,
                           double *__restrict__ out, double *__restrict__ e_out, int64_t *__restrict__ counts,
                           int *dev_status) {
  constexpr int W = !G ? 1 : (KIND == 2 ? kGroup : kPGroup);  // lanes per particle
  const int gl = static_cast<int>(threadIdx.x) & (W - 1);
  const unsigned mask = W == 1 ? 0u : (((1u << W) - 1u) << (threadIdx.x & 31 & ~(W - 1)));
  const int64_t stride = static_cast<int64_t>(gridDim.x) * (blockDim.x / W);
  for (int64_t p = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / W; p < n_particles; p += stride) {
    const int64_t off = offsets[p], L = offsets[p + 1] - off;
    const double E0 = energy[p];
    if (off < 0 || L < 1 || off + L > n_total || !(E0 > C.mass) || !isfinite(E0) || !isfinite(x0[p]) ||
        (y0 && !isfinite(y0[p])) || !isfinite(thx0[p]) || (thy0 && !isfinite(thy0[p]))) {
      if (gl == 0) atomicCAS(dev_status, 0, RAD_EDATA);
      continue;
    }
    const double *tp = times ? times + off : nullptr;
    auto t_of = [&](int64_t k) { return tp ? tp[k] : static_cast<double>(k) * dt; };
    bool bad_t = false;
    for (int64_t k = 0; k < L && tp; ++k)
      if (!isfinite(tp[k]) || (k > 0 && !(tp[k] > tp[k - 1]))) bad_t = true;
    if (bad_t) {
      if (gl == 0) atomicCAS(dev_status, 0, RAD_EDATA);
      continue;
    }
    const uint64_t pid = ids ? static_cast<uint64_t>(ids[p]) : static_cast<uint64_t>(p);
    const double g0 = E0 / C.mass;
    const double beta0 = 1.0 - 1.0 / (2.0 * g0 * g0);
    const double q0 = 1.0 / (4.0 * (g0 * g0) * (g0 * g0));
    State s{x0[p], y0 ? y0[p] : 0.0, thx0[p], thy0 ? thy0[p] : 0.0, 0.0, E0};
    double kx = 0.0, ky = 0.0;
    int level = 0;
    int64_t n_steps = 0, n_tries = 0;  // accepted sub-steps; all sub-steps (accepted or repeated)
    const int64_t unit = int64_t(1) << S.max_level;
    double *rec = out + off * kRec;
    bool stopped = false;
    for (int64_t k = 0; k < L && !stopped; ++k, rec += kRec) {
      const double g = s.E / C.mass;
      const double vp2 = s.vx * s.vx + s.vy * s.vy;
      double vz;
      const double dvz = dvz_of(g, g0, q0, beta0, vp2, vz);
      double Fx, Fy;
      field2<KIND, G>(C, P, A, s.x, s.y, Fx, Fy, gl, mask);
      const double ax = Fx / s.E + kx, ay = Fy / s.E + ky;
      const double gdot = C.ll ? C.ll_k * (g * g) * (Fx * Fx + Fy * Fy) / C.mass : 0.0;
      const double az = (gdot / (g * g * g) - (s.vx * ax + s.vy * ay)) / vz;
      // every lane of a group holds the record; lane f writes fields f, f + W, ...
      for (int f = gl; f < kRec; f += W) {
        double v;
        switch (f) {
          case F_T: v = t_of(k); break;
          case F_X: v = s.x; break;
          case F_Y: v = s.y; break;
          case F_DZ: v = s.dz; break;
          case F_VX: v = s.vx; break;
          case F_VY: v = s.vy; break;
          case F_DVZ: v = dvz; break;
          case F_AX: v = ax; break;
          case F_AY: v = ay; break;
          default: v = az; break;
        }
        rec[f] = v;
      }
      if (e_out && gl == 0) e_out[off + k] = s.E;
      kx = ky = 0.0;
      if (k == L - 1) break;
      const double H = t_of(k + 1) - t_of(k);
      int64_t pos = 0;
      while (pos < unit) {
        if (n_tries >= S.max_substeps) {  // the particle needs more sub-steps than allowed
          if (gl == 0) atomicCAS(dev_status, 0, RAD_EDATA);
          stopped = true;
          break;
        }
        const double h = H / static_cast<double>(int64_t(1) << level);
        State y5;
        const double err = dp5<KIND, G>(C, P, A, g0, q0, beta0, S, s, h, y5, gl, mask);
        ++n_tries;
        if (err > 1.0 && level < S.max_level) {
          ++level;
          continue;
        }
        s = y5;
        pos += int64_t(1) << (S.max_level - level);
        ++n_steps;
        if (err < 0.015625 && level > 0 && (pos % (int64_t(1) << (S.max_level - level + 1))) == 0) --level;
      }
      if (stopped) break;
      if (C.ms) {
        const double E = s.E;
        double n_nuc, n_el;
        if constexpr (KIND == 2) {
          if constexpr (G) axial_densities_group(A, s.x, s.y, gl, mask, n_nuc, n_el);
          else axial_densities(A, s.x, s.y, n_nuc, n_el);
        } else {
          n_nuc = plane_density(C, s.x);
          if constexpr (G && KIND == 1)
            n_el = P.el ? P.ecx * n_nuc + electron_density_group(C, P, s.x, gl, mask) : 0.0;
          else
            n_el = (KIND == 1 && P.el) ? electron_density_scaled(C, P, s.x, n_nuc) : 0.0;
        }
        // variances per unit length (the coefficients are built for a unit step), times H
        double var = C.var_k / (E * E) * n_nuc * H;
        const bool el = (KIND == 2) ? (A.el != 0) : (KIND == 1 && P.el);
        if (el) {
          const double lk = (KIND == 2) ? A.lk : P.lk;
          const double ge = E / C.mass, b2 = 1.0 - 1.0 / (ge * ge);
          const double br = fmax(log(lk * (ge * ge) * b2) - b2, 0.0);
          var += n_el * (br / ((ge * ge) * (b2 * b2))) * H;
        }
        double z0, z1;
        kick_normals(seed, pid, static_cast<uint64_t>(k), z0, z1);
        const double sd = sqrt(var);
        const double dthx = sd * z0, dthy = sd * z1;
        const double w = (k + 2 < L) ? 0.5 * (t_of(k + 2) - t_of(k)) : H;
        kx = dthx / w;
        ky = dthy / w;
        s.vx += dthx;
        s.vy += dthy;
        if (C.ms_loss) {
          const double gk = E / C.mass;
          s.E = E - C.loss_k * (gk * gk * gk) * (dthx * dthx + dthy * dthy);
        }
      }
    }
    if (counts && gl == 0) counts[p] = n_steps;
  }
}

// ------------------------------------------------------------------------------------
// Mixed precision (RAD_TRAJ_FP32): FP32 arithmetic with double-float state
// ------------------------------------------------------------------------------------
// GB300 issues FP32 at 64x its FP64 rate (72x measured), so this form evaluates the RK4 stages in
// FP32 and keeps every state variable as an unevaluated sum hi + lo of two floats (about 48
// bits), updated with error-free transformations (Knuth's two-sum, FMA two-product). The position is
// kept as (channel index m, offset s from the channel centre) so that s stays below d_p/2 in
// magnitude however far the particle drifts. The x and y increments h v use a double-float
// product of the step h and the double-float velocity; the other increments are FP32.
// Records are formed in FP64 from the double-float values.
struct Chan32 {
  float d_f, half_d, kf_hi, kf_lo, dt_hi, dt_lo, dt6_hi, dt6_lo, h2_6, h_half, ll_k, loss_k, dens_pref, nexp2_rho,
      var_k, inv_mass;
  double d_p, centre, dt, mass;
  int ms, ll, ms_loss;
};

// Doyle-Turner planar potential, FP32 form: the exponentials as exp2f with -1/(C ln 2) factors.
struct Planar32 {
  int nt, K, el;
  float fk[kMaxTerms], ck2[kMaxTerms], ek[kMaxTerms], eck2[kMaxTerms];
  float ecx, lk;
};

struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_of(double v) {
  const float h = static_cast<float>(v);
  return DF{h, static_cast<float>(v - static_cast<double>(h))};
}

__device__ __forceinline__ double df_val(const DF &a) { return static_cast<double>(a.hi) + static_cast<double>(a.lo); }

// a += d (two-sum, then renormalise)
__device__ __forceinline__ void df_add(DF &a, float d) {
  const float s = __fadd_rn(a.hi, d);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(d, bb));
  const float l = __fadd_rn(a.lo, err);
  const float h2 = __fadd_rn(s, l);
  a.lo = __fsub_rn(l, __fsub_rn(h2, s));
  a.hi = h2;
}

// a += (h_hi + h_lo) * (v.hi + v.lo), the product to about 46 bits (two-product of the high parts)
__device__ __forceinline__ void df_add_prod(DF &a, float h_hi, float h_lo, const DF &v) {
  const float p = __fmul_rn(h_hi, v.hi);
  const float pe = __fmaf_rn(h_hi, v.hi, -p);
  const float tail = __fmaf_rn(h_hi, v.lo, __fmaf_rn(h_lo, v.hi, pe));
  df_add(a, p);
  df_add(a, tail);
}

struct D32 {
  float vx, vy, a, dvz, dE;
};

// Planes relative to the channel centre, from the offset sw in [-d/2, d/2): the 2K planes of the
// cell that holds the particle, as in the FP64 form (positron channels are cells, with planes at
// (j - 1/2) d; an electron channel centre is a plane, and the cell is the one on sw's side).
// The nearest plane's distance sw - p is exact (Sterbenz), so the core of the plane is resolved
// to FP32 precision of the distance itself.
__device__ __forceinline__ void plane_frame(const Chan32 &C, const Planar32 &P, float sw, int &jlo, float &jofs) {
  if (C.centre != 0.0) {
    jlo = 1 - P.K;
    jofs = -0.5f;
  } else {
    jlo = sw >= 0.f ? 1 - P.K : -P.K;
    jofs = 0.f;
  }
}

__device__ __forceinline__ float planar_force32(const Chan32 &C, const Planar32 &P, float sw) {
  int jlo;
  float jofs;
  plane_frame(C, P, sw, jlo, jofs);
  float F = 0.f;
  for (int j = jlo; j < jlo + 2 * P.K; ++j) {
    const float r = sw - (static_cast<float>(j) + jofs) * C.d_f, r2 = r * r;
    float g = 0.f;
    for (int i = 0; i < P.nt; ++i) g = __fmaf_rn(P.fk[i], exp2f(r2 * P.ck2[i]), g);
    F = __fmaf_rn(r, g, F);
  }
  return F;
}

// (1/2) dt pi r0^2 n_el at offset sw, with n_nuc = n(x)/N
__device__ __forceinline__ float electron_density32(const Chan32 &C, const Planar32 &P, float sw, float n_nuc) {
  int jlo;
  float jofs;
  plane_frame(C, P, sw, jlo, jofs);
  float n = P.ecx * n_nuc;
  for (int j = jlo; j < jlo + 2 * P.K; ++j) {
    const float r = sw - (static_cast<float>(j) + jofs) * C.d_f, r2 = r * r;
    for (int i = 0; i < P.nt; ++i) n = __fmaf_rn(P.ek[i], exp2f(r2 * P.eck2[i]), n);
  }
  return n;
}

// stage derivative at offset s (any value; wrapped into the channel), velocity (vx, vy), energy
// offset dEoff from the entry energy E0 (for 1/gamma0^2 - 1/gamma^2), reciprocal of the step's
// energy (iE_hi, iE_lo) and the stage's energy change within the step dEs (radiation reaction:
// 1/(E + dEs) = (1/E)(1 - dEs/E) to first order, dEs/E ~ 1e-7)
template <bool DT>
__device__ __forceinline__ D32 deriv32(const Chan32 &C, const Planar32 &P, float s, float vx, float vy,
                                       float dEoff, float dEs, float g, float g0, float q0, float iE_hi,
                                       float iE_lo) {
  float sw = s;
  if (sw >= C.half_d) sw -= C.d_f;
  else if (sw < -C.half_d) sw += C.d_f;
  float F;
  if constexpr (DT) F = planar_force32(C, P, sw);
  else F = -__fmaf_rn(C.kf_hi, sw, C.kf_lo * sw);  // -8 U0 s / d_p^2, eV/m
  D32 d;
  d.vx = vx;
  d.vy = vy;
  // F (iE_hi + iE_lo)(1 - dEs/E), rounded once: the exact product F iE_hi inside the outer FMA
  const float corr = __fmaf_rn(-(F * iE_hi), dEs * iE_hi, F * iE_lo);
  d.a = __fmaf_rn(F, iE_hi, corr);
  // v_z - beta0 = ((1/g0^2 - 1/g^2) - v_perp^2 - 1/(4 g0^4)) / (v_z + beta0), with
  // v_z + beta0 = 2 - O(1e-8): the FP32 quotient is half the numerator
  const float dg = dEoff * C.inv_mass;  // gamma - gamma0
  const float dinv = (dg * (g + g0)) / ((g * g) * (g0 * g0));
  d.dvz = 0.5f * (dinv - __fmaf_rn(vx, vx, vy * vy) - q0);
  d.dE = C.ll ? C.ll_k * (g * g) * (F * F) : 0.f;
  return d;
}

template <bool DT>
__global__ void k_channel_mixed(const Chan32 C, const Planar32 P, int64_t n_particles, const int64_t *__restrict__ offsets,
                                int64_t n_total, const double *__restrict__ energy, const double *__restrict__ x0,
                                const double *__restrict__ thx0, const double *__restrict__ thy0,
                                const int64_t *__restrict__ ids, uint64_t seed, double *__restrict__ out,
                                double *__restrict__ e_out, int *dev_status) {
  for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < n_particles;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t off = offsets[p], L = offsets[p + 1] - off;
    const double E0 = energy[p];
    if (off < 0 || L < 1 || off + L > n_total || !(E0 > C.mass) || !isfinite(E0) || !isfinite(x0[p]) ||
        !isfinite(thx0[p]) || (thy0 && !isfinite(thy0[p]))) {
      atomicCAS(dev_status, 0, RAD_EDATA);
      continue;
    }
    const uint64_t pid = ids ? static_cast<uint64_t>(ids[p]) : static_cast<uint64_t>(p);
    const double g0d = E0 / C.mass;
    const float g0 = static_cast<float>(g0d);
    const float q0 = static_cast<float>(1.0 / (4.0 * (g0d * g0d) * (g0d * g0d)));
    // position as channel index and offset from its centre
    const double u = (x0[p] - C.centre) / C.d_p;
    double m = floor(u + 0.5);
    DF s = df_of((x0[p] - C.centre) - m * C.d_p);
    DF y{0.f, 0.f}, dz{0.f, 0.f};
    DF vx = df_of(thx0[p]), vy = df_of(thy0 ? thy0[p] : 0.0);
    DF E = df_of(E0);
    const DF E0f = E;
    float kx = 0.f, ky = 0.f;
    double *rec = out + off * kRec;
    for (int64_t k = 0; k < L; ++k, rec += kRec) {
      const float dEoff = __fadd_rn(__fsub_rn(E.hi, E0f.hi), __fsub_rn(E.lo, E0f.lo));
      const float g = __fmaf_rn(dEoff, C.inv_mass, g0);
      // 1/E to about 46 bits: one Newton correction of the FP32 reciprocal
      const float r = __frcp_rn(E.hi);
      const float res = __fmaf_rn(-E.lo, r, __fmaf_rn(-E.hi, r, 1.0f));
      const float iE_hi = r, iE_lo = res * r;
      // record k
      const D32 d0 = deriv32<DT>(C, P, s.hi + s.lo, vx.hi, vy.hi, dEoff, 0.f, g, g0, q0, iE_hi, iE_lo);
      const float ax = d0.a + kx, ay = ky;
      const float gdot = C.ll ? d0.dE * C.inv_mass : 0.f;
      rec[F_T] = static_cast<double>(k) * C.dt;
      rec[F_X] = (m * C.d_p + C.centre) + df_val(s);
      rec[F_Y] = df_val(y);
      rec[F_DZ] = df_val(dz);
      rec[F_VX] = df_val(vx);
      rec[F_VY] = df_val(vy);
      rec[F_DVZ] = static_cast<double>(d0.dvz);
      rec[F_AX] = static_cast<double>(ax);
      rec[F_AY] = static_cast<double>(ay);
      // a_z = (dgamma/dt / gamma^3 - v_perp . a_perp) / v_z with v_z = 1 to FP32 precision
      rec[F_AZ] = static_cast<double>(gdot / (g * g * g) - __fmaf_rn(vx.hi, ax, vy.hi * ay));
      if (e_out) e_out[off + k] = df_val(E);
      kx = ky = 0.f;
      if (k == L - 1) break;
      // RK4 stages in FP32 around the double-float state
      const float h2 = C.h_half, h = C.dt_hi;
      const D32 k1 = d0;
      const D32 k2 = deriv32<DT>(C, P, s.hi + (s.lo + h2 * k1.vx), vx.hi + (vx.lo + h2 * k1.a), vy.hi + vy.lo,
                             dEoff + h2 * k1.dE, h2 * k1.dE, g, g0, q0, iE_hi, iE_lo);
      const D32 k3 = deriv32<DT>(C, P, s.hi + (s.lo + h2 * k2.vx), vx.hi + (vx.lo + h2 * k2.a), vy.hi + vy.lo,
                             dEoff + h2 * k2.dE, h2 * k2.dE, g, g0, q0, iE_hi, iE_lo);
      const D32 k4 = deriv32<DT>(C, P, s.hi + (s.lo + h * k3.vx), vx.hi + (vx.lo + h * k3.a), vy.hi + vy.lo,
                             dEoff + h * k3.dE, h * k3.dE, g, g0, q0, iE_hi, iE_lo);
      // x' = v is linear in the stages: sum/6 = v + h (a1 + a2 + a3)/6. Every factor that
      // multiplies all steps alike (dt, dt/6) is a double-float pair: an FP32-rounded constant
      // would scale every increment by the same relative error and the oscillation's phase
      // would drift with it.
      df_add_prod(s, C.dt_hi, C.dt_lo, vx);
      df_add(s, C.h2_6 * (k1.a + k2.a + k3.a));
      df_add_prod(y, C.dt_hi, C.dt_lo, vy);
      const float sa = k1.a + 2.f * k2.a + 2.f * k3.a + k4.a;
      df_add(vx, __fmaf_rn(sa, C.dt6_hi, sa * C.dt6_lo));
      const float sz = k1.dvz + 2.f * k2.dvz + 2.f * k3.dvz + k4.dvz;
      df_add(dz, __fmaf_rn(sz, C.dt6_hi, sz * C.dt6_lo));
      if (C.ll) {
        const float se = k1.dE + 2.f * k2.dE + 2.f * k3.dE + k4.dE;
        df_add(E, __fmaf_rn(se, C.dt6_hi, se * C.dt6_lo));
      }
      // keep the offset inside the channel
      if (s.hi >= C.half_d) {
        m += 1.0;
        df_add(s, -C.d_f);
        df_add(s, -static_cast<float>(C.d_p - static_cast<double>(C.d_f)));
      } else if (s.hi < -C.half_d) {
        m -= 1.0;
        df_add(s, C.d_f);
        df_add(s, static_cast<float>(C.d_p - static_cast<double>(C.d_f)));
      }
      if (C.ms) {
        // distances to the two nearest planes from the offset (planes at +-d/2 around a
        // positron channel centre, at 0 and +-d around an electron channel centre)
        const float sc = s.hi + s.lo;
        float r1, r2;
        if (C.centre != 0.0) {
          r1 = C.half_d + sc;
          r2 = C.half_d - sc;
        } else {
          r1 = sc >= 0.f ? sc : C.d_f + sc;
          r2 = C.d_f - r1;
        }
        const float n = C.dens_pref * (exp2f(C.nexp2_rho * r1 * r1) + exp2f(C.nexp2_rho * r2 * r2));
        float var = (C.var_k * n) / (E.hi * E.hi);
        if (DT && P.el) {
          const float gk = E.hi * C.inv_mass, b2 = 1.f - 1.f / (gk * gk);
          const float br = fmaxf(logf(P.lk * (gk * gk) * b2) - b2, 0.f);
          var = __fmaf_rn(electron_density32(C, P, sc, n), br / ((gk * gk) * (b2 * b2)), var);
        }
        if (var > 0.f) {
          uint32_t c[4] = {static_cast<uint32_t>(pid), static_cast<uint32_t>(k), 1u, static_cast<uint32_t>(pid >> 32)};
          philox(c, static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
          // the 53-bit uniforms of the FP64 form, rounded to FP32 (never 0)
          const float u1 = __fmaf_rn(static_cast<float>(c[1] >> 6) + 0.5f, 1.1102230246251565e-16f,
                                     static_cast<float>(c[0] >> 5) * 7.450580596923828e-09f);
          const float u2 = __fmaf_rn(static_cast<float>(c[3] >> 6) + 0.5f, 1.1102230246251565e-16f,
                                     static_cast<float>(c[2] >> 5) * 7.450580596923828e-09f);
          const float rad = sqrtf(-2.0f * logf(u1));
          float sn, cs;
          sincospif(2.0f * u2, &sn, &cs);
          const float sd = sqrtf(var);
          const float dthx = sd * (rad * cs), dthy = sd * (rad * sn);
          kx = dthx / C.dt_hi;
          ky = dthy / C.dt_hi;
          df_add(vx, dthx);
          df_add(vy, dthy);
          if (C.ms_loss) {
            const float gk = E.hi * C.inv_mass;
            df_add(E, -C.loss_k * (gk * gk * gk) * __fmaf_rn(dthx, dthx, dthy * dthy));
          }
        }
      }
    }
  }
}

}  // namespace
}  // namespace rad

namespace rad {
namespace {

// Host checks of the planar potential; fills the FP64 and FP32 coefficient sets.
int make_planar(const rad_channel *ch, const rad_planar_potential *pot, double dt, Planar &P, Planar32 &P32) {
  P = Planar{};
  P32 = Planar32{};
  if (!pot) return RAD_OK;
  const bool el = (ch->flags & RAD_TRAJ_MS_EL) != 0;
  if (pot->n_terms < 1 || pot->n_terms > kMaxTerms || pot->n_neighbours < 1 || pot->n_neighbours > 8 ||
      !(pot->N > 0.0) || !isfinite(pot->N) || !isfinite(pot->cx) || !(ch->rho >= 0.0) || !isfinite(ch->rho))
    return RAD_EINVAL;
  if (el && !(pot->I_eV > 0.0 && isfinite(pot->I_eV))) return RAD_EINVAL;
  const double rho2 = ch->rho * ch->rho;
  // one plane: U = pref sum_i a_i / sqrt(C_i) exp(-r^2/C_i); -dU/dr = pref sum_i 2 a_i r / C_i^1.5 exp(..)
  const double pref = 2.0 * sqrt(kPi) * (kAlpha * kHbarC) * kA0 * pot->N * ch->d_p;
  const double el_pref = 0.5 * dt * kPi * kR0 * kR0;
  P.nt = P32.nt = pot->n_terms;
  P.K = P32.K = pot->n_neighbours;
  P.el = P32.el = el ? 1 : 0;
  for (int i = 0; i < pot->n_terms; ++i) {
    const double C = pot->b[i] / (4.0 * kPi * kPi) + rho2;
    if (!isfinite(pot->a[i]) || !isfinite(C) || !(C > 0.0)) return RAD_EINVAL;
    P.fk[i] = 2.0 * ch->charge_sign * pref * pot->a[i] / (C * sqrt(C));
    P.ck[i] = 1.0 / C;
    P.q[i] = exp(-2.0 * ch->d_p * ch->d_p / C);
    if (el) {
      const double CX = pot->bx[i] / (4.0 * kPi * kPi) + rho2;
      if (!isfinite(pot->ax[i]) || !isfinite(CX) || !(CX > 0.0)) return RAD_EINVAL;
      P.ek[i] = el_pref * pot->N * ch->d_p / sqrt(kPi) * pot->ax[i] / sqrt(CX);
      P.eck[i] = 1.0 / CX;
    }
    P32.fk[i] = static_cast<float>(P.fk[i]);
    P32.ck2[i] = static_cast<float>(-P.ck[i] / log(2.0));
    P32.ek[i] = static_cast<float>(P.ek[i]);
    P32.eck2[i] = static_cast<float>(-P.eck[i] / log(2.0));
  }
  P.ecx = el ? el_pref * pot->cx * pot->N : 0.0;
  P.lk = el ? 2.0 * kMe / pot->I_eV : 0.0;
  P32.ecx = static_cast<float>(P.ecx);
  P32.lk = static_cast<float>(P.lk);
  // every coefficient must be finite in the precision that uses it (an extreme fit, e.g. rho = 0
  // with a tiny b_i, overflows FP32 first)
  bool ok = isfinite(P.ecx) && isfinite(P.lk);
  for (int i = 0; i < pot->n_terms; ++i) ok = ok && isfinite(P.fk[i]) && isfinite(P.ck[i]) && isfinite(P.ek[i]) &&
                                              isfinite(P.eck[i]);
  if (ch->flags & RAD_TRAJ_FP32) {
    ok = ok && isfinite(P32.ecx) && isfinite(P32.lk);
    for (int i = 0; i < pot->n_terms; ++i)
      ok = ok && isfinite(P32.fk[i]) && isfinite(P32.ck2[i]) && isfinite(P32.ek[i]) && isfinite(P32.eck2[i]);
  }
  return ok ? RAD_OK : RAD_EINVAL;
}

int launch_trajectories(const rad_channel *ch, const rad_planar_potential *pot, int64_t n_particles,
                        const int64_t *offsets, int64_t n_samples_total, const double *energy_eV,
                        const double *x0, const double *thx0, const double *thy0, const int64_t *particle_ids,
                        double dt, uint64_t seed, double *out, double *energy_out, void *stream) {
  if (!ch || n_particles < 0 || n_samples_total < 0) return RAD_EINVAL;
  const int known = pot ? 31 : 15;
  if (!(dt > 0.0) || !isfinite(dt) || !(ch->d_p > 0.0) || !(ch->mass_eV > 0.0) ||
      (!pot && !(ch->U0_eV >= 0.0)) || (ch->charge_sign != 1 && ch->charge_sign != -1) || (ch->flags & ~known))
    return RAD_EINVAL;
  if ((ch->flags & RAD_TRAJ_MS) && !(ch->X0 > 0.0 && ch->rho > 0.0 && ch->eps_s_eV >= 0.0)) return RAD_EINVAL;
  if ((ch->flags & RAD_TRAJ_MS_EL) && !(ch->flags & RAD_TRAJ_MS)) return RAD_EINVAL;
  Planar P;
  Planar32 P32;
  const int pc = make_planar(ch, pot, dt, P, P32);
  if (pc != RAD_OK) return pc;
  if (n_particles == 0) return RAD_OK;
  if (!offsets || !energy_eV || !x0 || !thx0 || !out) return RAD_EINVAL;
  cudaError_t e;
  int *ds = device_status_word(&e);
  if (!ds) return cuda_status(e);
  Chan C;
  C.U0 = ch->U0_eV;
  C.d_p = ch->d_p;
  C.eps_s = ch->eps_s_eV;
  C.X0 = ch->X0;
  C.rho = ch->rho;
  C.mass = ch->mass_eV;
  C.centre = ch->charge_sign > 0 ? 0.5 * ch->d_p : 0.0;
  C.inv_d = 1.0 / ch->d_p;
  C.force_k = -8.0 * ch->U0_eV / (ch->d_p * ch->d_p);
  C.dens_pref = (ch->flags & RAD_TRAJ_MS) ? ch->d_p / (sqrt(kPi) * ch->rho) : 0.0;
  C.inv_rho2 = (ch->flags & RAD_TRAJ_MS) ? 1.0 / (ch->rho * ch->rho) : 0.0;
  C.var_k = (ch->flags & RAD_TRAJ_MS) ? 0.5 * ch->eps_s_eV * ch->eps_s_eV * (dt / ch->X0) : 0.0;
  C.loss_k = ch->mass_eV * kAlpha / (2.0 * kPi);
  C.ll_k = -(2.0 / 3.0) * kAlpha * kHbarC * ch->mass_eV / (ch->mass_eV * ch->mass_eV * ch->mass_eV);
  C.ms = (ch->flags & RAD_TRAJ_MS) != 0;
  C.ll = (ch->flags & RAD_TRAJ_LL) != 0;
  C.ms_loss = (ch->flags & RAD_TRAJ_MS_LOSS) != 0;
  // one thread per particle; small ensembles spread one warp per SM (the integration is a
  // dependent chain per thread), large ones fill the SMs with 128-thread blocks
  const int block = n_particles < 152 * 4 * 32 ? 32 : 128;
  int64_t grid = (n_particles + block - 1) / block;
  if (grid > 1 << 20) grid = 1 << 20;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (ch->flags & RAD_TRAJ_FP32) {
    Chan32 M;
    M.d_p = ch->d_p;
    M.centre = C.centre;
    M.dt = dt;
    M.mass = ch->mass_eV;
    M.d_f = static_cast<float>(ch->d_p);
    M.half_d = 0.5f * M.d_f;
    const double kf = 8.0 * ch->U0_eV / (ch->d_p * ch->d_p);
    M.kf_hi = static_cast<float>(kf);
    M.kf_lo = static_cast<float>(kf - static_cast<double>(M.kf_hi));
    M.dt_hi = static_cast<float>(dt);
    M.dt_lo = static_cast<float>(dt - static_cast<double>(M.dt_hi));
    M.h_half = static_cast<float>(0.5 * dt);
    M.dt6_hi = static_cast<float>(dt / 6.0);
    M.dt6_lo = static_cast<float>(dt / 6.0 - static_cast<double>(M.dt6_hi));
    M.h2_6 = static_cast<float>(dt * dt / 6.0);
    M.ll_k = static_cast<float>(C.ll_k);
    M.loss_k = static_cast<float>(C.loss_k);
    M.dens_pref = static_cast<float>(C.dens_pref);
    M.nexp2_rho = static_cast<float>(-C.inv_rho2 / log(2.0));
    M.var_k = static_cast<float>(C.var_k);
    M.inv_mass = static_cast<float>(1.0 / ch->mass_eV);
    M.ms = C.ms;
    M.ll = C.ll;
    M.ms_loss = C.ms_loss;
    if (pot)
      k_channel_mixed<true><<<static_cast<unsigned>(grid), block, 0, st>>>(
          M, P32, n_particles, offsets, n_samples_total, energy_eV, x0, thx0, thy0, particle_ids, seed, out,
          energy_out, ds);
    else
      k_channel_mixed<false><<<static_cast<unsigned>(grid), block, 0, st>>>(
          M, P32, n_particles, offsets, n_samples_total, energy_eV, x0, thx0, thy0, particle_ids, seed, out,
          energy_out, ds);
  } else if (pot && n_particles < kPGroupBelow) {  // lane groups share each particle's force evaluation
    const int64_t ggrid = (n_particles * kPGroup + 127) / 128;
    k_channel_group<<<static_cast<unsigned>(ggrid), 128, 0, st>>>(C, P, n_particles, offsets, n_samples_total,
                                                                 energy_eV, x0, thx0, thy0, particle_ids, dt, seed,
                                                                 out, energy_out, ds);
  } else if (pot) {
    k_channel<true><<<static_cast<unsigned>(grid), block, 0, st>>>(C, P, n_particles, offsets, n_samples_total,
                                                                   energy_eV, x0, thx0, thy0, particle_ids, dt,
                                                                   seed, out, energy_out, ds);
  } else {
    k_channel<false><<<static_cast<unsigned>(grid), block, 0, st>>>(C, P, n_particles, offsets, n_samples_total,
                                                                    energy_eV, x0, thx0, thy0, particle_ids, dt,
                                                                    seed, out, energy_out, ds);
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? RAD_OK : cuda_status(e);
}

// The axial potential's device coefficients; the electron term is scaled by the step length dt
// (the kick variance per angle over a step of dt).
int make_axial(const rad_channel *ch, const rad_axial_potential *pot, double dt, Axial &A) {
  if (!pot) return RAD_EINVAL;
  const bool ms = (ch->flags & RAD_TRAJ_MS) != 0, el = (ch->flags & RAD_TRAJ_MS_EL) != 0;
  if (!(ch->rho >= 0.0) || !isfinite(ch->rho)) return RAD_EINVAL;
  const rad_string_lattice &Lt = pot->lattice;
  if (pot->n_terms < 1 || pot->n_terms > kMaxTerms || pot->n_cells < 1 || pot->n_cells > 4 || Lt.n_strings < 1 ||
      Lt.n_strings > 8 || !(Lt.cell_x > 0.0) || !(Lt.cell_y > 0.0) || !(Lt.d > 0.0) || !isfinite(Lt.cell_x) ||
      !isfinite(Lt.cell_y) || !isfinite(Lt.d))
    return RAD_EINVAL;
  if (el && !(pot->I_eV > 0.0 && isfinite(pot->cx))) return RAD_EINVAL;
  A = Axial{};
  A.nt = pot->n_terms;
  A.nb = Lt.n_strings;
  A.K = pot->n_cells;
  A.el = el ? 1 : 0;
  A.Lx = Lt.cell_x;
  A.Ly = Lt.cell_y;
  for (int b = 0; b < A.nb; ++b) {
    if (!isfinite(Lt.sx[b]) || !isfinite(Lt.sy[b])) return RAD_EINVAL;
    A.sx[b] = Lt.sx[b];
    A.sy[b] = Lt.sy[b];
  }
  const double rho2 = ch->rho * ch->rho;
  const double N = A.nb / (Lt.d * Lt.cell_x * Lt.cell_y);
  const double e2 = kAlpha * kHbarC;
  const double el_pref = 0.5 * dt * kPi * kR0 * kR0;
  for (int i = 0; i < A.nt; ++i) {
    const double C = pot->b[i] / (4.0 * kPi * kPi) + rho2;
    if (!isfinite(pot->a[i]) || !isfinite(C) || !(C > 0.0)) return RAD_EINVAL;
    A.fk[i] = ch->charge_sign * (2.0 * e2 * kA0 / Lt.d) * (pot->a[i] / C) * (2.0 / C);
    A.ck[i] = 1.0 / C;
    if (el) {
      const double CX = pot->bx[i] / (4.0 * kPi * kPi) + rho2;
      if (!isfinite(pot->ax[i]) || !isfinite(CX) || !(CX > 0.0)) return RAD_EINVAL;
      A.ek[i] = el_pref * pot->ax[i] / (kPi * Lt.d * CX);
      A.eck[i] = 1.0 / CX;
    }
  }
  A.dens_k = ms ? 1.0 / (kPi * rho2 * N * Lt.d) : 0.0;
  A.inv_rho2 = ms ? 1.0 / rho2 : 0.0;
  for (int i = 0; i < A.nt; ++i) {
    A.qx[i] = exp(-2.0 * A.Lx * A.Lx * A.ck[i]);
    A.qy[i] = exp(-2.0 * A.Ly * A.Ly * A.ck[i]);
    A.eqx[i] = exp(-2.0 * A.Lx * A.Lx * A.eck[i]);
    A.eqy[i] = exp(-2.0 * A.Ly * A.Ly * A.eck[i]);
  }
  A.rqx = exp(-2.0 * A.Lx * A.Lx * A.inv_rho2);
  A.rqy = exp(-2.0 * A.Ly * A.Ly * A.inv_rho2);
  A.ecx = el ? el_pref * pot->cx * N : 0.0;
  A.lk = el ? 2.0 * kMe / pot->I_eV : 0.0;
  bool ok = isfinite(A.dens_k) && isfinite(A.inv_rho2) && isfinite(A.ecx) && isfinite(A.lk);
  for (int i = 0; i < A.nt; ++i) ok = ok && isfinite(A.fk[i]) && isfinite(A.ck[i]) && isfinite(A.ek[i]) && isfinite(A.eck[i]);
  return ok ? RAD_OK : RAD_EINVAL;
}

int launch_axial(const rad_channel *ch, const rad_axial_potential *pot, int64_t n_particles, const int64_t *offsets,
                 int64_t n_samples_total, const double *energy_eV, const double *x0, const double *y0,
                 const double *thx0, const double *thy0, const int64_t *particle_ids, double dt, uint64_t seed,
                 double *out, double *energy_out, void *stream) {
  if (!ch || !pot || n_particles < 0 || n_samples_total < 0) return RAD_EINVAL;
  if (!(dt > 0.0) || !isfinite(dt) || !(ch->mass_eV > 0.0) || (ch->charge_sign != 1 && ch->charge_sign != -1) ||
      (ch->flags & ~31))
    return RAD_EINVAL;
  if (ch->flags & RAD_TRAJ_FP32) return RAD_EUNSUPPORTED;
  const bool ms = (ch->flags & RAD_TRAJ_MS) != 0, el = (ch->flags & RAD_TRAJ_MS_EL) != 0;
  if (ms && !(ch->X0 > 0.0 && ch->rho > 0.0 && ch->eps_s_eV >= 0.0)) return RAD_EINVAL;
  if (el && !ms) return RAD_EINVAL;
  Axial A;
  const int ac = make_axial(ch, pot, dt, A);
  if (ac != RAD_OK) return ac;
  if (n_particles == 0) return RAD_OK;
  if (!offsets || !energy_eV || !x0 || !thx0 || !out) return RAD_EINVAL;
  cudaError_t e;
  int *ds = device_status_word(&e);
  if (!ds) return cuda_status(e);
  Chan C{};
  C.mass = ch->mass_eV;
  C.var_k = ms ? 0.5 * ch->eps_s_eV * ch->eps_s_eV * (dt / ch->X0) : 0.0;
  C.loss_k = ch->mass_eV * kAlpha / (2.0 * kPi);
  C.ll_k = -(2.0 / 3.0) * kAlpha * kHbarC * ch->mass_eV / (ch->mass_eV * ch->mass_eV * ch->mass_eV);
  C.ms = ms;
  C.ll = (ch->flags & RAD_TRAJ_LL) != 0;
  C.ms_loss = (ch->flags & RAD_TRAJ_MS_LOSS) != 0;
  if (n_particles < kGroupBelow) {  // lane groups share each particle's force evaluation
    const int block = 128;
    const int64_t grid = (n_particles * kGroup + block - 1) / block;
    k_axial_group<<<static_cast<unsigned>(grid), block, 0, static_cast<cudaStream_t>(stream)>>>(
        C, A, n_particles, offsets, n_samples_total, energy_eV, x0, y0, thx0, thy0, particle_ids, dt, seed, out,
        energy_out, ds);
  } else {
    const int block = 32;  // one-warp blocks spread the particles evenly over the SMs
    int64_t grid = (n_particles + block - 1) / block;
    if (grid > 1 << 20) grid = 1 << 20;
    k_axial<<<static_cast<unsigned>(grid), block, 0, static_cast<cudaStream_t>(stream)>>>(
        C, A, n_particles, offsets, n_samples_total, energy_eV, x0, y0, thx0, thy0, particle_ids, dt, seed, out,
        energy_out, ds);
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? RAD_OK : cuda_status(e);
}

int launch_adaptive(const rad_channel *ch, const rad_planar_potential *pot, const rad_axial_potential *axial,
                    const rad_step_control *sc, int64_t n_particles, const int64_t *offsets, int64_t n_samples_total,
                    const double *energy_eV, const double *x0, const double *y0, const double *thx0,
                    const double *thy0, const int64_t *particle_ids, const double *times, double dt, uint64_t seed,
                    double *out, double *energy_out, int64_t *substeps_out, void *stream) {
  if (!ch || !sc || n_particles < 0 || n_samples_total < 0 || (pot && axial)) return RAD_EINVAL;
  const int known = (pot || axial) ? 31 : 15;
  if (!(ch->mass_eV > 0.0) || (ch->charge_sign != 1 && ch->charge_sign != -1) || (ch->flags & ~known))
    return RAD_EINVAL;
  if (!times && !(dt > 0.0 && isfinite(dt))) return RAD_EINVAL;
  if (ch->flags & RAD_TRAJ_FP32) return RAD_EUNSUPPORTED;
  if (!axial && !(ch->d_p > 0.0)) return RAD_EINVAL;
  if (!pot && !axial && !(ch->U0_eV >= 0.0)) return RAD_EINVAL;
  const bool ms = (ch->flags & RAD_TRAJ_MS) != 0;
  if (ms && !(ch->X0 > 0.0 && ch->rho > 0.0 && ch->eps_s_eV >= 0.0)) return RAD_EINVAL;
  if ((ch->flags & RAD_TRAJ_MS_EL) && !ms) return RAD_EINVAL;
  if (!(sc->rtol > 0.0) || !(sc->atol_x > 0.0) || !(sc->atol_v > 0.0) || !isfinite(sc->rtol) || !isfinite(sc->atol_x) ||
      !isfinite(sc->atol_v) || sc->max_level < 0 || sc->max_level > 16 || sc->max_substeps < 1)
    return RAD_EINVAL;
  // coefficients per unit length: the kernel scales the kick variances by each interval's length
  Planar P;
  Planar32 P32;
  Axial A{};
  int rc = make_planar(ch, pot, 1.0, P, P32);
  if (rc != RAD_OK) return rc;
  if (axial) {
    rc = make_axial(ch, axial, 1.0, A);
    if (rc != RAD_OK) return rc;
  }
  if (n_particles == 0) return RAD_OK;
  if (!offsets || !energy_eV || !x0 || !thx0 || !out) return RAD_EINVAL;
  cudaError_t e;
  int *ds = device_status_word(&e);
  if (!ds) return cuda_status(e);
  Chan C{};
  C.U0 = ch->U0_eV;
  C.d_p = axial ? 1.0 : ch->d_p;
  C.mass = ch->mass_eV;
  C.rho = ch->rho;
  C.centre = ch->charge_sign > 0 ? 0.5 * C.d_p : 0.0;
  C.inv_d = 1.0 / C.d_p;
  C.force_k = axial ? 0.0 : -8.0 * ch->U0_eV / (ch->d_p * ch->d_p);
  C.dens_pref = (ms && !axial) ? ch->d_p / (sqrt(kPi) * ch->rho) : 0.0;
  C.inv_rho2 = ms ? 1.0 / (ch->rho * ch->rho) : 0.0;
  C.var_k = ms ? 0.5 * ch->eps_s_eV * ch->eps_s_eV / ch->X0 : 0.0;
  C.loss_k = ch->mass_eV * kAlpha / (2.0 * kPi);
  C.ll_k = -(2.0 / 3.0) * kAlpha * kHbarC * ch->mass_eV / (ch->mass_eV * ch->mass_eV * ch->mass_eV);
  C.ms = ms;
  C.ll = (ch->flags & RAD_TRAJ_LL) != 0;
  C.ms_loss = (ch->flags & RAD_TRAJ_MS_LOSS) != 0;
  StepCtl S{sc->rtol, sc->atol_x, sc->atol_v, sc->max_level, sc->max_substeps};
  const int block = n_particles < 152 * 4 * 32 ? 32 : 128;
  int64_t grid = (n_particles + block - 1) / block;
  if (grid > 1 << 20) grid = 1 << 20;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned gr = static_cast<unsigned>(grid);
  // small ensembles: lane groups share each particle's field sums (the thresholds of the RK4
  // integrators); 128-thread blocks of 8 or 16 groups
  const unsigned ggr8 = static_cast<unsigned>((n_particles * kPGroup + 127) / 128);
  const unsigned ggr16 = static_cast<unsigned>((n_particles * kGroup + 127) / 128);
  if (axial && n_particles < kGroupBelow)
    k_adaptive<2, true><<<ggr16, 128, 0, st>>>(C, P, A, S, n_particles, offsets, n_samples_total, energy_eV, x0, y0,
                                               thx0, thy0, particle_ids, times, dt, seed, out, energy_out,
                                               substeps_out, ds);
  else if (axial)
    k_adaptive<2, false><<<gr, block, 0, st>>>(C, P, A, S, n_particles, offsets, n_samples_total, energy_eV, x0, y0,
                                                thx0, thy0, particle_ids, times, dt, seed, out, energy_out,
                                                substeps_out, ds);
  else if (pot && n_particles < kPGroupBelow)
    k_adaptive<1, true><<<ggr8, 128, 0, st>>>(C, P, A, S, n_particles, offsets, n_samples_total, energy_eV, x0, y0,
                                              thx0, thy0, particle_ids, times, dt, seed, out, energy_out,
                                              substeps_out, ds);
  else if (pot)
    k_adaptive<1, false><<<gr, block, 0, st>>>(C, P, A, S, n_particles, offsets, n_samples_total, energy_eV, x0, y0,
                                                thx0, thy0, particle_ids, times, dt, seed, out, energy_out,
                                                substeps_out, ds);
  else
    k_adaptive<0, false><<<gr, block, 0, st>>>(C, P, A, S, n_particles, offsets, n_samples_total, energy_eV, x0, y0,
                                                thx0, thy0, particle_ids, times, dt, seed, out, energy_out,
                                                substeps_out, ds);
  e = cudaGetLastError();
  return e == cudaSuccess ? RAD_OK : cuda_status(e);
}

}  // namespace
}  // namespace rad

extern "C" int rad_trajectories_adaptive(const rad_channel *ch, const rad_planar_potential *pot,
                                         const rad_axial_potential *axial, const rad_step_control *sc,
                                         int64_t n_particles, const int64_t *offsets, int64_t n_samples_total,
                                         const double *energy_eV, const double *x0, const double *y0,
                                         const double *thx0, const double *thy0, const int64_t *particle_ids,
                                         const double *times, double dt, uint64_t seed, double *out,
                                         double *energy_out, int64_t *substeps_out, void *stream) {
  return rad::launch_adaptive(ch, pot, axial, sc, n_particles, offsets, n_samples_total, energy_eV, x0, y0, thx0, thy0,
                              particle_ids, times, dt, seed, out, energy_out, substeps_out, stream);
}

extern "C" int rad_axial_trajectories(const rad_channel *ch, const rad_axial_potential *pot, int64_t n_particles,
                                      const int64_t *offsets, int64_t n_samples_total, const double *energy_eV,
                                      const double *x0, const double *y0, const double *thx0, const double *thy0,
                                      const int64_t *particle_ids, double dt, uint64_t seed, double *out,
                                      double *energy_out, void *stream) {
  return rad::launch_axial(ch, pot, n_particles, offsets, n_samples_total, energy_eV, x0, y0, thx0, thy0,
                           particle_ids, dt, seed, out, energy_out, stream);
}

extern "C" int rad_channeling_trajectories(const rad_channel *ch, int64_t n_particles, const int64_t *offsets,
                                           int64_t n_samples_total, const double *energy_eV, const double *x0,
                                           const double *thx0, const double *thy0, const int64_t *particle_ids,
                                           double dt, uint64_t seed, double *out, double *energy_out,
                                           void *stream) {
  return rad::launch_trajectories(ch, nullptr, n_particles, offsets, n_samples_total, energy_eV, x0, thx0, thy0,
                                  particle_ids, dt, seed, out, energy_out, stream);
}

extern "C" int rad_crystal_trajectories(const rad_channel *ch, const rad_planar_potential *pot, int64_t n_particles,
                                        const int64_t *offsets, int64_t n_samples_total, const double *energy_eV,
                                        const double *x0, const double *thx0, const double *thy0,
                                        const int64_t *particle_ids, double dt, uint64_t seed, double *out,
                                        double *energy_out, void *stream) {
  if (!pot) return RAD_EINVAL;
  return rad::launch_trajectories(ch, pot, n_particles, offsets, n_samples_total, energy_eV, x0, thx0, thy0,
                                  particle_ids, dt, seed, out, energy_out, stream);
}
