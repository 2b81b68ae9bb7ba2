/*
 * FP64 CPU oracle for the radiation integral -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this library. The product path (the CUDA library) never calls it
 * and shares no code, header, table or constant with it.
 *
 * What it computes (C. F. Nielsen, arXiv:1910.10391, Sec. II):
 *   Eq. 1   d2I/(dw dOmega) = e^2/(4 pi^2) | int f(t,n) exp(i w (t - n.x(t))) dt |^2
 *   Eq. 2   f = n x ((n - beta) x beta_dot) / (1 - beta.n)^2
 *   expanded small-angle form (Sec. II, equations for f_x, f_y, f_z, g and the
 *   phase), evaluated literally as printed:
 *     f_x = {(vdz + ny vdy)(nx - vx) - [ny(ny - vy) + (-th2/2 - dvz + 1/(2g^2))] vdx} g
 *     f_y = {(vdz + nx vdx)(ny - vy) - [nx(nx - vx) + (-th2/2 - dvz + 1/(2g^2))] vdy} g
 *     f_z = {[-th2/2 - dvz + 1/(2g^2)](nx vdx + ny vdy) - [nx(nx - vx) + ny(ny - vy)] vdz} g
 *     g   = (1/(2g^2) + th2/2 - dvz - nx vx - ny vy)^-2
 *     phase = w ((1/(2g^2) + th2/2) t - dz - nx x - ny y)
 *   Lindhard substitution (spin 0, Eq. Lindhard_substi): w* = w/(1 - hw/E),
 *     dI_q/dhw(w) = (w/w*) dI_c/dhw(w*), applied per direction.
 *   BCK semiclassical spin 1/2 (Eqs. cue, Iterm, J):
 *     dI/dw dOmega = e^2/(4 pi^2) [ (E*^2 + E^2)/(2E^2) |I|^2 + hw^2/(2 E^2 g^2) |J|^2 ],
 *     E* = E - hw, I and J evaluated at w*, J integrand (n.beta_dot)/(1 - n.beta)^2
 *     taken in the same expansion: (nx vdx + ny vdy + vdz) g.
 *
 * Readings where the paper is silent (each stated once here):
 *   - time quadrature: trapezoid weights w_k = (t_{k+1} - t_{k-1})/2, one-sided at the ends;
 *   - units: c = 1, t and lengths in metres, w = hw/(hbar c) in 1/m; output is
 *     d2I/(d(hw) dOmega) = (alpha/(4 pi^2)) * S, dimensionless;
 *   - beta0 := 1 - 1/(2 gamma^2) exactly (the trajectory variables are defined from it);
 *   - ensemble: per-particle weights, incoherent sum over particles (Sec. IV);
 *   - the phase is evaluated in this fixed order with no fused operations:
 *       inv2g2 = 1/((2 gamma) gamma);  th2h = (nx nx + ny ny) * 0.5;  c = inv2g2 + th2h;
 *       A = ((c t - dz) - nx x) - ny y;  w = hw / hbar_c;
 *       w* = w / (1 - hw / E)  (quantum modes), w* = w (classical);  phi = w* A.
 *
 * Sums over time samples and over particles are Neumaier-compensated; sin and cos
 * are libm's, on the unreduced phase.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_HBARC_EV_M 1.973269804e-7 /* CODATA 2018 */
#define ORC_ALPHA 7.2973525693e-3     /* CODATA 2018 */
#define ORC_PI 3.14159265358979323846

enum { ORC_CLASSICAL = 0, ORC_SPIN0 = 1, ORC_SPIN_HALF = 2 };
enum { T_ = 0, X_, Y_, DZ_, VX_, VY_, DVZ_, AX_, AY_, AZ_ };
#define NREC 10

/* Test hook: a nonzero value plants one deliberate mistake (see orc_set_plant). */
static int g_plant = 0;
void orc_set_plant(int which) { g_plant = which; }

typedef struct {
  double s, c;
} nsum; /* Neumaier compensated sum */

static inline void nadd(nsum *a, double x) {
  const double t = a->s + x;
  if (fabs(a->s) >= fabs(x))
    a->c += (a->s - t) + x;
  else
    a->c += (x - t) + a->s;
  a->s = t;
}
static inline double nval(const nsum *a) { return a->s + a->c; }

/* trapezoid weight of sample k of a trajectory with L samples (Sec. II integral, reading c1) */
static double trap_weight(const double *smp, int64_t L, int64_t k) {
  if (L < 2) return 0.0;
  if (g_plant == 5) { /* planted: every step taken equal to the first */
    const double h = smp[1 * NREC + T_] - smp[0 * NREC + T_];
    return (k == 0 || k == L - 1) ? 0.5 * h : h;
  }
  if (g_plant == 6 && k > 0 && k < L - 1) /* planted: forward difference for interior samples */
    return smp[(k + 1) * NREC + T_] - smp[k * NREC + T_];
  if (k == 0) return 0.5 * (smp[1 * NREC + T_] - smp[0 * NREC + T_]);
  if (k == L - 1) return 0.5 * (smp[(L - 1) * NREC + T_] - smp[(L - 2) * NREC + T_]);
  return 0.5 * (smp[(k + 1) * NREC + T_] - smp[(k - 1) * NREC + T_]);
}

/*
 * Amplitudes of one particle at one (w*, n): out[0..5] = Re/Im of I_x, I_y, I_z,
 * out[6..7] = Re/Im of J, out[8] = sum_k w_k |f_k|, out[9] = sum_k w_k |j_k|.
 * omega_star in 1/m. Returns 0, or 1 for invalid input.
 */
int orc_amplitudes(const double *smp, int64_t L, double gamma, double omega_star, double nx,
                   double ny, double *out) {
  if (!smp || !out || L < 2 || !(gamma > 1.0)) return 1;
  const double inv2g2 = 1.0 / (2.0 * gamma * gamma);
  const double th2 = nx * nx + ny * ny;
  const double th2h = th2 * 0.5;
  const double c = inv2g2 + th2h;
  nsum acc[8] = {{0}};
  nsum af = {0}, aj = {0};
  for (int64_t k = 0; k < L; ++k) {
    const double *r = smp + k * NREC;
    const double t = r[T_], x = r[X_], y = r[Y_], dz = r[DZ_];
    const double vx = r[VX_], vy = r[VY_], dvz = r[DVZ_];
    const double ax = r[AX_], ay = r[AY_], az = r[AZ_];
    /* g (Sec. II) */
    const double D = inv2g2 + th2h - dvz - nx * vx - ny * vy;
    const double g = 1.0 / (D * D);
    /* bracket shared by f_x, f_y, f_z */
    const double br = -th2h - dvz + inv2g2;
    double fx = ((az + ny * ay) * (nx - vx) - (ny * (ny - vy) + br) * ax) * g;
    double fy = ((az + nx * ax) * (ny - vy) - (nx * (nx - vx) + br) * ay) * g;
    double fz = (br * (nx * ax + ny * ay) - (nx * (nx - vx) + ny * (ny - vy)) * az) * g;
    double jj = (nx * ax + ny * ay + az) * g;
    if (g_plant == 1) fx = ((az + ny * ay) * (nx - vx) - (ny * (ny - vy)) * ax) * g; /* drop br */
    if (g_plant == 2) jj = (nx * ax + ny * ay - az) * g;                              /* sign */
    if (g_plant == 3) fz = 0.0;                                                        /* drop f_z */
    /* phase, fixed evaluation order */
    double A = c * t;
    A = A - dz;
    A = A - nx * x;
    A = A - ny * y;
    if (g_plant == 4) A = A + 2.0 * ny * y; /* wrong sign of ny*y */
    const double phi = omega_star * A;
    const double cs = cos(phi), sn = sin(phi);
    const double w = trap_weight(smp, L, k);
    nadd(&acc[0], w * fx * cs);
    nadd(&acc[1], w * fx * sn);
    nadd(&acc[2], w * fy * cs);
    nadd(&acc[3], w * fy * sn);
    nadd(&acc[4], w * fz * cs);
    nadd(&acc[5], w * fz * sn);
    nadd(&acc[6], w * jj * cs);
    nadd(&acc[7], w * jj * sn);
    nadd(&af, w * sqrt(fx * fx + fy * fy + fz * fz));
    nadd(&aj, w * fabs(jj));
  }
  for (int i = 0; i < 8; ++i) out[i] = nval(&acc[i]);
  out[8] = nval(&af);
  out[9] = nval(&aj);
  return 0;
}

/* w* (1/m) for a photon energy hw (eV), particle energy E (eV) and mode */
static double omega_star_of(double hw, double E, int mode) {
  const double w = hw / ORC_HBARC_EV_M;
  if (mode == ORC_CLASSICAL) return w;
  const double u = hw / E;
  return w / (1.0 - u);
}

/*
 * S(w, n) for one particle: the bracket of Eq. 1 / Lindhard / Eq. cue without the
 * alpha/(4 pi^2) prefactor. cond receives the matching bound with |I| replaced by
 * sum_k w_k |f_k| (and |J| by sum_k w_k |j_k|).
 */
static int particle_S(const double *smp, int64_t L, double gamma, double E, double hw, double nx,
                      double ny, int mode, double *S, double *cond) {
  double a[10];
  const double ws = omega_star_of(hw, E, mode);
  if (orc_amplitudes(smp, L, gamma, ws, nx, ny, a)) return 1;
  const double I2 = a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3] + a[4] * a[4] + a[5] * a[5];
  const double J2 = a[6] * a[6] + a[7] * a[7];
  const double u = hw / E;
  if (mode == ORC_CLASSICAL) {
    *S = I2;
    *cond = a[8] * a[8];
  } else if (mode == ORC_SPIN0) {
    /* (w / w*) = 1 - u */
    *S = (1.0 - u) * I2;
    *cond = (1.0 - u) * a[8] * a[8];
  } else {
    /* (E*^2 + E^2)/(2 E^2) = (1 + (1-u)^2)/2 ;  hw^2/(2 E^2 gamma^2) = u^2/(2 gamma^2) */
    const double cI = 0.5 * (1.0 + (1.0 - u) * (1.0 - u));
    const double cJ = (u * u) / (2.0 * gamma * gamma);
    *S = cI * I2 + cJ * J2;
    *cond = cI * a[8] * a[8] + cJ * a[9] * a[9];
  }
  return 0;
}

static int check_common(const double *samples, const int64_t *offsets, int64_t n_particles,
                        const double *gamma, const double *energy, const double *hw,
                        int64_t n_omega, int mode) {
  if (!samples || !offsets || !gamma || !energy || !hw || n_particles < 0 || n_omega < 0) return 1;
  if (mode < 0 || mode > 2) return 1;
  for (int64_t p = 0; p < n_particles; ++p) {
    if (offsets[p + 1] - offsets[p] < 2) return 1;
    if (!(gamma[p] > 1.0)) return 1;
  }
  for (int64_t i = 0; i < n_omega; ++i) {
    if (!(hw[i] > 0.0)) return 1;
    if (mode != ORC_CLASSICAL)
      for (int64_t p = 0; p < n_particles; ++p)
        if (!(hw[i] < energy[p])) return 1;
  }
  return 0;
}

/*
 * Ensemble value at a list of bins (omega index, angle index):
 *   out_S[b] = alpha/(4 pi^2) * sum_p weight_p S_p(w_i, n_j)   (Neumaier over p)
 *   out_cond[b] = alpha/(4 pi^2) * sum_p weight_p cond_p        (may be NULL)
 * weight may be NULL (all ones). n_threads <= 0: OpenMP default.
 */
int orc_spectrum_bins(const double *samples, const int64_t *offsets, int64_t n_particles,
                      const double *gamma, const double *energy, const double *weight,
                      const double *hw, int64_t n_omega, const double *theta_x,
                      const double *theta_y, int64_t n_angles, int mode, const int64_t *bin_omega,
                      const int64_t *bin_angle, int64_t n_bins, double *out_S, double *out_cond,
                      int n_threads) {
  if (check_common(samples, offsets, n_particles, gamma, energy, hw, n_omega, mode)) return 1;
  if (!theta_x || !theta_y || !bin_omega || !bin_angle || !out_S || n_bins < 0) return 1;
  for (int64_t b = 0; b < n_bins; ++b)
    if (bin_omega[b] < 0 || bin_omega[b] >= n_omega || bin_angle[b] < 0 || bin_angle[b] >= n_angles)
      return 1;
  const double pref = ORC_ALPHA / (4.0 * ORC_PI * ORC_PI);
  int err = 0;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#endif
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
  for (int64_t b = 0; b < n_bins; ++b) {
    const double h = hw[bin_omega[b]];
    const double nx = theta_x[bin_angle[b]], ny = theta_y[bin_angle[b]];
    nsum sS = {0}, sC = {0};
    for (int64_t p = 0; p < n_particles; ++p) {
      double S, C;
      const int64_t L = offsets[p + 1] - offsets[p];
      err |= particle_S(samples + offsets[p] * NREC, L, gamma[p], energy[p], h, nx, ny, mode, &S, &C);
      const double wp = weight ? weight[p] : 1.0;
      nadd(&sS, wp * S);
      nadd(&sC, wp * C);
    }
    out_S[b] = pref * nval(&sS);
    if (out_cond) out_cond[b] = pref * nval(&sC);
  }
  return err;
}

/* Full cube out_cube[i * n_angles + j] (same definition as orc_spectrum_bins). */
int orc_spectrum_cube(const double *samples, const int64_t *offsets, int64_t n_particles,
                      const double *gamma, const double *energy, const double *weight,
                      const double *hw, int64_t n_omega, const double *theta_x,
                      const double *theta_y, int64_t n_angles, int mode, double *out_cube,
                      double *out_cond, int n_threads) {
  if (n_omega < 0 || n_angles < 0) return 1;
  const int64_t nb = n_omega * n_angles;
  int64_t *bi = (int64_t *)malloc((size_t)(nb > 0 ? nb : 1) * sizeof(int64_t));
  int64_t *bj = (int64_t *)malloc((size_t)(nb > 0 ? nb : 1) * sizeof(int64_t));
  if (!bi || !bj) {
    free(bi);
    free(bj);
    return 2;
  }
  for (int64_t i = 0; i < n_omega; ++i)
    for (int64_t j = 0; j < n_angles; ++j) {
      bi[i * n_angles + j] = i;
      bj[i * n_angles + j] = j;
    }
  const int rc = orc_spectrum_bins(samples, offsets, n_particles, gamma, energy, weight, hw, n_omega,
                                   theta_x, theta_y, n_angles, mode, bi, bj, nb, out_cube, out_cond,
                                   n_threads);
  free(bi);
  free(bj);
  return rc;
}

/*
 * Angle integration of the cube (Sec. IV: dI/dw = int dOmega d2I/dw dOmega, midpoint rule
 * with the caller's cell solid angles) and optional radial binning:
 *   out_spectrum[i]       = sum_j cube[i][j] dOmega_j
 *   out_bins[i*nb + b]    = sum_{j: bin_of_angle[j] == b} cube[i][j] dOmega_j
 */
int orc_reduce(const double *cube, int64_t n_omega, int64_t n_angles, const double *d_omega,
               const int32_t *bin_of_angle, int n_rbins, double *out_spectrum, double *out_bins) {
  if (!cube || !d_omega || n_omega < 0 || n_angles < 0) return 1;
  if (out_bins && (!bin_of_angle || n_rbins <= 0)) return 1;
  nsum *tmp = (nsum *)calloc((size_t)(n_rbins > 0 ? n_rbins : 1), sizeof(nsum));
  if (!tmp) return 2;
  for (int64_t i = 0; i < n_omega; ++i) {
    nsum s = {0};
    for (int b = 0; b < n_rbins; ++b) tmp[b].s = tmp[b].c = 0.0;
    for (int64_t j = 0; j < n_angles; ++j) {
      const double v = cube[i * n_angles + j] * d_omega[j];
      nadd(&s, v);
      if (out_bins) {
        const int32_t b = bin_of_angle[j];
        if (b >= 0 && b < n_rbins) nadd(&tmp[b], v);
      }
    }
    if (out_spectrum) out_spectrum[i] = nval(&s);
    if (out_bins)
      for (int b = 0; b < n_rbins; ++b) out_bins[i * n_rbins + b] = nval(&tmp[b]);
  }
  free(tmp);
  return 0;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
