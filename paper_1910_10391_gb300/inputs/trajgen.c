/*
 * Seeded synthetic trajectory generator for planar channeling (input side only).
 *
 * Produces the per-sample records the radiation integral consumes (Sec. II,
 * small-angle variables): t, x, y, dz, vx, vy, dvz, ax, ay, az with
 * dz = z - beta0*t, dvz = vz - beta0, beta0 := 1 - 1/(2 gamma^2), c = 1.
 *
 * Physics of the stand-in workload (Sec. III gives the real crystal model; its
 * Doyle-Turner tables are not in the paper, so a harmonic well replaces them):
 *   U(s) = U0 (2 s / d_p)^2, s = distance to the nearest channel centre.
 *   Positrons: channel centres mid-way between planes; electrons: on the planes.
 *   Transverse equation of motion d(v_perp)/dt = F_perp / E (ultra-relativistic).
 *   Multiple Coulomb scattering on nuclei (Sec. III, nuclear term only): after each
 *   step, Gaussian kicks in each transverse angle with variance
 *   0.5 (eps_s/E)^2 (dz/X0) n(r)/N, where n(r)/N sums the Gaussian plane density
 *   d_p/(sqrt(pi) rho) exp(-r^2/rho^2) over the two nearest planes.
 *   A kick rotates v_perp at fixed |beta|; the kicked sample's acceleration
 *   carries the kick as delta_v/dt so that the kick radiates.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), counter = (particle, step, stream, 0),
 * key = seed; uniforms from the top 53 bits of two outputs; normals by Box-Muller.
 *
 * Build: plain C, no FMA contraction (-ffp-contract=off) so x86-64 and aarch64
 * builds give the same bytes up to libm's last-ulp differences in log/cos.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define NREC 10
enum { R_T = 0, R_X, R_Y, R_DZ, R_VX, R_VY, R_DVZ, R_AX, R_AY, R_AZ };

/* ---------------- Philox4x32-10 ---------------- */
static void philox_round(uint32_t c[4], const uint32_t k[2]) {
  const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
  const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  uint32_t o[4];
  o[0] = hi1 ^ c[1] ^ k[0];
  o[1] = lo1;
  o[2] = hi0 ^ c[3] ^ k[1];
  o[3] = lo0;
  memcpy(c, o, sizeof o);
}

void tg_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    philox_round(c, k);
    k[0] += 0x9E3779B9u;
    k[1] += 0xBB67AE85u;
  }
  memcpy(out, c, sizeof c);
}

static double u53(uint32_t a, uint32_t b) { /* (0,1): never 0, never 1 */
  const uint64_t m = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6); /* 53 bits */
  return ((double)m + 0.5) * (1.0 / 9007199254740992.0);
}

/* Two independent standard normals for (particle, step, stream). */
static void normals2(uint64_t seed, uint64_t particle, uint64_t step, uint32_t stream,
                     double *z0, double *z1) {
  const uint32_t ctr[4] = {(uint32_t)particle, (uint32_t)step, stream,
                           (uint32_t)(particle >> 32)};
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t r[4];
  tg_philox4x32_10(ctr, key, r);
  const double u1 = u53(r[0], r[1]), u2 = u53(r[2], r[3]);
  const double rad = sqrt(-2.0 * log(u1));
  const double ang = 6.283185307179586 * u2;
  *z0 = rad * cos(ang);
  *z1 = rad * sin(ang);
}

/* Uniform (0,1) for (particle, stream). */
static void uniforms2(uint64_t seed, uint64_t particle, uint32_t stream, double *a, double *b) {
  const uint32_t ctr[4] = {(uint32_t)particle, 0xFFFFFFFFu, stream, (uint32_t)(particle >> 32)};
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t r[4];
  tg_philox4x32_10(ctr, key, r);
  *a = u53(r[0], r[1]);
  *b = u53(r[2], r[3]);
}

/* ---------------- channeling physics ---------------- */
typedef struct {
  double E_eV, gamma, beta0, U0_eV, d_p, charge_sign; /* +1 positron, -1 electron */
  double eps_s_eV, X0, rho;
  int ms;
} tg_params;

/* transverse force / E  (units 1/m), harmonic planar well */
static double accel_x(const tg_params *P, double x) {
  const double d = P->d_p;
  const double off = (P->charge_sign > 0) ? 0.5 * d : 0.0; /* channel centre */
  const double u = (x - off) / d;
  const double s = (u - floor(u + 0.5)) * d; /* s in [-d/2, d/2) */
  const double F = -8.0 * P->U0_eV * s / (d * d);   /* eV/m */
  return F / P->E_eV;
}

/* relative nuclear density n(r)/N summed over the two nearest planes (at m*d_p) */
static double nuc_density(const tg_params *P, double x) {
  const double d = P->d_p, rho = P->rho;
  const double m = floor(x / d);
  const double r1 = x - m * d, r2 = (m + 1.0) * d - x;
  const double pref = d / (sqrt(M_PI) * rho);
  return pref * (exp(-(r1 * r1) / (rho * rho)) + exp(-(r2 * r2) / (rho * rho)));
}

/* dvz from v_perp^2 with beta0 = 1 - 1/(2 g^2):  vz - beta0 = -(vp2 + 1/(4 g^4)) / (vz + beta0) */
static void longi(const tg_params *P, double vp2, double *vz, double *dvz) {
  const double g2 = P->gamma * P->gamma;
  *vz = sqrt(1.0 - 1.0 / g2 - vp2);
  *dvz = -(vp2 + 1.0 / (4.0 * g2 * g2)) / (*vz + P->beta0);
}

/* state: x, y, vx, vy, dz ; derivative */
static void deriv(const tg_params *P, const double s[5], double d[5]) {
  double vz, dvz;
  longi(P, s[2] * s[2] + s[3] * s[3], &vz, &dvz);
  d[0] = s[2];
  d[1] = s[3];
  d[2] = accel_x(P, s[0]);
  d[3] = 0.0;
  d[4] = dvz;
}

static void write_rec(const tg_params *P, double *rec, double t, const double s[5],
                      double kick_ax, double kick_ay) {
  double vz, dvz;
  longi(P, s[2] * s[2] + s[3] * s[3], &vz, &dvz);
  const double ax = accel_x(P, s[0]) + kick_ax;
  const double ay = 0.0 + kick_ay;
  rec[R_T] = t;
  rec[R_X] = s[0];
  rec[R_Y] = s[1];
  rec[R_DZ] = s[4];
  rec[R_VX] = s[2];
  rec[R_VY] = s[3];
  rec[R_DVZ] = dvz;
  rec[R_AX] = ax;
  rec[R_AY] = ay;
  rec[R_AZ] = -(s[2] * ax + s[3] * ay) / vz;
}

/*
 * Integrate one particle for L samples (L-1 RK4 steps of dt), writing L records.
 * Entry: x0, theta_x0, theta_y0 given; y0 = 0, dz0 = 0.
 */
static void run_particle(const tg_params *P, uint64_t seed, int64_t pid, double x0,
                         double thx0, double thy0, double dt, int64_t L, double *out) {
  double s[5] = {x0, 0.0, thx0, thy0, 0.0};
  double pend_ax = 0.0, pend_ay = 0.0;
  for (int64_t k = 0; k < L; ++k) {
    write_rec(P, out + k * NREC, (double)k * dt, s, pend_ax, pend_ay);
    pend_ax = pend_ay = 0.0;
    if (k == L - 1) break;
    double k1[5], k2[5], k3[5], k4[5], tmp[5];
    deriv(P, s, k1);
    for (int i = 0; i < 5; ++i) tmp[i] = s[i] + 0.5 * dt * k1[i];
    deriv(P, tmp, k2);
    for (int i = 0; i < 5; ++i) tmp[i] = s[i] + 0.5 * dt * k2[i];
    deriv(P, tmp, k3);
    for (int i = 0; i < 5; ++i) tmp[i] = s[i] + dt * k3[i];
    deriv(P, tmp, k4);
    for (int i = 0; i < 5; ++i)
      s[i] = s[i] + (dt / 6.0) * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    if (P->ms) {
      const double var = 0.5 * (P->eps_s_eV / P->E_eV) * (P->eps_s_eV / P->E_eV) *
                         (dt / P->X0) * nuc_density(P, s[0]);
      double z0, z1;
      normals2(seed, (uint64_t)pid, (uint64_t)k, 1u, &z0, &z1);
      const double dthx = sqrt(var) * z0, dthy = sqrt(var) * z1;
      /* rotate v_perp at fixed |beta|: small-angle kick of the direction */
      const double nvx = s[2] + dthx, nvy = s[3] + dthy;
      pend_ax = (nvx - s[2]) / dt;
      pend_ay = (nvy - s[3]) / dt;
      s[2] = nvx;
      s[3] = nvy;
    }
  }
}

/*
 * Public entry (ctypes): generate an ensemble.
 *   lengths[p]  samples of particle p (>= 2); records are written contiguously,
 *               particle p starting at offsets[p] (caller-computed prefix sum).
 *   entry: x0 ~ U[0, d_p) (absolute, so the channel phase is uniform),
 *          theta_x0 ~ N(0, (sigma_theta)^2), theta_y0 = 0.
 * Returns 0 on success.
 */
int tg_channeling(double E_eV, double mass_eV, int charge_sign, double U0_eV, double d_p,
                  double sigma_theta, double eps_s_eV, double X0, double rho, int ms,
                  double dt, uint64_t seed, int64_t n_particles, const int64_t *offsets,
                  double *out, double *entry_x0, double *entry_thx) {
  tg_params P;
  P.E_eV = E_eV;
  P.gamma = E_eV / mass_eV;
  P.beta0 = 1.0 - 1.0 / (2.0 * P.gamma * P.gamma);
  P.U0_eV = U0_eV;
  P.d_p = d_p;
  P.charge_sign = charge_sign > 0 ? 1.0 : -1.0;
  P.eps_s_eV = eps_s_eV;
  P.X0 = X0;
  P.rho = rho;
  P.ms = ms;
  if (!(P.gamma > 1.0) || n_particles < 0) return 1;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t p = 0; p < n_particles; ++p) {
    double ua, ub, z0, z1;
    uniforms2(seed, (uint64_t)p, 0u, &ua, &ub);
    normals2(seed, (uint64_t)p, 0xFFFFFFFEull, 2u, &z0, &z1);
    const double x0 = ua * d_p;
    const double thx0 = sigma_theta * z0;
    const int64_t L = offsets[p + 1] - offsets[p];
    if (entry_x0) entry_x0[p] = x0;
    if (entry_thx) entry_thx[p] = thx0;
    if (L >= 1) run_particle(&P, seed, p, x0, thx0, 0.0, dt, L, out + offsets[p] * NREC);
  }
  return 0;
}

/*
 * Same, with entry conditions given per particle (surrogate training data):
 * x0[p] absolute position, thx0[p] entry angle; energy per particle.
 */
int tg_channeling_given(const double *E_eV, double mass_eV, int charge_sign, double U0_eV,
                        double d_p, double eps_s_eV, double X0, double rho, int ms, double dt,
                        uint64_t seed, int64_t n_particles, const int64_t *offsets,
                        const double *x0, const double *thx0, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t p = 0; p < n_particles; ++p) {
    tg_params P;
    P.E_eV = E_eV[p];
    P.gamma = E_eV[p] / mass_eV;
    P.beta0 = 1.0 - 1.0 / (2.0 * P.gamma * P.gamma);
    P.U0_eV = U0_eV;
    P.d_p = d_p;
    P.charge_sign = charge_sign > 0 ? 1.0 : -1.0;
    P.eps_s_eV = eps_s_eV;
    P.X0 = X0;
    P.rho = rho;
    P.ms = ms;
    const int64_t L = offsets[p + 1] - offsets[p];
    if (L >= 1) run_particle(&P, seed, p, x0[p], thx0[p], 0.0, dt, L, out + offsets[p] * NREC);
  }
  return 0;
}

/* ---------------- energy loss and sections (Sec. II and III) ----------------
 *
 * Radiation reaction: the Landau-Lifshitz force's leading term for an ultra-relativistic
 * particle in a static transverse field is a drag along the velocity whose power is the
 * relativistic Larmor power, dE/dt = -(2/3) alpha hbar c gamma^2 F_perp^2 / (m c^2)^2
 * (c = 1, E in eV, t in m, F in eV/m). The drag leaves v_perp unchanged (d(gamma v_perp)/dt =
 * F_perp/m - (P/m) v_perp with d(gamma)/dt = -P/m), so the transverse equation of motion
 * stays d(v_perp)/dt = F_perp / E(t) with the current energy.
 * Multiple-scattering loss: each kick of angle theta costs dE = m alpha/(2 pi) gamma^3 theta^2.
 *
 * Sections: the trajectory is cut every (S - 1) steps into sections of S samples that share
 * their boundary sample (so trapezoid weights of the sections add up to the whole
 * trajectory's). Each section is its own entry for the radiation integral: its gamma and E
 * are the values when the particle enters it, and its records use that gamma:
 * t and dz restart at 0, dz = z - z_entry - beta0_s (t - t_entry), dvz = v_z - beta0_s.
 */
#define TG_ALPHA 7.2973525693e-3
#define TG_HBARC 1.973269804e-7
#define TG_PI 3.14159265358979323846

typedef struct {
  tg_params P;      /* field, scattering */
  double mass_eV;
  int ll, ms_loss;  /* radiation-reaction drag, scattering energy loss */
} tg_loss_params;

/* v_z and dvz = v_z - beta0_s at energy gamma, section gamma gs (cancellation-free):
 * v_z^2 - beta0_s^2 = (1/gs^2 - 1/g^2) - vp2 - 1/(4 gs^4). */
static void longi_s(double g, double gs, double beta0s, double vp2, double *vz, double *dvz) {
  const double g2 = g * g, gs2 = gs * gs;
  *vz = sqrt(1.0 - 1.0 / g2 - vp2);
  const double dg = ((g - gs) * (g + gs)) / (g2 * gs2);
  *dvz = -((vp2 + 1.0 / (4.0 * gs2 * gs2)) - dg) / (*vz + beta0s);
}

/* field-only transverse acceleration and Larmor energy loss rate at energy E */
static double accel_x_E(const tg_params *P, double x, double E) {
  return accel_x(P, x) * (P->E_eV / E);
}

/* state: x, y, vx, vy, dz_s, E */
static void deriv_loss(const tg_loss_params *Q, double gs, double beta0s, const double s[6],
                       double d[6]) {
  const double g = s[5] / Q->mass_eV;
  double vz, dvz;
  longi_s(g, gs, beta0s, s[2] * s[2] + s[3] * s[3], &vz, &dvz);
  const double ax = accel_x_E(&Q->P, s[0], s[5]);
  d[0] = s[2];
  d[1] = s[3];
  d[2] = ax;
  d[3] = 0.0;
  d[4] = dvz;
  if (Q->ll) {
    const double F = ax * s[5]; /* eV/m */
    d[5] = -(2.0 / 3.0) * TG_ALPHA * TG_HBARC * g * g * (F / Q->mass_eV) * (F / Q->mass_eV);
  } else {
    d[5] = 0.0;
  }
}

static void write_rec_s(const tg_loss_params *Q, double gs, double beta0s, double *rec, double t,
                        const double s[6], double kick_ax, double kick_ay) {
  const double g = s[5] / Q->mass_eV;
  double vz, dvz;
  longi_s(g, gs, beta0s, s[2] * s[2] + s[3] * s[3], &vz, &dvz);
  const double fax = accel_x_E(&Q->P, s[0], s[5]);
  const double ax = fax + kick_ax;
  const double ay = 0.0 + kick_ay;
  /* d(v_z)/dt from d(gamma)/dt (drag) and d(v_perp)/dt */
  double gdot = 0.0;
  if (Q->ll) {
    const double F = fax * s[5];
    gdot = -(2.0 / 3.0) * TG_ALPHA * TG_HBARC * g * g * (F / Q->mass_eV) * (F / Q->mass_eV) / Q->mass_eV;
  }
  rec[R_T] = t;
  rec[R_X] = s[0];
  rec[R_Y] = s[1];
  rec[R_DZ] = s[4];
  rec[R_VX] = s[2];
  rec[R_VY] = s[3];
  rec[R_DVZ] = dvz;
  rec[R_AX] = ax;
  rec[R_AY] = ay;
  rec[R_AZ] = (gdot / (g * g * g) - (s[2] * ax + s[3] * ay)) / vz;
}

/*
 * One particle of L samples (L - 1 RK4 steps of dt) cut into sections of S samples.
 * out: records of its sections, section after section (n_sec(L, S) * S - (shortening of the
 * last section) records, see tg_section_count); sec_E[j]: energy entering section j;
 * e_sample (optional, L values): energy at every sample.
 */
static void run_particle_loss(const tg_loss_params *Q, uint64_t seed, int64_t pid, double x0,
                              double thx0, double thy0, double dt, int64_t L, int64_t S,
                              double *out, double *sec_E, double *e_sample) {
  double s[6] = {x0, 0.0, thx0, thy0, 0.0, Q->P.E_eV};
  double pend_ax = 0.0, pend_ay = 0.0;
  double gs = s[5] / Q->mass_eV, beta0s = 1.0 - 1.0 / (2.0 * gs * gs), t0 = 0.0;
  int64_t sec = 0, r = 0; /* current section, next record slot */
  sec_E[0] = s[5];
  for (int64_t k = 0; k < L; ++k) {
    const double t = (double)k * dt;
    if (e_sample) e_sample[k] = s[5];
    write_rec_s(Q, gs, beta0s, out + (r++) * NREC, t - t0, s, pend_ax, pend_ay);
    if (k > 0 && k % (S - 1) == 0 && k < L - 1) { /* boundary: this sample also opens a section */
      ++sec;
      sec_E[sec] = s[5];
      gs = s[5] / Q->mass_eV;
      beta0s = 1.0 - 1.0 / (2.0 * gs * gs);
      t0 = t;
      s[4] = 0.0;
      write_rec_s(Q, gs, beta0s, out + (r++) * NREC, 0.0, s, pend_ax, pend_ay);
    }
    pend_ax = pend_ay = 0.0;
    if (k == L - 1) break;
    double k1[6], k2[6], k3[6], k4[6], tmp[6];
    deriv_loss(Q, gs, beta0s, s, k1);
    for (int i = 0; i < 6; ++i) tmp[i] = s[i] + 0.5 * dt * k1[i];
    deriv_loss(Q, gs, beta0s, tmp, k2);
    for (int i = 0; i < 6; ++i) tmp[i] = s[i] + 0.5 * dt * k2[i];
    deriv_loss(Q, gs, beta0s, tmp, k3);
    for (int i = 0; i < 6; ++i) tmp[i] = s[i] + dt * k3[i];
    deriv_loss(Q, gs, beta0s, tmp, k4);
    for (int i = 0; i < 6; ++i)
      s[i] = s[i] + (dt / 6.0) * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    if (Q->P.ms) {
      const double E = s[5];
      const double var = 0.5 * (Q->P.eps_s_eV / E) * (Q->P.eps_s_eV / E) * (dt / Q->P.X0) *
                         nuc_density(&Q->P, s[0]);
      double z0, z1;
      normals2(seed, (uint64_t)pid, (uint64_t)k, 1u, &z0, &z1);
      const double dthx = sqrt(var) * z0, dthy = sqrt(var) * z1;
      const double nvx = s[2] + dthx, nvy = s[3] + dthy;
      pend_ax = (nvx - s[2]) / dt;
      pend_ay = (nvy - s[3]) / dt;
      s[2] = nvx;
      s[3] = nvy;
      if (Q->ms_loss) {
        const double g = E / Q->mass_eV;
        s[5] = E - Q->mass_eV * TG_ALPHA / (2.0 * TG_PI) * g * g * g * (dthx * dthx + dthy * dthy);
      }
    }
  }
}

/* Number of sections of a particle of L >= 2 samples cut every S - 1 steps (S >= 2). */
int64_t tg_section_count(int64_t L, int64_t S) { return (L - 2) / (S - 1) + 1; }

/*
 * Ensemble with energy loss, cut into sections (ctypes). Entry conditions as tg_channeling
 * (same seed gives the same entries and, without losses, the same trajectories).
 *   lengths[p]: samples of particle p (>= 2); S: samples per section (>= 2).
 *   rec_off[p]: first record of particle p's sections (caller-computed: a particle has
 *   L + n_sec - 1 records); sec_off[p]: its first section; sec_E[sec_off[p] + j] energies;
 *   e_sample (optional): energy at every sample, particle p from samp_off[p].
 */
int tg_channeling_loss(double E_eV, double mass_eV, int charge_sign, double U0_eV, double d_p,
                       double sigma_theta, double eps_s_eV, double X0, double rho, int ms,
                       int ll, int ms_loss, double dt, uint64_t seed, int64_t n_particles,
                       const int64_t *lengths, int64_t S, const int64_t *rec_off,
                       const int64_t *sec_off, const int64_t *samp_off, double *out,
                       double *sec_E, double *e_sample, double *entry_x0, double *entry_thx) {
  tg_loss_params Q;
  Q.P.E_eV = E_eV;
  Q.P.gamma = E_eV / mass_eV;
  Q.P.beta0 = 1.0 - 1.0 / (2.0 * Q.P.gamma * Q.P.gamma);
  Q.P.U0_eV = U0_eV;
  Q.P.d_p = d_p;
  Q.P.charge_sign = charge_sign > 0 ? 1.0 : -1.0;
  Q.P.eps_s_eV = eps_s_eV;
  Q.P.X0 = X0;
  Q.P.rho = rho;
  Q.P.ms = ms;
  Q.mass_eV = mass_eV;
  Q.ll = ll;
  Q.ms_loss = ms_loss;
  if (!(Q.P.gamma > 1.0) || n_particles < 0 || S < 2) return 1;
  for (int64_t p = 0; p < n_particles; ++p)
    if (lengths[p] < 2) return 1;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t p = 0; p < n_particles; ++p) {
    double ua, ub, z0, z1;
    uniforms2(seed, (uint64_t)p, 0u, &ua, &ub);
    normals2(seed, (uint64_t)p, 0xFFFFFFFEull, 2u, &z0, &z1);
    const double x0 = ua * d_p;
    const double thx0 = sigma_theta * z0;
    if (entry_x0) entry_x0[p] = x0;
    if (entry_thx) entry_thx[p] = thx0;
    run_particle_loss(&Q, seed, p, x0, thx0, 0.0, dt, lengths[p], S, out + rec_off[p] * NREC,
                      sec_E + sec_off[p], e_sample ? e_sample + samp_off[p] : 0);
  }
  return 0;
}

/* Lognormal lengths: L = clip(round(exp(N(ln median, sigma))), lo, hi). */
int tg_lognormal_lengths(uint64_t seed, int64_t n, double median, double sigma, int64_t lo,
                         int64_t hi, int64_t *out) {
  for (int64_t p = 0; p < n; ++p) {
    double z0, z1;
    normals2(seed, (uint64_t)p, 0xFFFFFFFDull, 3u, &z0, &z1);
    double v = exp(log(median) + sigma * z0);
    int64_t L = (int64_t)floor(v + 0.5);
    if (L < lo) L = lo;
    if (L > hi) L = hi;
    out[p] = L;
  }
  return 0;
}
