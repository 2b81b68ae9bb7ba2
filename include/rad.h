/*
 * rad.h -- C ABI of the GB300 (sm_103a) radiation-integral library.
 *
 * The library evaluates the Lienard-Wiechert radiation integral of
 * C. F. Nielsen, "GPU Accelerated Simulation of Channeling Radiation of
 * Relativistic Particles" (arXiv:1910.10391), Sec. II:
 *
 *   d2I/(dw dOmega) = e^2/(4 pi^2) | int f(t, n) exp(i w (t - n.x(t))) dt |^2      (Eq. 1, 2)
 *
 * in the paper's small-angle expanded form (f_x, f_y, f_z, g and the phase of
 * Sec. II), for many trajectories at once, on a grid of photon energies hw_i and
 * emission directions n_j = (theta_x, theta_y), in three models:
 *   RAD_CLASSICAL  Eq. 1 as is;
 *   RAD_SPIN0      Lindhard substitution w -> w* = w/(1 - hw/E), intensity scaled by
 *                  w/w* (Sec. II, Eq. Lindhard_substi), applied per direction;
 *   RAD_SPIN_HALF  Belkacem-Cue-Kimball / Baier-Katkov semiclassical formula
 *                  (Sec. II, Eqs. cue, Iterm, J): (E*^2+E^2)/(2E^2) |I|^2 +
 *                  hw^2/(2 E^2 gamma^2) |J|^2 with I, J at w*, E* = E - hw.
 *
 * Conventions (all entry points):
 *   - c = 1; times and lengths in metres; photon energies in eV; w = hw/(hbar c).
 *   - Trajectory record: 10 float64 per time sample, in this order
 *       t, x, y, dz, vx, vy, dvz, ax, ay, az
 *     with dz = z - beta0 t, dvz = v_z - beta0, beta0 := 1 - 1/(2 gamma^2), and
 *     (ax, ay, az) = d(beta)/dt. Particle p owns records offsets[p] .. offsets[p+1]-1
 *     of one contiguous array; each particle needs at least 2 samples.
 *     Sections of a trajectory with different energies (Sec. II, energy loss) are
 *     passed as separate particles with their own gamma and energy.
 *   - Time integral: trapezoid weights (t_{k+1} - t_{k-1})/2, one-sided at the ends.
 *   - Output: d2I/(d(hw) dOmega), dimensionless, = alpha/(4 pi^2) * sum_p weight_p S_p,
 *     cube layout out_cube[i * n_angles + j] (i: photon energy, j: direction).
 *     out_spectrum[i] = sum_j cube[i][j] * d_omega[j]   (dI/d(hw), angle integral of Sec. IV)
 *     out_bins[i * n_bins + b] = sum over j with bin_of_angle[j] == b of cube[i][j] d_omega[j]
 *     (bin_of_angle[j] < 0 or >= n_bins excludes direction j).
 *   - Pointers named "device" must be device memory of the current CUDA device
 *     (cudaMalloc/torch); the caller owns them. samples must be 16-byte aligned.
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*; NULL is the
 *     legacy default stream). Host-side argument checks run before anything is
 *     enqueued: on failure nothing is enqueued and the error code is returned.
 *     Checks that need device data (finite values, offsets, gamma > 1, hw > 0,
 *     hw < E in quantum modes) run in a small kernel on the same stream; a failure
 *     skips the computation and is recorded in the per-device status word read by
 *     rad_device_status(). RAD_MIXED also bounds its in-tile phase offsets on the device
 *     and records RAD_EPRECISION when they exceed its error budget (see
 *     rad_plan_set_phase_budget). Outputs of a call whose device checks failed are left
 *     unchanged.
 *   - Each device-side wait in the kernels has an iteration limit; if it runs out
 *     the kernel records RAD_ETIMEOUT in the status word and returns.
 *   - There is no CPU fallback: without a usable sm_103a device every compute entry
 *     point returns RAD_ECUDA.
 */
#ifndef RAD_H
#define RAD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define RAD_OK 0
#define RAD_EINVAL 1       /* bad argument (null pointer, negative size, bad enum, ...)   */
#define RAD_ENOMEM 2       /* device allocation failed                                    */
#define RAD_ECUDA 3        /* a CUDA call failed; rad_status_string(RAD_ECUDA) has detail  */
#define RAD_ETIMEOUT 4     /* a bounded device-side wait ran out                          */
#define RAD_EUNSUPPORTED 5 /* valid request this build cannot serve (e.g. no sm_103a GPU) */
#define RAD_EDATA 6        /* device-side data check failed (see rad.h conventions)       */
#define RAD_ETOOBIG 7      /* request exceeds rad_spectrum_noalloc's fixed scratch        */
#define RAD_EPRECISION 8   /* RAD_MIXED: in-tile phase offsets beyond its error budget;   */
                           /* the same call in RAD_FP64_DF has no such limit              */

/* ---- enums ---- */
#define RAD_CLASSICAL 0
#define RAD_SPIN0 1
#define RAD_SPIN_HALF 2

#define RAD_FP64 0  /* every operation in FP64 (the paper's precision, Sec. IV)          */
#define RAD_MIXED 1 /* FP64 phase base and particle sums; FP32 sincos, f and tile sums   */
/* RAD_FP64_DF: FP64 accuracy with the FP64 phase product of RAD_FP64, reduced exactly by
 * fixed-point integer arithmetic, then double-float FP32 arithmetic (float pairs) for sin, cos,
 * f and compensated tile sums, and FP64 particle sums: the RAD_FP64 tolerance with a small
 * fraction of its FP64 instructions (GB300 runs FP64 at 1/64 of FP32). */
#define RAD_FP64_DF 2

#define RAD_NREC 10 /* float64 fields per trajectory record */

/*
 * rad_spectrum -- one call of the hot path (Sec. II integral, Sec. IV grid of
 * N_x x N_y x N_omega integrals per trajectory, angle sum and particle average).
 *
 *   samples          device, [n_samples_total][10] float64 records (layout above)
 *   offsets          device, [n_particles + 1] int64, offsets[0] = 0,
 *                    offsets[n_particles] = n_samples_total, nondecreasing with
 *                    offsets[p+1] - offsets[p] >= 2
 *   gamma            device, [n_particles] Lorentz factor (> 1) of each particle/section
 *   energy_eV        device, [n_particles] particle energy E (used by quantum modes)
 *   weight           device, [n_particles] ensemble weight, or NULL for all 1
 *   hbar_omega_eV    device, [n_omega] photon energies (> 0; < E in quantum modes)
 *   theta_x, theta_y device, [n_angles] transverse components of n (radians)
 *   d_omega          device, [n_angles] solid angle of each direction cell; may be NULL
 *                    when neither out_spectrum nor out_bins is requested
 *   mode             RAD_CLASSICAL | RAD_SPIN0 | RAD_SPIN_HALF
 *   precision        RAD_FP64 | RAD_MIXED | RAD_FP64_DF
 *   out_cube         device, [n_omega * n_angles] or NULL
 *   out_spectrum     device, [n_omega] or NULL
 *   bin_of_angle     device, [n_angles] int32 or NULL (required when out_bins != NULL)
 *   n_bins           number of radial/angular bins (>= 1 when out_bins != NULL)
 *   out_bins         device, [n_omega * n_bins] or NULL
 *   accumulate       0: outputs are overwritten; 1: results are added to them
 *   stream           cudaStream_t as void*
 * Returns RAD_OK when the work was enqueued. n_particles, n_omega or n_angles equal
 * to 0 is valid: outputs are zeroed (accumulate = 0) or left as they are. RAD_EINVAL when
 * n_omega or n_angles exceeds 2^31, or when the call would split into more than about 2^31
 * work items (RAD_FP64_DF takes one direction per item: at most about 2^31 directions per 256
 * photon energies).
 * Scratch memory is allocated by the library on first use of a shape and reused
 * (see rad_release). Thread-safe; concurrent calls on different streams are allowed.
 */
int rad_spectrum(const double *samples, int64_t n_samples_total, const int64_t *offsets,
                 int64_t n_particles, const double *gamma, const double *energy_eV,
                 const double *weight, const double *hbar_omega_eV, int64_t n_omega,
                 const double *theta_x, const double *theta_y, const double *d_omega,
                 int64_t n_angles, int mode, int precision, double *out_cube,
                 double *out_spectrum, const int32_t *bin_of_angle, int32_t n_bins,
                 double *out_bins, int accumulate, void *stream);

/*
 * rad_angular_distribution -- the energy radiated per solid angle over the photon-energy grid,
 * dI/dOmega (Sec. IV, the second integral test: the angular distribution integrated over a
 * photon-energy range): out[j] = sum_{i < n_omega - 1} (hw[i+1] - hw[i]) (cube[i][j] +
 * cube[i+1][j]) / 2, the trapezoid rule in photon energy over the cube rad_spectrum writes.
 *   cube           device, [n_omega * n_angles] (layout of rad_spectrum's out_cube)
 *   hbar_omega_eV  device, [n_omega], the cube's photon energies (eV), increasing
 *   out            device, [n_angles], overwritten (zero when n_omega < 2)
 * Asynchronous on `stream`; the sum over energies runs in a fixed order (deterministic).
 * RAD_EINVAL for negative sizes or a NULL pointer that is needed.
 */
int rad_angular_distribution(const double *cube, const double *hbar_omega_eV, int64_t n_omega,
                             int64_t n_angles, double *out, void *stream);

/*
 * rad_spectrum_host -- rad_spectrum on HOST arrays (same arguments, all pointers
 * host memory; pinned memory gives the fastest copies). Copies the inputs to the
 * device, computes, copies the requested outputs back and returns when they are
 * complete. Uses library-owned device buffers, grown as needed and reused.
 * Device-side data check failures are returned as RAD_EDATA.
 */
int rad_spectrum_host(const double *samples, int64_t n_samples_total, const int64_t *offsets,
                      int64_t n_particles, const double *gamma, const double *energy_eV,
                      const double *weight, const double *hbar_omega_eV, int64_t n_omega,
                      const double *theta_x, const double *theta_y, const double *d_omega,
                      int64_t n_angles, int mode, int precision, double *out_cube,
                      double *out_spectrum, const int32_t *bin_of_angle, int32_t n_bins,
                      double *out_bins, int accumulate, void *stream);

/*
 * rad_spectrum_noalloc -- the mixed-precision cube with no device allocation at all.
 * The paper has no counterpart; this serves callers that cannot allocate device memory:
 * processes whose GPU memory is already held by another framework's caching allocator
 * (a cudaMalloc of the library would fail there), and latency-critical loops in which
 * cudaMalloc/cudaFree would synchronize the device.
 *   Arguments as rad_spectrum (all device pointers), precision fixed to RAD_MIXED, output
 *   out_cube only ([n_omega * n_angles], overwritten). d_omega, spectrum and bins are not
 *   part of this entry point.
 *   Scratch: one fixed device array of 32 MiB inside the library, held by every GPU that
 *   loads the library until the process exits. Requests with n_omega * n_angles above
 *   (32 MiB - 256 B) / 8 = 4,194,272 bins return RAD_ETOOBIG before anything is enqueued.
 *   The first call on a device looks up the array's device address (once per device, with
 *   that device current) and keeps it for the life of the process; make that first call
 *   outside any stream capture. cudaDeviceReset unloads the library's device code, so the
 *   kept address is stale afterwards: a process that resets a device must not call this
 *   entry point on that device again.
 *   Every call shares the array: calls that overlap on the GPU (other streams, other host
 *   threads) race on it, so the caller must serialize them. Each call clears the control
 *   words it needs and leaves its partial sums in the array.
 *   Synchronous: returns after the cube is complete; device-side data check failures
 *   come back as RAD_EDATA and phase offsets beyond the mixed form's default error budget
 *   (see rad_plan_set_phase_budget) as RAD_EPRECISION (the cube is then left unchanged),
 *   bounded-wait expiry as RAD_ETIMEOUT. Calls no cudaMalloc, cudaFree or allocating library
 *   routine.
 */
int rad_spectrum_noalloc(const double *samples, int64_t n_samples_total, const int64_t *offsets,
                         int64_t n_particles, const double *gamma, const double *energy_eV,
                         const double *weight, const double *hbar_omega_eV, int64_t n_omega,
                         const double *theta_x, const double *theta_y, int64_t n_angles, int mode,
                         double *out_cube, void *stream);

/*
 * rad_spectrum_particles -- the same integral without the particle sum: one spectrum per
 * particle (Sec. IV's angle integral per trajectory), e.g. to build per-particle training sets.
 *   out_spectrum [n_particles][n_omega] (or NULL), out_bins [n_particles][n_omega][n_bins]
 *   (or NULL, n_bins <= 16): alpha/(4 pi^2) weight_p sum_j S_p(i, j) d_omega[j] (per bin).
 *   d_omega is required. Other arguments, checks and asynchrony as rad_spectrum; results
 *   overwrite the outputs. Scratch grows with n_particles * n_omega * n_angles doubles.
 */
int rad_spectrum_particles(const double *samples, int64_t n_samples_total, const int64_t *offsets,
                           int64_t n_particles, const double *gamma, const double *energy_eV,
                           const double *weight, const double *hbar_omega_eV, int64_t n_omega,
                           const double *theta_x, const double *theta_y, const double *d_omega,
                           int64_t n_angles, int mode, int precision, double *out_spectrum,
                           const int32_t *bin_of_angle, int32_t n_bins, double *out_bins, void *stream);

#define RAD_PER_PARTICLE 8 /* rad_plan_create `want` bit: per-particle spectrum/bins (no cube) */

/* ---- plans: bind a shape once, then execute, autotune or capture into a CUDA graph ---- */
typedef struct rad_plan_s *rad_plan;

/*
 * rad_plan_create -- validates the shape and allocates the scratch it needs.
 *   n_samples_total, n_particles, n_omega, n_angles, mode, precision: as rad_spectrum;
 *   want: bit mask of outputs (1 cube, 2 spectrum, 4 bins); n_bins for bins; with
 *   RAD_PER_PARTICLE (8) the spectrum and bins are per particle and the cube is not available
 *   (rad_plan_execute then writes [n_particles][...] outputs as rad_spectrum_particles does).
 * On success *plan receives a handle owned by the caller (rad_plan_destroy).
 * Allocation happens here, so a plan can be executed inside CUDA stream capture.
 */
int rad_plan_create(int64_t n_samples_total, int64_t n_particles, int64_t n_omega,
                    int64_t n_angles, int mode, int precision, int want, int32_t n_bins,
                    rad_plan *plan);

/* rad_plan_execute -- same pointer arguments as rad_spectrum, for the plan's shape. */
int rad_plan_execute(rad_plan plan, const double *samples, const int64_t *offsets,
                     const double *gamma, const double *energy_eV, const double *weight,
                     const double *hbar_omega_eV, const double *theta_x, const double *theta_y,
                     const double *d_omega, double *out_cube, double *out_spectrum,
                     const int32_t *bin_of_angle, double *out_bins, int accumulate, void *stream);

/*
 * rad_plan_autotune -- times the plan's candidate launch shapes (frequencies per
 * thread, warps per block, time-tile length, work split) on the given inputs for at
 * most about budget_ms milliseconds, keeps the fastest in the plan and in the
 * library's tuning cache (used by rad_spectrum for the same shape). Synchronous.
 * Writes to the outputs (they hold a valid result of the chosen shape on return).
 */
int rad_plan_autotune(rad_plan plan, const double *samples, const int64_t *offsets,
                      const double *gamma, const double *energy_eV, const double *weight,
                      const double *hbar_omega_eV, const double *theta_x, const double *theta_y,
                      const double *d_omega, double *out_cube, double *out_spectrum,
                      const int32_t *bin_of_angle, double *out_bins, int budget_ms, void *stream);

/*
 * rad_plan_set_shape -- selects the plan's launch shape explicitly:
 *   R           photon energies per thread (FP64: 1, 2, 4; FP64_DF: 1, 2; mixed: 1, 2, 4)
 *   NW          warps per block (4 or 8). FP64 and mixed: each warp takes its own direction
 *               (a work item is NW directions x 32 R energies). FP64_DF: the block takes one
 *               direction and each warp its own 32 R energies (NW x 32 R energies per item)
 *   T           time-tile length (FP64, FP64_DF: 64; mixed: 64, 128 or 256)
 *   chunk_mult  >= 1, multiplies the default number of work items (finer split)
 * Returns RAD_EINVAL for a shape this build does not provide (the plan is unchanged).
 * May reallocate scratch (waits for the device); not allowed during stream capture.
 */
int rad_plan_set_shape(rad_plan plan, int R, int NW, int T, int chunk_mult);

/*
 * rad_plan_set_prepass -- mixed precision only: enable != 0 selects the kernel fed by a
 * per-sample pre-pass (FP64 preparation once per sample, 48 bytes of scratch per sample),
 * 0 the kernel that prepares each time tile itself (no per-sample scratch). The current
 * (R, NW, T) must exist for the chosen kernel, else RAD_EINVAL (plan unchanged). When
 * rad_plan_set_shape asks for a shape only the other kernel provides, it switches kernels.
 */
int rad_plan_set_prepass(rad_plan plan, int enable);

/*
 * rad_plan_set_sincos_split -- pre-pass kernel only: every = 4 or 6 evaluates the sin/cos of the
 * terms whose index is every - 1 mod every in each group of 8 samples x R energies (R = 2: 1/4 or
 * 1/8 of them) on the FMA pipe (Cody-Waite reduction to |r| <= pi/4, Taylor polynomials; same
 * error bound as the SFU's on the in-tile phases) instead of the SFU, so that both pipes share
 * the work; 0 uses the SFU for every term. A new plan starts with 6 for the classical and spin-0
 * models and 0 for spin-1/2. RAD_EINVAL for other values, FP64 plans or the inline-preparation
 * kernel (plan unchanged). The autotuner also tries these.
 */
int rad_plan_set_sincos_split(rad_plan plan, int every);

/*
 * rad_plan_set_phase_budget -- RAD_MIXED plans only: the error-budget guard's limit, in radians
 * (default 8192). Every RAD_MIXED call bounds its in-tile phase offsets on the device,
 *   X = max over particles and samples of w*_max (c_max |t_k - t_ref| + |dz_k - dz_ref|
 *       + max|theta_x| |x_k - x_ref| + max|theta_y| |y_k - y_ref|),
 * with t_ref etc. the middle sample of the sample's time tile, c_max = 1/(2 gamma^2) + max
 * theta^2/2 over the grid and w*_max the particle's largest w* (Sec. II phase). The per-term phase
 * error of the FP32 offsets and the SFU sin/cos grows in proportion to X (about 2.7e-7 X rad); a
 * call with X above the limit records RAD_EPRECISION in the status word and leaves its outputs
 * unchanged. Raise the limit only where a larger error is acceptable; RAD_FP64_DF has no such
 * limit. RAD_EINVAL for a non-positive or non-finite value or a plan of another precision.
 */
int rad_plan_set_phase_budget(rad_plan plan, double radians);

/*
 * rad_plan_describe -- writes a short text description of the plan's chosen launch
 * shape into buf (at most len bytes, NUL-terminated). Returns RAD_OK.
 */
int rad_plan_describe(rad_plan plan, char *buf, int len);

/*
 * rad_plan_set_timing -- enable != 0 makes every later rad_plan_execute of this plan
 * record CUDA events on its stream just before and after the main integral kernel (after
 * the mixed kernel's per-sample pre-pass, which is not included);
 * rad_plan_last_kernel_ms waits for the last recorded pair and returns the main
 * kernel's duration in milliseconds in *ms. Do not enable timing on a plan that is
 * captured into a graph.
 */
int rad_plan_set_timing(rad_plan plan, int enable);
int rad_plan_last_kernel_ms(rad_plan plan, double *ms);

/* rad_plan_kernel_launches -- number of kernel launches one execute enqueues. */
int rad_plan_kernel_launches(rad_plan plan);

/* rad_plan_destroy -- frees the plan's scratch (waits for the device first). */
int rad_plan_destroy(rad_plan plan);

/*
 * CUDA graphs: rad_graph_create captures one rad_plan_execute with the given pointers
 * on `stream` into an executable graph; rad_graph_launch replays it on any stream.
 * The pointers are baked into the graph. The plan must outlive the graph.
 */
typedef struct rad_graph_s *rad_graph;
int rad_graph_create(rad_plan plan, const double *samples, const int64_t *offsets,
                     const double *gamma, const double *energy_eV, const double *weight,
                     const double *hbar_omega_eV, const double *theta_x, const double *theta_y,
                     const double *d_omega, double *out_cube, double *out_spectrum,
                     const int32_t *bin_of_angle, double *out_bins, int accumulate, void *stream,
                     rad_graph *graph);
int rad_graph_launch(rad_graph graph, void *stream);
int rad_graph_destroy(rad_graph graph);

/* ---- surrogate MLP (learned per-particle spectra; not part of the paper) ----
 *
 * A fully connected network x (n_in) -> depth x [Linear(width) -> GELU] -> Linear(n_out),
 * trained on spectra computed by rad_spectrum. The first layer is FP32; the others use BF16
 * weights and activations with FP32 accumulation on the tensor cores. FP32 master weights,
 * AdamW updates, mean-squared-error loss. All float pointers below are DEVICE pointers unless
 * named host_*; calls are asynchronous on `stream` except create/destroy/get/set.
 */
typedef struct rad_mlp_s *rad_mlp;

/* rad_mlp_create -- allocates a network for batches of up to max_batch rows (width and n_out
 * even, width <= 8192, n_out <= 65536, n_in <= 64, max_batch <= 4,194,240; RAD_EINVAL
 * otherwise); weights uniform in +-1/sqrt(fan_in) from `seed`, biases 0. */
int rad_mlp_create(int n_in, int width, int depth, int n_out, int64_t max_batch, uint64_t seed,
                   rad_mlp *out);
int rad_mlp_destroy(rad_mlp mlp);
int64_t rad_mlp_num_params(rad_mlp mlp);

/* rad_mlp_forward -- y [batch][n_out] = network(x [batch][n_in]); any batch size. */
int rad_mlp_forward(rad_mlp mlp, const float *x, int64_t batch, float *y, void *stream);

/* rad_mlp_backward -- forward pass, loss = mean(mask (y - target)^2) over all batch x n_out
 * elements written to *loss (device, may be NULL), and the gradient of the loss w.r.t. every
 * parameter kept in the network (batch <= max_batch). mask [batch][n_out] of nonnegative
 * weights m (loss = sum m (y - target)^2 / (batch n_out)), or NULL for all ones. */
int rad_mlp_backward(rad_mlp mlp, const float *x, const float *target, const float *mask, int64_t batch,
                     float *loss, void *stream);

/* rad_mlp_adamw -- one AdamW update of all parameters from the stored gradients. */
int rad_mlp_adamw(rad_mlp mlp, float lr, float beta1, float beta2, float eps, float weight_decay,
                  void *stream);

/* rad_mlp_train_step -- rad_mlp_backward then rad_mlp_adamw (beta 0.9/0.999, eps 1e-8). */
int rad_mlp_train_step(rad_mlp mlp, const float *x, const float *target, const float *mask, int64_t batch,
                       float lr, float weight_decay, float *loss, void *stream);

/* rad_mlp_get -- copies parameters (what 0), gradients (1) or Adam moments (2, 3) to host_out
 * [rad_mlp_num_params]. Layout per layer l = 0..depth: W_l [out][in] row-major, then b_l [out]. */
int rad_mlp_get(rad_mlp mlp, int what, float *host_out);
/* rad_mlp_set_params -- loads parameters (same layout) from host memory (checkpoint restore). */
int rad_mlp_set_params(rad_mlp mlp, const float *host_in);

/* rad_mlp_ensemble_estimate -- preds [n_models][batch][n_out] of log10 spectra -> mean
 * [batch][n_out] (mu_o) and err[batch] = ln(10) sqrt(sum_o s_o^2 var_o / sum_o s_o^2) with
 * s_o = 10^mu_o and var_o the unbiased variance over models: the relative L2 error of the
 * spectrum implied, to first order, by the ensemble spread (the surrogate's error estimate). */
int rad_mlp_ensemble_estimate(const float *preds, int n_models, int64_t batch, int n_out, float *mean,
                              float *err, void *stream);

/* rad_log_targets -- out[i] = log10(max(values[i], floor_value)) (FP64 in, FP32 out). */
int rad_log_targets(const double *values, int64_t n, double floor_value, float *out, void *stream);
/* rad_column_stats -- per-column mean and standard deviation of y [rows][cols]. */
int rad_column_stats(const float *y, int64_t rows, int cols, float *mean, float *stdv, void *stream);
/* rad_standardize -- y = (y - mean) / std per column, or the inverse when inverse != 0. */
int rad_standardize(float *y, int64_t rows, int cols, const float *mean, const float *stdv, int inverse,
                    void *stream);

/* ---- trajectories on the GPU (Sec. III) ---- */

/* Flags of rad_channel.flags */
#define RAD_TRAJ_MS 1      /* multiple Coulomb scattering kicks after every step            */
#define RAD_TRAJ_LL 2      /* radiation-reaction drag (leading Landau-Lifshitz term)        */
#define RAD_TRAJ_MS_LOSS 4 /* energy loss of each kick, m alpha/(2 pi) gamma^3 theta^2       */
#define RAD_TRAJ_FP32 8    /* FP32 arithmetic with double-float state (else FP64 throughout)  */
#define RAD_TRAJ_MS_EL 16  /* scattering on valence electrons too (rad_crystal_trajectories)  */

/* Planar channel of the trajectory integrator: a harmonic well U(s) = U0 (2 s / d_p)^2 in the
 * distance s to the nearest channel centre (a stand-in for the planar continuum potential of
 * Sec. III, whose Doyle-Turner tables the paper does not print), and the nuclear
 * multiple-scattering model of Sec. III. rad_crystal_trajectories replaces the well by the
 * Doyle-Turner planar potential with the caller's fit (rad_planar_potential, below), and may add
 * scattering on valence electrons. */
typedef struct {
  double U0_eV;    /* well depth, eV (>= 0)                                                 */
  double d_p;      /* interplanar distance, m (> 0)                                         */
  double eps_s_eV; /* scattering energy constant (10.6 MeV in Sec. III), eV                 */
  double X0;       /* radiation length, m (> 0 with RAD_TRAJ_MS)                             */
  double rho;      /* thermal amplitude of the Gaussian plane density, m (> 0 with MS)       */
  double mass_eV;  /* rest energy of the particle, eV (> 0)                                  */
  int charge_sign; /* +1: channel centres mid-way between planes; -1: centres on the planes */
  int flags;       /* RAD_TRAJ_* bits                                                        */
} rad_channel;

/* Thermally averaged Doyle-Turner continuum potential of a family of planes (Sec. III, Eq. plane)
 * and the valence-electron density of the same planes (Sec. III). The fit coefficients are the
 * caller's (the paper prints no tables). Planes sit at x = m d_p; a unit positive charge feels
 *   U(x) = 2 sqrt(pi) e^2 a0 N d_p sum_planes sum_i a[i] / sqrt(C_i) exp(-r^2 / C_i),
 *   C_i = b[i] / (4 pi^2) + rho^2 (rho of rad_channel), r = distance to the plane,
 * summed over the 2 n_neighbours planes m0 - n_neighbours + 1 .. m0 + n_neighbours around the
 * cell m0 = floor(x / d_p) that holds x. A particle of charge sign q feels q U. With
 * RAD_TRAJ_MS_EL the electron density
 *   n_el(x) = (N d_p / sqrt(pi)) sum_planes sum_i ax[i] / sqrt(CX_i) exp(-r^2 / CX_i)
 *             + cx N n(x)/N,   CX_i = bx[i] / (4 pi^2) + rho^2,
 * (n(x)/N the nuclear plane density of rad_channel's scattering model) sets a second kick
 * variance per angle, (1/2) dt pi r0^2 / (gamma^2 beta^4) max(ln(2 m_e gamma^2 beta^2 / I) -
 * beta^2, 0) n_el(x) (Sec. III, the paper's electron term with its factor 2 removed). */
typedef struct {
  int n_terms;      /* Gaussian terms of each fit, 1 .. 8 (the paper's fits have 4)              */
  int n_neighbours; /* planes summed on each side of the particle's cell, 1 .. 8                */
  double N;         /* atom density, m^-3 (> 0)                                                 */
  double a[8];      /* potential fit a_i, m (finite)                                            */
  double b[8];      /* potential fit b_i, m^2 (C_i must be > 0)                                 */
  double ax[8];     /* X-ray fit a_i^(X), electrons (finite; used with RAD_TRAJ_MS_EL)          */
  double bx[8];     /* X-ray fit b_i^(X), m^2 (CX_i > 0 with RAD_TRAJ_MS_EL)                    */
  double cx;        /* X-ray constant c^(X), electrons at the nucleus (finite)                  */
  double I_eV;      /* mean ionisation energy of the target, eV (> 0 with RAD_TRAJ_MS_EL)        */
} rad_planar_potential;

/*
 * rad_channeling_trajectories -- integrates n_particles trajectories in the channel `ch` and
 * writes their records in the layout every rad_spectrum* entry point reads (Sec. II
 * variables), one thread per particle.
 *   Equations (c = 1, metres, eV): dx/dt = v_x, dy/dt = v_y, dv_x/dt = F(x)/E with
 *   F = -8 U0 s/d_p^2, dv_y/dt = 0, d(dz)/dt = v_z - beta0 with beta0 = 1 - 1/(2 gamma0^2)
 *   from the entry energy, v_z = sqrt(1 - 1/gamma^2 - v_perp^2), and with RAD_TRAJ_LL
 *   dE/dt = -(2/3) alpha hbar c gamma^2 F^2/m^2 (Sec. III, Landau-Lifshitz force). One
 *   classical Runge-Kutta (RK4) step of dt between samples. With RAD_TRAJ_MS, after every
 *   step both angles get Gaussian kicks of variance (1/2)(eps_s/E)^2 (dt/X0) n(x)/N, n(x)/N =
 *   d_p/(sqrt(pi) rho) sum over the two nearest planes of exp(-r^2/rho^2); the next sample's
 *   acceleration carries the kick as delta_v/dt; with RAD_TRAJ_MS_LOSS the kick costs
 *   m alpha/(2 pi) gamma^3 theta^2 of energy (Sec. III). Normals: Philox4x32-10 (Salmon et
 *   al., SC'11), counter (id low word, step, 1, id high word), key (seed low, seed high);
 *   u = ((a >> 5) 2^26 + (b >> 6) + 1/2) 2^-53 from output words (0,1) and (2,3); Box-Muller
 *   z0 = r cos(2 pi u2), z1 = r sin(2 pi u2), r = sqrt(-2 ln u1).
 *   Records: t = k dt, x, y, dz, v_x, v_y, dvz = v_z - beta0, a_x = F/E + kick, a_y = kick,
 *   a_z = (dgamma/dt / gamma^3 - v_perp . a_perp)/v_z. Particle p owns records
 *   offsets[p] .. offsets[p+1]-1 (device int64, n_particles + 1 values, within
 *   [0, n_samples_total]) and starts at x0[p], v_x = thx0[p], v_y = thy0[p] (thy0 may be NULL
 *   for 0), y = dz = 0, energy energy_eV[p] (> mass); particle_ids[p] (device, may be NULL for
 *   p) selects its random stream. All arrays are device memory; out holds n_samples_total
 *   records; energy_out (optional, n_samples_total doubles) receives the energy at every
 *   sample. Asynchronous on `stream`; host checks (null pointers, dt > 0, channel values,
 *   unknown flags) return RAD_EINVAL before anything is enqueued; a particle with bad
 *   offsets, non-finite entry values or energy <= mass is skipped and RAD_EDATA is recorded
 *   for rad_device_status().
 */
/*   Precision: FP64 throughout by default. With RAD_TRAJ_FP32 the stages are evaluated in FP32
 *   and every state variable is kept as a double-float (hi + lo, about 48 bits) updated with
 *   error-free sums and products; the channel offset replaces the absolute position (channel
 *   index + offset); records are then within about 1e-7 relative of the FP64 form for
 *   channeled motion (dvz, a_x, a_y, a_z carry FP32 precision). */
int rad_channeling_trajectories(const rad_channel *ch, int64_t n_particles, const int64_t *offsets,
                                int64_t n_samples_total, const double *energy_eV, const double *x0,
                                const double *thx0, const double *thy0, const int64_t *particle_ids,
                                double dt, uint64_t seed, double *out, double *energy_out, void *stream);

/*
 * rad_crystal_trajectories -- rad_channeling_trajectories in the Doyle-Turner planar potential
 * `pot` (host struct, read during the call) instead of the harmonic well: F = -q dU/dx with U
 * above, q = ch->charge_sign (U0_eV is ignored). Every other argument, the records, the random
 * streams and both precisions are those of rad_channeling_trajectories. Flags may add
 * RAD_TRAJ_MS_EL (needs RAD_TRAJ_MS). Host checks (null ch or pot, n_terms or n_neighbours out of
 * range, N <= 0, a non-finite coefficient, C_i <= 0, with RAD_TRAJ_MS_EL CX_i <= 0 or I_eV <= 0,
 * a derived force or density coefficient that is not finite in the precision used (with
 * RAD_TRAJ_FP32: in FP32), and the checks of rad_channeling_trajectories) return RAD_EINVAL before
 * anything is enqueued.
 */
int rad_crystal_trajectories(const rad_channel *ch, const rad_planar_potential *pot, int64_t n_particles,
                             const int64_t *offsets, int64_t n_samples_total, const double *energy_eV,
                             const double *x0, const double *thx0, const double *thy0,
                             const int64_t *particle_ids, double dt, uint64_t seed, double *out,
                             double *energy_out, void *stream);

/* ---- crystal geometry (Sec. IV: the placement of strings and planes in FCC and BCC crystals,
 *      in the (100), (110), (111) planes and <100>, <110>, <111> axes) ---- */
#define RAD_DIAMOND 0 /* diamond cubic (FCC lattice, two-atom basis): Si, C, Ge */
#define RAD_BCC 1     /* body-centred cubic: W                                  */
#define RAD_SI 0
#define RAD_C 1
#define RAD_GE 2
#define RAD_W 3

/* Element presets: structure, cubic lattice constant a (m), atomic number, mean ionisation energy
 * (eV) and radiation length (m): standard tabulated material constants, not values from the paper
 * (the Doyle-Turner fit coefficients stay the caller's). */
typedef struct {
  int structure; /* RAD_DIAMOND or RAD_BCC */
  double a;      /* lattice constant, m   */
  int Z;
  double I_eV;
  double X0;
} rad_element;

/* The strings of an axis seen in the transverse plane: a rectangular cell cell_x x cell_y
 * repeated over the plane, with n_strings strings at (sx[k], sy[k]) in it; d is the mean distance
 * between atoms along a string, so the atom density is n_strings / (d cell_x cell_y). */
typedef struct {
  int n_strings;          /* 1 .. 8 */
  double cell_x, cell_y;  /* m      */
  double sx[8], sy[8];    /* m      */
  double d;               /* m      */
} rad_string_lattice;

/* The planes of a family along its normal: n_planes planes at offset[k] in every period, each
 * holding areal[k] atoms per unit area. Equidistant families have n_planes = 1 (the planar
 * potential's d_p is then the period and N d_p the areal density). */
typedef struct {
  int n_planes;      /* 1 .. 4 */
  double period;     /* m      */
  double offset[4];  /* m, in [0, period) */
  double areal[4];   /* m^-2   */
} rad_plane_stack;

/* rad_crystal_element -- the preset of element RAD_SI, RAD_C, RAD_GE or RAD_W. RAD_EINVAL for
 * another value or a NULL out. Host only. */
int rad_crystal_element(int element, rad_element *out);

/* rad_crystal_string_lattice -- the string lattice of the axis <100>, <110> or <111> (axis =
 * 100, 110, 111) of a crystal of the given structure and lattice constant a (> 0), in the frame
 * x along [010], y along [001] (<100>); x along [001], y along [1-10] (<110>); x along [1-10], y
 * along [11-2] (<111>). RAD_EINVAL for another structure or axis, a <= 0 or a NULL out. Host only. */
int rad_crystal_string_lattice(int structure, double a, int axis, rad_string_lattice *out);

/* rad_crystal_plane_stack -- the plane family (100), (110) or (111) (plane = 100, 110, 111) of
 * a crystal of the given structure and lattice constant. Diamond (111) is a stack of pairs of
 * planes (n_planes = 2); the others are equidistant. RAD_EINVAL as above. Host only. */
int rad_crystal_plane_stack(int structure, double a, int plane, rad_plane_stack *out);

/* Thermally averaged Doyle-Turner continuum potential of the strings of an axis (Sec. III,
 * Eq. string) and their electron density (Sec. III). A unit positive charge feels
 *   U(x, y) = sum_strings (2 e^2 a0 / d) sum_i a[i] / C_i exp(-r^2 / C_i),
 *   C_i = b[i] / (4 pi^2) + rho^2 (rho of rad_channel), r = distance to the string,
 * summed over the strings of the (2 n_cells + 1)^2 cells around the cell (floor(x / cell_x),
 * floor(y / cell_y)) that holds the particle. With RAD_TRAJ_MS the kicks take the strings'
 * nuclear density, n(x, y)/N = sum_strings exp(-r^2 / rho^2) / (pi rho^2 N d) with N =
 * n_strings / (d cell_x cell_y); with RAD_TRAJ_MS_EL also the electron density
 *   n_el = (1 / (pi d)) sum_strings sum_i ax[i] / CX_i exp(-r^2 / CX_i) + cx N n(x, y)/N,
 * CX_i = bx[i] / (4 pi^2) + rho^2, in the electron term of rad_planar_potential. */
typedef struct {
  int n_terms;      /* Gaussian terms of each fit, 1 .. 8 */
  int n_cells;      /* cells summed on each side of the particle's cell in x and y, 1 .. 4 */
  double a[8];      /* potential fit a_i, m (finite) */
  double b[8];      /* potential fit b_i, m^2 (C_i > 0) */
  double ax[8];     /* X-ray fit a_i^(X), electrons (used with RAD_TRAJ_MS_EL) */
  double bx[8];     /* X-ray fit b_i^(X), m^2 (CX_i > 0 with RAD_TRAJ_MS_EL) */
  double cx;        /* X-ray constant c^(X) */
  double I_eV;      /* mean ionisation energy, eV (> 0 with RAD_TRAJ_MS_EL) */
  rad_string_lattice lattice;
} rad_axial_potential;

/*
 * rad_axial_trajectories -- rad_crystal_trajectories for axial channeling: the force is
 * -q grad U(x, y) of the string potential `pot` (host struct, read during the call), in both
 * transverse directions; particle p enters at (x0[p], y0[p]) (device; y0 may be NULL for 0) with
 * angles (thx0[p], thy0[p]). The records, the random streams, the radiation reaction and the
 * scattering options are those of rad_channeling_trajectories, with the string densities in place
 * of the plane densities (U0_eV and d_p of rad_channel are ignored). FP64 only: RAD_TRAJ_FP32
 * returns RAD_EUNSUPPORTED. Host checks (null ch or pot, n_terms, n_cells or n_strings out of
 * range, a cell side or d <= 0, a non-finite coefficient or position, C_i <= 0, with
 * RAD_TRAJ_MS_EL CX_i <= 0 or I_eV <= 0, rho <= 0 with RAD_TRAJ_MS, and the checks of
 * rad_channeling_trajectories) return RAD_EINVAL before anything is enqueued.
 */
int rad_axial_trajectories(const rad_channel *ch, const rad_axial_potential *pot, int64_t n_particles,
                           const int64_t *offsets, int64_t n_samples_total, const double *energy_eV,
                           const double *x0, const double *y0, const double *thx0, const double *thy0,
                           const int64_t *particle_ids, double dt, uint64_t seed, double *out,
                           double *energy_out, void *stream);

/* Step control of rad_trajectories_adaptive. */
typedef struct {
  double rtol;          /* relative tolerance of the embedded error estimate (> 0)                 */
  double atol_x;        /* absolute tolerance of x, y and dz, m (> 0)                              */
  double atol_v;        /* absolute tolerance of the angles v_x, v_y (> 0)                          */
  int max_level;        /* 0 .. 16: the smallest sub-step is an output interval / 2^max_level      */
  int64_t max_substeps; /* per particle, >= 1: a particle that needs more stops, RAD_EDATA          */
} rad_step_control;

/*
 * rad_trajectories_adaptive -- the trajectory integrators with adaptive steps between output
 * times the caller sets (Sec. IV: an RK45 solver with step-size control and a lower bound on the
 * step, returning the trajectory at the times the caller asks for). The field is the harmonic
 * well of `ch` (pot and axial NULL), the planar potential `pot`, or the axial potential `axial`
 * (at most one of them). Each output interval H = t_{k+1} - t_k is integrated with Dormand-Prince
 * 5(4) sub-steps H / 2^m (Dormand and Prince, J. Comput. Appl. Math. 6 (1980) 19): a sub-step
 * whose error estimate, the RMS over (x, y, v_x, v_y, dz, E) of (y5 - y4) / (atol_i + rtol
 * max(|y_i|, |y5_i|)) with atol = (atol_x, atol_x, atol_v, atol_v, atol_x, 0), exceeds 1 is
 * repeated at half the size unless m = max_level (the lower bound), where it is kept; after an
 * accepted sub-step with error below 2^-6 the size doubles when the interval position allows it.
 * The level starts at 0 and carries over between intervals; each interval ends exactly at its
 * output time. Kicks (RAD_TRAJ_MS) follow each interval with variances for its length H; the next
 * record's acceleration carries the kick as delta_v / w, w = (t_{k+2} - t_k)/2, or H for the last
 * record (delta_v / dt for uniform times, as in rad_channeling_trajectories). times: device,
 * [n_samples_total], the output times of every record of every particle (increasing within a
 * particle), or NULL for t_k = k dt. substeps_out: device int64 [n_particles] (may be NULL), the
 * accepted sub-steps of each particle. Records, entry values (y0, thy0 may be NULL), streams and
 * flags as in rad_channeling_trajectories / rad_axial_trajectories; FP64 only (RAD_TRAJ_FP32:
 * RAD_EUNSUPPORTED). Host checks return RAD_EINVAL before anything is enqueued; a particle with
 * non-increasing or non-finite times, or that exceeds max_substeps, records RAD_EDATA (its
 * records after that point are not written).
 */
int rad_trajectories_adaptive(const rad_channel *ch, const rad_planar_potential *pot,
                              const rad_axial_potential *axial, const rad_step_control *sc, int64_t n_particles,
                              const int64_t *offsets, int64_t n_samples_total, const double *energy_eV,
                              const double *x0, const double *y0, const double *thx0, const double *thy0,
                              const int64_t *particle_ids, const double *times, double dt, uint64_t seed,
                              double *out, double *energy_out, int64_t *substeps_out, void *stream);

/*
 * rad_device_status -- waits for the current device to finish, returns the first
 * device-side error recorded since the last reset (RAD_OK, RAD_EDATA or RAD_ETIMEOUT)
 * and clears it when reset != 0.
 */
int rad_device_status(int reset);

/*
 * rad_selftest_bounded_wait -- failure-detection self-test (the paper has no counterpart):
 * enqueues on `stream` a one-thread kernel that waits, with the same bounded wait the staging
 * kernels use for their bulk copies, on an mbarrier phase that nothing completes. After the
 * wait's time limit (about 2 s) the kernel records RAD_ETIMEOUT in the device status word and
 * returns; the context stays usable. Returns RAD_OK when the kernel was enqueued; read the
 * outcome with rad_device_status. Shows that a stalled copy ends in an error status, not a hang.
 */
int rad_selftest_bounded_wait(void *stream);

/* rad_status_string -- static description of a status code (RAD_ECUDA: last CUDA error). */
const char *rad_status_string(int status);

/* rad_version -- library version string. */
const char *rad_version(void);

/* rad_release -- frees library-owned buffers and the tuning cache (after a device sync). */
void rad_release(void);

#ifdef __cplusplus
}
#endif
#endif /* RAD_H */
