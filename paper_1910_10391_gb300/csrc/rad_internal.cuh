// Internal definitions shared by the CUDA translation units of the radiation library.
//
// Work decomposition (both precisions):
//   bin tile   = NW directions (one per warp) x (32 * R) photon energies (R per lane)
//   chunk      = S mode:   a contiguous range of whole particles; the item adds the
//                          particles' |amplitude|^2 (Sec. II) and writes FP64 partial sums
//                AMP mode: one time piece of one particle; the item writes the piece's
//                          complex amplitudes so pieces combine coherently (few particles)
//   work item  = (chunk, direction tile, energy tile); a persistent grid pulls items
//                from an atomic counter.
// Trajectory time tiles of T samples (+1 halo sample each side for the trapezoid
// weights) are staged into shared memory with cp.async.bulk, double-buffered, each
// buffer guarded by an mbarrier whose waits are bounded.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rad.h"

namespace rad {

constexpr double kHbarC = 1.973269804e-7;  // eV m (CODATA 2018)
constexpr double kAlpha = 7.2973525693e-3;  // fine-structure constant (CODATA 2018)
constexpr double kPi = 3.141592653589793238462643383279502884;

// record fields
enum { F_T = 0, F_X, F_Y, F_DZ, F_VX, F_VY, F_DVZ, F_AX, F_AY, F_AZ };
constexpr int kRec = RAD_NREC;

// FP64 sincos table: kTabN entries of (cos, sin)(2 pi j / kTabN)
constexpr int kTabBits = 12;
constexpr int kTabN = 1 << kTabBits;

// Bounded waits: give up after this many nanoseconds of %globaltimer (and a
// backstop iteration count), record RAD_ETIMEOUT and return.
// Largest grid y extent; kernels with a y dimension stride over y beyond it.
constexpr int64_t kMaxGridY = 65535;
inline unsigned grid_y(int64_t n) { return static_cast<unsigned>(n < kMaxGridY ? n : kMaxGridY); }
constexpr unsigned long long kWaitLimitNs = 2000000000ull;
constexpr unsigned long long kWaitLimitIter = 400000000ull;

struct Params {
  const double *samples;
  int64_t n_samples_total;
  const int64_t *offsets;
  int64_t n_particles;
  const double *gamma;
  const double *energy;
  const double *weight;  // may be null
  const double *hw;
  int64_t n_omega;
  const double *theta_x;
  const double *theta_y;
  int64_t n_angles;
  int mode;
  // decomposition
  int n_wt;        // energy tiles
  int n_nt;        // direction tiles
  int64_t n_chunks;
  int amp_mode;    // 0: S partials, 1: amplitude partials
  int n_q;         // AMP mode: time pieces per particle
  int64_t n_items;
  // scratch
  double *part;    // S: [n_chunks][n_angles][n_omega]; AMP: [n_chunks][ncomp][n_angles][n_omega]
  int *counter;    // work counter (zeroed before launch)
  int *status;     // per-call status word (zeroed before launch)
  const double2 *table;  // FP64 sincos table in global memory (kTabN entries)
  // RAD_MIXED only (else null): grid maxima filled by the validation kernel, as the bit patterns
  // of non-negative doubles (zeroed before launch): [0] max |theta_x|, [1] max |theta_y|,
  // [2] max (theta_x^2 + theta_y^2)/2, [3] max hw (eV). They bound the in-tile phase offsets.
  unsigned long long *grid_max;
  double phase_budget;  // RAD_MIXED: largest accepted in-tile phase-offset bound (radians)
};

// RAD_MIXED's error budget: the largest in-tile phase-offset bound w*_max B_k (radians) it accepts,
// B_k = c_max |t_k - t_ref| + |dz_k - dz_ref| + max|theta_x| |x_k - x_ref| + max|theta_y| |y_k - y_ref|
// with c_max = 1/(2 gamma^2) + max theta^2/2 and w*_max the largest w* of the particle. The sum of
// magnitudes bounds both the FP32 rounding of the offset (about 2^-23 of it per operand) and the SFU
// sin/cos error (which grows as 2.5e-7 |x|). Calls above it record RAD_EPRECISION; a plan can
// set another budget (rad_plan_set_phase_budget).
constexpr double kMixedPhaseBudget = 8192.0;
constexpr int kGridMaxWords = 4;

// ------------------------------------------------------------------------------------
// PTX wrappers (sm_90+ mbarrier / bulk async copy), all CTA-scoped
// ------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// 1-D bulk copy global -> shared, completion signalled on bar (bytes % 16 == 0, both
// addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase `parity` of bar to complete; false when the wait limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned long long it = 0; it < kWaitLimitIter; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255ull) == 0 && global_ns() - t0 > kWaitLimitNs) break;
  }
  return false;
}

__device__ __forceinline__ void set_status(int *status, int code) {
  atomicCAS(status, 0, code);
}

// ------------------------------------------------------------------------------------
// Tile iterator over the samples a work item covers (uniform across the block)
// ------------------------------------------------------------------------------------
struct TileCursor {
  int64_t p, p_end;  // particle, one past last particle of the chunk
  int64_t k0;        // first sample of the current tile (particle-local)
  int64_t kb, ke;    // sample range of the current particle covered by this item
  int64_t L;         // samples of the current particle
  bool valid;
};

__device__ __forceinline__ void cursor_particle(const Params &P, TileCursor &c, int q) {
  c.L = P.offsets[c.p + 1] - P.offsets[c.p];
  if (P.amp_mode) {
    c.kb = (c.L * q) / P.n_q;
    c.ke = (c.L * (q + 1)) / P.n_q;
  } else {
    c.kb = 0;
    c.ke = c.L;
  }
  c.k0 = c.kb;
}

// First non-empty tile at or after the cursor's particle.
__device__ __forceinline__ void cursor_settle(const Params &P, TileCursor &c, int q) {
  while (c.p < c.p_end) {
    cursor_particle(P, c, q);
    if (c.kb < c.ke) {
      c.valid = true;
      return;
    }
    ++c.p;
  }
  c.valid = false;
}

template <int T>
__device__ __forceinline__ void cursor_next(const Params &P, TileCursor &c, int q) {
  c.k0 += T;
  if (c.k0 < c.ke) return;
  ++c.p;
  cursor_settle(P, c, q);
}

// Chunk -> particle range / time piece
__device__ __forceinline__ void chunk_range(const Params &P, int64_t chunk, int64_t &p0, int64_t &p1,
                                            int &q) {
  if (P.amp_mode) {
    p0 = chunk / P.n_q;
    p1 = p0 + 1;
    q = static_cast<int>(chunk % P.n_q);
  } else {
    p0 = (P.n_particles * chunk) / P.n_chunks;
    p1 = (P.n_particles * (chunk + 1)) / P.n_chunks;
    q = 0;
  }
}

// Issue the bulk copy of one tile: records [k0-1, k0+n+1) clipped to [0, L) of particle p
// into stage buffer slots (k - k0 + 1). Returns bytes requested.
template <int T>
__device__ __forceinline__ uint32_t issue_tile(const Params &P, const TileCursor &c, double *stage,
                                               uint64_t *bar) {
  const int64_t n = (c.ke - c.k0) < T ? (c.ke - c.k0) : T;
  const int64_t lo = c.k0 > 0 ? c.k0 - 1 : 0;
  const int64_t hi = (c.k0 + n + 1) < c.L ? (c.k0 + n + 1) : c.L;
  const uint32_t bytes = static_cast<uint32_t>((hi - lo) * kRec * sizeof(double));
  double *dst = stage + (lo - c.k0 + 1) * kRec;
  const double *src = P.samples + (P.offsets[c.p] + lo) * kRec;
  fence_proxy_async();
  mbar_arrive_expect_tx(bar, bytes);
  bulk_g2s(dst, src, bytes, bar);
  return bytes;
}

// ------------------------------------------------------------------------------------
// Launch interface of the two main kernels
// ------------------------------------------------------------------------------------
struct LaunchShape {
  int R;        // photon energies per lane
  int NW;       // warps per block (= directions per tile)
  int T;        // time-tile length
  int grid;     // persistent grid size
  int smem;     // dynamic shared memory bytes
  int pe = 0;   // mixed pre-pass kernel: 1/pe of the terms take sincos on the FMA pipe (0: none)
};

// Returns cudaSuccess or the launch error. Fills shape->smem.
cudaError_t launch_fp64(const Params &P, LaunchShape *shape, cudaStream_t st);
cudaError_t launch_mixed(const Params &P, LaunchShape *shape, cudaStream_t st);
// Occupancy (resident blocks per SM) of a shape for a mode (default: spin 1/2, the largest
// footprint); 0 if unsupported.
int occupancy_fp64(const LaunchShape &s, int mode = RAD_SPIN_HALF);
int occupancy_mixed(const LaunchShape &s, int mode = RAD_SPIN_HALF);
bool shape_supported_fp64(int R, int NW, int T);
bool shape_supported_mixed(int R, int NW, int T);
// mixed kernel fed by the per-sample pre-pass (rad_mixed_pp.cu); prep holds 12 floats per sample
bool shape_supported_mixed_pp(int R, int NW, int T);
int occupancy_mixed_pp(const LaunchShape &s, int mode = RAD_SPIN_HALF);
cudaError_t launch_prep_samples(const Params &P, int T, float *prep, cudaStream_t st);
cudaError_t launch_mixed_pp(const Params &P, const float *prep, LaunchShape *shape, cudaStream_t st);

// FP64-accurate kernel with double-float FP32 arithmetic after the FP64 phase (rad_df.cu)
bool shape_supported_df(int R, int NW, int T);
int occupancy_df(const LaunchShape &s, int mode = RAD_SPIN_HALF);
cudaError_t launch_df(const Params &P, LaunchShape *shape, cudaStream_t st);

// post-processing kernels (rad_post.cu)
cudaError_t launch_validate(const Params &P, const double *d_omega, bool need_domega,
                            const int32_t *bin_of_angle, cudaStream_t st);
cudaError_t launch_finalize(const Params &P, double *cube_new, double *out_cube, int accumulate,
                            cudaStream_t st);
// k_finalize (S-mode partials) publishing a failed call status into *publish_status.
cudaError_t launch_finalize_status(const Params &P, double *cube_new, double *out_cube, int accumulate,
                                   int *publish_status, cudaStream_t st);
cudaError_t launch_reduce(const Params &P, const double *cube_new, const double *d_omega,
                          double *out_spectrum, const int32_t *bin_of_angle, int n_bins,
                          double *out_bins, int accumulate, cudaStream_t st);
// Per-particle spectrum / radial bins from S-mode partials with one chunk per particle
// (n_bins <= 16).
cudaError_t launch_reduce_particles(const Params &P, const double *d_omega, double *out_spectrum,
                                   const int32_t *bin_of_angle, int n_bins, double *out_bins, cudaStream_t st);
cudaError_t launch_zero_outputs(const Params &P, double *out_cube, double *out_spectrum,
                                int n_bins, double *out_bins, cudaStream_t st);
const double2 *device_table(cudaError_t *err);  // per-device FP64 sincos table
int *device_status_word(cudaError_t *err);      // per-device sticky status word
cudaError_t launch_wait_selftest(cudaStream_t st);  // a bounded wait that runs out (RAD_ETIMEOUT)
int cuda_status(cudaError_t e);                 // records e for rad_status_string; RAD_ENOMEM or RAD_ECUDA

inline int ncomp_of(int mode) { return mode == RAD_SPIN_HALF ? 8 : 6; }

}  // namespace rad
