// Device-side input checks, the deterministic combine of per-item partials into the
// d2I/(d hw dOmega) cube (particle sum of Sec. IV), and the angle integral and radial
// binning of the cube (spectrum dI/d hw of Sec. IV). Fixed summation orders: results are
// bitwise reproducible run to run.
#include <math.h>

#include <mutex>
#include <vector>

#include "rad_internal.cuh"

namespace rad {
namespace {

__device__ __forceinline__ bool finite_d(double v) { return isfinite(v); }

// One grid-stride pass over every device input; any violation sets RAD_EDATA.
__global__ void k_validate(const Params P, const double *d_omega, int need_domega,
                           double max_hw_unused) {
  (void)max_hw_unused;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t t0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  bool bad = false;
  // particles
  for (int64_t p = t0; p < P.n_particles; p += stride) {
    const int64_t a = P.offsets[p], b = P.offsets[p + 1];
    if (b - a < 2 || a < 0 || b > P.n_samples_total) bad = true;
    const double g = P.gamma[p], E = P.energy[p];
    if (!(finite_d(g) && g > 1.0)) bad = true;
    if (!(finite_d(E) && E > 0.0)) bad = true;
    if (P.weight && !finite_d(P.weight[p])) bad = true;
  }
  if (t0 == 0 && P.n_particles >= 0) {
    if (P.offsets[0] != 0 || P.offsets[P.n_particles] != P.n_samples_total) bad = true;
  }
  // photon energies (and hw < E for every particle in the quantum modes)
  for (int64_t i = t0; i < P.n_omega; i += stride) {
    const double h = P.hw[i];
    if (!(finite_d(h) && h > 0.0)) bad = true;
  }
  if (P.mode != RAD_CLASSICAL) {
    const int64_t npairs = P.n_omega * P.n_particles;
    for (int64_t e = t0; e < npairs; e += stride) {
      const int64_t i = e % P.n_omega, p = e / P.n_omega;
      if (!(P.hw[i] < P.energy[p])) bad = true;
    }
  }
  // directions
  for (int64_t j = t0; j < P.n_angles; j += stride) {
    if (!finite_d(P.theta_x[j]) || !finite_d(P.theta_y[j])) bad = true;
    if (need_domega && !finite_d(d_omega[j])) bad = true;
  }
  // trajectory records
  const int64_t nv = P.n_samples_total * kRec;
  for (int64_t e = t0; e < nv; e += stride)
    if (!finite_d(P.samples[e])) bad = true;
  if (bad) set_status(P.status, RAD_EDATA);
  // RAD_MIXED: grid maxima for the error-budget guard (non-negative doubles order as their bits)
  if (P.grid_max) {
    double m[kGridMaxWords] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t j = t0; j < P.n_angles; j += stride) {
      const double ux = P.theta_x[j], uy = P.theta_y[j];
      m[0] = fmax(m[0], fabs(ux));
      m[1] = fmax(m[1], fabs(uy));
      m[2] = fmax(m[2], (ux * ux + uy * uy) * 0.5);
    }
    for (int64_t i = t0; i < P.n_omega; i += stride) m[3] = fmax(m[3], fabs(P.hw[i]));
#pragma unroll
    for (int w = 0; w < kGridMaxWords; ++w) {
      double v = m[w];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
      // NaN inputs were flagged above; fmax drops them here
      if ((threadIdx.x & 31) == 0 && v > 0.0)
        atomicMax(&P.grid_max[w], static_cast<unsigned long long>(__double_as_longlong(v)));
    }
  }
}

// Combine partials into the cube, tile-transposed: part layout [chunk][..][j][i] (i fastest),
// cube layout [i][j] (j fastest). Block = 32 x 8 threads over a 32 x 32 tile.
template <bool AMP, int NC>
__global__ void k_finalize(const Params P, double *cube_new, double *out_cube, int accumulate,
                           int *dev_status) {
  __shared__ double tile[32][33];
  const int st = *reinterpret_cast<volatile int *>(P.status);
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0 && st != 0)
    atomicCAS(dev_status, 0, st);
  if (st != 0) return;  // leave the outputs untouched
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * 32;  // energy tile
  const double pref = kAlpha / (4.0 * kPi * kPi);
  const int64_t n_jt = (P.n_angles + 31) / 32;
  for (int64_t jt = blockIdx.y; jt < n_jt; jt += gridDim.y) {  // direction tiles
  const int64_t j0 = jt * 32;
  // read phase: thread (x, y) reads i = i0 + x, j = j0 + y + 8k
  for (int kk = 0; kk < 32; kk += 8) {
    const int64_t i = i0 + threadIdx.x, j = j0 + threadIdx.y + kk;
    double v = 0.0;
    if (i < P.n_omega && j < P.n_angles) {
      if (!AMP) {
        for (int64_t c = 0; c < P.n_chunks; ++c) v += P.part[(c * P.n_angles + j) * P.n_omega + i];
      } else {
        const double h = P.hw[i];
        for (int64_t p = 0; p < P.n_particles; ++p) {
          double a[NC];
#pragma unroll
          for (int c = 0; c < NC; ++c) a[c] = 0.0;
          for (int q = 0; q < P.n_q; ++q) {
            const int64_t ch = p * P.n_q + q;
#pragma unroll
            for (int c = 0; c < NC; ++c) a[c] += P.part[((ch * NC + c) * P.n_angles + j) * P.n_omega + i];
          }
          double I2 = 0.0;
#pragma unroll
          for (int c = 0; c < 6; ++c) I2 = fma(a[c], a[c], I2);
          double S;
          if (P.mode == RAD_CLASSICAL) {
            S = I2;
          } else {
            const double u = h / P.energy[p];
            if (P.mode == RAD_SPIN0) {
              S = (1.0 - u) * I2;
            } else {
              const double g = P.gamma[p];
              const double J2 = (NC == 8) ? a[NC - 2] * a[NC - 2] + a[NC - 1] * a[NC - 1] : 0.0;
              S = 0.5 * (1.0 + (1.0 - u) * (1.0 - u)) * I2 + (u * u) / (2.0 * g * g) * J2;
            }
          }
          v = fma(P.weight ? P.weight[p] : 1.0, S, v);
        }
      }
    }
    tile[threadIdx.y + kk][threadIdx.x] = pref * v;
  }
  __syncthreads();
  // write phase: thread (x, y) writes j = j0 + x, i = i0 + y + 8k
  for (int kk = 0; kk < 32; kk += 8) {
    const int64_t j = j0 + threadIdx.x, i = i0 + threadIdx.y + kk;
    if (i < P.n_omega && j < P.n_angles) {
      const double v = tile[threadIdx.x][threadIdx.y + kk];
      const int64_t e = i * P.n_angles + j;
      cube_new[e] = v;
      if (out_cube) out_cube[e] = accumulate ? out_cube[e] + v : v;
    }
  }
  __syncthreads();  // the tile is rewritten by the next direction tile
  }
}

// One block per photon energy: spectrum and radial bins with fixed-order tree sums.
__global__ void k_reduce(const Params P, const double *cube_new, const double *d_omega,
                         double *out_spectrum, const int32_t *bin_of_angle, int n_bins,
                         double *out_bins, int accumulate) {
  if (*reinterpret_cast<volatile int *>(P.status) != 0) return;
  __shared__ double red[256];
  const int64_t i = blockIdx.x;
  const double *row = cube_new + i * P.n_angles;
  auto block_sum = [&](double v) -> double {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
      if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
  };
  if (out_spectrum) {
    double v = 0.0;
    for (int64_t j = threadIdx.x; j < P.n_angles; j += 256) v += row[j] * d_omega[j];
    const double tot = block_sum(v);
    if (threadIdx.x == 0) out_spectrum[i] = accumulate ? out_spectrum[i] + tot : tot;
  }
  if (out_bins) {
    for (int b = 0; b < n_bins; ++b) {
      double v = 0.0;
      for (int64_t j = threadIdx.x; j < P.n_angles; j += 256)
        if (bin_of_angle[j] == b) v += row[j] * d_omega[j];
      const double tot = block_sum(v);
      if (threadIdx.x == 0) {
        const int64_t e = i * n_bins + b;
        out_bins[e] = accumulate ? out_bins[e] + tot : tot;
      }
    }
  }
}

// Per-particle angle integral and radial bins (S-mode partials, one chunk per particle).
// Block (32 energies) x (8 direction lanes); grid (energy tiles, particles).
constexpr int kMaxBinsPP = 16;
__global__ void k_reduce_particles(const Params P, const double *d_omega, double *out_spectrum,
                                   const int32_t *bin_of_angle, int n_bins, double *out_bins,
                                   int *dev_status) {
  __shared__ double acc[kMaxBinsPP + 1][8][32];
  const int st = *reinterpret_cast<volatile int *>(P.status);
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0 && st != 0)
    atomicCAS(dev_status, 0, st);
  if (st != 0) return;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * 32 + tx;
  const double pref = kAlpha / (4.0 * kPi * kPi);
  for (int64_t p = blockIdx.y; p < P.n_particles; p += gridDim.y) {
  for (int b = 0; b <= kMaxBinsPP; ++b) acc[b][ty][tx] = 0.0;
  if (i < P.n_omega) {
    for (int64_t j = ty; j < P.n_angles; j += 8) {
      const double v = P.part[(p * P.n_angles + j) * P.n_omega + i] * d_omega[j];
      acc[kMaxBinsPP][ty][tx] += v;
      if (bin_of_angle) {
        const int32_t b = bin_of_angle[j];
        if (b >= 0 && b < n_bins) acc[b][ty][tx] += v;
      }
    }
  }
  __syncthreads();
  if (ty == 0 && i < P.n_omega) {
    double s = 0.0;
    for (int l = 0; l < 8; ++l) s += acc[kMaxBinsPP][l][tx];
    if (out_spectrum) out_spectrum[p * P.n_omega + i] = pref * s;
    if (out_bins)
      for (int b = 0; b < n_bins; ++b) {
        double sb = 0.0;
        for (int l = 0; l < 8; ++l) sb += acc[b][l][tx];
        out_bins[(p * P.n_omega + i) * n_bins + b] = pref * sb;
      }
  }
  __syncthreads();  // acc is cleared for the next particle
  }
}

std::mutex g_mu;
struct DevRes {
  double2 *table = nullptr;
  int *status = nullptr;
};
std::vector<DevRes> g_dev;

void fill_table_host(std::vector<double2> &t) {
  // (cos, sin)(2 pi j / N): first quadrant from long double libm, others by exact symmetry
  t.resize(kTabN);
  const int Q = kTabN / 4;
  const long double pi_l = 3.141592653589793238462643383279502884L;
  for (int m = 0; m < Q; ++m) {
    const long double th = 2.0L * pi_l * static_cast<long double>(m) / static_cast<long double>(kTabN);
    const double c = static_cast<double>(cosl(th)), s = static_cast<double>(sinl(th));
    t[m] = make_double2(c, s);
    t[m + Q] = make_double2(-s, c);
    t[m + 2 * Q] = make_double2(-c, -s);
    t[m + 3 * Q] = make_double2(s, -c);
  }
}

DevRes *dev_res(cudaError_t *err) {
  int dev = 0;
  *err = cudaGetDevice(&dev);
  if (*err != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (static_cast<int>(g_dev.size()) <= dev) g_dev.resize(dev + 1);
  DevRes &r = g_dev[dev];
  if (!r.table) {
    std::vector<double2> h;
    fill_table_host(h);
    double2 *d = nullptr;
    *err = cudaMalloc(&d, sizeof(double2) * kTabN);
    if (*err != cudaSuccess) return nullptr;
    *err = cudaMemcpy(d, h.data(), sizeof(double2) * kTabN, cudaMemcpyHostToDevice);
    if (*err != cudaSuccess) {
      cudaFree(d);
      return nullptr;
    }
    int *s = nullptr;
    *err = cudaMalloc(&s, sizeof(int));
    if (*err != cudaSuccess) {
      cudaFree(d);
      return nullptr;
    }
    *err = cudaMemset(s, 0, sizeof(int));
    if (*err != cudaSuccess) {
      cudaFree(d);
      cudaFree(s);
      return nullptr;
    }
    r.table = d;
    r.status = s;
  }
  *err = cudaSuccess;
  return &r;
}

// Self-test of the bounded mbarrier wait that every staging kernel uses to wait for its bulk
// copies: one thread waits on a phase of an mbarrier that nothing ever completes. The wait gives
// up after its time limit (kWaitLimitNs), the kernel records RAD_ETIMEOUT in the device status
// word and returns, and the context stays usable.
__global__ void k_wait_selftest(int *dev_status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_mbar_init();
  if (!mbar_wait_bounded(&bar, 0u)) set_status(dev_status, RAD_ETIMEOUT);
}

}  // namespace

cudaError_t launch_wait_selftest(cudaStream_t st) {
  cudaError_t e;
  int *ds = device_status_word(&e);
  if (!ds) return e;
  k_wait_selftest<<<1, 32, 0, st>>>(ds);
  return cudaGetLastError();
}

const double2 *device_table(cudaError_t *err) {
  DevRes *r = dev_res(err);
  return r ? r->table : nullptr;
}

int *device_status_word(cudaError_t *err) {
  DevRes *r = dev_res(err);
  return r ? r->status : nullptr;
}

cudaError_t launch_validate(const Params &P, const double *d_omega, bool need_domega,
                            const int32_t *bin_of_angle, cudaStream_t st) {
  (void)bin_of_angle;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t work = P.n_samples_total * kRec + P.n_particles + P.n_angles + P.n_omega * (1 + P.n_particles);
  int64_t blocks = (work + 255) / 256;
  const int64_t cap = static_cast<int64_t>(sms > 0 ? sms : 1) * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  k_validate<<<static_cast<int>(blocks), 256, 0, st>>>(P, d_omega, need_domega ? 1 : 0, 0.0);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const Params &P, double *cube_new, double *out_cube, int accumulate,
                            cudaStream_t st) {
  cudaError_t e;
  int *ds = device_status_word(&e);
  if (!ds) return e;
  dim3 blk(32, 8);
  dim3 grd(static_cast<unsigned>((P.n_omega + 31) / 32), grid_y((P.n_angles + 31) / 32));
  if (grd.x == 0 || grd.y == 0) return cudaSuccess;
  if (!P.amp_mode)
    k_finalize<false, 6><<<grd, blk, 0, st>>>(P, cube_new, out_cube, accumulate, ds);
  else if (P.mode == RAD_SPIN_HALF)
    k_finalize<true, 8><<<grd, blk, 0, st>>>(P, cube_new, out_cube, accumulate, ds);
  else
    k_finalize<true, 6><<<grd, blk, 0, st>>>(P, cube_new, out_cube, accumulate, ds);
  return cudaGetLastError();
}

cudaError_t launch_finalize_status(const Params &P, double *cube_new, double *out_cube, int accumulate,
                                   int *publish_status, cudaStream_t st) {
  dim3 blk(32, 8);
  dim3 grd(static_cast<unsigned>((P.n_omega + 31) / 32), grid_y((P.n_angles + 31) / 32));
  if (grd.x == 0 || grd.y == 0) return cudaSuccess;
  if (P.amp_mode) return cudaErrorInvalidValue;
  k_finalize<false, 6><<<grd, blk, 0, st>>>(P, cube_new, out_cube, accumulate, publish_status);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const Params &P, const double *cube_new, const double *d_omega,
                          double *out_spectrum, const int32_t *bin_of_angle, int n_bins,
                          double *out_bins, int accumulate, cudaStream_t st) {
  if (P.n_omega == 0 || (!out_spectrum && !out_bins)) return cudaSuccess;
  k_reduce<<<static_cast<unsigned>(P.n_omega), 256, 0, st>>>(P, cube_new, d_omega, out_spectrum,
                                                           bin_of_angle, n_bins, out_bins, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_reduce_particles(const Params &P, const double *d_omega, double *out_spectrum,
                                   const int32_t *bin_of_angle, int n_bins, double *out_bins, cudaStream_t st) {
  if (P.amp_mode || n_bins > kMaxBinsPP) return cudaErrorInvalidValue;
  if (P.n_omega == 0 || P.n_particles == 0) return cudaSuccess;
  cudaError_t e;
  int *ds = device_status_word(&e);
  if (!ds) return e;
  dim3 blk(32, 8);
  dim3 grd(static_cast<unsigned>((P.n_omega + 31) / 32), grid_y(P.n_particles));
  k_reduce_particles<<<grd, blk, 0, st>>>(P, d_omega, out_spectrum, bin_of_angle, n_bins, out_bins, ds);
  return cudaGetLastError();
}

cudaError_t launch_zero_outputs(const Params &P, double *out_cube, double *out_spectrum, int n_bins,
                                double *out_bins, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (out_cube && P.n_omega * P.n_angles > 0)
    e = cudaMemsetAsync(out_cube, 0, sizeof(double) * P.n_omega * P.n_angles, st);
  if (e == cudaSuccess && out_spectrum && P.n_omega > 0)
    e = cudaMemsetAsync(out_spectrum, 0, sizeof(double) * P.n_omega, st);
  if (e == cudaSuccess && out_bins && P.n_omega * n_bins > 0)
    e = cudaMemsetAsync(out_bins, 0, sizeof(double) * P.n_omega * n_bins, st);
  return e;
}

// dI/dOmega over a photon-energy range: out[j] = sum_i w_i cube[i][j], trapezoid weights in hw
// (Sec. IV, the energy radiated per solid angle). One thread per direction, the energies summed in
// order (deterministic); lanes along j read the cube rows coalesced.
__global__ void k_angular(const double *__restrict__ cube, const double *__restrict__ hw, int64_t n_omega,
                          int64_t n_angles, double *__restrict__ out) {
  for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < n_angles;
       j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double acc = 0.0;
    for (int64_t i = 0; i + 1 < n_omega; ++i) {
      const double h = hw[i + 1] - hw[i];
      acc += 0.5 * h * (cube[i * n_angles + j] + cube[(i + 1) * n_angles + j]);
    }
    out[j] = acc;
  }
}

}  // namespace rad

extern "C" int rad_angular_distribution(const double *cube, const double *hbar_omega_eV, int64_t n_omega,
                                        int64_t n_angles, double *out, void *stream) {
  if (n_omega < 0 || n_angles < 0) return RAD_EINVAL;
  if (n_angles == 0) return RAD_OK;
  if (!out || (n_omega > 0 && (!cube || !hbar_omega_eV))) return RAD_EINVAL;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (n_omega < 2) {
    e = cudaMemsetAsync(out, 0, sizeof(double) * n_angles, st);
  } else {
    int64_t blocks = (n_angles + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    rad::k_angular<<<static_cast<unsigned>(blocks), 256, 0, st>>>(cube, hbar_omega_eV, n_omega, n_angles, out);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? RAD_OK : rad::cuda_status(e);
}
