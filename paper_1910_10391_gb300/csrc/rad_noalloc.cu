// rad_spectrum_noalloc: the mixed-precision spectrum without any device allocation.
//
// Some callers cannot let a library call cudaMalloc: a process whose device memory is
// already reserved by another framework's caching allocator (the library's own cudaMalloc
// then fails although the framework holds free blocks), or a latency-critical loop where
// cudaMalloc/cudaFree would synchronize the whole device. This entry point serves them: its
// scratch is one file-scope device array of fixed size (kNoallocBytes), present on every GPU
// that loads the library until the process exits. The caller still provides every input
// and the output.
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "rad_internal.cuh"

namespace {

constexpr size_t kNoallocBytes = size_t(32) << 20;  // 32 MiB
constexpr size_t kCtrlBytes = 256;  // work counter, call status, publish word; grid maxima from byte 16

// Device-resident scratch. In host code this name is only a host-side stand-in for the
// symbol: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_mu;
std::vector<unsigned char *> g_addr;  // per device: device address of g_noalloc_scratch

// Set-up, once per device, with that device current.
int scratch_address(int dev, unsigned char **out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (static_cast<int>(g_addr.size()) <= dev) g_addr.resize(dev + 1, nullptr);
  if (!g_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return RAD_ECUDA;
    g_addr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_addr[dev];
  return RAD_OK;
}

}  // namespace

extern "C" int rad_spectrum_noalloc(const double *samples, int64_t n_samples_total, const int64_t *offsets,
                                    int64_t n_particles, const double *gamma, const double *energy_eV,
                                    const double *weight, const double *hbar_omega_eV, int64_t n_omega,
                                    const double *theta_x, const double *theta_y, int64_t n_angles, int mode,
                                    double *out_cube, void *stream) {
  using namespace rad;
  // host-side checks: nothing is enqueued when they fail
  if (n_samples_total < 0 || n_particles < 0 || n_omega < 0 || n_angles < 0) return RAD_EINVAL;
  if (mode < RAD_CLASSICAL || mode > RAD_SPIN_HALF) return RAD_EINVAL;
  if (n_particles > 0 && n_samples_total < 2 * n_particles) return RAD_EINVAL;
  if (n_particles == 0 && n_samples_total != 0) return RAD_EINVAL;
  if (n_omega == 0 || n_angles == 0) return RAD_OK;
  if (!out_cube || !offsets || !hbar_omega_eV || !theta_x || !theta_y) return RAD_EINVAL;
  if (n_particles > 0 && (!samples || !gamma || !energy_eV)) return RAD_EINVAL;
  if (samples && (reinterpret_cast<uintptr_t>(samples) & 15u)) return RAD_EINVAL;
  // the bin count is compared without forming a product that could overflow
  const int64_t max_bins = static_cast<int64_t>((kNoallocBytes - kCtrlBytes) / sizeof(double));
  if (n_omega > max_bins || n_angles > max_bins / n_omega) return RAD_ETOOBIG;
  const int64_t bins = n_omega * n_angles;

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return RAD_ECUDA;
  int major = 0, sms = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) return RAD_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return RAD_ECUDA;
  if (major < 10) return RAD_EUNSUPPORTED;
  unsigned char *base = nullptr;
  if (scratch_address(dev, &base) != RAD_OK) return RAD_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // launch shape: the mixed kernel, 2 energies per lane, 8 warps, 128-sample tiles;
  // particle chunks as many as the fixed scratch holds (up to 4 work items per resident block)
  LaunchShape sh{2, 8, 128, 0, 0};
  const int occ = occupancy_mixed(sh);
  if (occ <= 0) return RAD_EUNSUPPORTED;
  const int64_t resident = static_cast<int64_t>(sms) * occ;
  const int n_wt = static_cast<int>((n_omega + 63) / 64);
  const int n_nt = static_cast<int>((n_angles + 7) / 8);
  const int64_t tiles = static_cast<int64_t>(n_wt) * n_nt;
  int64_t chunks = 1;
  if (tiles < 4 * resident) chunks = (4 * resident + tiles - 1) / tiles;
  if (chunks > n_particles) chunks = n_particles > 0 ? n_particles : 1;
  const int64_t fit = max_bins / bins;
  if (chunks > fit) chunks = fit;

  Params P{};
  P.samples = samples;
  P.n_samples_total = n_samples_total;
  P.offsets = offsets;
  P.n_particles = n_particles;
  P.gamma = gamma;
  P.energy = energy_eV;
  P.weight = weight;
  P.hw = hbar_omega_eV;
  P.n_omega = n_omega;
  P.theta_x = theta_x;
  P.theta_y = theta_y;
  P.n_angles = n_angles;
  P.mode = mode;
  P.n_wt = n_wt;
  P.n_nt = n_nt;
  P.n_chunks = chunks;
  P.amp_mode = 0;
  P.n_q = 1;
  P.n_items = tiles * chunks;
  int *ctrl = reinterpret_cast<int *>(base);
  P.counter = ctrl;
  P.status = ctrl + 1;
  P.part = reinterpret_cast<double *>(base + kCtrlBytes);
  P.table = nullptr;  // the mixed kernel has no table
  // grid maxima of the mixed form's error-budget guard, after the three control ints
  P.grid_max = reinterpret_cast<unsigned long long *>(base + 16);
  P.phase_budget = kMixedPhaseBudget;
  sh.grid = static_cast<int>(P.n_items < resident ? P.n_items : resident);
  if (sh.grid < 1) sh.grid = 1;

  // the work counter and status words must start at zero on every call
  e = cudaMemsetAsync(ctrl, 0, kCtrlBytes, st);
  if (e == cudaSuccess) e = launch_validate(P, nullptr, false, nullptr, st);
  if (e == cudaSuccess) e = launch_mixed(P, &sh, st);
  // combine: the cube is written once (cube_new and the output are the same array)
  if (e == cudaSuccess) e = launch_finalize_status(P, out_cube, out_cube, 0, ctrl + 2, st);
  // the status word comes back on the caller's stream: one wait, for this call's work only
  int status = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, ctrl + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return RAD_ECUDA;
  return status;
}
