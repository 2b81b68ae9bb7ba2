// Host side of the C ABI declared in include/rad.h: argument checks, plans (shape +
// scratch + launch shape), the per-(shape, stream) plan cache behind rad_spectrum, the
// autotuner, CUDA-graph capture and the host-buffer entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "rad_internal.cuh"

using namespace rad;

namespace {

thread_local char g_cuda_msg[256] = "no CUDA error recorded";

int cuda_fail(cudaError_t e) {
  std::snprintf(g_cuda_msg, sizeof g_cuda_msg, "CUDA error %d: %s", static_cast<int>(e),
                cudaGetErrorString(e));
  return (e == cudaErrorMemoryAllocation) ? RAD_ENOMEM : RAD_ECUDA;
}

struct Choice {
  int R, NW, T;
  int chunk_mult;  // multiplies the default number of work items
  int pp;          // mixed precision: 1 = per-sample pre-pass kernel, 0 = in-kernel preparation
  int pe = 0;      // pre-pass kernel: 1/pe of the terms take sincos on the FMA pipe (0, 4 or 6)
};

}  // namespace

namespace rad {
int cuda_status(cudaError_t e) { return cuda_fail(e); }
}  // namespace rad

struct rad_plan_s {
  int device = 0;
  int sms = 0;
  int64_t n_samples_total = 0, n_particles = 0, n_omega = 0, n_angles = 0;
  int mode = 0, precision = 0, want = 0;
  int32_t n_bins = 0;
  Choice choice{};
  LaunchShape shape{};
  int n_wt = 0, n_nt = 0, amp_mode = 0, n_q = 1;
  int64_t n_chunks = 1, n_items = 0;
  double *part = nullptr;
  size_t part_cap = 0;  // doubles
  double *cube_new = nullptr;
  float *prep = nullptr;  // pre-pass records (mixed precision with pp = 1), 12 floats per sample
  int *ctrl = nullptr;    // [0] work counter, [1] call status, then RAD_MIXED's grid maxima
  double phase_budget = rad::kMixedPhaseBudget;  // RAD_MIXED error-budget guard (radians)
  std::string desc;
  bool timing = false;
  bool timed_once = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

struct rad_graph_s {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

std::mutex g_mu;
using ShapeKey = std::tuple<int, int64_t, int64_t, int64_t, int64_t, int, int, int, int>;
std::map<ShapeKey, Choice> g_tuned;                                  // autotuned choices
std::map<std::tuple<ShapeKey, void *>, rad_plan> g_plans;            // rad_spectrum cache

constexpr size_t kCtrlBytes = 16 + sizeof(unsigned long long) * kGridMaxWords;

ShapeKey key_of(int dev, int64_t ns, int64_t np, int64_t no, int64_t na, int mode, int prec, int want,
                int nb) {
  return ShapeKey{dev, ns, np, no, na, mode, prec, want, nb};
}

// Defaults before any autotuning: the fastest shapes on the 10 GeV positron ensemble (512 hw x
// 64 x 64 directions, 32 particles per launch). The mixed kernel runs 8 warps per block, 2 blocks
// per SM; spin-1/2 keeps every sin/cos on the SFU, classical and spin-0 (two fewer sums per term)
// take 1/8 of them on the FMA pipe. k_df's blocks of 4 warps take 256 energies of one direction
// (128 when the grid has no more).
Choice default_choice(int precision, int mode, int64_t n_omega) {
  if (precision == RAD_FP64) return Choice{2, 8, 64, 1, 0};
  if (precision == RAD_FP64_DF) return Choice{n_omega <= 128 ? 1 : 2, 4, 64, 1, 0};
  if (mode == RAD_SPIN_HALF) return Choice{2, 8, 256, 1, 1, 0};
  return Choice{2, 8, 256, 1, 1, 6};
}

bool supported(int precision, const Choice &c) {
  if (c.pe != 0 && (precision != RAD_MIXED || !c.pp || (c.pe != 4 && c.pe != 6))) return false;
  if (precision == RAD_FP64) return c.pp == 0 && shape_supported_fp64(c.R, c.NW, c.T);
  if (precision == RAD_FP64_DF) return c.pp == 0 && shape_supported_df(c.R, c.NW, c.T);
  return c.pp ? shape_supported_mixed_pp(c.R, c.NW, c.T) : shape_supported_mixed(c.R, c.NW, c.T);
}

bool same_choice(const Choice &a, const Choice &b) {
  return a.R == b.R && a.NW == b.NW && a.T == b.T && a.chunk_mult == b.chunk_mult && a.pp == b.pp && a.pe == b.pe;
}

// Work decomposition for a choice; (re)allocates scratch when it grows.
int configure(rad_plan p, const Choice &c) {
  if (!supported(p->precision, c)) return RAD_EINVAL;
  LaunchShape sh{c.R, c.NW, c.T, 0, 0, c.pe};
  const int occ = p->precision == RAD_FP64      ? occupancy_fp64(sh, p->mode)
                  : p->precision == RAD_FP64_DF ? occupancy_df(sh, p->mode)
                  : c.pp                        ? occupancy_mixed_pp(sh, p->mode)
                                                : occupancy_mixed(sh, p->mode);
  if (occ <= 0) return RAD_EUNSUPPORTED;
  const int64_t resident = static_cast<int64_t>(p->sms) * occ;
  if (p->precision == RAD_FP64_DF) {  // k_df: one direction and NW 32 R energies per work item
    if (p->n_angles > INT32_MAX) return RAD_EINVAL;
    const int64_t per_block = 32LL * c.R * c.NW;
    p->n_wt = static_cast<int>((p->n_omega + per_block - 1) / per_block);
    p->n_nt = static_cast<int>(p->n_angles);
  } else {  // NW directions and 32 R energies per work item
    p->n_wt = static_cast<int>((p->n_omega + 32 * c.R - 1) / (32 * c.R));
    p->n_nt = static_cast<int>((p->n_angles + c.NW - 1) / c.NW);
  }
  const int64_t tiles = static_cast<int64_t>(p->n_wt) * p->n_nt;
  const int64_t target = resident * 4 * std::max(1, c.chunk_mult);
  p->amp_mode = 0;
  p->n_q = 1;
  p->n_chunks = 1;
  const bool per_particle = (p->want & RAD_PER_PARTICLE) != 0;
  if (per_particle) {
    p->n_chunks = std::max<int64_t>(p->n_particles, 1);  // one chunk per particle: partials are per particle
  } else if (tiles > 0 && tiles < target) {
    const int64_t factor = (target + tiles - 1) / tiles;
    if (p->n_particles >= factor || p->n_particles >= 64) {
      p->n_chunks = std::min<int64_t>(factor, std::max<int64_t>(p->n_particles, 1));
    } else if (p->n_particles > 0) {
      p->amp_mode = 1;
      const int64_t avg_len = p->n_samples_total / p->n_particles;
      int64_t nq = (factor + p->n_particles - 1) / p->n_particles;
      nq = std::min<int64_t>(nq, std::max<int64_t>(avg_len / (2 * c.T), 1));  // pieces of >= 2 tiles
      p->n_q = static_cast<int>(std::max<int64_t>(nq, 1));
      p->n_chunks = p->n_particles * p->n_q;
    }
  }
  const int ncomp = ncomp_of(p->mode);
  // keep the partials within 4 GiB
  const int64_t per_chunk = p->n_omega * p->n_angles * (p->amp_mode ? ncomp : 1);
  const int64_t cap_chunks = per_chunk > 0 ? std::max<int64_t>(1, (int64_t(1) << 29) / per_chunk) : 1;
  if (per_particle && p->n_chunks > cap_chunks) return RAD_ENOMEM;
  if (p->n_chunks > cap_chunks) {
    if (p->amp_mode) {
      p->n_q = static_cast<int>(std::max<int64_t>(1, cap_chunks / std::max<int64_t>(p->n_particles, 1)));
      p->n_chunks = p->n_particles * p->n_q;
      if (p->n_chunks > cap_chunks) return RAD_ENOMEM;
    } else {
      p->n_chunks = cap_chunks;
    }
  }
  p->n_items = tiles * p->n_chunks;
  // the kernels take work items from a 32-bit counter that every resident block advances once
  // past the last item
  if (p->n_items > static_cast<int64_t>(INT32_MAX) - resident) return RAD_EINVAL;
  sh.grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(p->n_items, resident)));
  p->shape = sh;
  p->choice = c;
  const size_t need = static_cast<size_t>(std::max<int64_t>(per_chunk * p->n_chunks, 1));
  if (need > p->part_cap) {
    if (p->part) cudaFree(p->part);
    p->part = nullptr;
    p->part_cap = 0;
    cudaError_t e = cudaMalloc(&p->part, need * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(e);
    p->part_cap = need;
  }
  if (c.pp && !p->prep && p->n_samples_total > 0) {
    cudaError_t e = cudaMalloc(&p->prep, sizeof(float) * 12 * static_cast<size_t>(p->n_samples_total));
    if (e != cudaSuccess) return cuda_fail(e);
  }
  char buf[256];
  std::snprintf(buf, sizeof buf,
                "precision=%s mode=%d R=%d NW=%d T=%d grid=%d occ=%d items=%lld chunks=%lld amp=%d nq=%d pp=%d "
                "pe=%d",
                p->precision == RAD_FP64 ? "fp64" : p->precision == RAD_FP64_DF ? "fp64_df" : "mixed", p->mode, c.R,
                c.NW, c.T, sh.grid, occ,
                static_cast<long long>(p->n_items), static_cast<long long>(p->n_chunks), p->amp_mode,
                p->n_q, c.pp, c.pe);
  p->desc = buf;
  return RAD_OK;
}

int check_shape(int64_t ns, int64_t np, int64_t no, int64_t na, int mode, int prec, int want,
                int32_t nb) {
  if (ns < 0 || np < 0 || no < 0 || na < 0) return RAD_EINVAL;
  if (mode < RAD_CLASSICAL || mode > RAD_SPIN_HALF) return RAD_EINVAL;
  if (prec != RAD_FP64 && prec != RAD_MIXED && prec != RAD_FP64_DF) return RAD_EINVAL;
  if (want < 0 || want > 15) return RAD_EINVAL;
  if ((want & 4) && nb < 1) return RAD_EINVAL;
  if (want & RAD_PER_PARTICLE) {
    if ((want & 1) || !(want & 6)) return RAD_EINVAL;  // per particle: spectrum and/or bins, no cube
    if ((want & 4) && nb > 16) return RAD_EINVAL;
  }
  if (np > 0 && ns < 2 * np) return RAD_EINVAL;
  if (np == 0 && ns != 0) return RAD_EINVAL;
  if (no > (int64_t(1) << 31) || na > (int64_t(1) << 31)) return RAD_EINVAL;
  return RAD_OK;
}

Params make_params(rad_plan p, const double *samples, const int64_t *offsets, const double *gamma,
                   const double *energy, const double *weight, const double *hw, const double *tx,
                   const double *ty, const double2 *table) {
  Params P{};
  P.samples = samples;
  P.n_samples_total = p->n_samples_total;
  P.offsets = offsets;
  P.n_particles = p->n_particles;
  P.gamma = gamma;
  P.energy = energy;
  P.weight = weight;
  P.hw = hw;
  P.n_omega = p->n_omega;
  P.theta_x = tx;
  P.theta_y = ty;
  P.n_angles = p->n_angles;
  P.mode = p->mode;
  P.n_wt = p->n_wt;
  P.n_nt = p->n_nt;
  P.n_chunks = p->n_chunks;
  P.amp_mode = p->amp_mode;
  P.n_q = p->n_q;
  P.n_items = p->n_items;
  P.part = p->part;
  P.counter = p->ctrl;
  P.status = p->ctrl + 1;
  P.table = table;
  // control block: [0] work counter, [1] status, bytes 16..47 the grid maxima of RAD_MIXED's guard
  P.phase_budget = p->phase_budget;
  P.grid_max = p->precision == RAD_MIXED
                   ? reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(p->ctrl) + 16)
                   : nullptr;
  return P;
}

int execute(rad_plan p, const double *samples, const int64_t *offsets, const double *gamma,
            const double *energy, const double *weight, const double *hw, const double *tx,
            const double *ty, const double *d_omega, double *out_cube, double *out_spectrum,
            const int32_t *bin_of_angle, double *out_bins, int accumulate, cudaStream_t st) {
  // host-side pointer checks for the plan's shape
  const bool need_dom = (out_spectrum != nullptr) || (out_bins != nullptr);
  if (accumulate != 0 && accumulate != 1) return RAD_EINVAL;
  if (out_bins && (!bin_of_angle || p->n_bins < 1)) return RAD_EINVAL;
  if ((out_cube && !(p->want & 1)) || (out_spectrum && !(p->want & 2)) || (out_bins && !(p->want & 4)))
    return RAD_EINVAL;
  if ((p->want & RAD_PER_PARTICLE) && accumulate) return RAD_EINVAL;
  if (p->n_omega > 0 && p->n_angles > 0) {
    if (p->n_particles > 0 && (!samples || !offsets || !gamma || !energy)) return RAD_EINVAL;
    if (!offsets) return RAD_EINVAL;
    if (!hw || !tx || !ty) return RAD_EINVAL;
    if (need_dom && !d_omega) return RAD_EINVAL;
    if (samples && (reinterpret_cast<uintptr_t>(samples) & 15u)) return RAD_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  if (dev != p->device) return RAD_EINVAL;
  if (p->n_omega == 0) return RAD_OK;
  if (p->n_angles == 0 && (p->want & RAD_PER_PARTICLE)) {
    cudaError_t e2 = cudaSuccess;
    if (out_spectrum && p->n_particles > 0)
      e2 = cudaMemsetAsync(out_spectrum, 0, sizeof(double) * p->n_particles * p->n_omega, st);
    if (e2 == cudaSuccess && out_bins && p->n_particles > 0)
      e2 = cudaMemsetAsync(out_bins, 0, sizeof(double) * p->n_particles * p->n_omega * p->n_bins, st);
    return e2 == cudaSuccess ? RAD_OK : cuda_fail(e2);
  }
  if (p->n_angles == 0) {
    // no directions: spectrum and bins are empty sums
    Params Z = make_params(p, samples, offsets, gamma, energy, weight, hw, tx, ty, nullptr);
    if (!accumulate) {
      e = launch_zero_outputs(Z, nullptr, out_spectrum, p->n_bins, out_bins, st);
      if (e != cudaSuccess) return cuda_fail(e);
    }
    return RAD_OK;
  }
  const double2 *table = device_table(&e);
  if (!table) return cuda_fail(e);
  Params P = make_params(p, samples, offsets, gamma, energy, weight, hw, tx, ty, table);
  e = cudaMemsetAsync(p->ctrl, 0, kCtrlBytes, st);
  if (e != cudaSuccess) return cuda_fail(e);
  e = launch_validate(P, d_omega, need_dom, bin_of_angle, st);
  if (e != cudaSuccess) return cuda_fail(e);
  LaunchShape sh = p->shape;
  if (p->precision == RAD_MIXED && p->choice.pp) {
    e = launch_prep_samples(P, sh.T, p->prep, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  if (p->timing) {  // events bracket the integral kernel alone
    e = cudaEventRecord(p->ev0, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  if (p->precision == RAD_FP64) {
    e = launch_fp64(P, &sh, st);
  } else if (p->precision == RAD_FP64_DF) {
    e = launch_df(P, &sh, st);
  } else if (p->choice.pp) {
    e = launch_mixed_pp(P, p->prep, &sh, st);
  } else {
    e = launch_mixed(P, &sh, st);
  }
  if (e != cudaSuccess) return cuda_fail(e);
  if (p->timing) {
    e = cudaEventRecord(p->ev1, st);
    if (e != cudaSuccess) return cuda_fail(e);
    p->timed_once = true;
  }
  if (p->want & RAD_PER_PARTICLE) {
    e = launch_reduce_particles(P, d_omega, out_spectrum, bin_of_angle, p->n_bins, out_bins, st);
    return e == cudaSuccess ? RAD_OK : cuda_fail(e);
  }
  e = launch_finalize(P, p->cube_new, out_cube, accumulate, st);
  if (e != cudaSuccess) return cuda_fail(e);
  e = launch_reduce(P, p->cube_new, d_omega, out_spectrum, bin_of_angle, p->n_bins, out_bins,
                    accumulate, st);
  if (e != cudaSuccess) return cuda_fail(e);
  return RAD_OK;
}

int plan_create(int64_t ns, int64_t np, int64_t no, int64_t na, int mode, int prec, int want, int32_t nb,
                rad_plan *out) {
  if (!out) return RAD_EINVAL;
  *out = nullptr;
  int rc = check_shape(ns, np, no, na, mode, prec, want, nb);
  if (rc) return rc;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return cuda_fail(e);
  if (prop.major * 10 + prop.minor < 100) return RAD_EUNSUPPORTED;
  rad_plan p = new rad_plan_s();
  p->device = dev;
  p->sms = prop.multiProcessorCount;
  p->n_samples_total = ns;
  p->n_particles = np;
  p->n_omega = no;
  p->n_angles = na;
  p->mode = mode;
  p->precision = prec;
  p->want = want;
  p->n_bins = (want & 4) ? nb : 0;
  e = cudaMalloc(&p->ctrl, kCtrlBytes);
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e);
  }
  const size_t cube_n = static_cast<size_t>(std::max<int64_t>(no * na, 1));
  e = cudaMalloc(&p->cube_new, cube_n * sizeof(double));
  if (e != cudaSuccess) {
    cudaFree(p->ctrl);
    delete p;
    return cuda_fail(e);
  }
  Choice c = default_choice(prec, mode, no);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_tuned.find(key_of(dev, ns, np, no, na, mode, prec, want, p->n_bins));
    if (it != g_tuned.end()) c = it->second;
  }
  rc = configure(p, c);
  if (rc) {
    cudaFree(p->ctrl);
    cudaFree(p->cube_new);
    if (p->part) cudaFree(p->part);
    delete p;
    return rc;
  }
  *out = p;
  return RAD_OK;
}

void plan_free(rad_plan p) {
  if (!p) return;
  cudaDeviceSynchronize();
  if (p->prep) cudaFree(p->prep);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  if (p->part) cudaFree(p->part);
  if (p->cube_new) cudaFree(p->cube_new);
  if (p->ctrl) cudaFree(p->ctrl);
  delete p;
}

// library-owned device buffers of rad_spectrum_host, per device
struct HostBufs {
  void *ptr[12] = {nullptr};
  size_t cap[12] = {0};
};
std::map<int, HostBufs> g_hbufs;

int ensure(HostBufs &b, int slot, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.cap[slot] >= bytes) return RAD_OK;
  if (b.ptr[slot]) cudaFree(b.ptr[slot]);
  b.ptr[slot] = nullptr;
  b.cap[slot] = 0;
  cudaError_t e = cudaMalloc(&b.ptr[slot], bytes);
  if (e != cudaSuccess) return cuda_fail(e);
  b.cap[slot] = bytes;
  return RAD_OK;
}

}  // namespace

extern "C" {

const char *rad_version(void) { return "radspec-gb300 0.1 (sm_103a)"; }

const char *rad_status_string(int status) {
  switch (status) {
    case RAD_OK: return "ok";
    case RAD_EINVAL: return "invalid argument";
    case RAD_ENOMEM: return "device allocation failed";
    case RAD_ECUDA: return g_cuda_msg;
    case RAD_ETIMEOUT: return "a bounded device-side wait ran out";
    case RAD_EUNSUPPORTED: return "unsupported request (needs an sm_100-class or newer GPU)";
    case RAD_EDATA: return "device-side input check failed (non-finite value, bad offsets, gamma <= 1, hw <= 0 or hw >= E)";
    case RAD_ETOOBIG: return "n_omega * n_angles exceeds the no-allocation entry point's fixed 32 MiB scratch";
    case RAD_EPRECISION:
      return "RAD_MIXED: the in-tile phase offsets exceed its error budget (directions far outside the emission "
             "cone, coarse time steps or hw close to E); use RAD_FP64_DF";
    default: return "unknown status";
  }
}

int rad_plan_create(int64_t n_samples_total, int64_t n_particles, int64_t n_omega, int64_t n_angles,
                    int mode, int precision, int want, int32_t n_bins, rad_plan *plan) {
  return plan_create(n_samples_total, n_particles, n_omega, n_angles, mode, precision, want, n_bins, plan);
}

int rad_plan_execute(rad_plan plan, const double *samples, const int64_t *offsets, const double *gamma,
                     const double *energy_eV, const double *weight, const double *hbar_omega_eV,
                     const double *theta_x, const double *theta_y, const double *d_omega,
                     double *out_cube, double *out_spectrum, const int32_t *bin_of_angle,
                     double *out_bins, int accumulate, void *stream) {
  if (!plan) return RAD_EINVAL;
  return execute(plan, samples, offsets, gamma, energy_eV, weight, hbar_omega_eV, theta_x, theta_y,
                 d_omega, out_cube, out_spectrum, bin_of_angle, out_bins, accumulate,
                 static_cast<cudaStream_t>(stream));
}

int rad_plan_set_prepass(rad_plan plan, int enable) {
  if (!plan || plan->precision != RAD_MIXED) return RAD_EINVAL;
  Choice c = plan->choice;
  c.pp = enable ? 1 : 0;
  if (!c.pp) c.pe = 0;
  if (!supported(plan->precision, c)) return RAD_EINVAL;
  const Choice old = plan->choice;
  int rc = configure(plan, c);
  if (rc) configure(plan, old);
  return rc;
}

int rad_plan_set_shape(rad_plan plan, int R, int NW, int T, int chunk_mult) {
  if (!plan || chunk_mult < 1) return RAD_EINVAL;
  Choice c{R, NW, T, chunk_mult, plan->choice.pp, plan->choice.pe};
  if (plan->precision == RAD_MIXED && !supported(plan->precision, c)) {
    c.pp = 1 - c.pp;
    if (!c.pp) c.pe = 0;
  }
  if (!supported(plan->precision, c)) return RAD_EINVAL;
  const Choice old = plan->choice;
  int rc = configure(plan, c);
  if (rc) configure(plan, old);
  return rc;
}

int rad_plan_set_sincos_split(rad_plan plan, int every) {
  if (!plan || plan->precision != RAD_MIXED || !plan->choice.pp) return RAD_EINVAL;
  Choice c = plan->choice;
  c.pe = every;
  if (!supported(plan->precision, c)) return RAD_EINVAL;
  const Choice old = plan->choice;
  int rc = configure(plan, c);
  if (rc) configure(plan, old);
  return rc;
}

int rad_plan_set_phase_budget(rad_plan plan, double radians) {
  if (!plan || plan->precision != RAD_MIXED) return RAD_EINVAL;
  if (!(radians > 0.0) || !(radians < 1e300)) return RAD_EINVAL;
  plan->phase_budget = radians;
  return RAD_OK;
}

int rad_plan_describe(rad_plan plan, char *buf, int len) {
  if (!plan || !buf || len <= 0) return RAD_EINVAL;
  std::snprintf(buf, static_cast<size_t>(len), "%s", plan->desc.c_str());
  return RAD_OK;
}

int rad_plan_set_timing(rad_plan plan, int enable) {
  if (!plan) return RAD_EINVAL;
  if (enable && !plan->ev0) {
    cudaError_t e = cudaEventCreate(&plan->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&plan->ev1);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  plan->timing = enable != 0;
  plan->timed_once = false;
  return RAD_OK;
}

int rad_plan_last_kernel_ms(rad_plan plan, double *ms) {
  if (!plan || !ms || !plan->timed_once) return RAD_EINVAL;
  cudaError_t e = cudaEventSynchronize(plan->ev1);
  if (e != cudaSuccess) return cuda_fail(e);
  float f = 0.f;
  e = cudaEventElapsedTime(&f, plan->ev0, plan->ev1);
  if (e != cudaSuccess) return cuda_fail(e);
  *ms = static_cast<double>(f);
  return RAD_OK;
}

int rad_plan_kernel_launches(rad_plan plan) {
  if (!plan) return 0;
  if (plan->n_omega == 0 || plan->n_angles == 0) return 0;
  const int pre = (plan->precision == RAD_MIXED && plan->choice.pp) ? 1 : 0;  // pre-pass
  if (plan->want & RAD_PER_PARTICLE) return 3 + pre;  // validate, main, per-particle reduce
  int n = 3 + pre;  // validate, main, finalize
  if (plan->want & 6) n += 1;
  return n;
}

int rad_plan_destroy(rad_plan plan) {
  plan_free(plan);
  return RAD_OK;
}

int rad_plan_autotune(rad_plan plan, const double *samples, const int64_t *offsets, const double *gamma,
                      const double *energy_eV, const double *weight, const double *hbar_omega_eV,
                      const double *theta_x, const double *theta_y, const double *d_omega,
                      double *out_cube, double *out_spectrum, const int32_t *bin_of_angle,
                      double *out_bins, int budget_ms, void *stream) {
  if (!plan || budget_ms < 0) return RAD_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<Choice> cands;
  const int Rs[] = {1, 2, 4};
  const int NWs[] = {4, 8};
  const int Ts[] = {64, 128, 256};
  const int mults[] = {1, 2, 4};
  const int pes[] = {0, 4, 6};
  for (int pp = 0; pp <= 1; ++pp)
    for (int pe : pes)
      for (int R : Rs)
        for (int NW : NWs)
          for (int T : Ts)
            for (int m : mults) {
              Choice c{R, NW, T, m, pp, pe};
              if (supported(plan->precision, c)) cands.push_back(c);
            }
  const Choice start = plan->choice;
  Choice best = start;
  float best_ms = 1e30f;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return cuda_fail(cudaGetLastError());
  const auto t_start = std::chrono::steady_clock::now();
  int rc = RAD_OK;
  for (const Choice &c : cands) {
    const double spent = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    if (spent > budget_ms && best_ms < 1e30f) break;
    rc = configure(plan, c);
    if (rc) continue;
    // one untimed run (module load, caches), one timed run
    rc = execute(plan, samples, offsets, gamma, energy_eV, weight, hbar_omega_eV, theta_x, theta_y, d_omega,
                 out_cube, out_spectrum, bin_of_angle, out_bins, 0, st);
    if (rc) break;
    cudaEventRecord(e0, st);
    rc = execute(plan, samples, offsets, gamma, energy_eV, weight, hbar_omega_eV, theta_x, theta_y, d_omega,
                 out_cube, out_spectrum, bin_of_angle, out_bins, 0, st);
    cudaEventRecord(e1, st);
    if (rc) break;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      rc = cuda_fail(e);
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int rc2 = configure(plan, best_ms < 1e30f ? best : start);
  if (rc == RAD_OK) rc = rc2;
  if (rc == RAD_OK) {
    std::lock_guard<std::mutex> lk(g_mu);
    // cached rad_spectrum plans of this shape pick up the choice on their next call
    g_tuned[key_of(plan->device, plan->n_samples_total, plan->n_particles, plan->n_omega, plan->n_angles,
                   plan->mode, plan->precision, plan->want, plan->n_bins)] = plan->choice;
  }
  // leave a result of the chosen shape in the outputs
  if (rc == RAD_OK)
    rc = execute(plan, samples, offsets, gamma, energy_eV, weight, hbar_omega_eV, theta_x, theta_y, d_omega,
                 out_cube, out_spectrum, bin_of_angle, out_bins, 0, st);
  if (rc == RAD_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e);
  }
  return rc;
}

int rad_spectrum(const double *samples, int64_t n_samples_total, const int64_t *offsets, int64_t n_particles,
                 const double *gamma, const double *energy_eV, const double *weight,
                 const double *hbar_omega_eV, int64_t n_omega, const double *theta_x, const double *theta_y,
                 const double *d_omega, int64_t n_angles, int mode, int precision, double *out_cube,
                 double *out_spectrum, const int32_t *bin_of_angle, int32_t n_bins, double *out_bins,
                 int accumulate, void *stream) {
  const int want = (out_cube ? 1 : 0) | (out_spectrum ? 2 : 0) | (out_bins ? 4 : 0);
  int rc = check_shape(n_samples_total, n_particles, n_omega, n_angles, mode, precision, want, n_bins);
  if (rc) return rc;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  const int32_t nb = (want & 4) ? n_bins : 0;
  const ShapeKey k = key_of(dev, n_samples_total, n_particles, n_omega, n_angles, mode, precision, want, nb);
  rad_plan p = nullptr;
  Choice tuned{};
  bool have_tuned = false;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_plans.find({k, stream});
    if (it != g_plans.end()) p = it->second;
    auto tt = g_tuned.find(k);
    if (tt != g_tuned.end()) {
      tuned = tt->second;
      have_tuned = true;
    }
  }
  if (p && have_tuned && !same_choice(tuned, p->choice)) {
    // a newer autotuned shape: reconfigure (scratch growth frees with cudaFree, which waits
    // for the device, so work still using the old scratch has finished)
    rc = configure(p, tuned);
    if (rc) return rc;
  }
  if (!p) {
    rc = plan_create(n_samples_total, n_particles, n_omega, n_angles, mode, precision, want, nb, &p);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_mu);
    auto ins = g_plans.emplace(std::make_tuple(k, stream), p);
    if (!ins.second) {  // another thread created it first
      plan_free(p);
      p = ins.first->second;
    }
  }
  return execute(p, samples, offsets, gamma, energy_eV, weight, hbar_omega_eV, theta_x, theta_y, d_omega,
                 out_cube, out_spectrum, bin_of_angle, out_bins, accumulate, static_cast<cudaStream_t>(stream));
}

int rad_spectrum_particles(const double *samples, int64_t n_samples_total, const int64_t *offsets,
                           int64_t n_particles, const double *gamma, const double *energy_eV, const double *weight,
                           const double *hbar_omega_eV, int64_t n_omega, const double *theta_x,
                           const double *theta_y, const double *d_omega, int64_t n_angles, int mode, int precision,
                           double *out_spectrum, const int32_t *bin_of_angle, int32_t n_bins, double *out_bins,
                           void *stream) {
  const int want = RAD_PER_PARTICLE | (out_spectrum ? 2 : 0) | (out_bins ? 4 : 0);
  int rc = check_shape(n_samples_total, n_particles, n_omega, n_angles, mode, precision, want, n_bins);
  if (rc) return rc;
  if (n_angles > 0 && !d_omega) return RAD_EINVAL;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  const int32_t nb = (want & 4) ? n_bins : 0;
  const ShapeKey k = key_of(dev, n_samples_total, n_particles, n_omega, n_angles, mode, precision, want, nb);
  rad_plan p = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_plans.find({k, stream});
    if (it != g_plans.end()) p = it->second;
  }
  if (!p) {
    rc = plan_create(n_samples_total, n_particles, n_omega, n_angles, mode, precision, want, nb, &p);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_mu);
    auto ins = g_plans.emplace(std::make_tuple(k, stream), p);
    if (!ins.second) {
      plan_free(p);
      p = ins.first->second;
    }
  }
  return execute(p, samples, offsets, gamma, energy_eV, weight, hbar_omega_eV, theta_x, theta_y, d_omega,
                 nullptr, out_spectrum, bin_of_angle, out_bins, 0, static_cast<cudaStream_t>(stream));
}

int rad_spectrum_host(const double *samples, int64_t n_samples_total, const int64_t *offsets,
                      int64_t n_particles, const double *gamma, const double *energy_eV, const double *weight,
                      const double *hbar_omega_eV, int64_t n_omega, const double *theta_x,
                      const double *theta_y, const double *d_omega, int64_t n_angles, int mode, int precision,
                      double *out_cube, double *out_spectrum, const int32_t *bin_of_angle, int32_t n_bins,
                      double *out_bins, int accumulate, void *stream) {
  const int want = (out_cube ? 1 : 0) | (out_spectrum ? 2 : 0) | (out_bins ? 4 : 0);
  int rc = check_shape(n_samples_total, n_particles, n_omega, n_angles, mode, precision, want, n_bins);
  if (rc) return rc;
  if (n_particles > 0 && (!samples || !gamma || !energy_eV)) return RAD_EINVAL;
  if (!offsets || (n_omega > 0 && !hbar_omega_eV) || (n_angles > 0 && (!theta_x || !theta_y))) return RAD_EINVAL;
  const bool need_dom = out_spectrum || out_bins;
  if (need_dom && n_angles > 0 && !d_omega) return RAD_EINVAL;
  if (out_bins && !bin_of_angle) return RAD_EINVAL;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t nb = (want & 4) ? n_bins : 0;
  const size_t sz[12] = {
      sizeof(double) * n_samples_total * kRec, sizeof(int64_t) * (n_particles + 1),
      sizeof(double) * n_particles,           sizeof(double) * n_particles,
      sizeof(double) * n_particles,           sizeof(double) * n_omega,
      sizeof(double) * n_angles,              sizeof(double) * n_angles,
      sizeof(double) * n_angles,              sizeof(double) * n_omega * n_angles,
      sizeof(double) * n_omega,               sizeof(double) * n_omega * nb};
  const void *src[9] = {samples, offsets, gamma, energy_eV, weight, hbar_omega_eV, theta_x, theta_y, d_omega};
  std::lock_guard<std::mutex> lk_host([]() -> std::mutex & {
    static std::mutex m;
    return m;
  }());
  HostBufs *b;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    b = &g_hbufs[dev];
  }
  for (int i = 0; i < 12; ++i) {
    rc = ensure(*b, i, sz[i]);
    if (rc) return rc;
  }
  void *bins_slot = nullptr;
  int32_t *d_boa = nullptr;
  if (out_bins) {
    rc = ensure(*b, 11, sz[11] + sizeof(int32_t) * n_angles + 64);
    if (rc) return rc;
    bins_slot = b->ptr[11];
    d_boa = reinterpret_cast<int32_t *>(static_cast<char *>(b->ptr[11]) + ((sz[11] + 63) / 64) * 64);
  }
  for (int i = 0; i < 9; ++i) {
    if (!src[i] || sz[i] == 0) continue;
    e = cudaMemcpyAsync(b->ptr[i], src[i], sz[i], cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  if (out_bins) {
    e = cudaMemcpyAsync(d_boa, bin_of_angle, sizeof(int32_t) * n_angles, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  double *d_cube = out_cube ? static_cast<double *>(b->ptr[9]) : nullptr;
  double *d_spec = out_spectrum ? static_cast<double *>(b->ptr[10]) : nullptr;
  double *d_bins = out_bins ? static_cast<double *>(bins_slot) : nullptr;
  if (accumulate) {  // bring the caller's current values over so the result adds to them
    if (d_cube) e = cudaMemcpyAsync(d_cube, out_cube, sz[9], cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && d_spec) e = cudaMemcpyAsync(d_spec, out_spectrum, sz[10], cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && d_bins) e = cudaMemcpyAsync(d_bins, out_bins, sz[11], cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  rc = rad_spectrum(static_cast<const double *>(b->ptr[0]), n_samples_total,
                    static_cast<const int64_t *>(b->ptr[1]), n_particles, static_cast<const double *>(b->ptr[2]),
                    static_cast<const double *>(b->ptr[3]), weight ? static_cast<const double *>(b->ptr[4]) : nullptr,
                    static_cast<const double *>(b->ptr[5]), n_omega, static_cast<const double *>(b->ptr[6]),
                    static_cast<const double *>(b->ptr[7]), d_omega ? static_cast<const double *>(b->ptr[8]) : nullptr,
                    n_angles, mode, precision, d_cube, d_spec, d_boa, n_bins, d_bins, accumulate, stream);
  if (rc) return rc;
  // read the call's device status through the cached plan's control word
  if (d_cube) e = cudaMemcpyAsync(out_cube, d_cube, sz[9], cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && d_spec) e = cudaMemcpyAsync(out_spectrum, d_spec, sz[10], cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && d_bins) e = cudaMemcpyAsync(out_bins, d_bins, sz[11], cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e);
  int call_status = 0;
  {
    rad_plan p = nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_plans.find({key_of(dev, n_samples_total, n_particles, n_omega, n_angles, mode, precision, want,
                                   static_cast<int>(nb)),
                            stream});
    if (it != g_plans.end()) p = it->second;
    if (p && n_omega > 0 && n_angles > 0) {
      e = cudaMemcpyAsync(&call_status, p->ctrl + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) return cuda_fail(e);
    }
  }
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  return call_status;
}

int rad_graph_create(rad_plan plan, const double *samples, const int64_t *offsets, const double *gamma,
                     const double *energy_eV, const double *weight, const double *hbar_omega_eV,
                     const double *theta_x, const double *theta_y, const double *d_omega, double *out_cube,
                     double *out_spectrum, const int32_t *bin_of_angle, double *out_bins, int accumulate,
                     void *stream, rad_graph *graph) {
  if (!plan || !graph) return RAD_EINVAL;
  *graph = nullptr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!st) return RAD_EINVAL;  // capture needs a non-default stream
  cudaError_t e;
  if (!device_table(&e)) return cuda_fail(e);  // allocate per-device resources before capture
  if (!device_status_word(&e)) return cuda_fail(e);
  e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e);
  int rc = execute(plan, samples, offsets, gamma, energy_eV, weight, hbar_omega_eV, theta_x, theta_y, d_omega,
                   out_cube, out_spectrum, bin_of_angle, out_bins, accumulate, st);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(st, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e);
  cudaGraphExec_t x = nullptr;
  e = cudaGraphInstantiate(&x, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(e);
  }
  rad_graph h = new rad_graph_s();
  h->graph = g;
  h->exec = x;
  *graph = h;
  return RAD_OK;
}

int rad_graph_launch(rad_graph graph, void *stream) {
  if (!graph) return RAD_EINVAL;
  cudaError_t e = cudaGraphLaunch(graph->exec, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? RAD_OK : cuda_fail(e);
}

int rad_graph_destroy(rad_graph graph) {
  if (!graph) return RAD_OK;
  if (graph->exec) cudaGraphExecDestroy(graph->exec);
  if (graph->graph) cudaGraphDestroy(graph->graph);
  delete graph;
  return RAD_OK;
}

int rad_selftest_bounded_wait(void *stream) {
  const cudaError_t e = launch_wait_selftest(static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? RAD_OK : cuda_fail(e);
}

int rad_device_status(int reset) {
  cudaError_t e;
  int *ds = device_status_word(&e);
  if (!ds) return cuda_fail(e);
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e);
  int v = 0;
  e = cudaMemcpy(&v, ds, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e);
  if (reset) {
    e = cudaMemset(ds, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return v;
}

void rad_release(void) {
  cudaDeviceSynchronize();
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto &kv : g_plans) plan_free(kv.second);
  g_plans.clear();
  g_tuned.clear();
  for (auto &kv : g_hbufs)
    for (int i = 0; i < 12; ++i)
      if (kv.second.ptr[i]) cudaFree(kv.second.ptr[i]);
  g_hbufs.clear();
}

}  // extern "C"
