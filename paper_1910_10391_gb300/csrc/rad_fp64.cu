// Plain FP64 radiation-integral kernel for sm_103a (Sec. II integrand, Sec. IV decomposition).
//
// Every operation is FP64, as the paper requires for this sum (Sec. IV). The phase
//   A_k(n) = ((c t_k - dz_k) - nx x_k) - ny y_k,  c = 1/((2 gamma) gamma) + (nx nx + ny ny) 0.5,
//   phi    = w* A_k,  w* = (hw/hbar_c) / (1 - hw/E)  (quantum modes)  or  hw/hbar_c,
// is evaluated in exactly this IEEE order with no fused operations, so it is the same
// double as any other implementation that follows that order. sin/cos of phi use a
// table-driven method (P. T. P. Tang, "Table-driven implementation of the exponential
// function", ACM TOMS 15 (1989), applied to sin/cos): phi is split into j * 2pi/4096 + r
// with a two-part Cody-Waite reduction (W. J. Cody, W. Waite, "Software Manual for the
// Elementary Functions", 1980), (cos, sin)(2 pi j/4096) is read from a shared-memory table
// and sin r, cos r - 1 come from their Taylor series (|r| <= pi/4096: truncation below
// 3e-18). About 14 FP64 operations per sin/cos pair, 18 (classical) or 20 (spin 1/2) per term
// with the accumulation: the expanded f of Sec. II satisfies n_x f_x + n_y f_y + f_z = 0
// identically, so I_z = -(n_x I_x + n_y I_y) is formed from the particle amplitudes instead of
// being summed.
#include <cstdio>

#include "rad_internal.cuh"

namespace rad {
namespace {

// 2 pi / kTabN = pi * 2^-11 split into the double nearest pi and its remainder, both
// scaled by 2^-11 (exact): C1 + C2 = 2 pi / 4096 to about 106 bits.
constexpr double kPiHi = 3.141592653589793116;        // nearest double to pi
constexpr double kPiLo = 1.2246467991473531772e-16;   // pi - kPiHi (rounded)
constexpr double kC1 = kPiHi / 2048.0;
constexpr double kC2 = kPiLo / 2048.0;
constexpr double kInvStep = 2048.0 / 3.141592653589793238462643383279502884;  // 4096/(2 pi)
constexpr double kMagic = 6755399441055744.0;  // 1.5 * 2^52: adding it rounds to an integer

__device__ __forceinline__ void sincos_table(double phi, const double2 *__restrict__ tab, double &s,
                                             double &c) {
  const double y = fma(phi, kInvStep, kMagic);  // round(phi * 4096/(2 pi)) + magic
  const int j = __double2loint(y);              // low word holds the integer (two's complement)
  const double jd = y - kMagic;                 // exact
  double r = fma(-jd, kC1, phi);
  r = fma(-jd, kC2, r);
  const double2 t = tab[j & (kTabN - 1)];       // (cos, sin)(2 pi j / 4096)
  const double r2 = r * r;
  const double sr = fma(r2 * r, -1.0 / 6.0, r);           // sin r
  const double cm = r2 * fma(r2, 1.0 / 24.0, -0.5);       // cos r - 1
  s = fma(t.x, sr, fma(t.y, cm, t.y));                    // sin(a + r)
  c = fma(-t.y, sr, fma(t.x, cm, t.x));                   // cos(a + r)
}

template <int MODE>
struct Ncomp {
  static constexpr int value = (MODE == RAD_SPIN_HALF) ? 8 : 6;  // components that leave the kernel
};

// component c of the NC output components (I_x, I_y, I_z, J as re, im) from the NC - 2 summed ones
// (I_x, I_y, J): I_z = -(n_x I_x + n_y I_y)
template <typename V>
__device__ __forceinline__ double out_component(const V &a, int c, double nx, double ny) {
  if (c < 4) return a[c];
  if (c < 6) return -fma(nx, a[c - 4], ny * a[c - 2]);
  return a[c - 2];
}

template <int MODE, int R, int NW, int T>
struct Fp64Layout {
  static constexpr int NARR = (MODE == RAD_SPIN_HALF) ? 4 : 3;  // A, fx, fy (, j)
  static constexpr int kStageDoubles = (T + 2) * kRec;
  static constexpr int kTable = 0;
  static constexpr int kStage = kTable + kTabN * 16;
  static constexpr int kNk = kStage + 2 * kStageDoubles * 8;
  static constexpr int kBar = kNk + NW * NARR * T * 8;
  static constexpr int kMisc = kBar + 16;
  static constexpr int kTotal = kMisc + 16;
};

template <int MODE, int R, int NW, int T>
__global__ void __launch_bounds__(NW * 32) k_fp64(const Params P) {
  using L = Fp64Layout<MODE, R, NW, T>;
  constexpr int NC = Ncomp<MODE>::value;
  constexpr int NA = NC - 2;  // summed components
  constexpr int NARR = L::NARR;
  extern __shared__ __align__(128) unsigned char sm[];
  double2 *tab = reinterpret_cast<double2 *>(sm + L::kTable);
  double *stage_base = reinterpret_cast<double *>(sm + L::kStage);
  double *nk = reinterpret_cast<double *>(sm + L::kNk);
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + L::kBar);
  int *s_item = reinterpret_cast<int *>(sm + L::kMisc);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // a failed device data check skips the computation (one read per block, shared by all threads)
  if (tid == 0) s_item[1] = *reinterpret_cast<volatile int *>(P.status);
  __syncthreads();
  if (s_item[1] != 0) return;

  for (int i = tid; i < kTabN; i += NW * 32) tab[i] = P.table[i];
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t parity[2] = {0u, 0u};
  double *myA = nk + warp * NARR * T;
  double *myFx = myA + T, *myFy = myA + 2 * T;
  double *myJ = myA + 3 * T;  // spin-1/2 only

  const int64_t per_chunk = static_cast<int64_t>(P.n_wt) * P.n_nt;
  int s = 0;  // stage of the next tile to consume

  for (;;) {
    if (tid == 0) s_item[0] = atomicAdd(P.counter, 1);
    __syncthreads();
    const int64_t item = s_item[0];
    __syncthreads();
    if (item >= P.n_items) break;
    const int64_t chunk = item / per_chunk;
    const int64_t rem = item % per_chunk;
    const int nt = static_cast<int>(rem / P.n_wt), wt = static_cast<int>(rem % P.n_wt);
    const int64_t jdir = static_cast<int64_t>(nt) * NW + warp;
    const bool jvalid = jdir < P.n_angles;
    const double nx = jvalid ? P.theta_x[jdir] : 0.0;
    const double ny = jvalid ? P.theta_y[jdir] : 0.0;
    const double th2h = __dmul_rn(__dadd_rn(__dmul_rn(nx, nx), __dmul_rn(ny, ny)), 0.5);

    int64_t iw[R];
    double hwv[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      iw[r] = static_cast<int64_t>(wt) * 32 * R + r * 32 + lane;
      hwv[r] = iw[r] < P.n_omega ? P.hw[iw[r]] : 1.0;
    }
    double S_acc[R];
    double amp[R][NA];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      S_acc[r] = 0.0;
#pragma unroll
      for (int c = 0; c < NA; ++c) amp[r][c] = 0.0;
    }

    int64_t p0, p1;
    int q;
    chunk_range(P, chunk, p0, p1, q);
    TileCursor cur;
    cur.p = p0;
    cur.p_end = p1;
    cursor_settle(P, cur, q);

    if (cur.valid) {
      if (tid == 0) issue_tile<T>(P, cur, stage_base + s * L::kStageDoubles, &bar[s]);
      int64_t cur_p = -1;
      double ws[R];
      double inv2g2 = 0.0, cn = 0.0, wp = 1.0, gam = 2.0, En = 1.0;
      for (;;) {
        TileCursor nxt = cur;
        cursor_next<T>(P, nxt, q);
        if (nxt.valid && tid == 0)
          issue_tile<T>(P, nxt, stage_base + (s ^ 1) * L::kStageDoubles, &bar[s ^ 1]);
        if (cur.p != cur_p) {  // new particle: per-particle constants, fresh amplitudes
          cur_p = cur.p;
          gam = P.gamma[cur_p];
          En = P.energy[cur_p];
          wp = P.weight ? P.weight[cur_p] : 1.0;
          inv2g2 = __ddiv_rn(1.0, __dmul_rn(__dmul_rn(2.0, gam), gam));
          cn = __dadd_rn(inv2g2, th2h);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const double w = __ddiv_rn(hwv[r], kHbarC);
            if (MODE == RAD_CLASSICAL) {
              ws[r] = w;
            } else {
              const double u = __ddiv_rn(hwv[r], En);
              ws[r] = __ddiv_rn(w, __dsub_rn(1.0, u));
            }
#pragma unroll
            for (int c = 0; c < NA; ++c) amp[r][c] = 0.0;
          }
        }
        const bool ok = mbar_wait_bounded(&bar[s], parity[s]);
        parity[s] ^= 1u;
        if (__syncthreads_or(!ok)) {  // bounded wait ran out: record, drain, leave
          if (tid == 0) {
            set_status(P.status, RAD_ETIMEOUT);
            mbar_wait_bounded(&bar[s], parity[s] ^ 1u);                 // the stalled copy, again
            if (nxt.valid) mbar_wait_bounded(&bar[s ^ 1], parity[s ^ 1]);  // the prefetched one
          }
          return;
        }
        const double *st = stage_base + s * L::kStageDoubles;
        const int n = static_cast<int>((cur.ke - cur.k0) < T ? (cur.ke - cur.k0) : T);

        // per (n, k): phase A (fixed IEEE order), weighted f and j
        for (int k = lane; k < n; k += 32) {
          const double *rc = st + (k + 1) * kRec;
          const int64_t K = cur.k0 + k;
          double tm, tp;
          tm = (K == 0) ? rc[F_T] : st[k * kRec + F_T];
          tp = (K == cur.L - 1) ? rc[F_T] : st[(k + 2) * kRec + F_T];
          const double w = 0.5 * (tp - tm);
          double A = __dmul_rn(cn, rc[F_T]);
          A = __dsub_rn(A, rc[F_DZ]);
          A = __dsub_rn(A, __dmul_rn(nx, rc[F_X]));
          A = __dsub_rn(A, __dmul_rn(ny, rc[F_Y]));
          const double vx = rc[F_VX], vy = rc[F_VY], dvz = rc[F_DVZ];
          const double ax = rc[F_AX], ay = rc[F_AY], az = rc[F_AZ];
          const double D = cn - dvz - nx * vx - ny * vy;          // 1 - n.beta (Sec. II, g)
          const double gw = w / (D * D);
          const double a = nx - vx, b = ny - vy;
          const double m = az + nx * ax + ny * ay;                 // n.beta_dot
          myA[k] = A;
          myFx[k] = (a * m - ax * D) * gw;
          myFy[k] = (b * m - ay * D) * gw;
          if (MODE == RAD_SPIN_HALF) myJ[k] = m * gw;
        }
        __syncwarp();

        double tpart[R][NA];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int c = 0; c < NA; ++c) tpart[r][c] = 0.0;
        for (int k = 0; k < n; ++k) {
          const double A = myA[k], fx = myFx[k], fy = myFy[k];
          double jj = 0.0;
          if (MODE == RAD_SPIN_HALF) jj = myJ[k];
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const double phi = __dmul_rn(ws[r], A);
            double sn, cs;
            sincos_table(phi, tab, sn, cs);
            tpart[r][0] = fma(fx, cs, tpart[r][0]);
            tpart[r][1] = fma(fx, sn, tpart[r][1]);
            tpart[r][2] = fma(fy, cs, tpart[r][2]);
            tpart[r][3] = fma(fy, sn, tpart[r][3]);
            if (MODE == RAD_SPIN_HALF) {
              tpart[r][4] = fma(jj, cs, tpart[r][4]);
              tpart[r][5] = fma(jj, sn, tpart[r][5]);
            }
          }
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int c = 0; c < NA; ++c) amp[r][c] += tpart[r][c];

        const bool last_of_particle = !nxt.valid || nxt.p != cur.p;
        if (last_of_particle && !P.amp_mode) {
#pragma unroll
          for (int r = 0; r < R; ++r) {
            double I2 = 0.0;
#pragma unroll
            for (int c = 0; c < 6; ++c) {
              const double v = out_component(amp[r], c, nx, ny);
              I2 = fma(v, v, I2);
            }
            double Sv;
            if (MODE == RAD_CLASSICAL) {
              Sv = I2;
            } else {
              const double u = hwv[r] / En;
              if (MODE == RAD_SPIN0) {
                Sv = (1.0 - u) * I2;
              } else {
                const double J2 = amp[r][4] * amp[r][4] + amp[r][5] * amp[r][5];
                Sv = 0.5 * (1.0 + (1.0 - u) * (1.0 - u)) * I2 + (u * u) / (2.0 * gam * gam) * J2;
              }
            }
            S_acc[r] = fma(wp, Sv, S_acc[r]);
          }
        }
        __syncthreads();  // stage s and the per-warp arrays are free again
        s ^= 1;
        if (!nxt.valid) break;
        cur = nxt;
      }
    }
    // partial results of this item (layout [chunk][(comp)][direction][energy])
    if (jvalid) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (iw[r] >= P.n_omega) continue;
        if (!P.amp_mode) {
          P.part[(chunk * P.n_angles + jdir) * P.n_omega + iw[r]] = S_acc[r];
        } else {
#pragma unroll
          for (int c = 0; c < NC; ++c)
            P.part[((chunk * NC + c) * P.n_angles + jdir) * P.n_omega + iw[r]] = out_component(amp[r], c, nx, ny);
        }
      }
    }
  }
}

template <int MODE, int R, int NW>
cudaError_t launch_t(const Params &P, LaunchShape *shape, cudaStream_t st) {
  constexpr int T = 64;
  using L = Fp64Layout<MODE, R, NW, T>;
  auto kern = k_fp64<MODE, R, NW, T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kTotal);
  if (e != cudaSuccess) return e;
  shape->smem = L::kTotal;
  if (shape->grid <= 0) return cudaErrorInvalidConfiguration;
  kern<<<shape->grid, NW * 32, L::kTotal, st>>>(P);
  return cudaGetLastError();
}

template <int MODE, int R, int NW>
int occ_t() {
  constexpr int T = 64;
  using L = Fp64Layout<MODE, R, NW, T>;
  auto kern = k_fp64<MODE, R, NW, T>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kTotal) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NW * 32, L::kTotal) != cudaSuccess) return 0;
  return nb;
}

template <int MODE>
cudaError_t dispatch_mode(const Params &P, LaunchShape *sh, cudaStream_t st, int *occ) {
#define RAD_FP64_CASE(RR, WW)                                      \
  if (sh->R == RR && sh->NW == WW) {                               \
    if (occ) {                                                     \
      *occ = occ_t<MODE, RR, WW>();                                \
      return cudaSuccess;                                          \
    }                                                              \
    return launch_t<MODE, RR, WW>(P, sh, st);                      \
  }
  RAD_FP64_CASE(1, 4)
  RAD_FP64_CASE(1, 8)
  RAD_FP64_CASE(2, 4)
  RAD_FP64_CASE(2, 8)
  RAD_FP64_CASE(4, 4)
  RAD_FP64_CASE(4, 8)
#undef RAD_FP64_CASE
  return cudaErrorInvalidValue;
}

cudaError_t dispatch(const Params &P, LaunchShape *sh, cudaStream_t st, int *occ) {
  if (sh->T != 64) return cudaErrorInvalidValue;
  switch (P.mode) {
    case RAD_CLASSICAL: return dispatch_mode<RAD_CLASSICAL>(P, sh, st, occ);
    case RAD_SPIN0: return dispatch_mode<RAD_SPIN0>(P, sh, st, occ);
    case RAD_SPIN_HALF: return dispatch_mode<RAD_SPIN_HALF>(P, sh, st, occ);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool shape_supported_fp64(int R, int NW, int T) {
  return T == 64 && (R == 1 || R == 2 || R == 4) && (NW == 4 || NW == 8);
}

cudaError_t launch_fp64(const Params &P, LaunchShape *shape, cudaStream_t st) {
  return dispatch(P, shape, st, nullptr);
}

int occupancy_fp64(const LaunchShape &s, int mode) {
  Params P{};
  P.mode = mode;
  LaunchShape sh = s;
  int occ = 0;
  if (dispatch(P, &sh, nullptr, &occ) != cudaSuccess) return 0;
  return occ;
}

}  // namespace rad
