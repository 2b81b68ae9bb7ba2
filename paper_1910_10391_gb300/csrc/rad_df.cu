// FP64-accurate radiation-integral kernel that spends the FP64 pipe only where the result needs
// it (sm_103a). GB300 executes FP64 at 1/64 of its FP32 rate, and the plain FP64 kernel
// (rad_fp64.cu) spends about 20 FP64 instructions per term. Here a term costs one FP64 instruction:
//   phi = w* A_k(n)                      one FP64 multiply: the same double as the oracle's phase
//                                        (A_k(n) is formed in the oracle's IEEE order, FP64)
//   phi = j 2 pi/2048 + r                the table index j and the reduced phase by a fixed-point
//                                        (Payne-Hanek) reduction of phi's bits with 32-bit integer
//                                        multiplies (rad_df_reduce.cuh)
// and everything after the reduction runs in double-float FP32 arithmetic (T. J. Dekker, Numer.
// Math. 18 (1971); error-free products by FMA, sums by Knuth's TwoSum or Dekker's Fast2Sum):
//   r = (r_hi, r_lo)                     the reduction's fraction times pi/1024 as a float pair
//   sin r, cos r - 1                     Taylor series on |r| <= pi/2048, FP32 beyond the leading
//                                        term of sin
//   sin phi, cos phi                     with a (cos, sin)(2 pi j/2048) table held as float pairs,
//                                        one error-free product and one Fast2Sum each
//   sum_k f_k e^{i phi_k}                 f as float pairs, accumulated with the compensated dot
//                                        product of Ogita, Rump and Oishi ("Accurate sum and dot
//                                        product", SIAM J. Sci. Comput. 26 (2005), Dot2): per term
//                                        and component an error-free product, a TwoSum and the
//                                        errors summed in FP32; f_z is not summed: the expanded f
//                                        of Sec. II satisfies n_x f_x + n_y f_y + f_z = 0
//                                        identically, so I_z = -(n_x I_x + n_y I_y) is formed from
//                                        the particle amplitudes
// The sums over runs of two 64-sample tiles are added into FP64 particle amplitudes. The per-term error is about 1e-14
// of |f|, far inside the FP64 form's tolerance (1e-9 of a bin, floor 1e-6 of the peak).
// Work split: a block takes one direction and NW 32 R energies. The per-(direction, sample)
// preparation (the FP64 phase A_k(n), 1 - n.beta, f and j) is computed once per block and time
// tile and shared by all NW 32 R energies, so that the FP64 pipe carries little beyond the phase
// products.
#include <cstdio>

#include "rad_df_reduce.cuh"
#include "rad_internal.cuh"

namespace rad {
namespace {

constexpr int kDfTabN = 2048;  // table of (cos, sin)(2 pi j / 2048): every other FP64 table entry
using dfr::reduce_phase;
using dfr::split_df;

// s + t = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &t) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + t = a + b exactly when |a| >= |b| or a = 0 (Dekker)
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &t) {
  s = __fadd_rn(a, b);
  t = __fsub_rn(b, __fsub_rn(s, a));
}

// one Dot2 step: (S, C) += (fh + fl)(eh + el)
__device__ __forceinline__ void dot2(float &S, float &C, float fh, float fl, float eh, float el) {
  const float p = __fmul_rn(fh, eh);
  float q = __fmaf_rn(fh, eh, -p);                 // exact error of the product
  q = __fmaf_rn(fh, el, __fmaf_rn(fl, eh, q));     // cross terms
  float s, t;
  two_sum(S, p, s, t);
  S = s;
  C = __fadd_rn(C, __fadd_rn(t, q));
}

template <int MODE>
struct DfNcomp {
  static constexpr int value = (MODE == RAD_SPIN_HALF) ? 8 : 6;  // components that leave the kernel
};

// component c of the NC output components (I_x, I_y, I_z, J as re, im) from the NC - 2 summed ones
// (I_x, I_y, J): I_z = -(n_x I_x + n_y I_y)
__device__ __forceinline__ double df_component(const double *a, int c, double nx, double ny) {
  if (c < 4) return a[c];
  if (c < 6) return -fma(nx, a[c - 4], ny * a[c - 2]);
  return a[c - 2];
}

// Shared memory of a block: the float-pair table, the double-buffered stage of trajectory records
// and the per-sample preparation of the block's direction (A [T] double, Fa [T] float4 and, for
// spin 1/2, Fj [T] float2), written once per tile by the block and read by all its warps.
template <int MODE, int R, int NW, int T>
struct DfLayout {
  static constexpr int kStageDoubles = (T + 2) * kRec;
  static constexpr int kTable = 0;                                   // float4 [kDfTabN]
  static constexpr int kStage = kTable + kDfTabN * 16;
  static constexpr int kNk = kStage + 2 * kStageDoubles * 8;
  static constexpr int kNkBytes = T * 8 + T * 16 + ((MODE == RAD_SPIN_HALF) ? T * 8 : 0);
  static constexpr int kBar = kNk + kNkBytes;
  static constexpr int kMisc = kBar + 16;
  static constexpr int kTotal = kMisc + 16;
};

// Tile sums (FP32 Dot2 pairs) are added into the FP64 particle amplitudes every kConvTiles tiles
// and at the end of a particle. Ogita, Rump and Oishi bound the Dot2 error of n terms by
// gamma_n^2 times the sum of the products' magnitudes (gamma_n = n u / (1 - n u), u = 2^-24), which
// for 2 x 64 terms is below 1e-10 of that sum; each conversion costs 4 FP64 instructions per
// component and energy.
constexpr int kConvTiles = 2;

// Blocks of 4 warps run 5 per SM (46 KB of shared memory each; registers held to 96, for which the
// compiler spills 12-152 bytes per thread at R = 2): 20 warps per SM hide the float-pair chains'
// latency better than 16 at 122-128 registers without spills (723 / 839 ms against 754 / 865 ms per
// 4-particle launch of the positron ensemble, classical / spin-1/2). Blocks of 8 warps run 2 per SM.
template <int MODE, int R, int NW, int T>
__global__ void __launch_bounds__(NW * 32, NW == 4 ? 5 : 2) k_df(const Params P) {
  using L = DfLayout<MODE, R, NW, T>;
  constexpr int NC = DfNcomp<MODE>::value;
  constexpr int NA = NC - 2;  // summed components
  extern __shared__ __align__(128) unsigned char sm[];
  float4 *tab = reinterpret_cast<float4 *>(sm + L::kTable);
  double *stage_base = reinterpret_cast<double *>(sm + L::kStage);
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + L::kBar);
  int *s_item = reinterpret_cast<int *>(sm + L::kMisc);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_item[1] = *reinterpret_cast<volatile int *>(P.status);
  __syncthreads();
  if (s_item[1] != 0) return;

  // (cos, sin)(2 pi j / 2048) as float pairs (c_hi, c_lo, s_hi, s_lo) from every other entry of the
  // FP64 table (2048 entries, 32 KB)
  for (int i = tid; i < kDfTabN; i += NW * 32) {
    const double2 t = P.table[2 * i];
    const float ch = __double2float_rn(t.x), sh = __double2float_rn(t.y);
    tab[i] = make_float4(ch, __double2float_rn(t.x - static_cast<double>(ch)), sh,
                         __double2float_rn(t.y - static_cast<double>(sh)));
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t parity[2] = {0u, 0u};
  double *sA = reinterpret_cast<double *>(sm + L::kNk);
  float4 *sFa = reinterpret_cast<float4 *>(sm + L::kNk + T * 8);   // (fx_hi, fx_lo, fy_hi, fy_lo)
  float2 *sFj = reinterpret_cast<float2 *>(sm + L::kNk + T * 24);  // (j_hi, j_lo), spin 1/2 only

  const int64_t per_chunk = static_cast<int64_t>(P.n_wt) * P.n_nt;
  int s = 0;

  for (;;) {
    if (tid == 0) s_item[0] = atomicAdd(P.counter, 1);
    __syncthreads();
    const int64_t item = s_item[0];
    __syncthreads();
    if (item >= P.n_items) break;
    const int64_t chunk = item / per_chunk;
    const int64_t rem = item % per_chunk;
    // one direction per item, shared by the block's warps (the per-sample preparation is done
    // once for all of them); warp w takes the energies (wt NW + w) 32 R + 32 r + lane
    const int64_t jdir = rem / P.n_wt;
    const int wt = static_cast<int>(rem % P.n_wt);
    const double nx = P.theta_x[jdir];
    const double ny = P.theta_y[jdir];
    const double th2h = __dmul_rn(__dadd_rn(__dmul_rn(nx, nx), __dmul_rn(ny, ny)), 0.5);

    // energy indices; the energies themselves are read where they are used
    const int64_t iw0 = (static_cast<int64_t>(wt) * NW + warp) * 32 * R + lane;
    auto hw_of = [&](int r) { return iw0 + 32 * r < P.n_omega ? __ldg(P.hw + iw0 + 32 * r) : 1.0; };
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
      // compensated sums (S + C per component) since the last conversion into amp
      float tS[R][NA], tC[R][NA];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < NA; ++c) tS[r][c] = tC[r][c] = 0.f;
      int since = 0;
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
            const double hwr = hw_of(r);
            const double w = __ddiv_rn(hwr, kHbarC);
            if (MODE == RAD_CLASSICAL) {
              ws[r] = w;
            } else {
              const double u = __ddiv_rn(hwr, En);
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
            mbar_wait_bounded(&bar[s], parity[s] ^ 1u);
            if (nxt.valid) mbar_wait_bounded(&bar[s ^ 1], parity[s ^ 1]);
          }
          return;
        }
        const double *st = stage_base + s * L::kStageDoubles;
        const int n = static_cast<int>((cur.ke - cur.k0) < T ? (cur.ke - cur.k0) : T);

        // per (n, k), once per block: phase A in the oracle's IEEE order (FP64), weighted f and j
        // as float pairs
        for (int k = tid; k < n; k += NW * 32) {
          const double *rc = st + (k + 1) * kRec;
          const int64_t K = cur.k0 + k;
          const double tm = (K == 0) ? rc[F_T] : st[k * kRec + F_T];
          const double tp = (K == cur.L - 1) ? rc[F_T] : st[(k + 2) * kRec + F_T];
          const double w = 0.5 * (tp - tm);
          double A = __dmul_rn(cn, rc[F_T]);
          A = __dsub_rn(A, rc[F_DZ]);
          A = __dsub_rn(A, __dmul_rn(nx, rc[F_X]));
          A = __dsub_rn(A, __dmul_rn(ny, rc[F_Y]));
          const double vx = rc[F_VX], vy = rc[F_VY], dvz = rc[F_DVZ];
          const double ax = rc[F_AX], ay = rc[F_AY], az = rc[F_AZ];
          const double D = cn - dvz - nx * vx - ny * vy;  // 1 - n.beta (Sec. II, g)
          const double gw = w / (D * D);
          const double a = nx - vx, b = ny - vy;
          const double m = az + nx * ax + ny * ay;         // n.beta_dot
          const double fx = (a * m - ax * D) * gw, fy = (b * m - ay * D) * gw;
          const float fxh = __double2float_rn(fx), fyh = __double2float_rn(fy);
          sA[k] = A;
          sFa[k] = make_float4(fxh, __double2float_rn(fx - fxh), fyh, __double2float_rn(fy - fyh));
          if (MODE == RAD_SPIN_HALF) {
            const double fj = m * gw;
            const float fjh = __double2float_rn(fj);
            sFj[k] = make_float2(fjh, __double2float_rn(fj - fjh));
          }
        }
        __syncthreads();

        // compensated sums over the tile
#pragma unroll 2
        for (int k = 0; k < n; ++k) {
          const double A = sA[k];
          const float4 Fa = sFa[k];
          const float2 Fj = (MODE == RAD_SPIN_HALF) ? sFj[k] : make_float2(0.f, 0.f);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const double phi = __dmul_rn(ws[r], A);
            float xh, xl;
            const int j = reduce_phase(phi, xh, xl);
            const float4 t = tab[j & (kDfTabN - 1)];  // (C_hi, C_lo, S_hi, S_lo)
            const float x2 = __fmul_rn(xh, xh);
            const float x2e = __fmaf_rn(xh, xh, -x2);  // xh^2 = x2 + x2e exactly
            // cos x - 1 and the part of sin x below xh
            const float cm = __fmaf_rn(-0.5f, x2e, __fmaf_rn(-xh, xl, __fmul_rn(x2, __fmaf_rn(x2, 1.0f / 24.0f, -0.5f))));
            const float sxl = __fmaf_rn(__fmul_rn(-xh, x2), __fmaf_rn(x2, -1.0f / 120.0f, 1.0f / 6.0f), xl);
            // sin(phi) = S + S cm + C xh + C sxl. The table's leading parts are 0 at multiples of pi/2
            // (filled by exact symmetry) and at least sin(2 pi/2048) = 3.07e-3 in magnitude elsewhere,
            // twice |C xh| <= pi/2048, so Fast2Sum gives the exact sum of S and C xh
            float sh, sl;
            {
              const float p = __fmul_rn(t.x, xh);
              const float pe = __fmaf_rn(t.x, xh, -p);
              float v;
              fast_two_sum(t.z, p, sh, v);
              sl = __fadd_rn(v, __fadd_rn(pe, __fmaf_rn(t.y, xh, __fmaf_rn(t.x, sxl, __fmaf_rn(t.z, cm, t.w)))));
            }
            // cos(phi) = C + C cm - S xh - S sxl
            float ch, cl;
            {
              const float p = __fmul_rn(-t.z, xh);
              const float pe = __fmaf_rn(-t.z, xh, -p);
              float v;
              fast_two_sum(t.x, p, ch, v);
              cl = __fadd_rn(v, __fadd_rn(pe, __fmaf_rn(-t.w, xh, __fmaf_rn(-t.z, sxl, __fmaf_rn(t.x, cm, t.y)))));
            }
            dot2(tS[r][0], tC[r][0], Fa.x, Fa.y, ch, cl);
            dot2(tS[r][1], tC[r][1], Fa.x, Fa.y, sh, sl);
            dot2(tS[r][2], tC[r][2], Fa.z, Fa.w, ch, cl);
            dot2(tS[r][3], tC[r][3], Fa.z, Fa.w, sh, sl);
            if (MODE == RAD_SPIN_HALF) {
              dot2(tS[r][4], tC[r][4], Fj.x, Fj.y, ch, cl);
              dot2(tS[r][5], tC[r][5], Fj.x, Fj.y, sh, sl);
            }
          }
        }
        const bool last_of_particle = !nxt.valid || nxt.p != cur.p;
        if (last_of_particle || ++since == kConvTiles) {
#pragma unroll
          for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c < NA; ++c) {
              amp[r][c] += static_cast<double>(tS[r][c]) + static_cast<double>(tC[r][c]);
              tS[r][c] = tC[r][c] = 0.f;
            }
          since = 0;
        }
        if (last_of_particle && !P.amp_mode) {
#pragma unroll
          for (int r = 0; r < R; ++r) {
            double I2 = 0.0;
#pragma unroll
            for (int c = 0; c < 6; ++c) {
              const double v = df_component(amp[r], c, nx, ny);
              I2 = fma(v, v, I2);
            }
            double Sv;
            if (MODE == RAD_CLASSICAL) {
              Sv = I2;
            } else {
              const double u = hw_of(r) / En;
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
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t iw = iw0 + 32 * r;
      if (iw >= P.n_omega) continue;
      if (!P.amp_mode) {
        P.part[(chunk * P.n_angles + jdir) * P.n_omega + iw] = S_acc[r];
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c)
          P.part[((chunk * NC + c) * P.n_angles + jdir) * P.n_omega + iw] = df_component(amp[r], c, nx, ny);
      }
    }
  }
}

template <int MODE, int R, int NW>
cudaError_t launch_t(const Params &P, LaunchShape *shape, cudaStream_t st, int *occ) {
  constexpr int T = 64;
  using L = DfLayout<MODE, R, NW, T>;
  auto kern = k_df<MODE, R, NW, T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kTotal);
  if (e != cudaSuccess) return e;
  shape->smem = L::kTotal;
  if (occ) {
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NW * 32, L::kTotal);
    *occ = (e == cudaSuccess) ? nb : 0;
    return e;
  }
  if (shape->grid <= 0) return cudaErrorInvalidConfiguration;
  kern<<<shape->grid, NW * 32, L::kTotal, st>>>(P);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t dispatch_mode(const Params &P, LaunchShape *sh, cudaStream_t st, int *occ) {
  if (sh->T != 64) return cudaErrorInvalidValue;
  if (sh->R == 1 && sh->NW == 4) return launch_t<MODE, 1, 4>(P, sh, st, occ);
  if (sh->R == 1 && sh->NW == 8) return launch_t<MODE, 1, 8>(P, sh, st, occ);
  if (sh->R == 2 && sh->NW == 4) return launch_t<MODE, 2, 4>(P, sh, st, occ);
  if (sh->R == 2 && sh->NW == 8) return launch_t<MODE, 2, 8>(P, sh, st, occ);
  return cudaErrorInvalidValue;
}

cudaError_t dispatch(const Params &P, LaunchShape *sh, cudaStream_t st, int *occ) {
  switch (P.mode) {
    case RAD_CLASSICAL: return dispatch_mode<RAD_CLASSICAL>(P, sh, st, occ);
    case RAD_SPIN0: return dispatch_mode<RAD_SPIN0>(P, sh, st, occ);
    case RAD_SPIN_HALF: return dispatch_mode<RAD_SPIN_HALF>(P, sh, st, occ);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool shape_supported_df(int R, int NW, int T) {
  return T == 64 && (R == 1 || R == 2) && (NW == 4 || NW == 8);
}

cudaError_t launch_df(const Params &P, LaunchShape *shape, cudaStream_t st) {
  return dispatch(P, shape, st, nullptr);
}

int occupancy_df(const LaunchShape &s, int mode) {
  Params P{};
  P.mode = mode;
  LaunchShape sh = s;
  int occ = 0;
  if (dispatch(P, &sh, nullptr, &occ) != cudaSuccess) return 0;
  return occ;
}

}  // namespace rad
