// Mixed-precision radiation-integral kernel for sm_103a (Sec. II integrand).
//
// Precision split (the method is unchanged: the same trapezoid sum of Eq. 1 in the
// expanded variables of Sec. II):
//   - FP64: the phase A at the middle sample of each time tile and the per-sample inputs
//     (the longitudinal term q = -(dvz + v_perp^2/2), tile-relative differences of t, dz,
//     x, y); the particle sum of |amplitude|^2.
//   - double-float FP32 (T. J. Dekker, "A floating-point technique for extending the
//     available precision", Numer. Math. 18 (1971)): the tile's base phase (w*/2pi) A_ref in
//     turns and its exact reduction to [-1/2, 1/2] (magic-number rounding).
//   - FP32: the phase offset within the tile, x_k = w* (A_k - A_ref), sin/cos of x_k on
//     the SFU, f(t, n) and j(t, n) (Sec. II, with
//     1 - n.beta = 1/(2 gamma^2) + |n_perp - v_perp|^2/2 + q, algebraically equal to the
//     paper's g base and free of cancellation), tile sums of f e^{i phi}.
//   - Tile sums are rotated by e^{i Phi0} and added to Kahan-compensated FP32 running sums
//     (W. Kahan, "Further remarks on reducing truncation errors", CACM 8 (1965)).
// Per term: 2 SFU ops (sin, cos) and 6 (classical/spin-0) or 8 (spin-1/2) FMA-pipe ops. f_z is
// not summed: the expanded f of Sec. II satisfies n_x f_x + n_y f_y + f_z = 0 identically, so
// I_z = -(n_x I_x + n_y I_y) is formed from the running sums.
#include "rad_mixed_common.cuh"

namespace rad {
namespace {

template <int MODE, int R, int NW, int T>
struct MixLayout {
  static constexpr int kStageDoubles = (T + 2) * kRec;
  static constexpr int NS = 10;  // per-sample FP32 arrays: dt ddz dx dy vx vy axw ayw azw s0
  static constexpr int kStage = 0;
  static constexpr int kSamp = kStage + 2 * kStageDoubles * 8;
  static constexpr int kRef = kSamp + NS * T * 4;          // per warp: FP64 phase at the reference sample
  static constexpr int kNk = kRef + 16 * NW;                // per warp: float4 [T] (dA, fx, fy, j)
  static constexpr int kNkWarp = T * 16;
  static constexpr int kBar = kNk + NW * kNkWarp;
  static constexpr int kMisc = kBar + 16;
  static constexpr int kGuard = kMisc + 16;  // error-budget guard: w*_max, c_max, max|theta_x|, max|theta_y|
  static constexpr int kTotal = kGuard + 16;
};

template <int MODE, int R, int NW, int T>
__global__ void __launch_bounds__(NW * 32) k_mixed(const Params P) {
  using L = MixLayout<MODE, R, NW, T>;
  constexpr int NC = (MODE == RAD_SPIN_HALF) ? 8 : 6;  // I_x, I_y, I_z (, J) as re, im
  constexpr int NA = NC - 2;                             // summed: I_x, I_y (, J)
  extern __shared__ __align__(128) unsigned char sm[];
  double *stage_base = reinterpret_cast<double *>(sm + L::kStage);
  float *samp = reinterpret_cast<float *>(sm + L::kSamp);
  float *sDt = samp, *sDdz = samp + T, *sDx = samp + 2 * T, *sDy = samp + 3 * T;
  float *sVx = samp + 4 * T, *sVy = samp + 5 * T, *sAx = samp + 6 * T, *sAy = samp + 7 * T;
  float *sAz = samp + 8 * T, *sS0 = samp + 9 * T;
  double *sRef = reinterpret_cast<double *>(sm + L::kRef);
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + L::kBar);
  int *s_item = reinterpret_cast<int *>(sm + L::kMisc);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float4 *myF = reinterpret_cast<float4 *>(sm + L::kNk + warp * L::kNkWarp);  // dA, fx, fy, j
  // a failed device data check skips the computation (one read per block, shared by all threads)
  if (tid == 0) s_item[1] = *reinterpret_cast<volatile int *>(P.status);
  __syncthreads();
  if (s_item[1] != 0) return;

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t parity[2] = {0u, 0u};
  const int64_t per_chunk = static_cast<int64_t>(P.n_wt) * P.n_nt;
  int s = 0;
  // error-budget guard (see kMixedPhaseBudget): the current particle's w*_max and c_max and the
  // grid's max |theta_x|, |theta_y| (from the validation kernel) in shared memory, in units of
  // the budget
  float *s_guard = reinterpret_cast<float *>(sm + L::kGuard);
  bool over = false;

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
    const double th2h = (nx * nx + ny * ny) * 0.5;
    const float nxf = static_cast<float>(nx), nyf = static_cast<float>(ny);

    int64_t iw[R];
    double hwv[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      iw[r] = static_cast<int64_t>(wt) * 32 * R + r * 32 + lane;
      hwv[r] = iw[r] < P.n_omega ? P.hw[iw[r]] : 1.0;
    }
    double S_acc[R];
    float ks[R][NA], kc[R][NA];  // Kahan running sums of the current particle
#pragma unroll
    for (int r = 0; r < R; ++r) {
      S_acc[r] = 0.0;
#pragma unroll
      for (int c = 0; c < NA; ++c) ks[r][c] = kc[r][c] = 0.f;
    }
    // output component c (0..NC-1) of energy r from the compensated sums
    auto component = [&](int r, int c) -> double {
      auto v = [&](int i) { return static_cast<double>(ks[r][i]) - static_cast<double>(kc[r][i]); };
      if (c < 4) return v(c);
      if (c < 6) return -fma(nx, v(c - 4), ny * v(c - 2));
      return v(c - 2);
    };

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
      double ws[R];              // w* (1/m), FP64
      float ws_f[R];             // w* in FP32 (radians per metre)
      float wt_hi[R], wt_lo[R];  // w*/(2 pi) split into two floats (turns per metre)
      double inv2g2 = 0.0, cn = 0.0, wp = 1.0, gam = 2.0, En = 1.0;
      float cn_hi = 0.f, cn_lo = 0.f;
      for (;;) {
        TileCursor nxt = cur;
        cursor_next<T>(P, nxt, q);
        if (nxt.valid && tid == 0)
          issue_tile<T>(P, nxt, stage_base + (s ^ 1) * L::kStageDoubles, &bar[s ^ 1]);
        if (cur.p != cur_p) {
          cur_p = cur.p;
          gam = P.gamma[cur_p];
          En = P.energy[cur_p];
          wp = P.weight ? P.weight[cur_p] : 1.0;
          inv2g2 = 1.0 / (2.0 * gam * gam);
          cn = inv2g2 + th2h;
          cn_hi = static_cast<float>(cn);
          cn_lo = static_cast<float>(cn - static_cast<double>(cn_hi));
          if (tid == 0 && P.grid_max) {
            const double hmax = __longlong_as_double(static_cast<long long>(P.grid_max[3]));
            const double wsm = (hmax / kHbarC) / (MODE == RAD_CLASSICAL ? 1.0 : (1.0 - hmax / En));
            const double scale = wsm / P.phase_budget;
            s_guard[0] = static_cast<float>(scale * (inv2g2 + __longlong_as_double(static_cast<long long>(P.grid_max[2]))));
            s_guard[1] = static_cast<float>(scale);
            s_guard[2] = static_cast<float>(scale * __longlong_as_double(static_cast<long long>(P.grid_max[0])));
            s_guard[3] = static_cast<float>(scale * __longlong_as_double(static_cast<long long>(P.grid_max[1])));
          }
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const double w = hwv[r] / kHbarC;
            ws[r] = (MODE == RAD_CLASSICAL) ? w : w / (1.0 - hwv[r] / En);
            ws_f[r] = static_cast<float>(ws[r]);
            const double wtd = ws[r] * kInvTwoPi;
            wt_hi[r] = static_cast<float>(wtd);
            wt_lo[r] = static_cast<float>(wtd - static_cast<double>(wt_hi[r]));
#pragma unroll
            for (int c = 0; c < NA; ++c) ks[r][c] = kc[r][c] = 0.f;
          }
        }
        const bool ok = mbar_wait_bounded(&bar[s], parity[s]);
        parity[s] ^= 1u;
        if (__syncthreads_or(!ok)) {
          if (tid == 0) {
            set_status(P.status, RAD_ETIMEOUT);
            mbar_wait_bounded(&bar[s], parity[s] ^ 1u);
            if (nxt.valid) mbar_wait_bounded(&bar[s ^ 1], parity[s ^ 1]);
          }
          return;
        }
        const double *st = stage_base + s * L::kStageDoubles;
        const int n = static_cast<int>((cur.ke - cur.k0) < T ? (cur.ke - cur.k0) : T);

        // per-sample preparation (direction independent), FP64 -> FP32; offsets are taken
        // from the tile's middle sample so that in-tile phases stay small
        const int km = (n - 1) >> 1;
        const double *r0 = st + (km + 1) * kRec;
        for (int k = tid; k < n; k += NW * 32) {
          const double *rc = st + (k + 1) * kRec;
          const int64_t K = cur.k0 + k;
          const double tm = (K == 0) ? rc[F_T] : st[k * kRec + F_T];
          const double tp = (K == cur.L - 1) ? rc[F_T] : st[(k + 2) * kRec + F_T];
          const double w = 0.5 * (tp - tm);
          const double vx = rc[F_VX], vy = rc[F_VY];
          sDt[k] = static_cast<float>(rc[F_T] - r0[F_T]);
          sDdz[k] = static_cast<float>(rc[F_DZ] - r0[F_DZ]);
          sDx[k] = static_cast<float>(rc[F_X] - r0[F_X]);
          sDy[k] = static_cast<float>(rc[F_Y] - r0[F_Y]);
          sVx[k] = static_cast<float>(vx);
          sVy[k] = static_cast<float>(vy);
          sAx[k] = static_cast<float>(rc[F_AX] * w);
          sAy[k] = static_cast<float>(rc[F_AY] * w);
          sAz[k] = static_cast<float>(rc[F_AZ] * w);
          sS0[k] = static_cast<float>(inv2g2 - (rc[F_DVZ] + 0.5 * (vx * vx + vy * vy)));
          if (P.grid_max) {  // w*_max B_k / budget, B_k as in kMixedPhaseBudget
            const float X = fmaf(s_guard[3], fabsf(sDy[k]),
                                 fmaf(s_guard[2], fabsf(sDx[k]), fmaf(s_guard[0], fabsf(sDt[k]), s_guard[1] * fabsf(sDdz[k]))));
            if (!(X <= 1.0f)) over = true;
          }
        }
        if (tid < NW) {  // FP64 phase A at the reference sample, one per warp's direction
          const int64_t jd = static_cast<int64_t>(nt) * NW + tid;
          const double ux = jd < P.n_angles ? P.theta_x[jd] : 0.0;
          const double uy = jd < P.n_angles ? P.theta_y[jd] : 0.0;
          const double c_u = inv2g2 + (ux * ux + uy * uy) * 0.5;
          const double A0 = ((c_u * r0[F_T] - r0[F_DZ]) - ux * r0[F_X]) - uy * r0[F_Y];
          sRef[2 * tid] = A0;
        }
        __syncthreads();

        // per (n, k): weighted f, j and the FP32 phase offset
        for (int k = lane; k < n; k += 32) {
          const float a = nxf - sVx[k], b = nyf - sVy[k];
          const float axw = sAx[k], ayw = sAy[k], azw = sAz[k];
          const float m = fmaf(nyf, ayw, fmaf(nxf, axw, azw));            // w n.beta_dot
          const float D = fmaf(0.5f, fmaf(a, a, b * b), sS0[k]);          // 1 - n.beta
          const float rD = __frcp_rn(D);
          const float g = rD * rD;
          float4 o;
          o.x = fmaf(-nyf, sDy[k], fmaf(-nxf, sDx[k], fmaf(cn_hi, sDt[k], fmaf(cn_lo, sDt[k], -sDdz[k]))));
          o.y = fmaf(a, m, -axw * D) * g;
          o.z = fmaf(b, m, -ayw * D) * g;
          o.w = (MODE == RAD_SPIN_HALF) ? m * g : 0.f;
          myF[k] = o;
        }
        __syncwarp();

        // base phase of the tile: (w*/2pi) A0 in double-float FP32 (Dekker products with
        // fmaf), reduced to [-1/2, 1/2] turns; FP64 for phases beyond 2^21 turns
        const double A0 = sRef[2 * warp];
        const float a0h = static_cast<float>(A0);
        const float a0l = static_cast<float>(A0 - static_cast<double>(a0h));
        float c0[R], s0[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float p = wt_hi[r] * a0h;
          float e = fmaf(wt_hi[r], a0h, -p);
          e = fmaf(wt_hi[r], a0l, e);
          e = fmaf(wt_lo[r], a0h, e);
          float rr;
          if (fabsf(p) < 2097152.0f) {
            const float nr = __fsub_rn(__fadd_rn(p, kMagicF), kMagicF);
            rr = __fadd_rn(__fsub_rn(p, nr), e);
          } else {
            const double ph = ws[r] * A0 * kInvTwoPi;
            rr = static_cast<float>(ph - rint(ph));
          }
          __sincosf(rr * kTwoPiF, &s0[r], &c0[r]);
        }

        float tpart[R][NA];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int c = 0; c < NA; ++c) tpart[r][c] = 0.f;
        // per term: phase offset x = w* (A_k - A_ref) in radians (the reference is the tile's
        // middle sample, so |x| stays below ~1e3 rad), SFU sin/cos with the unit's own
        // periodic argument handling (absolute error ~2e-7 |x|, random per term; bounded by
        // tests/test_sfu.py), and the amplitude FMAs
#pragma unroll 4
        for (int k = 0; k < n; ++k) {
          const float4 F = myF[k];
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const float x = ws_f[r] * F.x;
            float sn, cs;
            __sincosf(x, &sn, &cs);
            tpart[r][0] = fmaf(F.y, cs, tpart[r][0]);
            tpart[r][1] = fmaf(F.y, sn, tpart[r][1]);
            tpart[r][2] = fmaf(F.z, cs, tpart[r][2]);
            tpart[r][3] = fmaf(F.z, sn, tpart[r][3]);
            if (MODE == RAD_SPIN_HALF) {
              tpart[r][4] = fmaf(F.w, cs, tpart[r][4]);
              tpart[r][5] = fmaf(F.w, sn, tpart[r][5]);
            }
          }
        }
        // rotate the tile sums by e^{i Phi0} and add them to the running sums
#pragma unroll
        for (int r = 0; r < R; ++r) {
#pragma unroll
          for (int c = 0; c < NA; c += 2) {
            const float re = fmaf(c0[r], tpart[r][c], -s0[r] * tpart[r][c + 1]);
            const float im = fmaf(s0[r], tpart[r][c], c0[r] * tpart[r][c + 1]);
            kahan_add(ks[r][c], kc[r][c], re);
            kahan_add(ks[r][c + 1], kc[r][c + 1], im);
          }
        }

        const bool last_of_particle = !nxt.valid || nxt.p != cur.p;
        if (last_of_particle && !P.amp_mode) {
#pragma unroll
          for (int r = 0; r < R; ++r) {
            double I2 = 0.0;
#pragma unroll
            for (int c = 0; c < 6; ++c) {
              const double v = component(r, c);
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
                const double jr = component(r, 6);
                const double ji = component(r, 7);
                Sv = 0.5 * (1.0 + (1.0 - u) * (1.0 - u)) * I2 + (u * u) / (2.0 * gam * gam) * (jr * jr + ji * ji);
              }
            }
            S_acc[r] = fma(wp, Sv, S_acc[r]);
          }
        }
        __syncthreads();
        s ^= 1;
        if (!nxt.valid) break;
        cur = nxt;
      }
    }
    if (over) {  // the finalize then leaves the outputs untouched
      set_status(P.status, RAD_EPRECISION);
      over = false;
    }
    if (jvalid) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (iw[r] >= P.n_omega) continue;
        if (!P.amp_mode) {
          P.part[(chunk * P.n_angles + jdir) * P.n_omega + iw[r]] = S_acc[r];
        } else {
#pragma unroll
          for (int c = 0; c < NC; ++c)
            P.part[((chunk * NC + c) * P.n_angles + jdir) * P.n_omega + iw[r]] = component(r, c);
        }
      }
    }
  }
}

template <int MODE, int R, int NW, int T>
cudaError_t launch_t(const Params &P, LaunchShape *shape, cudaStream_t st, int *occ) {
  using L = MixLayout<MODE, R, NW, T>;
  auto kern = k_mixed<MODE, R, NW, T>;
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
#define RAD_MIX_CASE(RR, WW, TT) \
  if (sh->R == RR && sh->NW == WW && sh->T == TT) return launch_t<MODE, RR, WW, TT>(P, sh, st, occ);
  RAD_MIX_CASE(1, 8, 64)
  RAD_MIX_CASE(2, 4, 64)
  RAD_MIX_CASE(2, 8, 64)
  RAD_MIX_CASE(2, 8, 128)
  RAD_MIX_CASE(4, 4, 64)
  RAD_MIX_CASE(4, 8, 64)
  RAD_MIX_CASE(4, 8, 128)
  RAD_MIX_CASE(2, 4, 256)
  RAD_MIX_CASE(2, 8, 256)
#undef RAD_MIX_CASE
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

bool shape_supported_mixed(int R, int NW, int T) {
  if (T == 64) return (R == 1 && NW == 8) || ((R == 2 || R == 4) && (NW == 4 || NW == 8));
  if (T == 128) return (R == 2 || R == 4) && NW == 8;
  if (T == 256) return R == 2 && (NW == 4 || NW == 8);
  return false;
}

cudaError_t launch_mixed(const Params &P, LaunchShape *shape, cudaStream_t st) {
  return dispatch(P, shape, st, nullptr);
}

int occupancy_mixed(const LaunchShape &s, int mode) {
  Params P{};
  P.mode = mode;
  LaunchShape sh = s;
  int occ = 0;
  if (dispatch(P, &sh, nullptr, &occ) != cudaSuccess) return 0;
  return occ;
}

}  // namespace rad
