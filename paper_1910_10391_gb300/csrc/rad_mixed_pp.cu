// Mixed-precision radiation-integral kernel fed by a per-sample pre-pass (sm_103a).
//
// Same method and precision split as k_mixed (rad_mixed.cu), reorganised so that the FP64
// per-sample work runs once per call instead of once per work item:
//   k_prep_samples  one pass over the trajectory records: for every sample, FP32 offsets of t,
//                   dz, x, y from the middle sample of its time tile (the tiling is the main
//                   kernel's), the transverse velocity, the trapezoid-weighted acceleration and
//                   s0 = 1/(2 gamma^2) - (dvz + v_perp^2/2), written as 48-byte records.
//   k_mixed_pp      stages those records with cp.async.bulk (48 B x T per tile, no halo),
//                   each warp computes f, j and the in-tile phase for its own direction, releases
//                   the stage through an mbarrier, and runs its term loop. There is no block-wide
//                   barrier per tile: warps only meet when a new work item is fetched.
#include "rad_mixed_common.cuh"

namespace rad {
namespace {

// Tile geometry shared by the pre-pass and the kernel: sample k of particle p (length L)
// belongs to the tile starting at k0 with n samples; its reference is the tile's middle sample.
__device__ __forceinline__ void tile_of(const Params &P, int64_t L, int64_t k, int T, int64_t &k0,
                                        int64_t &km) {
  int64_t kb = 0, ke = L;
  if (P.amp_mode) {
    int64_t q = (k * P.n_q) / L;
    while (q + 1 < P.n_q && (L * (q + 1)) / P.n_q <= k) ++q;
    while (q > 0 && (L * q) / P.n_q > k) --q;
    kb = (L * q) / P.n_q;
    ke = (L * (q + 1)) / P.n_q;
  }
  k0 = kb + ((k - kb) / T) * T;
  const int64_t n = (ke - k0) < T ? (ke - k0) : T;
  km = k0 + (n - 1) / 2;
}

// w*_max of particle p and the grid maxima of the error-budget guard (see kMixedPhaseBudget).
struct PhaseBound {
  double ws_max, c_max, tx_max, ty_max;
};

__device__ __forceinline__ PhaseBound phase_bound(const Params &P, double inv2g2, double E) {
  PhaseBound b;
  const double hmax = __longlong_as_double(static_cast<long long>(P.grid_max[3]));
  b.ws_max = (hmax / kHbarC) / (P.mode == RAD_CLASSICAL ? 1.0 : (1.0 - hmax / E));
  b.c_max = inv2g2 + __longlong_as_double(static_cast<long long>(P.grid_max[2]));
  b.tx_max = __longlong_as_double(static_cast<long long>(P.grid_max[0]));
  b.ty_max = __longlong_as_double(static_cast<long long>(P.grid_max[1]));
  return b;
}

// One particle's records: grid x strides over its samples. Returns true when a sample's
// in-tile phase-offset bound exceeds the mixed form's error budget.
__device__ __forceinline__ bool prep_particle(const Params &P, int T, int64_t p, float *__restrict__ out) {
  const int64_t off = P.offsets[p];
  const int64_t L = P.offsets[p + 1] - off;
  const double g = P.gamma[p];
  const double inv2g2 = 1.0 / (2.0 * g * g);
  const double *S = P.samples + off * kRec;
  const bool guard = P.grid_max != nullptr;
  PhaseBound pb{0.0, 0.0, 0.0, 0.0};
  if (guard) pb = phase_bound(P, inv2g2, P.energy[p]);
  bool over = false;
  for (int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < L;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int64_t k0, km;
    tile_of(P, L, k, T, k0, km);
    const double *rc = S + k * kRec;
    const double *r0 = S + km * kRec;
    const double tm = (k == 0) ? rc[F_T] : S[(k - 1) * kRec + F_T];
    const double tp = (k == L - 1) ? rc[F_T] : S[(k + 1) * kRec + F_T];
    const double w = 0.5 * (tp - tm);
    const double vx = rc[F_VX], vy = rc[F_VY];
    float *o = out + (off + k) * kPP;
    const double dt = rc[F_T] - r0[F_T], ddz = rc[F_DZ] - r0[F_DZ];
    const double dx = rc[F_X] - r0[F_X], dy = rc[F_Y] - r0[F_Y];
    if (guard) {
      const double B = pb.c_max * fabs(dt) + fabs(ddz) + pb.tx_max * fabs(dx) + pb.ty_max * fabs(dy);
      if (!(pb.ws_max * B <= P.phase_budget)) over = true;
    }
    float4 a, b, c;
    a.x = static_cast<float>(dt);
    a.y = static_cast<float>(ddz);
    a.z = static_cast<float>(dx);
    a.w = static_cast<float>(dy);
    b.x = static_cast<float>(vx);
    b.y = static_cast<float>(vy);
    b.z = static_cast<float>(rc[F_AX] * w);
    b.w = static_cast<float>(rc[F_AY] * w);
    c.x = static_cast<float>(rc[F_AZ] * w);
    c.y = static_cast<float>(inv2g2 - (rc[F_DVZ] + 0.5 * (vx * vx + vy * vy)));
    c.z = 0.f;
    c.w = 0.f;
    reinterpret_cast<float4 *>(o)[0] = a;
    reinterpret_cast<float4 *>(o)[1] = b;
    reinterpret_cast<float4 *>(o)[2] = c;
  }
  return over;
}

__global__ void k_prep_samples(const Params P, int T, float *__restrict__ out) {
  if (*reinterpret_cast<volatile int *>(P.status) != 0) return;  // device data check failed
  bool over = false;
  for (int64_t p = blockIdx.y; p < P.n_particles; p += gridDim.y) over |= prep_particle(P, T, p, out);
  if (over) set_status(P.status, RAD_EPRECISION);  // the integral kernel and the finalize skip
}

template <int MODE, int R, int NW, int T>
struct PPLayout {
  static constexpr int kStageBytes = T * kPP * 4;
  static constexpr int kStage = 0;
  static constexpr int kNk = kStage + 2 * kStageBytes;
  static constexpr int kNkWarp = T * 16;  // (phase offset, f_x, f_y, j) per sample
  static constexpr int kBar = kNk + NW * kNkWarp;  // full[2], empty[2]
  static constexpr int kMisc = kBar + 32;
  static constexpr int kTotal = kMisc + 16;
};

// sin and cos of x (radians) on the FMA pipe, to take part of the terms off the SFU:
// x = j pi/2 + r with j = rint(2x/pi) formed by adding 1.5 2^23 (the integer lands in the low
// mantissa bits), r by a three-term Cody-Waite reduction (each step one FMA, so the product
// j * (pi/2)_i is exact inside it), |r| <= pi/4; Taylor polynomials of degree 9 (sin) and 8
// (cos) in r (truncation below 3e-8 on |r| <= pi/4); the quadrant j mod 4 rotates the pair.
// Valid for |2x/pi| < 2^22.
__device__ __forceinline__ void sincos_fma(float x, float &s, float &c) {
  constexpr float kMagic = 12582912.0f;             // 1.5 * 2^23
  const float t = __fmaf_rn(x, 0.636619772367581343f, kMagic);
  const float j = __fsub_rn(t, kMagic);
  float r = __fmaf_rn(-j, 1.57079637050628662f, x);   // (pi/2)_1 = fl(pi/2)
  r = __fmaf_rn(-j, -4.37113900018624283e-08f, r);    // (pi/2)_2 = fl(pi/2 - (pi/2)_1)
  r = __fmaf_rn(-j, -1.70899169742600938e-15f, r);    // (pi/2)_3
  const float r2 = r * r;
  float ps = __fmaf_rn(r2, 2.75573192239858907e-06f, -1.98412698412698413e-04f);
  ps = __fmaf_rn(r2, ps, 8.33333333333333333e-03f);
  ps = __fmaf_rn(r2, ps, -1.66666666666666667e-01f);
  const float sr = __fmaf_rn(r * r2, ps, r);
  float pc = __fmaf_rn(r2, 2.48015873015873016e-05f, -1.38888888888888889e-03f);
  pc = __fmaf_rn(r2, pc, 4.16666666666666667e-02f);
  pc = __fmaf_rn(r2, pc, -0.5f);
  const float cr = __fmaf_rn(r2, pc, 1.0f);
  const int q = __float_as_int(t);  // = 2^22 + j: its low two bits are j mod 4
  const float a = (q & 1) ? cr : sr;
  const float b = (q & 1) ? sr : cr;
  s = (q & 2) ? -a : a;
  c = ((q + 1) & 2) ? -b : b;
}

// PE: with PE > 0, the term with index (q R + r) % PE == PE - 1 in every group of 8 samples x R
// energies takes sincos_fma instead of the SFU (about 1/PE of the terms), balancing the SFU
// against the FMA pipe and the issue slots.
template <int MODE, int R, int NW, int T, int PE>
__global__ void __launch_bounds__(NW * 32, NW == 8 ? (R <= 2 ? 2 : 1) : 3) k_mixed_pp(const Params P, const float *__restrict__ prep) {
  using L = PPLayout<MODE, R, NW, T>;
  // NC components leave the kernel (I_x, I_y, I_z and, for spin 1/2, J, each re and im); NA are
  // summed: the expanded f of Sec. II satisfies n_x f_x + n_y f_y + f_z = 0 identically, so
  // I_z = -(n_x I_x + n_y I_y) is formed from the sums at the end instead of being summed.
  constexpr int NC = (MODE == RAD_SPIN_HALF) ? 8 : 6;
  constexpr int NA = NC - 2;
  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t *full = reinterpret_cast<uint64_t *>(sm + L::kBar);
  uint64_t *empty = full + 2;
  int *s_item = reinterpret_cast<int *>(sm + L::kMisc);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float4 *myF = reinterpret_cast<float4 *>(sm + L::kNk + warp * L::kNkWarp);

  if (tid == 0) s_item[1] = *reinterpret_cast<volatile int *>(P.status);
  __syncthreads();
  if (s_item[1] != 0) return;
  if (tid == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_init(&empty[0], NW);
    mbar_init(&empty[1], NW);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t full_par[2] = {0u, 0u};   // consumers: next parity of full[s]
  uint32_t uses[2] = {0u, 0u};       // producer (thread 0): copies issued into stage s so far
  const int64_t per_chunk = static_cast<int64_t>(P.n_wt) * P.n_nt;
  int s = 0;

  // thread 0: wait until every warp released stage st's previous tile, then fill it
  auto produce = [&](const TileCursor &c, int st) -> bool {
    if (uses[st] > 0 && !mbar_wait_bounded(&empty[st], (uses[st] - 1) & 1u)) return false;
    const int64_t n = (c.ke - c.k0) < T ? (c.ke - c.k0) : T;
    const uint32_t bytes = static_cast<uint32_t>(n * kPP * 4);
    const float *src = prep + (P.offsets[c.p] + c.k0) * kPP;
    fence_proxy_async();
    mbar_arrive_expect_tx(&full[st], bytes);
    bulk_g2s(sm + L::kStage + st * L::kStageBytes, src, bytes, &full[st]);
    uses[st] += 1;
    return true;
  };

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
    float ks[R][NA], kc[R][NA];
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
    bool failed = false;
    if (cur.valid) {
      if (tid == 0 && !produce(cur, s)) failed = true;
      int64_t cur_p = -1;
      double ws[R];
      float ws_f[R], wt_hi[R], wt_lo[R];
      double inv2g2 = 0.0, cn = 0.0, wp = 1.0, gam = 2.0, En = 1.0;
      float cn_hi = 0.f, cn_lo = 0.f;
      for (;;) {
        TileCursor nxt = cur;
        cursor_next<T>(P, nxt, q);
        if (tid == 0 && nxt.valid && !failed && !produce(nxt, s ^ 1)) failed = true;
        if (cur.p != cur_p) {
          cur_p = cur.p;
          gam = P.gamma[cur_p];
          En = P.energy[cur_p];
          wp = P.weight ? P.weight[cur_p] : 1.0;
          inv2g2 = 1.0 / (2.0 * gam * gam);
          cn = inv2g2 + th2h;
          cn_hi = static_cast<float>(cn);
          cn_lo = static_cast<float>(cn - static_cast<double>(cn_hi));
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
        const bool ok = !failed && mbar_wait_bounded(&full[s], full_par[s]);
        full_par[s] ^= 1u;
        if (__any_sync(0xffffffffu, !ok)) {  // bounded wait ran out (or the producer gave up)
          if (lane == 0) set_status(P.status, RAD_ETIMEOUT);
          if (tid == 0) {
            mbar_wait_bounded(&full[s], full_par[s] ^ 1u);
            if (nxt.valid) mbar_wait_bounded(&full[s ^ 1], full_par[s ^ 1]);
          }
          return;
        }
        const float *st = reinterpret_cast<const float *>(sm + L::kStage + s * L::kStageBytes);
        const int n = static_cast<int>((cur.ke - cur.k0) < T ? (cur.ke - cur.k0) : T);
        const int km = (n - 1) >> 1;

        // base phase at the reference (middle) sample, FP64 by lane 0, as a double-float pair;
        // started here and consumed after the term loop, so its global load and FP64 chain overlap
        // the tile's FP32 work
        float a0h = 0.f, a0l = 0.f;
        if (lane == 0) {
          const double *r0 = P.samples + (P.offsets[cur.p] + cur.k0 + km) * kRec;
          const double A0 = ((cn * r0[F_T] - r0[F_DZ]) - nx * r0[F_X]) - ny * r0[F_Y];
          a0h = static_cast<float>(A0);
          a0l = static_cast<float>(A0 - static_cast<double>(a0h));
        }

        // per (n, k): weighted f_x, f_y, j and the FP32 phase offset for this warp's direction
        for (int k = lane; k < n; k += 32) {
          const float4 ra = reinterpret_cast<const float4 *>(st + k * kPP)[0];
          const float4 rb = reinterpret_cast<const float4 *>(st + k * kPP)[1];
          const float2 rcz = reinterpret_cast<const float2 *>(st + k * kPP)[4];
          const float a = nxf - rb.x, b = nyf - rb.y;
          const float axw = rb.z, ayw = rb.w, azw = rcz.x;
          const float m = fmaf(nyf, ayw, fmaf(nxf, axw, azw));
          const float D = fmaf(0.5f, fmaf(a, a, b * b), rcz.y);
          const float rD = __frcp_rn(D);
          const float g = rD * rD;
          float4 o;
          o.x = fmaf(-nyf, ra.w, fmaf(-nxf, ra.z, fmaf(cn_hi, ra.x, fmaf(cn_lo, ra.x, -ra.y))));
          o.y = fmaf(a, m, -axw * D) * g;
          o.z = fmaf(b, m, -ayw * D) * g;
          o.w = (MODE == RAD_SPIN_HALF) ? m * g : 0.f;
          myF[k] = o;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);  // this warp is done with the stage

        float tpart[R][NA];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int c = 0; c < NA; ++c) tpart[r][c] = 0.f;
        auto term = [&](const float4 &F, int r, bool on_fma) {
          const float x = ws_f[r] * F.x;
          float sn, cs;
          if (on_fma)
            sincos_fma(x, sn, cs);
          else
            __sincosf(x, &sn, &cs);
          tpart[r][0] = fmaf(F.y, cs, tpart[r][0]);
          tpart[r][1] = fmaf(F.y, sn, tpart[r][1]);
          tpart[r][2] = fmaf(F.z, cs, tpart[r][2]);
          tpart[r][3] = fmaf(F.z, sn, tpart[r][3]);
          if (MODE == RAD_SPIN_HALF) {
            tpart[r][4] = fmaf(F.w, cs, tpart[r][4]);
            tpart[r][5] = fmaf(F.w, sn, tpart[r][5]);
          }
        };
        int k = 0;
        for (; k + 8 <= n; k += 8) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 F = myF[k + q];
#pragma unroll
            for (int r = 0; r < R; ++r) term(F, r, PE > 0 && (q * R + r) % (PE > 0 ? PE : 1) == PE - 1);
          }
        }
        for (; k < n; ++k) {
          const float4 F = myF[k];
#pragma unroll
          for (int r = 0; r < R; ++r) term(F, r, false);
        }
        a0h = __shfl_sync(0xffffffffu, a0h, 0);
        a0l = __shfl_sync(0xffffffffu, a0l, 0);
        float c0[R], s0[R];
#pragma unroll
        for (int r = 0; r < R; ++r) tile_base_sincos(wt_hi[r], wt_lo[r], a0h, a0l, ws[r], s0[r], c0[r]);
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
        s ^= 1;
        if (!nxt.valid) break;
        cur = nxt;
      }
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
  // drain: the last copies of every stage were consumed; nothing is in flight here
}

template <int MODE, int R, int NW, int T, int PE>
cudaError_t launch_t(const Params &P, const float *prep, LaunchShape *shape, cudaStream_t st, int *occ) {
  using L = PPLayout<MODE, R, NW, T>;
  auto kern = k_mixed_pp<MODE, R, NW, T, PE>;
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
  kern<<<shape->grid, NW * 32, L::kTotal, st>>>(P, prep);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t dispatch_mode(const Params &P, const float *prep, LaunchShape *sh, cudaStream_t st, int *occ) {
#define RAD_PP_CASE(RR, WW, TT)                                                          \
  if (sh->R == RR && sh->NW == WW && sh->T == TT) {                                      \
    if (sh->pe == 4) return launch_t<MODE, RR, WW, TT, 4>(P, prep, sh, st, occ);         \
    if (sh->pe == 6) return launch_t<MODE, RR, WW, TT, 6>(P, prep, sh, st, occ);         \
    if (sh->pe == 0) return launch_t<MODE, RR, WW, TT, 0>(P, prep, sh, st, occ);         \
    return cudaErrorInvalidValue;                                                        \
  }
  RAD_PP_CASE(2, 8, 128)
  RAD_PP_CASE(2, 8, 256)
  RAD_PP_CASE(2, 4, 256)
  RAD_PP_CASE(4, 8, 128)
  RAD_PP_CASE(4, 8, 256)
#undef RAD_PP_CASE
  return cudaErrorInvalidValue;
}

cudaError_t dispatch(const Params &P, const float *prep, LaunchShape *sh, cudaStream_t st, int *occ) {
  switch (P.mode) {
    case RAD_CLASSICAL: return dispatch_mode<RAD_CLASSICAL>(P, prep, sh, st, occ);
    case RAD_SPIN0: return dispatch_mode<RAD_SPIN0>(P, prep, sh, st, occ);
    case RAD_SPIN_HALF: return dispatch_mode<RAD_SPIN_HALF>(P, prep, sh, st, occ);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool shape_supported_mixed_pp(int R, int NW, int T) {
  if (T == 128) return (R == 2 || R == 4) && NW == 8;
  if (T == 256) return (R == 2 && (NW == 4 || NW == 8)) || (R == 4 && NW == 8);
  return false;
}

cudaError_t launch_prep_samples(const Params &P, int T, float *prep, cudaStream_t st) {
  if (P.n_particles == 0) return cudaSuccess;
  dim3 grd(8, grid_y(P.n_particles));
  k_prep_samples<<<grd, 256, 0, st>>>(P, T, prep);
  return cudaGetLastError();
}

cudaError_t launch_mixed_pp(const Params &P, const float *prep, LaunchShape *shape, cudaStream_t st) {
  return dispatch(P, prep, shape, st, nullptr);
}

int occupancy_mixed_pp(const LaunchShape &s, int mode) {
  Params P{};
  P.mode = mode;
  LaunchShape sh = s;
  int occ = 0;
  if (dispatch(P, nullptr, &sh, nullptr, &occ) != cudaSuccess) return 0;
  return occ;
}

}  // namespace rad
