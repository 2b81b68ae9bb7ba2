// Mixed-precision radiation-integral kernel for direction grids that are tensor products
// (sm_103a). Same inputs (the pre-pass records of rad_mixed_pp.cu), precision split and
// outputs as k_mixed_pp; it differs in how e^{i phi} is formed.
//
// The in-tile phase offset of Sec. II, with c(n) = 1/(2 gamma^2) + (n_x^2 + n_y^2)/2,
//   dA(n, k) = c(n) dt_k - ddz_k - n_x dx_k - n_y dy_k,
// separates in the two direction components: for directions (X_j, Y_l) of a tensor grid
//   dA(j, l, k) = dA(0, 0, k) + P_j(k) + Q_l(k),
//   P_j(k) = (X_j - X_0) [ (X_j + X_0)/2 dt_k - dx_k ],  Q_l(k) = (Y_l - Y_0) [ (Y_l + Y_0)/2 dt_k - dy_k ],
// an exact identity. So for a 2 x 2 block of directions
//   e^{i w* dA(j, l)} = e^{i w* dA00} e^{i w* P_j} e^{i w* Q_l}:
// three sin/cos pairs (SFU) and three complex products give the four phase factors of one
// (energy, sample), instead of four sin/cos pairs. Per term this is ~1.5 SFU operations and ~10.5
// FMA-pipe operations (the 6 or 8 accumulations included) against 2 and 8 for k_mixed_pp, which
// is bound by the SFU; this kernel is bound by the issue slots.
//
// Work decomposition: a warp owns one 2 x 2 direction block and 32 photon energies (one per
// lane); a block of NW warps owns NW consecutive direction blocks; work items (chunk, block
// tile, energy tile) are pulled from an atomic counter by a persistent grid. Staging and the
// per-tile FP64 base phase are those of k_mixed_pp, per direction of the block.
#include "rad_mixed_common.cuh"

namespace rad {
namespace {

template <int MODE, int NW, int T>
struct SepLayout {
  static constexpr int kStageBytes = T * kPP * 4;
  static constexpr int kStage = 0;
  static constexpr int kPh = kStage + 2 * kStageBytes;   // per warp: float4 [T] (dA00, P, Q, -)
  static constexpr int kF = kPh + NW * T * 16;           // per warp: float4 [T][4] (f_x, f_y, f_z, j)
  static constexpr int kBar = kF + NW * T * 64;          // full[2], empty[2]
  static constexpr int kMisc = kBar + 32;
  static constexpr int kTotal = kMisc + 16;
};

template <int MODE, int NW, int T>
__global__ void __launch_bounds__(NW * 32, NW == 8 ? 1 : 2) k_mixed_sep(const Params P, const float *__restrict__ prep) {
  using L = SepLayout<MODE, NW, T>;
  constexpr int NC = (MODE == RAD_SPIN_HALF) ? 8 : 6;
  constexpr int ND = 4;  // directions per warp: (0,0), (1,0), (0,1), (1,1)
  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t *full = reinterpret_cast<uint64_t *>(sm + L::kBar);
  uint64_t *empty = full + 2;
  int *s_item = reinterpret_cast<int *>(sm + L::kMisc);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float4 *myPh = reinterpret_cast<float4 *>(sm + L::kPh + warp * T * 16);
  float4 *myF = reinterpret_cast<float4 *>(sm + L::kF + warp * T * 64);

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
  uint32_t full_par[2] = {0u, 0u};
  uint32_t uses[2] = {0u, 0u};
  const int64_t per_chunk = static_cast<int64_t>(P.n_wt) * P.n_nt;
  const int64_t nbx = (P.grid_nx + 1) / 2;
  const int64_t nby = (P.n_angles / P.grid_nx + 1) / 2;
  const int64_t ny = P.n_angles / P.grid_nx;
  int s = 0;

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
    // this warp's 2 x 2 direction block; a block past the end computes block 0 and writes nothing
    const int64_t blk = static_cast<int64_t>(nt) * NW + warp;
    const bool bvalid = blk < nbx * nby;
    const int64_t bb = bvalid ? blk : 0;
    const int64_t ix0 = 2 * (bb % nbx), iy0 = 2 * (bb / nbx);
    const bool vx1 = ix0 + 1 < P.grid_nx, vy1 = iy0 + 1 < ny;
    const int64_t ix1 = vx1 ? ix0 + 1 : ix0, iy1 = vy1 ? iy0 + 1 : iy0;
    int64_t jdir[ND];
    bool dvalid[ND];
    jdir[0] = iy0 * P.grid_nx + ix0;
    jdir[1] = iy0 * P.grid_nx + ix1;
    jdir[2] = iy1 * P.grid_nx + ix0;
    jdir[3] = iy1 * P.grid_nx + ix1;
    dvalid[0] = bvalid;
    dvalid[1] = bvalid && vx1;
    dvalid[2] = bvalid && vy1;
    dvalid[3] = bvalid && vx1 && vy1;
    // theta_x depends on the column only and theta_y on the row only (checked by k_validate)
    const double X0 = P.theta_x[jdir[0]], X1 = P.theta_x[jdir[1]];
    const double Y0 = P.theta_y[jdir[0]], Y1 = P.theta_y[jdir[2]];
    const float dXf = static_cast<float>(X1 - X0), hXf = static_cast<float>(0.5 * (X1 + X0));
    const float dYf = static_cast<float>(Y1 - Y0), hYf = static_cast<float>(0.5 * (Y1 + Y0));
    const float X0f = static_cast<float>(X0), X1f = static_cast<float>(X1);
    const float Y0f = static_cast<float>(Y0), Y1f = static_cast<float>(Y1);
    const double th2h00 = (X0 * X0 + Y0 * Y0) * 0.5;
    // this lane's direction for the FP64 base phase (lanes 0..3)
    const int dl = lane & 3;
    const double nxl = (dl & 1) ? X1 : X0, nyl = (dl & 2) ? Y1 : Y0;
    const double th2hl = (nxl * nxl + nyl * nyl) * 0.5;

    const int64_t iw = static_cast<int64_t>(wt) * 32 + lane;
    const double hwv = iw < P.n_omega ? P.hw[iw] : 1.0;
    double S_acc[ND];
    float ks[ND][NC], kc[ND][NC];
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      S_acc[d] = 0.0;
#pragma unroll
      for (int c = 0; c < NC; ++c) ks[d][c] = kc[d][c] = 0.f;
    }
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
      double ws = 1.0, inv2g2 = 0.0, wp = 1.0, gam = 2.0, En = 1.0;
      float ws_f = 0.f, wt_hi = 0.f, wt_lo = 0.f, cn_hi = 0.f, cn_lo = 0.f;
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
          const double cn = inv2g2 + th2h00;
          cn_hi = static_cast<float>(cn);
          cn_lo = static_cast<float>(cn - static_cast<double>(cn_hi));
          const double w = hwv / kHbarC;
          ws = (MODE == RAD_CLASSICAL) ? w : w / (1.0 - hwv / En);
          ws_f = static_cast<float>(ws);
          const double wtd = ws * kInvTwoPi;
          wt_hi = static_cast<float>(wtd);
          wt_lo = static_cast<float>(wtd - static_cast<double>(wt_hi));
#pragma unroll
          for (int d = 0; d < ND; ++d)
#pragma unroll
            for (int c = 0; c < NC; ++c) ks[d][c] = kc[d][c] = 0.f;
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

        // per (block, k): the three phase pieces and the weighted f, j of the four directions
        for (int k = lane; k < n; k += 32) {
          const float4 ra = reinterpret_cast<const float4 *>(st + k * kPP)[0];
          const float4 rb = reinterpret_cast<const float4 *>(st + k * kPP)[1];
          const float2 rcz = reinterpret_cast<const float2 *>(st + k * kPP)[4];
          float4 ph;
          ph.x = fmaf(-Y0f, ra.w, fmaf(-X0f, ra.z, fmaf(cn_hi, ra.x, fmaf(cn_lo, ra.x, -ra.y))));
          ph.y = dXf * fmaf(hXf, ra.x, -ra.z);
          ph.z = dYf * fmaf(hYf, ra.x, -ra.w);
          ph.w = 0.f;
          myPh[k] = ph;
          const float axw = rb.z, ayw = rb.w, azw = rcz.x;
#pragma unroll
          for (int d = 0; d < ND; ++d) {
            const float nxf = (d & 1) ? X1f : X0f, nyf = (d & 2) ? Y1f : Y0f;
            const float a = nxf - rb.x, b = nyf - rb.y;
            const float m = fmaf(nyf, ayw, fmaf(nxf, axw, azw));
            const float D = fmaf(0.5f, fmaf(a, a, b * b), rcz.y);
            const float rD = __frcp_rn(D);
            const float g = rD * rD;
            const float cz = fmaf(-nyf, b, fmaf(-nxf, a, D));
            float4 o;
            o.x = fmaf(a, m, -axw * D) * g;
            o.y = fmaf(b, m, -ayw * D) * g;
            o.z = fmaf(cz, m, -azw * D) * g;
            o.w = (MODE == RAD_SPIN_HALF) ? m * g : 0.f;
            myF[k * ND + d] = o;
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);  // this warp is done with the stage

        // FP64 phase of each direction at the reference (middle) sample, lanes 0..3
        float a0h = 0.f, a0l = 0.f;
        if (lane < ND) {
          const double *r0 = P.samples + (P.offsets[cur.p] + cur.k0 + km) * kRec;
          const double A0 = (((inv2g2 + th2hl) * r0[F_T] - r0[F_DZ]) - nxl * r0[F_X]) - nyl * r0[F_Y];
          a0h = static_cast<float>(A0);
          a0l = static_cast<float>(A0 - static_cast<double>(a0h));
        }

        float tp[ND][NC];
#pragma unroll
        for (int d = 0; d < ND; ++d)
#pragma unroll
          for (int c = 0; c < NC; ++c) tp[d][c] = 0.f;
        auto acc = [&](float (&t)[NC], const float4 &F, float er, float ei) {
          t[0] = fmaf(F.x, er, t[0]);
          t[1] = fmaf(F.x, ei, t[1]);
          t[2] = fmaf(F.y, er, t[2]);
          t[3] = fmaf(F.y, ei, t[3]);
          t[4] = fmaf(F.z, er, t[4]);
          t[5] = fmaf(F.z, ei, t[5]);
          if (MODE == RAD_SPIN_HALF) {
            t[6] = fmaf(F.w, er, t[6]);
            t[7] = fmaf(F.w, ei, t[7]);
          }
        };
#pragma unroll 2
        for (int k = 0; k < n; ++k) {
          const float4 ph = myPh[k];
          float s0, c0, sp, cp, sq, cq;
          __sincosf(ws_f * ph.x, &s0, &c0);
          __sincosf(ws_f * ph.y, &sp, &cp);
          __sincosf(ws_f * ph.z, &sq, &cq);
          const float e1r = fmaf(c0, cp, -s0 * sp), e1i = fmaf(c0, sp, s0 * cp);
          const float e2r = fmaf(c0, cq, -s0 * sq), e2i = fmaf(c0, sq, s0 * cq);
          const float e3r = fmaf(e1r, cq, -e1i * sq), e3i = fmaf(e1r, sq, e1i * cq);
          acc(tp[0], myF[k * ND + 0], c0, s0);
          acc(tp[1], myF[k * ND + 1], e1r, e1i);
          acc(tp[2], myF[k * ND + 2], e2r, e2i);
          acc(tp[3], myF[k * ND + 3], e3r, e3i);
        }
        // rotate each direction's tile sums by its base phase factor, add to the running sums
#pragma unroll
        for (int d = 0; d < ND; ++d) {
          const float bh = __shfl_sync(0xffffffffu, a0h, d);
          const float bl = __shfl_sync(0xffffffffu, a0l, d);
          float sb, cb;
          tile_base_sincos(wt_hi, wt_lo, bh, bl, ws, sb, cb);
#pragma unroll
          for (int c = 0; c < NC; c += 2) {
            const float re = fmaf(cb, tp[d][c], -sb * tp[d][c + 1]);
            const float im = fmaf(sb, tp[d][c], cb * tp[d][c + 1]);
            kahan_add(ks[d][c], kc[d][c], re);
            kahan_add(ks[d][c + 1], kc[d][c + 1], im);
          }
        }
        const bool last_of_particle = !nxt.valid || nxt.p != cur.p;
        if (last_of_particle && !P.amp_mode) {
          const double u = hwv / En;
#pragma unroll
          for (int d = 0; d < ND; ++d) {
            double I2 = 0.0;
#pragma unroll
            for (int c = 0; c < 6; ++c) {
              const double v = static_cast<double>(ks[d][c]) - static_cast<double>(kc[d][c]);
              I2 = fma(v, v, I2);
            }
            double Sv;
            if (MODE == RAD_CLASSICAL) {
              Sv = I2;
            } else if (MODE == RAD_SPIN0) {
              Sv = (1.0 - u) * I2;
            } else {
              const double jr = static_cast<double>(ks[d][6]) - static_cast<double>(kc[d][6]);
              const double ji = static_cast<double>(ks[d][7]) - static_cast<double>(kc[d][7]);
              Sv = 0.5 * (1.0 + (1.0 - u) * (1.0 - u)) * I2 + (u * u) / (2.0 * gam * gam) * (jr * jr + ji * ji);
            }
            S_acc[d] = fma(wp, Sv, S_acc[d]);
          }
        }
        s ^= 1;
        if (!nxt.valid) break;
        cur = nxt;
      }
    }
    if (iw < P.n_omega) {
#pragma unroll
      for (int d = 0; d < ND; ++d) {
        if (!dvalid[d]) continue;
        if (!P.amp_mode) {
          P.part[(chunk * P.n_angles + jdir[d]) * P.n_omega + iw] = S_acc[d];
        } else {
#pragma unroll
          for (int c = 0; c < NC; ++c)
            P.part[((chunk * NC + c) * P.n_angles + jdir[d]) * P.n_omega + iw] =
                static_cast<double>(ks[d][c]) - static_cast<double>(kc[d][c]);
        }
      }
    }
  }
}

template <int MODE, int NW, int T>
cudaError_t launch_t(const Params &P, const float *prep, LaunchShape *shape, cudaStream_t st, int *occ) {
  using L = SepLayout<MODE, NW, T>;
  auto kern = k_mixed_sep<MODE, NW, T>;
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
  if (P.grid_nx <= 0 || P.n_angles % P.grid_nx != 0) return cudaErrorInvalidValue;
  kern<<<shape->grid, NW * 32, L::kTotal, st>>>(P, prep);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t dispatch_mode(const Params &P, const float *prep, LaunchShape *sh, cudaStream_t st, int *occ) {
  if (sh->R != 1) return cudaErrorInvalidValue;
  if (sh->NW == 4 && sh->T == 128) return launch_t<MODE, 4, 128>(P, prep, sh, st, occ);
  if (sh->NW == 8 && sh->T == 128) return launch_t<MODE, 8, 128>(P, prep, sh, st, occ);
  if (sh->NW == 4 && sh->T == 256) return launch_t<MODE, 4, 256>(P, prep, sh, st, occ);
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

bool shape_supported_mixed_sep(int R, int NW, int T) {
  return R == 1 && ((NW == 4 && (T == 128 || T == 256)) || (NW == 8 && T == 128));
}

cudaError_t launch_mixed_sep(const Params &P, const float *prep, LaunchShape *shape, cudaStream_t st) {
  return dispatch(P, prep, shape, st, nullptr);
}

int occupancy_mixed_sep(const LaunchShape &s) {
  Params P{};
  P.mode = RAD_SPIN_HALF;
  LaunchShape sh = s;
  int occ = 0;
  if (dispatch(P, nullptr, &sh, nullptr, &occ) != cudaSuccess) return 0;
  return occ;
}

}  // namespace rad
