// Pieces shared by the mixed-precision kernels (rad_mixed.cu, rad_mixed_pp.cu).
#pragma once
#include "rad_internal.cuh"

namespace rad {

constexpr int kPP = 12;                   // floats per pre-pass record (10 used + 2 pad: 48 B)
constexpr float kMagicF = 12582912.0f;    // 1.5 * 2^23: adding it rounds |x| < 2^22 to an integer
constexpr float kTwoPiF = 6.28318530717958647692f;
constexpr double kInvTwoPi = 0.159154943091895335768883763372514362;

// Kahan-compensated FP32 running sum (W. Kahan, "Further remarks on reducing truncation
// errors", CACM 8 (1965)); the value is s - c.
__device__ __forceinline__ void kahan_add(float &s, float &c, float v) {
  const float y = __fsub_rn(v, c);
  const float t = __fadd_rn(s, y);
  c = __fsub_rn(__fsub_rn(t, s), y);
  s = t;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// e^{i 2 pi (wt_hi + wt_lo)(a0h + a0l)} of a tile's base phase, the photon-energy factor
// w*/2pi and the FP64 phase A at the reference sample both as double-float pairs
// (T. J. Dekker, Numer. Math. 18 (1971)): the product in turns is formed as p + e with p the
// rounded product and e its error plus the cross terms, then reduced exactly by magic-number
// rounding. Beyond 2^21 turns the FP64 product (ws_d * A) / 2pi is reduced instead.
__device__ __forceinline__ void tile_base_sincos(float wt_hi, float wt_lo, float a0h, float a0l, double ws_d,
                                                 float &s0, float &c0) {
  const float p = wt_hi * a0h;
  float e = fmaf(wt_hi, a0h, -p);
  e = fmaf(wt_hi, a0l, e);
  e = fmaf(wt_lo, a0h, e);
  float rr;
  if (fabsf(p) < 2097152.0f) {
    const float nr = __fsub_rn(__fadd_rn(p, kMagicF), kMagicF);
    rr = __fadd_rn(__fsub_rn(p, nr), e);
  } else {
    const double ph = ws_d * (static_cast<double>(a0h) + static_cast<double>(a0l)) * kInvTwoPi;
    rr = static_cast<float>(ph - rint(ph));
  }
  __sincosf(rr * kTwoPiF, &s0, &c0);
}

}  // namespace rad
