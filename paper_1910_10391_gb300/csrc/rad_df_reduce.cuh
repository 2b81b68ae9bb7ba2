// Exact reduction of an FP64 phase to a 2048-entry table index and a float-pair remainder, used by
// the FP64-accurate double-float kernel (rad_df.cu): phi = j 2 pi/2048 + r, |r| <= pi/2048, with an
// absolute error of r below 3e-16 rad (Payne-Hanek with integer multiplies for 2^-10 <= |phi| <
// 2^22, FP64 Cody-Waite above, r = phi below). Device functions only; internal to the library.
#pragma once

#include <cstdint>

namespace rad {
namespace dfr {

constexpr double kPiHi = 3.141592653589793116;
constexpr double kPiLo = 1.2246467991473531772e-16;
constexpr double kC1 = kPiHi / 1024.0;
constexpr double kC2 = kPiLo / 1024.0;
constexpr double kInvStep = 1024.0 / 3.141592653589793238462643383279502884;  // 2048/(2 pi)
constexpr double kMagic = 6755399441055744.0;  // 1.5 * 2^52

// hi = r rounded to FP32, lo = (r - hi) rounded to FP32, from r's bits with integer operations.
// Valid for |r| < 2^100; |r| < 2^-126 gives (0, 0), an error below 1.2e-38.
__device__ __forceinline__ void split_df(double r, float &hi, float &lo) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(r));
  const unsigned sign = static_cast<unsigned>(u >> 32) & 0x80000000u;
  const int e = static_cast<int>((u >> 52) & 0x7ffull);
  if (e < 1023 - 126) {
    hi = 0.f;
    lo = 0.f;
    return;
  }
  const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);  // 53-bit significand
  unsigned long long mh = (m + (1ull << 28)) >> 29;                      // rounded to 24 bits
  const long long d = static_cast<long long>(m) - static_cast<long long>(mh << 29);  // |d| <= 2^28
  int eh = e;
  if (mh >> 24) {  // rounding carried into a 25th bit
    mh >>= 1;
    ++eh;
  }
  hi = __int_as_float(static_cast<int>(sign | (static_cast<unsigned>(eh - 1023 + 127) << 23) |
                                       (static_cast<unsigned>(mh) & 0x7FFFFFu)));
  // r - hi = sign * d * 2^(e - 1075) exactly; its FP32 rounding (0 when below 2^-98)
  if (e >= 949) {
    const float scale = __int_as_float((e - 948) << 23);  // 2^(e - 1075)
    const float l = __int2float_rn(static_cast<int>(d)) * scale;
    lo = sign ? -l : l;
  } else {
    lo = 0.f;
  }
}

// 1024/pi = kKH + kKL 2^-64 (fixed point, truncation below 2^-64) and pi/1024 = kChf + kClf
// (float pair, residual 3e-18 relative)
constexpr unsigned long long kKH = 325ull;
constexpr unsigned long long kKL = 17511926765934236664ull;
constexpr float kChf = 0.003067961661145091f;
constexpr float kClf = -8.537380524753502e-11f;

// 1024/pi 2^64 = kK2 2^64 + kK1 2^32 + kK0 as 32-bit words, and the float-pair constants of pi/1024
// times 2^-24 and 2^-48 (exact power-of-two scalings, all normal), which take the fraction's two
// 24-bit parts as plain integers
constexpr unsigned kK2 = static_cast<unsigned>(kKH);
constexpr unsigned kK1 = static_cast<unsigned>(kKL >> 32);
constexpr unsigned kK0 = static_cast<unsigned>(kKL & 0xFFFFFFFFull);
constexpr float kChf24 = kChf * 5.9604644775390625e-8f;
constexpr float kClf24 = kClf * 5.9604644775390625e-8f;
constexpr float kChf48 = kChf * 3.552713678800501e-15f;

// phi = j pi/1024 + r with |r| <= pi/2048; returns j mod 2^16 (the table takes it mod 2048) and r
// as the float pair (xh, xl).
// For 2^-10 <= |phi| < 2^22 by a fixed-point (Payne-Hanek) reduction of phi's bits with integer
// multiplies: |phi| = m 2^(e-1075) with the 53-bit significand m = m1 2^32 + m0 (m1 of 21 bits), and
// phi 1024/pi = m K 2^(e-1139) with K = 1024/pi 2^64 as a 73-bit integer. m K is formed from 32-bit
// products without its lowest word (nothing else lands below bit 32, so every bit from 32 up is
// exact); X = m K >> (a + 16), a = 1075 - e in [31, 62], taken by funnel shifts, holds the low bits
// of the integer part from bit 48 (rounded to nearest by the fraction's top bit) and the fraction's
// top 48 bits F below, so r = F pi/1024 with absolute error below 3e-16 rad. Below 2^-10, r = phi;
// from 2^22 on, the FP64 Cody-Waite reduction.
__device__ __forceinline__ int reduce_phase(double phi, float &xh, float &xl) {
  const unsigned hi = static_cast<unsigned>(__double2hiint(phi));
  const unsigned m0 = static_cast<unsigned>(__double2loint(phi));
  const int e = static_cast<int>((hi >> 20) & 0x7ffu);
  if (static_cast<unsigned>(e - 1013) > 31u) {
    if (e < 1013) {  // |phi| < 2^-10 < pi/2048
      split_df(phi, xh, xl);
      return 0;
    }
    // |phi| >= 2^22
    const double y = fma(phi, kInvStep, kMagic);
    const double jd = y - kMagic;
    split_df(fma(-jd, kC2, fma(-jd, kC1, phi)), xh, xl);
    return __double2loint(y);
  }
  const unsigned m1 = (hi & 0xFFFFFu) | 0x100000u;
  const unsigned long long a01 = static_cast<unsigned long long>(m0) * kK1;
  const unsigned long long a10 = static_cast<unsigned long long>(m1) * kK0;
  const unsigned long long s1 = static_cast<unsigned long long>(__umulhi(m0, kK0)) + static_cast<unsigned>(a01) +
                                static_cast<unsigned>(a10);  // bits 32.. of m K
  const unsigned long long h = static_cast<unsigned long long>(m0) * kK2 + static_cast<unsigned long long>(m1) * kK1 +
                               (a01 >> 32) + (a10 >> 32) + (s1 >> 32) +
                               (static_cast<unsigned long long>(m1 * kK2) << 32);  // bits 64.. of m K
  const unsigned w0 = static_cast<unsigned>(s1), w1 = static_cast<unsigned>(h), w2 = static_cast<unsigned>(h >> 32);
  const int sh = 1059 - e;  // a - 16 in [15, 46]: X = (w2 w1 w0) >> sh
  const bool big = sh >= 32;
  const unsigned v0 = big ? w1 : w0, v1 = big ? w2 : w1, v2 = big ? 0u : w2;
  const unsigned x0 = __funnelshift_r(v0, v1, sh);  // shift taken mod 32
  const unsigned x1 = __funnelshift_r(v1, v2, sh);
  const int t24 = static_cast<int>(__funnelshift_r(x0, x1, 24) << 8) >> 8;  // F's signed top 24 bits
  const int low24 = static_cast<int>(x0 & 0xFFFFFFu);                       // F's next 24 bits
  int j = static_cast<int>((x1 + 0x8000u) >> 16);
  const float fa = __int2float_rn(t24), fb = __int2float_rn(low24);
  float p = __fmul_rn(fa, kChf24);
  float lo = __fadd_rn(__fmaf_rn(fa, kChf24, -p), __fmaf_rn(fa, kClf24, __fmul_rn(fb, kChf48)));
  if (hi >> 31) {
    p = -p;
    lo = -lo;
    j = -j;
  }
  xh = p;
  xl = lo;
  return j;
}

}  // namespace dfr
}  // namespace rad
