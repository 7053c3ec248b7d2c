// fixed.cuh -- signed 64-bit fixed-point arithmetic for the FP64 sweep.
//
// B300's binary64 pipe issues about 1.7 operations per clock per SM, against
// about 64 for 32-bit integer operations, so a binary64 sweep is bound by
// arithmetic at a quarter of the HBM roofline.  The fixed-point sweep keeps
// binary64 storage and does its arithmetic on integers instead: a value x is
// represented by round(x * 2^S) with one scale S per call, chosen so that
// every sum of the sweep stays below 2^58 in magnitude.  Sums are then exact,
// the division by 6 is rounded to the nearest unit 2^-S, and the result is
// rounded to binary64 once per pass.
#pragma once

#include <stdint.h>

namespace stencil {

// Biased representation used by the sweep kernels: a value x is held as the
// unsigned integer U = K + round(x * 2^S) with K = 2^59 and |x * 2^S| < 2^58,
// so six neighbours plus the source term sum to a positive number below
// 2^63 and the division by 6 needs no sign handling:
//   (sum of 6 (K + q_i) + G + 3) / 6 = K + round((sum q_i + G) / 6).
constexpr uint64_t kFxBias = 1ull << 59;

// Per-launch constants, computed identically by every thread from max|u|
// and max|f| (see fx_params).
struct FixedParams {
  int S;        // values are q * 2^-S
  int Cu;       // 1085 - S: shift base of the u conversion
  int Cg;       // 1085 - S - eh: shift base of the source conversion
  uint64_t H;   // mh * 2^64 where hh = mh * 2^eh, mh in [0.5, 1)
  int bad;      // 1: input not finite, 2: beyond range -> write NaN
};

// 64-bit logical right shift with PTX semantics: amounts >= 64 give 0.
__device__ __forceinline__ uint64_t shr64(uint64_t v, unsigned n) {
  uint64_t r;
  asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(v), "r"(n));
  return r;
}

// binary64 -> K + round(x * 2^S), ties up.  The 53-bit significand is
// left-aligned at bit 63 and shifted right by (1085 - S - e), keeping one
// extra bit for the rounding; zeros and subnormals (e = 0) shift out to 0.
__device__ __forceinline__ uint64_t fx_in(double x, int Cu) {
  const uint64_t b = static_cast<uint64_t>(__double_as_longlong(x));
  const int e = static_cast<int>((b >> 52) & 0x7ffu);
  const uint64_t m63 = (b << 11) | 0x8000000000000000ull;
  const uint64_t t = shr64(m63, static_cast<unsigned>(Cu - e));  // 2|x| 2^S
  const uint64_t sgn = static_cast<uint64_t>(static_cast<int64_t>(b) >> 63);
  const uint64_t w = ((t ^ sgn) - sgn) + (2 * kFxBias + 1);
  return w >> 1;
}

// Source term G = round(f * hh * 2^S) (signed, unbiased), ties up: the
// significand of f times the significand of hh (high 64 bits of the
// product), then the same aligned shift.
__device__ __forceinline__ int64_t fx_source(double f, int Cg, uint64_t H) {
  const uint64_t b = static_cast<uint64_t>(__double_as_longlong(f));
  const int e = static_cast<int>((b >> 52) & 0x7ffu);
  const uint64_t m63 = (b << 11) | 0x8000000000000000ull;
  const uint64_t t = shr64(__umul64hi(m63, H), static_cast<unsigned>(Cg - e));
  const uint64_t sgn = static_cast<uint64_t>(static_cast<int64_t>(b) >> 63);
  const int64_t w = static_cast<int64_t>((t ^ sgn) - sgn) + 1;
  return w >> 1;
}

// (sum + 3) / 6 for 0 <= sum + 3 < 2^64: multiply by ceil(2^65 / 3), take
// the high word, shift by 2 (exact floor division for every 64-bit input).
__device__ __forceinline__ uint64_t fx_div6(uint64_t sum_plus_3) {
  return __umul64hi(sum_plus_3, 0xAAAAAAAAAAAAAAABull) >> 2;
}

// Biased U -> binary64 (U - K) * 2^-S, rounded to nearest even: hardware
// conversion of the signed integer, then an exact exponent shift (S <= 1022
// keeps every nonzero result normal).
__device__ __forceinline__ double fx_out(uint64_t U, int S) {
  const int64_t q = static_cast<int64_t>(U - kFxBias);
  const double d = __ll2double_rn(q);
  const long long bits = __double_as_longlong(d) - (static_cast<long long>(S) << 52);
  return q == 0 ? 0.0 : __longlong_as_double(bits);
}

// Scale selection.  maxu = max|u| over every cell (halo included), maxf =
// max|f| over the interior, n = sweeps this call does, lmin = (smallest
// extent + 1) * h.  Bound on every iterate (maximum principle of the sweep):
//   |u_n| <= M = min(maxu + n hh maxf / 6,  3 maxu + maxf lmin^2 / 4);
// the largest magnitude before the division by 6 is B = 6 M + hh maxf, and
// S = 58 - ceil(log2 B) keeps it below 2^58 (capped at 1022).
__device__ __forceinline__ FixedParams fx_params(double maxu, double maxf, double hh, double n,
                                                 double lmin) {
  FixedParams p;
  p.bad = 0;
  p.S = 0; p.Cu = 0; p.Cg = 0; p.H = 0;
  if (!(maxu <= 1.0e300) || !(maxf <= 1.0e300)) {  // NaN, Inf or absurdly large
    p.bad = 1;
    return p;
  }
  const double lin = maxu + n * hh * maxf / 6.0;
  const double cmp = 3.0 * maxu + maxf * lmin * lmin / 4.0;
  const double M = lin < cmp ? lin : cmp;
  const double B = 6.0 * M + hh * maxf;
  int e = 0;
  if (B > 0.0) frexp(B, &e);  // B = m 2^e, m in [0.5, 1), so B <= 2^e
  int S = 58 - e;
  if (S > 1022) S = 1022;
  if (S < -900) p.bad = 2;
  int eh = 0;
  const double mh = frexp(hh, &eh);
  p.S = S;
  p.Cu = 1085 - S;
  p.Cg = 1085 - S - eh;
  p.H = (static_cast<uint64_t>(__double_as_longlong(mh)) << 11) | 0x8000000000000000ull;
  return p;
}

}  // namespace stencil
