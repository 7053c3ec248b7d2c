// fixed.cuh -- signed 64-bit fixed-point arithmetic for the FP64 sweep.
//
// B300's binary64 pipe issues about 1.7 operations per clock per SM, against
// about 64 for 32-bit integer operations, so a binary64 sweep is bound by
// arithmetic at a quarter of the HBM roofline.  The fixed-point sweep keeps
// binary64 storage and does its arithmetic on integers instead: a value x is
// represented by round(x * 2^S).  The scale S is chosen afresh for every pass
// from a bound on the magnitudes that pass can produce (the largest value the
// previous pass wrote, the Dirichlet values and the source's contribution),
// so the resolution 2^-S follows the iterate rather than an a-priori bound
// for the whole call.  Sums of six neighbours and the source then stay below
// 2^58 and are exact, the division by 6 is rounded to the nearest unit
// 2^-S, and the result is rounded to binary64 once per call (or per pass).
#pragma once

#include <stdint.h>

namespace stencil {

// Biased representation used by the sweep kernels: a value x is held as the
// unsigned integer U = K + round(x * 2^S) with K = 2^59 and |x * 2^S| < 2^58,
// so six neighbours plus the source term sum to a positive number below
// 2^63 and the division by 6 needs no sign handling:
//   (sum of 6 (K + q_i) + G + 3) / 6 = K + round((sum q_i + G) / 6).
constexpr uint64_t kFxBias = 1ull << 59;
// Scale marking a failed call: set once a pass sees a non-finite input or a
// bound beyond the representable range; every later pass keeps it.
constexpr int kFxBadScale = 4000;

// Per-pass constants, computed identically by every thread (policies.cuh).
struct FixedParams {
  int S;          // values of this pass are q * 2^-S (resident: its output's scale)
  int Cu;         // 1085 - S: shift base of the u conversion (resident: of the
                  // computing scale, that of the stored input)
  int Cg;         // 1085 - S - eh: shift base of the per-pass source conversion
  uint64_t H;     // mh * 2^64 where hh = mh * 2^eh, mh in [0.5, 1)
  int bad;        // 1: input not finite, 2: beyond range -> write NaN
  int dshift;     // resident: S - (scale of the stored input); 0 almost always
  int fpath;      // resident: the stored source is not at the computing scale;
                  // this pass reads f itself and stores the source afresh
};

// 64-bit logical right shift with PTX semantics: amounts >= 64 give 0.
__device__ __forceinline__ uint64_t shr64(uint64_t v, unsigned n) {
  uint64_t r;
  asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(v), "r"(n));
  return r;
}

// Rounding of y = |x| 2^S to nearest, halves away from zero, with the sign
// of x, from t = floor(2y) and the sign mask s (all ones if x < 0):
//   x >= 0:  floor((t + 1) / 2) = (t + 1) >> 1
//   x <  0: -floor((t + 1) / 2) = floor(-t / 2) = (~t + 1) >> 1 (arithmetic)
// i.e. ((t ^ s) + 1) >> 1 in both cases; with the bias K folded in,
// ((t ^ s) + 2K + 1) >> 1 (logical: the sum is positive).
__device__ __forceinline__ uint64_t fx_sign_mask(uint64_t b) {
  return static_cast<uint64_t>(static_cast<int64_t>(b) >> 63);
}

// binary64 -> K + round(x * 2^S), halves away from zero.  The 53-bit
// significand is left-aligned at bit 63 and shifted right by (1085 - S - e),
// which leaves t = floor(2 |x| 2^S).  Zeros and subnormals (e = 0) shift out
// to 0.
__device__ __forceinline__ uint64_t fx_in(double x, int Cu) {
  const uint64_t b = static_cast<uint64_t>(__double_as_longlong(x));
  const int e = static_cast<int>((b >> 52) & 0x7ffu);
  const uint64_t m63 = (b << 11) | 0x8000000000000000ull;
  const uint64_t t = shr64(m63, static_cast<unsigned>(Cu - e));  // floor(2|x| 2^S)
  return ((t ^ fx_sign_mask(b)) + (2 * kFxBias + 1)) >> 1;
}

// Source term G = round(f * hh * 2^S) (signed, unbiased), halves away from
// zero: the significand of f times the significand of hh (high 64 bits of
// the product), then the same aligned shift.
__device__ __forceinline__ int64_t fx_source(double f, int Cg, uint64_t H) {
  const uint64_t b = static_cast<uint64_t>(__double_as_longlong(f));
  const int e = static_cast<int>((b >> 52) & 0x7ffu);
  const uint64_t m63 = (b << 11) | 0x8000000000000000ull;
  const uint64_t t = shr64(__umul64hi(m63, H), static_cast<unsigned>(Cg - e));
  return static_cast<int64_t>((t ^ fx_sign_mask(b)) + 1) >> 1;
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

// A stored iterate U at scale S_old, brought to scale S_old + d: an exact
// left shift (d > 0) or a right shift rounded to nearest, halves up (d < 0).
__device__ __forceinline__ uint64_t fx_rescale(uint64_t U, int d) {
  const int64_t q = static_cast<int64_t>(U - kFxBias);
  int64_t r;
  if (d > 0) {
    r = static_cast<int64_t>(static_cast<uint64_t>(q) << d);
  } else {
    const int n = -d;
    r = (q + (1ll << (n - 1))) >> n;
  }
  return static_cast<uint64_t>(r) + kFxBias;
}

// Scale for a pass whose values (and six-neighbour sums plus the source) are
// bounded by B: S = 58 - ceil(log2 B), capped at 1022; bad = 2 if B is out
// of range, 1 if it is not a number.
__device__ __forceinline__ int fx_scale_for(double B, int* bad) {
  if (!(B <= 1.0e300)) {
    *bad = (B != B) ? 1 : 2;
    return 0;
  }
  int e = 0;
  if (B > 0.0) frexp(B, &e);  // B = m 2^e, m in [0.5, 1), so B <= 2^e
  int S = 58 - e;
  if (S > 1022) S = 1022;
  if (S < -900) *bad = 2;
  return S;
}

// Conversion constants for scale S and source factor hh.
__device__ __forceinline__ void fx_conv(FixedParams& p, int S, double hh) {
  int eh = 0;
  const double mh = frexp(hh, &eh);
  p.S = S;
  p.Cu = 1085 - S;
  p.Cg = 1085 - S - eh;
  p.H = (static_cast<uint64_t>(__double_as_longlong(mh)) << 11) | 0x8000000000000000ull;
}

}  // namespace stencil
