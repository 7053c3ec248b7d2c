// advect.cu -- Piacsek-Williams flux-form momentum advection (Section 4.1:
// the three stencils over u, v, w fused into one region, 63 operations per
// cell).
//
// B300 issues binary64 arithmetic at about 1/64 of its binary32 rate, so a
// binary64 evaluation of the 63 operations is bound by the FP64 pipe at a
// few percent of the HBM roofline.  The kernel therefore evaluates the
// tendencies in 64-bit integer fixed point:
//   * one scale S per call from max |u|, |v|, |w| (halos included):
//     X = trunc(x 2^S) with |X| <= 2^61, so every sum of two or three is
//     exact;
//   * each product a (b + c) is a s / 2^64 from three 32 x 32-bit products
//     (mh: within [-1/4, 9/4) of the exact value, 2^-57 of the largest
//     product), a function of (a, s) alone, so equal fluxes cancel exactly;
//     the self terms um (u + um) - up (u + up) are taken as the one product
//     (um - up)(u + um + up), the same value in exact arithmetic;
//   * the factors tcx, tcy, tzc1[k], tzc2[k] use one scale T from their
//     maximum (|C| <= 2^62; exact for the binary64 inputs in use); the
//     factor products are mh again (power-of-two tcx, tcy: exact shifts),
//     the three terms are summed in 64 bits and the sum is rounded to
//     binary64 once.
// The error is a few units of 2^-57 of the largest product per output, the
// order of the rounding error of a binary64 evaluation of the same formula.
// When the fields' magnitudes differ by more than 2^8, or the factors' do,
// or a value is not finite, a single scale would cost the smaller field its
// precision, so the launch evaluates the formula in binary64 instead (the
// decision is taken on the device from the magnitudes the pass read: the
// call stays asynchronous).
//
// Each CTA owns a 32 x (RPT BY) column of cells and marches up a chunk of
// z planes (48 by default): every plane of u, v, w is loaded once
// (coalesced, one plane ahead in registers), quantised once into a ring of
// four shared-memory plane slots, and each thread computes su, sv, sw of
// its RPT cells from the three slots around them -- one CTA barrier per
// plane.  48 algorithmic bytes per cell (three fields in, three out).  The quantisation and the final
// rounding run as 64-bit conversions on B300's FP64 pipe (about two per
// clock per SM), so the integer pipes keep the products.
// (Computing sw in binary64 on the FP64 pipe while su and sv use the
// integer pipes was measured slower: 21 binary64 operations per cell keep
// that pipe busy on their own.)
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace stencil {

namespace {

constexpr unsigned long long kAbsMask = 0x7fffffffffffffffull;
constexpr unsigned long long kInfBits = 0x7ff0000000000000ull;

// Bits of max |u|, |v|, |w| over every cell (halos included) into
// r[0..2] (zeroed first).  Non-negative doubles order as their bit patterns.
__global__ void advect_range_kernel(const double* __restrict__ u, const double* __restrict__ v,
                                    const double* __restrict__ w, int64_t nx, int64_t ny, int64_t nz, int64_t sy,
                                    int64_t sz, unsigned long long* r) {
  const int64_t rows = (ny + 2) * (nz + 2);
  unsigned long long m[3] = {0, 0, 0};
  for (int64_t row = blockIdx.x * int64_t(blockDim.y) + threadIdx.y; row < rows;
       row += int64_t(gridDim.x) * blockDim.y) {
    const int64_t k = row / (ny + 2), j = row - k * (ny + 2);
    for (int64_t i = threadIdx.x; i < nx + 2; i += blockDim.x) {
      const int64_t c = i + j * sy + k * sz;
      const unsigned long long b[3] = {static_cast<unsigned long long>(__double_as_longlong(u[c])) & kAbsMask,
                                       static_cast<unsigned long long>(__double_as_longlong(v[c])) & kAbsMask,
                                       static_cast<unsigned long long>(__double_as_longlong(w[c])) & kAbsMask};
#pragma unroll
      for (int f = 0; f < 3; ++f) m[f] = b[f] > m[f] ? b[f] : m[f];
    }
  }
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long a = __shfl_xor_sync(0xffffffffu, m[f], o);
      m[f] = a > m[f] ? a : m[f];
    }
    if ((threadIdx.x & 31) == 0) atomicMax(&r[f], m[f]);
  }
}

// A magnitude record (5 x uint64, zeroed = nothing recorded, every entry
// raised with atomicMax): the bits of max |u|, |v|, |w| (high words, see
// adv_scales), the bits of the largest |factor| (tcx, tcy, tzc1[], tzc2[])
// and the complement of the bits of the smallest nonzero |factor|.
//
// The factors' entries of a context's first record (one warp; the fields'
// entries come from advect_range_kernel).
__global__ void advect_factor_kernel(const double* __restrict__ tzc1, const double* __restrict__ tzc2, int64_t nz,
                                     double tcx, double tcy, unsigned long long* rec) {
  unsigned long long cmax = 0, cmin = ~0ull;
  auto take = [&](double x) {
    const unsigned long long v = static_cast<unsigned long long>(__double_as_longlong(x)) & kAbsMask;
    cmax = v > cmax ? v : cmax;
    if (v != 0) cmin = v < cmin ? v : cmin;
  };
  if (threadIdx.x == 0) {
    take(tcx);
    take(tcy);
  }
  for (int64_t k = threadIdx.x; k < nz; k += 32) {
    take(tzc1[k]);
    take(tzc2[k]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long x = __shfl_xor_sync(0xffffffffu, cmax, o);
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, cmin, o);
    cmax = x > cmax ? x : cmax;
    cmin = y < cmin ? y : cmin;
  }
  if (threadIdx.x == 0) {
    rec[3] = cmax;
    rec[4] = ~cmin;
  }
}

// ceil(log2 x) for the positive normal double with these bits.
__device__ __forceinline__ int ceil_log2_bits(unsigned long long b) {
  const int e = static_cast<int>(b >> 52) - 1023;
  return (b & 0xfffffffffffffull) ? e + 1 : e;
}

struct AdvScales {
  int S, T, Q;
  bool fixed;
};

// The scales of this launch (the same in every thread) and whether the
// fixed-point evaluation applies.
// The fields' magnitudes count by their high words only (rounded up to the
// largest double with that high word; a zero high word counts as zero), so
// the maxima a pass records from high words give the same decision as the
// exact maxima of a range pass.
__device__ __forceinline__ AdvScales adv_scales(const unsigned long long* rb) {
  AdvScales sc{0, 0, 0, false};
  unsigned long long r[5];
  for (int f = 0; f < 3; ++f) r[f] = (rb[f] >> 32) ? (rb[f] | 0xffffffffull) : 0ull;
  r[3] = rb[3];
  r[4] = rb[4];
  unsigned long long M = 0;
  for (int f = 0; f < 3; ++f) {
    if (r[f] >= kInfBits) return sc;
    M = r[f] > M ? r[f] : M;
  }
  if (r[3] >= kInfBits || M < (1ull << 52) || r[3] < (1ull << 52)) return sc;  // zero / subnormal extremes
  const int eM = static_cast<int>(M >> 52);
  for (int f = 0; f < 3; ++f)
    if (r[f] != 0 && eM - static_cast<int>(r[f] >> 52) > 8) return sc;
  if (static_cast<int>(r[3] >> 52) - static_cast<int>(r[4] >> 52) > 8) return sc;
  sc.S = 61 - ceil_log2_bits(M);
  sc.T = 62 - ceil_log2_bits(r[3]);
  if (sc.S > 1000 || sc.T > 1000) return sc;  // magnitudes below 2^-939: binary64
  sc.Q = 2 * sc.S + sc.T - 128;
  sc.fixed = true;
  return sc;
}

// The scales a magnitude record gives.
__device__ __forceinline__ AdvScales adv_scales_rec(const unsigned long long* rec) {
  const unsigned long long r[5] = {rec[0], rec[1], rec[2], rec[3], ~rec[4]};
  return adv_scales(r);
}

// round(x 2^S) for |x| 2^S <= 2^62 (half away from zero; zero and subnormal
// inputs give 0).
__device__ __forceinline__ long long fx_quant(double x, int S) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const int e = static_cast<int>((b >> 52) & 0x7ff);
  if (e == 0) return 0;
  const unsigned long long m = (b & 0xfffffffffffffull) | (1ull << 52);
  const int sh = e - 1075 + S;  // x 2^S = m 2^sh
  unsigned long long q;
  if (sh >= 0) {
    q = m << sh;
  } else if (sh > -64) {
    const int k = -sh;
    q = (m + (1ull << (k - 1))) >> k;
  } else {
    q = 0;
  }
  return (b >> 63) ? -static_cast<long long>(q) : static_cast<long long>(q);
}

// x 2^-Q rounded to binary64 (nearest, ties up; results below the normal
// range flush to zero).
__device__ __forceinline__ double fx64_to_double(long long x, int Q) {
  if (x == 0) return 0.0;
  const bool neg = x < 0;
  const unsigned long long m = neg ? 0ull - static_cast<unsigned long long>(x) : static_cast<unsigned long long>(x);
  const int lz = __clzll(static_cast<long long>(m));
  const unsigned long long top = m << lz;   // leading bit at 63
  const long long E = 63 - lz - Q + 1023;   // biased exponent of the leading bit
  if (E <= 0) return neg ? -0.0 : 0.0;
  if (E >= 2047) return neg ? -__longlong_as_double(kInfBits) : __longlong_as_double(kInfBits);
  const unsigned long long bits =
      (static_cast<unsigned long long>(E) << 52) + ((top >> 11) & 0xfffffffffffffull) + ((top >> 10) & 1ull);
  return __longlong_as_double(static_cast<long long>(bits | (neg ? (1ull << 63) : 0ull)));
}

// The binary64 evaluation (the fallback): every operation rounded on its
// own, in the order of the definition (no fused multiply-add), so equal
// fluxes cancel exactly and the result is the plain evaluation's, bit for
// bit.
__device__ __forceinline__ double flux64(double a, double b, double c, double d, double e, double f) {
  return __dsub_rn(__dmul_rn(a, __dadd_rn(b, c)), __dmul_rn(d, __dadd_rn(e, f)));
}

// c1 a (b + c) - c2 d (e + f), the products taken left to right.
__device__ __forceinline__ double zflux64(double c1, double a, double b, double c, double c2, double d, double e,
                                          double f) {
  return __dsub_rn(__dmul_rn(__dmul_rn(c1, a), __dadd_rn(b, c)), __dmul_rn(__dmul_rn(c2, d), __dadd_rn(e, f)));
}

__device__ __forceinline__ double advect_sw_f64(const double* __restrict__ u, const double* __restrict__ v,
                                                const double* __restrict__ w, int64_t c, int64_t sy, int64_t sz,
                                                double tcx, double tcy, double c1, double c2) {
  const double u0 = u[c], v0 = v[c], w0 = w[c];
  const double wm = w[c - sz], wp = w[c + sz];
  const double tx = __dmul_rn(tcx, flux64(w[c - 1], u[c - 1], u[c - 1 + sz], w[c + 1], u0, u[c + sz]));
  const double ty = __dmul_rn(tcy, flux64(w[c - sy], v[c - sy], v[c - sy + sz], w[c + sy], v0, v[c + sz]));
  const double tz = zflux64(c1, wm, w0, wm, c2, wp, w0, wp);
  return __dadd_rn(__dadd_rn(tx, ty), tz);
}

__device__ __forceinline__ void advect_cell_f64(const double* __restrict__ u, const double* __restrict__ v,
                                                const double* __restrict__ w, int64_t c, int64_t sy, int64_t sz,
                                                double tcx, double tcy, double c1, double c2, double& osu,
                                                double& osv, double& osw) {
  const double u0 = u[c], v0 = v[c], w0 = w[c];
  const double um = u[c - 1], up = u[c + 1];
  double tx = __dmul_rn(tcx, flux64(um, u0, um, up, u0, up));
  double ty = __dmul_rn(tcy, flux64(u[c - sy], v[c - sy], v[c - sy + 1], u[c + sy], v0, v[c + 1]));
  double tz = zflux64(c1, u[c - sz], w[c - sz], w[c - sz + 1], c2, u[c + sz], w0, w[c + 1]);
  osu = __dadd_rn(__dadd_rn(tx, ty), tz);
  const double vm = v[c - sy], vp = v[c + sy];
  tx = __dmul_rn(tcx, flux64(v[c - 1], u[c - 1], u[c - 1 + sy], v[c + 1], u0, u[c + sy]));
  ty = __dmul_rn(tcy, flux64(vm, v0, vm, vp, v0, vp));
  tz = zflux64(c1, v[c - sz], w[c - sz], w[c - sz + sy], c2, v[c + sz], w0, w[c + sy]);
  osv = __dadd_rn(__dadd_rn(tx, ty), tz);
  osw = advect_sw_f64(u, v, w, c, sy, sz, tcx, tcy, c1, c2);
}

// a s / 2^64 for |a| <= 2^62 and |s| < 2^63 - 2^32, from three 32 x 32-bit
// products: with a = ah 2^32 + al and s = sh 2^32 + sl, the low words taken
// as SIGNED 32-bit values (so every limb product is a plain signed multiply),
//   a s = ah sh 2^64 + (ah sl + al sh) 2^32 + al sl,
// and the result is ah sh + floor(ah sl / 2^32) + floor(al sh / 2^32).  It
// lies within [-1/4, 9/4) of the exact a s / 2^64 (the dropped al sl / 2^64
// is below 1/4 in magnitude, the two floors drop less than 2): the same
// order as keeping the exact product's high half, at a third of the integer
// instructions.  It is a function of (a, s) alone, so equal fluxes still
// cancel exactly.
__device__ __forceinline__ long long mh(long long a, long long s) {
  const int al = static_cast<int>(a);
  const int ah = static_cast<int>(a >> 32) + static_cast<int>(static_cast<unsigned>(al) >> 31);
  const int sl = static_cast<int>(s);
  const int sh = static_cast<int>(s >> 32) + static_cast<int>(static_cast<unsigned>(sl) >> 31);
  const int t = __mulhi(ah, sl) + __mulhi(al, sh);  // |t| < 2^31 for the stated ranges
  return static_cast<long long>(ah) * sh + t;
}

// The factor product of a horizontal factor c with a flux difference d.
// POW2: c = 2^m exactly (tcx, tcy positive powers of two, as 1/4 is), so
// c d / 2^64 is d shifted right by sh = 64 - m (floor).
// On the fixed-point path sh lies in 2..11 (the factors' magnitudes are
// within 2^8 of each other), so the shift is one 32-bit funnel shift of the
// low word and one arithmetic shift of the high word.
template <bool POW2>
__device__ __forceinline__ long long hfactor(long long c, int sh, long long d) {
  if constexpr (POW2) {
    const unsigned lo = static_cast<unsigned>(d);
    const int hi = static_cast<int>(d >> 32);
    return static_cast<long long>((static_cast<unsigned long long>(static_cast<unsigned>(hi >> sh)) << 32) |
                                  __funnelshift_r(lo, static_cast<unsigned>(hi), sh));
  } else {
    return mh(c, d);
  }
}

// 64 - log2(c) for c a positive power of two (the shift of hfactor), else -1.
__device__ __forceinline__ int pow2_shift(long long c) {
  return (c > 0 && (c & (c - 1)) == 0) ? 64 - (63 - __clzll(c)) : -1;
}

// trunc(x 2^S) (toward zero) for |x| 2^S <= 2^61 and S <= 1000: zero and
// subnormal inputs give 0, and quant(-x) = -quant(x).  The significand with
// its leading bit at 62 is shifted right by 1085 - e - S >= 1 (clamped at
// 63, which gives 0), then the sign is applied.
__device__ __forceinline__ long long fx_trunc(double x, int S) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const int e = static_cast<int>((b >> 52) & 0x7ff);
  const unsigned long long m = ((b & 0xfffffffffffffull) | (1ull << 52)) << 10;
  const int r = min(1085 - e - S, 63);
  const long long q = static_cast<long long>(m >> r);
  const long long s = static_cast<long long>(b) >> 63;
  return (q ^ s) - s;
}

// Tile geometry of the z-marching kernel: a CTA of 32 x BY threads owns a
// 32 x BY column of cells and marches up a chunk of z planes.  Each plane of
// u, v, w is quantised once, with its one-cell x/y margin (34 x (BY + 2)
// values per field), into a ring of four plane slots in shared memory: the
// cell at plane k reads slots k - 1, k, k + 1 while plane k + 2 is written
// into the fourth and plane k + 3 is loaded into registers.
template <int BY, int RPT = 1>
struct AdvGeom {
  static constexpr int BX = 32;
  // RPT rows per thread: thread row ty computes rows ty, ty + BY, ...
  static constexpr int PX = BX + 2, PY = RPT * BY + 2, PL = PX * PY;  // one quantised field plane
  static constexpr int NT = BX * BY;
  static constexpr int NE = (PL + NT - 1) / NT;  // plane values a thread loads per field
  static constexpr int kSlot = 3 * PL;            // u, v, w of one plane
  static constexpr int kSmem = 4 * kSlot * 8;
};
constexpr int kAdvZcMax = 128;  // z planes per CTA at most (factor table size)

// The fixed-point z march of one CTA.  FAST: the conversions leave the
// integer pipes -- a value is quantised as trunc(x 2^S) by adding S to its
// exponent field and converting to a 64-bit integer toward zero (the same
// integer fx_trunc gives; valid for 0 <= S <= 1000), and a sum is converted
// to binary64 (nearest) and scaled by 2^-Q through its exponent field (valid
// for -960 <= Q <= 1022, where every nonzero result is normal).  B300 runs
// these conversions on its FP64 pipe, about two per clock per SM.
template <bool POW2, int BY, bool FAST, int QF = 3, int RPT = 1>
__device__ __forceinline__ void advect_march(const double* __restrict__ u, const double* __restrict__ v,
                                             const double* __restrict__ w, double* __restrict__ su,
                                             double* __restrict__ sv, double* __restrict__ sw,
                                             const double* __restrict__ tzc1, const double* __restrict__ tzc2,
                                             double tcx, double tcy, int64_t nx, int64_t ny, int64_t sy, int64_t sz,
                                             int64_t osy, int64_t osz, int64_t i0, int64_t j0, int64_t k0, int kn,
                                             const AdvScales& sc, long long* zfac, uint32_t (&mx)[3]) {
  using G = AdvGeom<BY, RPT>;
  extern __shared__ long long adv_ring[];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * G::BX + tx;
  const int64_t i = i0 + 1 + tx, j = j0 + 1 + ty;
  const int sadd = sc.S << 20;  // FAST: x 2^S through the high word's exponent field
  const int qsub = sc.Q << 20;  // FAST: s 2^-Q likewise (s != 0: the exponent stays in range)
  auto quant = [&](double x) -> long long {
    if constexpr (FAST) return __double2ll_rz(__hiloint2double(__double2hiint(x) + sadd, __double2loint(x)));
    else return fx_trunc(x, sc.S);
  };
  auto quant_i = [&](double x) -> long long { return fx_trunc(x, sc.S); };
  auto outv = [&](long long s) -> double {
    if constexpr (FAST) {
      const double d = __ll2double_rn(s);
      const int hi = __double2hiint(d);  // 0 only for s = 0
      return __hiloint2double(hi == 0 ? 0 : hi - qsub, __double2loint(d));
    } else {
      return fx64_to_double(s, sc.Q);
    }
  };
  // the plane values this thread loads: offsets within a plane, validity
  int64_t goff[G::NE];
  int soff[G::NE];
  bool ok[G::NE];
#pragma unroll
  for (int n = 0; n < G::NE; ++n) {
    const int e = tid + n * G::NT;
    const int xx = e % G::PX, yy = e / G::PX;
    soff[n] = e < G::PL ? e : -1;
    ok[n] = e < G::PL && i0 + xx <= nx + 1 && j0 + yy <= ny + 1;
    goff[n] = (i0 + xx) + (j0 + yy) * sy;
  }
  double raw[3][G::NE];
  auto load = [&](int p) {  // plane k0 + p of u, v, w into registers
    const int64_t base = (k0 + p) * sz;
#pragma unroll
    for (int n = 0; n < G::NE; ++n) {
      raw[0][n] = ok[n] ? __ldg(u + base + goff[n]) : 0.0;
      raw[1][n] = ok[n] ? __ldg(v + base + goff[n]) : 0.0;
      raw[2][n] = ok[n] ? __ldg(w + base + goff[n]) : 0.0;
    }
  };
  auto store = [&](int p) {  // the registers, quantised, into plane p's slot
    long long* d = adv_ring + (p & 3) * G::kSlot;
#pragma unroll
    for (int n = 0; n < G::NE; ++n) {
      if (soff[n] >= 0) {
#pragma unroll
        for (int f = 0; f < 3; ++f)
          mx[f] = max(mx[f], static_cast<uint32_t>(__double2hiint(raw[f][n])) & 0x7fffffffu);
        // the first QF fields on the FP64 pipe's conversion, the rest in
        // integer instructions (the same integers either way)
        d[soff[n]] = QF >= 1 ? quant(raw[0][n]) : quant_i(raw[0][n]);
        d[G::PL + soff[n]] = QF >= 2 ? quant(raw[1][n]) : quant_i(raw[1][n]);
        d[2 * G::PL + soff[n]] = QF >= 3 ? quant(raw[2][n]) : quant_i(raw[2][n]);
      }
    }
  };
  // planes k0 .. k0 + kn + 1 are read; the first three fill slots 0..2
#pragma unroll 1
  for (int p = 0; p < 3 && p <= kn + 1; ++p) {
    load(p);
    store(p);
  }
  if (3 <= kn + 1) load(3);
  if (tid < 2 * kn) {
    const int64_t k = k0 + 1 + (tid >> 1);
    zfac[tid] = fx_quant((tid & 1) ? tzc2[k - 1] : tzc1[k - 1], sc.T);
  }
  const long long cx = fx_quant(tcx, sc.T), cy = fx_quant(tcy, sc.T);
  const int shx = pow2_shift(cx), shy = pow2_shift(cy);
  __syncthreads();
  constexpr int DX = 1, DY = G::PX;
#pragma unroll 1
  for (int kk = 0; kk < kn; ++kk) {
    // plane kk + 3 (in registers) into the slot that plane kk - 1 freed;
    // plane kk + 4 starts loading
    if (kk + 3 <= kn + 1) store(kk + 3);
    if (kk + 4 <= kn + 1) load(kk + 4);
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) {
    const int t = (ty + rr * BY + 1) * DY + tx + 1;
    if (i <= nx && j + rr * BY <= ny) {
      const long long* Um = adv_ring + (kk & 3) * G::kSlot;  // plane k - 1
      const long long* U0 = adv_ring + ((kk + 1) & 3) * G::kSlot;
      const long long* Up = adv_ring + ((kk + 2) & 3) * G::kSlot;
      const long long *Vm = Um + G::PL, *Wm = Um + 2 * G::PL;
      const long long *V0 = U0 + G::PL, *W0 = U0 + 2 * G::PL;
      const long long *Vp = Up + G::PL, *Wp = Up + 2 * G::PL;
      const long long c1 = zfac[2 * kk], c2 = zfac[2 * kk + 1];
      const long long u0 = U0[t], v0 = V0[t], w0 = W0[t];
      const int64_t k = k0 + 1 + kk;
      const int64_t o = i + (j + rr * BY) * osy + k * osz;
      // su at (i+1/2, j, k); its x term um (u0 + um) - up (u0 + up) taken as
      // (um - up)(u0 + um + up), exact in integers
      {
        const long long um = U0[t - DX], up = U0[t + DX];
        const long long dx = mh(um - up, u0 + um + up);
        const long long dy = mh(U0[t - DY], V0[t - DY] + V0[t - DY + DX]) - mh(U0[t + DY], v0 + V0[t + DX]);
        const long long p3 = mh(Um[t], Wm[t] + Wm[t + DX]);
        const long long p4 = mh(Up[t], w0 + W0[t + DX]);
        su[o] = outv(hfactor<POW2>(cx, shx, dx) + hfactor<POW2>(cy, shy, dy) + mh(c1, p3) - mh(c2, p4));
      }
      // sv at (i, j+1/2, k)
      {
        const long long vm = V0[t - DY], vp = V0[t + DY];
        const long long dx = mh(V0[t - DX], U0[t - DX] + U0[t - DX + DY]) - mh(V0[t + DX], u0 + U0[t + DY]);
        const long long dy = mh(vm - vp, v0 + vm + vp);
        const long long p3 = mh(Vm[t], Wm[t] + Wm[t + DY]);
        const long long p4 = mh(Vp[t], w0 + W0[t + DY]);
        sv[o] = outv(hfactor<POW2>(cx, shx, dx) + hfactor<POW2>(cy, shy, dy) + mh(c1, p3) - mh(c2, p4));
      }
      // sw at (i, j, k+1/2)
      {
        const long long wm = Wm[t], wp = Wp[t];
        const long long dx = mh(W0[t - DX], U0[t - DX] + Up[t - DX]) - mh(W0[t + DX], u0 + Up[t]);
        const long long dy = mh(W0[t - DY], V0[t - DY] + Vp[t - DY]) - mh(W0[t + DY], v0 + Vp[t]);
        const long long p3 = mh(wm, w0 + wm);
        const long long p4 = mh(wp, w0 + wp);
        sw[o] = outv(hfactor<POW2>(cx, shx, dx) + hfactor<POW2>(cy, shy, dy) + mh(c1, p3) - mh(c2, p4));
      }
    }
    }
    __syncthreads();
  }
}

// One pass of the advection.  The first pass takes its scales from the
// record `prev` (the previous call's, or the range pass's on a context's
// first call) and records into `cur` the magnitudes it reads: the fields'
// and the factors' (tcx, tcy and the tzc entries, recorded by the CTAs of
// column (0, 0), whose chunks cover every plane).  The
// second pass compares the decision (fixed point or binary64) and the
// scales that `prev` gave with those of what the first pass read, and
// runs only when they differ, with the scales of `cur`; it records nothing
// and clears `next`, the record the next call's first pass fills.
struct AdvPass {
  const unsigned long long* prev;
  unsigned long long* cur;
  unsigned long long* next;
  int second;
};

// Each CTA owns one column of 32 x (BY RPT) cells (blockIdx.x, blockIdx.y)
// and one chunk of zc planes (blockIdx.z).
template <bool POW2, int BY, int MINB, bool FASTCVT, int QF = 3, int RPT = 1>
__global__ void __launch_bounds__(32 * BY, MINB)
    advect_kernel(const double* __restrict__ u, const double* __restrict__ v, const double* __restrict__ w,
                  double* __restrict__ su, double* __restrict__ sv, double* __restrict__ sw,
                  const double* __restrict__ tzc1, const double* __restrict__ tzc2, double tcx, double tcy,
                  int64_t nx, int64_t ny, int64_t nz, int64_t sy, int64_t sz, int64_t osy, int64_t osz,
                  int zc, const AdvPass ps) {
  __shared__ long long zfac[2 * kAdvZcMax];  // tzc1, tzc2 of the chunk's planes at scale T
  __shared__ unsigned long long fac[2];      // largest |factor| read, complement of the smallest nonzero (bits)
  const int tid = threadIdx.y * 32 + threadIdx.x;
  AdvScales sc;
  if (ps.second) {
    const AdvScales x = adv_scales_rec(ps.prev), y = adv_scales_rec(ps.cur);
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && tid == 0)
      for (int f = 0; f < 5; ++f) ps.next[f] = 0ull;
    if (x.fixed == y.fixed && (!x.fixed || (x.S == y.S && x.T == y.T))) return;  // uniform
    sc = y;
  } else {
    sc = adv_scales_rec(ps.prev);
  }
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * 32;  // halo index of the plane box's first column
  const int64_t j0 = static_cast<int64_t>(blockIdx.y) * BY * RPT;
  const int64_t k0 = static_cast<int64_t>(blockIdx.z) * zc;
  const int kn = static_cast<int>(min(static_cast<int64_t>(zc), nz - k0));  // cells of this chunk along z
  uint32_t mx[3] = {0u, 0u, 0u};  // largest high words of |u|, |v|, |w| read
  if (!sc.fixed) {  // uniform over the launch
    // the magnitudes of the cells the fixed-point path would have loaded
    // (this CTA's box, halo included), then binary64 cell by cell
    const int PXb = 34, PYb = BY * RPT + 2;
    for (int e = tid; e < PXb * PYb; e += 32 * BY) {
      const int64_t gi = i0 + e % PXb, gj = j0 + e / PXb;
      if (gi > nx + 1 || gj > ny + 1) continue;
      for (int kk = 0; kk <= kn + 1; ++kk) {
        const int64_t c = gi + gj * sy + (k0 + kk) * sz;
        mx[0] = max(mx[0], static_cast<uint32_t>(__double2hiint(u[c])) & 0x7fffffffu);
        mx[1] = max(mx[1], static_cast<uint32_t>(__double2hiint(v[c])) & 0x7fffffffu);
        mx[2] = max(mx[2], static_cast<uint32_t>(__double2hiint(w[c])) & 0x7fffffffu);
      }
    }
    const int64_t i = i0 + 1 + threadIdx.x;
    for (int rr = 0; rr < RPT; ++rr) {
      const int64_t j = j0 + 1 + threadIdx.y + rr * BY;
      if (i > nx || j > ny) continue;
      for (int kk = 0; kk < kn; ++kk) {
        const int64_t k = k0 + 1 + kk;
        const int64_t o = i + j * osy + k * osz;
        advect_cell_f64(u, v, w, i + j * sy + k * sz, sy, sz, tcx, tcy, tzc1[k - 1], tzc2[k - 1], su[o], sv[o],
                        sw[o]);
      }
    }
  } else if (FASTCVT && sc.S >= 0 && sc.S <= 1000 && sc.Q >= -960 && sc.Q <= 1022) {
    advect_march<POW2, BY, FASTCVT, QF, RPT>(u, v, w, su, sv, sw, tzc1, tzc2, tcx, tcy, nx, ny, sy, sz, osy, osz,
                                             i0, j0, k0, kn, sc, zfac, mx);
  } else {
    advect_march<POW2, BY, false, 3, RPT>(u, v, w, su, sv, sw, tzc1, tzc2, tcx, tcy, nx, ny, sy, sz, osy, osz, i0,
                                          j0, k0, kn, sc, zfac, mx);
  }
  if (ps.second) return;  // uniform
  // record (every thread of every warp arrives here)
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    const uint32_t m = __reduce_max_sync(0xffffffffu, mx[f]);
    if ((threadIdx.x & 31) == 0 && m)
      atomicMax(ps.cur + f, (static_cast<unsigned long long>(m) << 32) | 0xffffffffull);
  }
  // the factors (tcx, tcy, tzc1, tzc2): the chunks of column (0, 0) read
  // every plane's between them, so they alone record the factors' range,
  // after their march (uniform per CTA), gathered in shared memory first
  if (blockIdx.x == 0 && blockIdx.y == 0) {
    const int t = threadIdx.y * 32 + threadIdx.x;
    auto take = [&](double x) {
      const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x)) & kAbsMask;
      atomicMax(&fac[0], b);
      if (b != 0) atomicMax(&fac[1], ~b);
    };
    if (t == 0) fac[0] = fac[1] = 0ull;
    __syncthreads();
    if (t == 0) {
      take(tcx);
      take(tcy);
    }
    const int64_t kb = static_cast<int64_t>(blockIdx.z) * zc;
    const int kc = static_cast<int>(min(static_cast<int64_t>(zc), nz - kb));
    if (t < 2 * kc) take((t & 1) ? tzc2[kb + (t >> 1)] : tzc1[kb + (t >> 1)]);
    __syncthreads();
    if (t == 0) {
      if (fac[0]) atomicMax(ps.cur + 3, fac[0]);
      if (fac[1]) atomicMax(ps.cur + 4, fac[1]);
    }
  }
}

// Compiled tile shapes (thread rows BY, CTAs per SM, fields quantised on
// the FP64 pipe QF, rows per thread RPT) and the longest z chunk (zc, at
// most kAdvZcMax), fastest first at 512 x 512 x 256: two rows per thread
// and one field quantised in integer instructions gained 5% over one row
// and three fields (four rows per thread lost 30%); chunks of 48 or 64
// planes beat 32 by 1% (each chunk re-reads and re-quantises two planes and
// fills its ring before its first output plane; that outweighs the last,
// partly filled round of CTAs), 16 to 30 planes were slower than 32.
using AdvKernel = void (*)(const double*, const double*, const double*, double*, double*, double*, const double*,
                           const double*, double, double, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t,
                           int64_t, int, AdvPass);
struct AdvVariant {
  int BY, minb, rpt;  // thread rows, CTAs per SM, rows per thread
  int zc;             // longest z chunk
  AdvKernel kern[2];  // tcx, tcy general / powers of two
  int smem;
};
#define STENCIL_ADV_VARIANT(BY, MINB, QF, RPT, ZC)                                                          \
  {BY, MINB, RPT, ZC, {advect_kernel<false, BY, MINB, true, QF, RPT>, advect_kernel<true, BY, MINB, true, QF, RPT>}, \
   AdvGeom<BY, RPT>::kSmem}
const AdvVariant kAdvVariants[] = {
    STENCIL_ADV_VARIANT(8, 3, 2, 2, 48), STENCIL_ADV_VARIANT(8, 3, 2, 2, 64), STENCIL_ADV_VARIANT(8, 3, 2, 2, 32),
    STENCIL_ADV_VARIANT(8, 3, 2, 2, 128), STENCIL_ADV_VARIANT(8, 3, 3, 2, 64), STENCIL_ADV_VARIANT(8, 3, 1, 2, 64),
    STENCIL_ADV_VARIANT(8, 3, 2, 1, 64), STENCIL_ADV_VARIANT(4, 6, 2, 2, 64),
};
#undef STENCIL_ADV_VARIANT
constexpr int kNumAdvVariants = sizeof(kAdvVariants) / sizeof(kAdvVariants[0]);

}  // namespace

int advect_config_count() { return kNumAdvVariants; }

int launch_advect(stencil_ctx* ctx, const Grid& u, const Grid& v, const Grid& w, const Grid& su,
                  const Grid& sv, const Grid& sw, const double* tzc1, const double* tzc2,
                  double tcx, double tcy, cudaStream_t st) {
  if (u.sy != v.sy || u.sy != w.sy || u.sz != v.sz || u.sz != w.sz)
    return set_error(STENCIL_ERR_ARG, "advect: u, v, w must share strides");
  if (su.sy != sv.sy || su.sy != sw.sy || su.sz != sv.sz || su.sz != sw.sz)
    return set_error(STENCIL_ERR_ARG, "advect: su, sv, sw must share strides");
  const AdvVariant& av =
      kAdvVariants[(ctx->advect_choice >= 0 && ctx->advect_choice < kNumAdvVariants) ? ctx->advect_choice : 0];
  const int64_t gx = (u.nx + 31) / 32, gy = (u.ny + av.BY * av.rpt - 1) / (av.BY * av.rpt);
  // z chunk: the longest of these lengths (up to the shape's, and to what
  // the factor table holds when one thread fills each entry) that still
  // gives four rounds of resident CTAs (on smaller grids the last, partly
  // filled round costs more than the two planes each chunk re-reads)
  const int zmax = std::min(av.zc, std::min(kAdvZcMax, 16 * av.BY));
  static const int kChunks[] = {128, 64, 48, 32, 24, 16, 12, 8, 6, 4};
  int zc = 4;
  for (int c : kChunks)
    if (c <= zmax && gx * gy * ((u.nz + c - 1) / c) >= int64_t(4) * av.minb * ctx->num_sms) {
      zc = c;
      break;
    }
  const int64_t gz = (u.nz + zc - 1) / zc;
  if (gx > 0x7fffffff || gy > 65535 || gz > 65535) return set_error(STENCIL_ERR_ARG, "advect: grid too large");
  // tcx and tcy positive powers of two (within the fixed-point range): their
  // factor products are shifts (the quantised factor is then exactly
  // 2^(m + T), see hfactor)
  auto pow2 = [](double c) {
    int e = 0;
    return c > 0.0 && std::frexp(c, &e) == 0.5 && e > -900 && e < 900;
  };
  const bool p2 = pow2(tcx) && pow2(tcy);
  auto kern = av.kern[p2 ? 1 : 0];
  int rc = check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, av.smem),
                      "advect smem attribute");
  if (rc) return rc;
  // The scales.  Each call's first pass takes them from the previous call's
  // record (a context's first call measures the magnitudes with a range
  // pass and a one-warp pass over the factors) and records what it reads;
  // its second pass (launched every call, returning at once when not
  // needed) recomputes with the recorded magnitudes when they lead to
  // another decision or other scales -- the output is a function of the
  // input alone, and a call whose magnitudes keep the previous scales reads
  // u, v, w once.  Three records rotate: the previous call's, this call's,
  // and the next call's (cleared by this call's second pass).
  unsigned char* scr = ctx->scratch;
  auto* rec = reinterpret_cast<unsigned long long*>(scr + kScratchAdvRec);
  const int pos = ctx->advect_pos;
  unsigned long long* cur = rec + 5 * pos;
  unsigned long long* next = rec + 5 * ((pos + 1) % 3);
  const unsigned long long* prev = rec + 5 * ((pos + 2) % 3);
  if (!ctx->advect_guess) {
    unsigned long long* range = reinterpret_cast<unsigned long long*>(scr + kScratchAdvRange);
    rc = check_cuda(cudaMemsetAsync(rec, 0, 15 * sizeof(unsigned long long), st), "advect record init");
    if (rc) return rc;
    rc = check_cuda(cudaMemsetAsync(range, 0, 5 * sizeof(unsigned long long), st), "advect range init");
    if (rc) return rc;
    const int64_t rows = (u.ny + 2) * (u.nz + 2);
    const int rblocks = static_cast<int>(std::min<int64_t>((rows + 7) / 8, 8 * ctx->num_sms));
    advect_range_kernel<<<rblocks, dim3(32, 8), 0, st>>>(
        static_cast<const double*>(u.data), static_cast<const double*>(v.data), static_cast<const double*>(w.data),
        u.nx, u.ny, u.nz, u.sy, u.sz, range);
    rc = check_cuda(cudaGetLastError(), "advect range kernel");
    if (rc) return rc;
    advect_factor_kernel<<<1, 32, 0, st>>>(tzc1, tzc2, u.nz, tcx, tcy, range);
    rc = check_cuda(cudaGetLastError(), "advect factor kernel");
    if (rc) return rc;
    prev = range;
  }
  ctx->advect_guess = 0;  // until both passes are enqueued
  const dim3 block(32, av.BY);
  const dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy), static_cast<unsigned>(gz));
  auto launch = [&](const AdvPass& ps) {
    kern<<<grid, block, av.smem, st>>>(
        static_cast<const double*>(u.data), static_cast<const double*>(v.data),
        static_cast<const double*>(w.data), static_cast<double*>(su.data), static_cast<double*>(sv.data),
        static_cast<double*>(sw.data), tzc1, tzc2, tcx, tcy, u.nx, u.ny, u.nz, u.sy, u.sz, su.sy, su.sz, zc, ps);
    return check_cuda(cudaGetLastError(), "advect kernel");
  };
  rc = launch(AdvPass{prev, cur, next, 0});
  if (rc) return rc;
  rc = launch(AdvPass{prev, cur, next, 1});
  if (rc) return rc;
  ctx->advect_pos = (pos + 1) % 3;
  ctx->advect_guess = 1;
  return STENCIL_OK;
}

}  // namespace stencil
