// policies.cuh -- numeric policies of the sweep kernel (jacobi.cu).
//
// A policy fixes the storage type T of u and f, the register type C the
// sweep computes in, and four operations: `in` (storage -> register), `out`
// (register -> storage), `update` (one Jacobi update from the six
// neighbours and the source value) and `make` (per-launch constants,
// evaluated on the device by every thread).  Every `update` adds the two x
// neighbours first (xm + xp): the red-black kernel relies on it to pass
// them in either order.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "fixed.cuh"

namespace stencil {

// Arguments every sweep launch passes to its policy's `make`.
struct SweepArgs {
  double hh;                              // h*h
  const unsigned long long* maxbits;      // fixed point: bit patterns of [max|u| over the halo,
                                          //   max|f| over the interior, max|u| over the interior]
  uint32_t* status;                       // device status word
  uint32_t* fxmag;                        // fixed point: [3] magnitude keys of recent passes' outputs
  int32_t* fxscale;                       // fixed point: [3] scales of recent passes' outputs
  int32_t* fxgscale;                      // resident fixed point: [3] scale of the stored source
                                          //   after recent passes
  int pass;                               // fixed point: index of this pass in the call (1, 2, ...)
  int stages;                             // sweeps (Jacobi) or colour stages (red-black) per pass
  const double* fsrc64;                   // resident fixed point: the binary64 source f ...
  int64_t fsy, fsz;                       //   ... and its strides (host side: its tensor map)
  unsigned long long* gdst;               // resident fixed point: the stored source (work grid) ...
  int64_t gsy, gsz;                       //   ... and its strides
  int write_r;                            // residual: store r
  unsigned long long* rpart;              // residual: [CTA count, then 4 words per CTA] partial sums
  const uint32_t* run_flag;               // residual: if set, the pass runs only when *run_flag != 0
  unsigned long long* seen;               // residual: [3] bounds (bits) of max|u|, max|f|, max|u| read
};

__device__ __forceinline__ double bits_as_double(unsigned long long b) {
  return __longlong_as_double(static_cast<long long>(b));
}

// Scale of pass a.pass of a fixed-point call.  Pass p reads slot (p-1) mod 3
// of the state (the scale its input is stored at and the magnitude key of
// that input -- what the previous pass wrote; the set-up kernel fills slot 0
// for pass 1) and publishes slot p mod 3.  Every value the pass produces is
// bounded by
//   M = max(bound of its input, max|halo|) + stages * hh max|f| / 6
// (one sweep, or one colour stage, averages values below the running bound
// and adds at most hh max|f| / 6: the maximum principle of the update), and
// a six-neighbour sum plus the source by B = 6 M + hh max|f|, which fixes
// S = fx_scale_for(B).
// PER-PASS (not RESIDENT): the pass converts its binary64 input and the
// source at S, computes and rounds back to binary64.
// RESIDENT: the pass computes at the scale its input is stored at (Sprev)
// and writes its output at S, the scale the next pass computes at:
// S = Sprev unless the bound needs a coarser scale or allows one at least
// two steps finer (most passes rescale nothing: dshift = 0); a pass that
// does rescale shifts each value it writes.  The source is stored in the
// work grid at one scale (slot's fxgscale); when that is not the computing
// scale (fpath: the pass after a rescale), every tile of the pass loads the
// binary64 f instead, converts it at the computing scale, and stores the
// source afresh for its own cells -- no tile reads the work grid during that
// pass, so rewriting it races with nothing.  Computing at Sprev cannot overflow: Sprev leaves
// room for values up to 2^58 / 6 (a bound B_prev >= 6 M_prev + hh max|f|
// below 2^(58 - Sprev)), the biased sums hold up to 2^60 / 6, and this
// pass's values stay below M_prev + stages hh max|f| / 6 <= 2 M_prev.
template <bool RESIDENT>
__device__ __forceinline__ FixedParams fx_pass_params(const SweepArgs& a) {
  FixedParams p;
  p.bad = 0; p.dshift = 0; p.fpath = 0;
  const int prev = (a.pass + 2) % 3;
  const int Sprev = a.fxscale[prev];
  const double mh = bits_as_double(a.maxbits[0]);
  const double mf = bits_as_double(a.maxbits[1]);
  if (Sprev >= kFxBadScale) {  // an earlier pass (or the set-up) failed
    p.bad = Sprev - kFxBadScale;
    fx_conv(p, 0, a.hh);
    return p;
  }
  if (!(mh <= 1.0e300) || !(mf <= 1.0e300)) {
    p.bad = (mh - mh == 0.0 && mf - mf == 0.0) ? 2 : 1;
    fx_conv(p, 0, a.hh);
    return p;
  }
  const uint32_t key = a.fxmag[prev];
  const double mi = RESIDENT ? ldexp(static_cast<double>(key) + 1.0, 32 - Sprev)
                             : bits_as_double((static_cast<unsigned long long>(key) << 32) | 0xffffffffull);
  const double hmf = a.hh * mf;
  const double M = fmax(mi, mh) + static_cast<double>(a.stages) * hmf / 6.0;
  int S = fx_scale_for(6.0 * M + hmf, &p.bad);
  if (RESIDENT && !p.bad) {
    if (S >= Sprev && S < Sprev + 2) S = Sprev;
    p.dshift = max(-62, min(62, S - Sprev));
    p.fpath = a.fxgscale[prev] != Sprev;
    fx_conv(p, Sprev, a.hh);  // conversions (Dirichlet values, source) at the computing scale
    p.S = S;                  // the output's scale
    return p;
  }
  fx_conv(p, S, a.hh);
  return p;
}

// Block 0, thread 0 of pass a.pass: publish its scale (or the failure), clear
// the magnitude slot the next pass accumulates into, report a new failure.
__device__ __forceinline__ void fx_pass_publish(const SweepArgs& a, const FixedParams& p) {
  if (blockIdx.x != 0 || threadIdx.x != 0 || threadIdx.y != 0) return;
  const int prev = (a.pass + 2) % 3;
  const bool sticky = a.fxscale[prev] >= kFxBadScale;
  a.fxscale[a.pass % 3] = p.bad ? kFxBadScale + p.bad : p.S;
  if (a.fxgscale) a.fxgscale[a.pass % 3] = p.fpath ? 1085 - p.Cu : a.fxgscale[prev];
  a.fxmag[(a.pass + 1) % 3] = 0u;
  if (p.bad && !sticky) atomicOr(a.status, p.bad == 1 ? kStatusNonFinite : kStatusRange);
}

// Combine the magnitude keys of a warp's active lanes into the pass's slot.
__device__ __forceinline__ void fx_track_commit(const SweepArgs& a, uint32_t key) {
  const uint32_t mask = __activemask();
  const uint32_t m = __reduce_max_sync(mask, key);
  if ((threadIdx.x & 31) == static_cast<uint32_t>(__ffs(mask) - 1) && m) atomicMax(a.fxmag + a.pass % 3, m);
}

// Output magnitude tracking of the policies that do not track.
template <class T>
struct NoTrack {
  __device__ __forceinline__ void add(T) {}
  __device__ __forceinline__ void add2(T, T) {}
  __device__ __forceinline__ uint32_t key() const { return 0u; }
};

// binary64 storage and arithmetic: adds in the order of the definition,
// the source term fused (h*h*f + s), then a multiply by the rounded 1/6.
struct PolF64 {
  using T = double;
  using C = double;
  static constexpr int kElem = 8;
  static constexpr bool kFixed = false;
  static constexpr bool kTrack = false;
  static constexpr bool kResident = false;
  static constexpr bool kResidual = false;
  using Track = NoTrack<double>;
  struct K { double hh; };
  __device__ static __forceinline__ K make(const SweepArgs& a) { return K{a.hh}; }
  __device__ static __forceinline__ C in(T v, const K&) { return v; }
  __device__ static __forceinline__ C in_halo(T v, const K& k) { return in(v, k); }
  __device__ static __forceinline__ T out(C v, const K&) { return v; }
  __device__ static __forceinline__ C update(C xm, C xp, C ym, C yp, C zm, C zp, T f, const K& k) {
    C s = xm + xp;
    s += ym;
    s += yp;
    s += zm;
    s += zp;
    return fma(k.hh, f, s) * (1.0 / 6.0);
  }
};

// binary32 storage and arithmetic (hh rounded once to binary32).
struct PolF32 {
  using T = float;
  using C = float;
  static constexpr int kElem = 4;
  static constexpr bool kFixed = false;
  static constexpr bool kTrack = false;
  static constexpr bool kResident = false;
  static constexpr bool kResidual = false;
  using Track = NoTrack<float>;
  struct K { float hh; };
  __device__ static __forceinline__ K make(const SweepArgs& a) { return K{static_cast<float>(a.hh)}; }
  __device__ static __forceinline__ C in(T v, const K&) { return v; }
  __device__ static __forceinline__ C in_halo(T v, const K& k) { return in(v, k); }
  __device__ static __forceinline__ T out(C v, const K&) { return v; }
  // The sum as a tree (x pair, y pair, z pair plus the source): four
  // dependent operations instead of seven, for the latency-bound passes.
  __device__ static __forceinline__ C update(C xm, C xp, C ym, C yp, C zm, C zp, T f, const K& k) {
    const C sx = xm + xp, sy = ym + yp, sz = fmaf(k.hh, f, zm + zp);
    return ((sx + sy) + sz) * (1.0f / 6.0f);
  }
};

// bfloat16 storage, binary32 arithmetic, round-to-nearest-even stores.
// Intermediate sweeps of a temporally blocked pass stay in binary32.
struct PolBF16 {
  using T = __nv_bfloat16;
  using C = float;
  static constexpr int kElem = 2;
  static constexpr bool kFixed = false;
  static constexpr bool kTrack = false;
  static constexpr bool kResident = false;
  static constexpr bool kResidual = false;
  using Track = NoTrack<__nv_bfloat16>;
  struct K { float hh; };
  __device__ static __forceinline__ K make(const SweepArgs& a) { return K{static_cast<float>(a.hh)}; }
  __device__ static __forceinline__ C in(T v, const K&) { return __bfloat162float(v); }
  __device__ static __forceinline__ C in_halo(T v, const K& k) { return in(v, k); }
  __device__ static __forceinline__ T out(C v, const K&) { return __float2bfloat16_rn(v); }
  // The sum as a tree, as PolF32.
  __device__ static __forceinline__ C update(C xm, C xp, C ym, C yp, C zm, C zp, T f, const K& k) {
    const C sx = xm + xp, sy = ym + yp, sz = fmaf(k.hh, __bfloat162float(f), zm + zp);
    return ((sx + sy) + sz) * (1.0f / 6.0f);
  }
};

// binary64 storage, 64-bit fixed-point arithmetic (fixed.cuh), converted in
// every pass at that pass's scale.  The magnitude key of an output is the
// high word of |x|'s bit pattern: the pass's largest |x| is at most the
// double with that high word and an all-ones low word.
struct PolFixed {
  using T = double;
  using C = uint64_t;
  static constexpr int kElem = 8;
  static constexpr bool kFixed = true;
  static constexpr bool kTrack = true;
  static constexpr bool kResident = false;
  static constexpr bool kResidual = false;
  using K = FixedParams;
  struct Track {
    uint32_t m = 0;
    __device__ __forceinline__ void add(double o) {
      m = max(m, static_cast<uint32_t>(static_cast<unsigned long long>(__double_as_longlong(o)) >> 32) &
                     0x7fffffffu);
    }
    __device__ __forceinline__ void add2(double a, double b) {
      add(a);
      add(b);
    }
    __device__ __forceinline__ uint32_t key() const { return m; }
  };
  __device__ static __forceinline__ K make(const SweepArgs& a) { return fx_pass_params<false>(a); }
  __device__ static __forceinline__ void publish(const SweepArgs& a, const K& k) { fx_pass_publish(a, k); }
  __device__ static __forceinline__ C in(T v, const K& k) { return fx_in(v, k.Cu); }
  __device__ static __forceinline__ C in_halo(T v, const K& k) { return in(v, k); }
  __device__ static __forceinline__ T out(C v, const K& k) {
    return k.bad ? __longlong_as_double(0x7ff8000000000000ll) : fx_out(v, k.S);
  }
  __device__ static __forceinline__ C update(C xm, C xp, C ym, C yp, C zm, C zp, T f, const K& k) {
    const uint64_t sum = xm + xp + ym + yp + zm + zp +
                         static_cast<uint64_t>(fx_source(f, k.Cg, k.H)) + 3ull;
    return fx_div6(sum);
  }
};

// binary64 storage, 64-bit fixed point resident for the whole call: the
// interior of the iterate buffers holds the biased integers U (fixed.cuh) at
// the scale the pass that wrote them chose, and the work buffer holds the
// source G = round(h*h*f*2^S) at that same scale (written by the set-up,
// rewritten by every pass that changes the scale).  Halo cells stay binary64
// (the Dirichlet values are never rewritten); the kernel converts them as it
// loads them.  The magnitude key of a pass: the largest and smallest high
// word of its outputs U (two 32-bit min/max per output); the largest |q| is
// below (max(hi_max - 2^27, 2^27 - hi_min) + 1) * 2^32.
struct PolResident {
  using T = uint64_t;
  using C = uint64_t;
  static constexpr int kElem = 8;
  static constexpr bool kFixed = true;
  static constexpr bool kTrack = true;
  static constexpr bool kResident = true;
  static constexpr bool kResidual = false;
  using K = FixedParams;
  struct Track {
    uint32_t mx = 0u, mn = 0xffffffffu;
    __device__ __forceinline__ void add(uint64_t U) {
      const uint32_t hi = static_cast<uint32_t>(U >> 32);
      mx = max(mx, hi);
      mn = min(mn, hi);
    }
    // two outputs: one three-way max and one three-way min
    __device__ __forceinline__ void add2(uint64_t a, uint64_t b) {
      const uint32_t ha = static_cast<uint32_t>(a >> 32), hb = static_cast<uint32_t>(b >> 32);
      mx = __vimax3_u32(mx, ha, hb);
      mn = __vimin3_u32(mn, ha, hb);
    }
    __device__ __forceinline__ uint32_t key() const {
      constexpr int32_t kb = static_cast<int32_t>(kFxBias >> 32);
      if (mx < mn) return 0u;  // wrote nothing
      const int32_t a = static_cast<int32_t>(mx) - kb, b = kb - static_cast<int32_t>(mn);
      return static_cast<uint32_t>(max(0, max(a, b)));
    }
  };
  __device__ static __forceinline__ K make(const SweepArgs& a) { return fx_pass_params<true>(a); }
  __device__ static __forceinline__ void publish(const SweepArgs& a, const K& k) { fx_pass_publish(a, k); }
  __device__ static __forceinline__ C in(T v, const K&) { return v; }
  __device__ static __forceinline__ C in_halo(T v, const K& k) {
    return fx_in(__longlong_as_double(static_cast<long long>(v)), k.Cu);
  }
  __device__ static __forceinline__ bool needs_rescale(const K& k) { return k.dshift != 0 || k.fpath != 0; }
  // an fpath pass: the staged binary64 source (its bit pattern) at the computing scale
  __device__ static __forceinline__ T source_at(T f_bits, const K& k) {
    return static_cast<uint64_t>(fx_source(__longlong_as_double(static_cast<long long>(f_bits)), k.Cg, k.H));
  }
  __device__ static __forceinline__ C rescale(C v, const K& k) { return fx_rescale(v, k.dshift); }
  __device__ static __forceinline__ T out(C v, const K&) { return v; }
  __device__ static __forceinline__ C update(C xm, C xp, C ym, C yp, C zm, C zp, T g, const K&) {
    return fx_div6(xm + xp + ym + yp + zm + zp + g + 3ull);
  }
};

// The residual r = f - (6u - sum of the six neighbours) / h^2 and its
// squared norm (Section 4.1's operator; the residual decides convergence),
// in 64-bit fixed point.  One scale S for the call: u -> U = K + round(u 2^S)
// and h*h*f -> G = round(h*h*f 2^S) with 12 max|u| + h*h max|f| below
// 2^(62 - S), so D = 6U - (sum of the six neighbours' U) = 6q - sum q is
// exact (the bias K cancels) and R = G - D = round(h^2 r 2^S) up to the
// conversions (at most 6.5 units of 2^-S: about 2^-55 of 12 max|u|, finer
// than a binary64 evaluation of the same expression).  The squared norm of
// R is summed exactly in 192-bit integers (so it is the same whatever the
// order), that of f in binary64; r, when asked for, is R 2^-S / h^2.
struct PolResid {
  using T = double;
  using C = uint64_t;
  static constexpr int kElem = 8;
  static constexpr bool kFixed = true;
  static constexpr bool kTrack = false;
  static constexpr bool kResident = false;
  static constexpr bool kResidual = true;
  struct K {
    int S, Cu, Cg;
    uint64_t H;
    int bad;     // 1: input not finite, 2: beyond range
    int write;   // store r
    double rs;   // 2^-S / h^2
  };
  // exact sums: s = s2 2^128 + s1 2^64 + s0 of R^2, and ff of f^2; the
  // largest high words of |u| and |f| the lane converted
  struct Track {
    uint64_t s0 = 0, s1 = 0, s2 = 0;
    double ff = 0.0;
    uint32_t mu = 0, mf = 0;
    __device__ __forceinline__ void see_u(double u) {
      mu = max(mu, static_cast<uint32_t>(__double2hiint(u)) & 0x7fffffffu);
    }
    __device__ __forceinline__ void add_sq(int64_t R) {
      const uint64_t a = static_cast<uint64_t>(R < 0 ? -R : R);
      const uint64_t lo = a * a, hi = __umul64hi(a, a);
      // (s2, s1, s0) += (0, hi, lo) as one carry chain
      asm("add.cc.u64 %0, %0, %3;\n\taddc.cc.u64 %1, %1, %4;\n\taddc.u64 %2, %2, 0;"
          : "+l"(s0), "+l"(s1), "+l"(s2)
          : "l"(lo), "l"(hi));
    }
    __device__ __forceinline__ void add(uint64_t R, double f) {
      add_sq(static_cast<int64_t>(R));
      ff = fma(f, f, ff);
      mf = max(mf, static_cast<uint32_t>(__double2hiint(f)) & 0x7fffffffu);
    }
    // this + o (exactly for the integer part)
    __device__ __forceinline__ void merge(uint64_t o0, uint64_t o1, uint64_t o2, double off) {
      s0 += o0;
      const uint64_t c0 = s0 < o0;
      const uint64_t t = s1 + o1;
      const uint64_t c1 = t < o1;
      s1 = t + c0;
      s2 += o2 + c1 + (s1 < c0);
      ff += off;
    }
  };
  // The scale follows from the magnitudes' high words (each rounded up to
  // the largest double with that high word), so a bound measured from high
  // words alone gives the same scale as the exact maxima.
  __device__ static __forceinline__ K make(const SweepArgs& a) {
    K k;
    k.bad = 0;
    k.write = a.write_r;
    const double mh = bits_as_double(a.maxbits[0] | 0xffffffffull), mf = bits_as_double(a.maxbits[1] | 0xffffffffull),
                 mu = bits_as_double(a.maxbits[2] | 0xffffffffull);
    int S = 0;
    if (!(mh <= 1.0e300) || !(mf <= 1.0e300) || !(mu <= 1.0e300)) {
      k.bad = (mh - mh == 0.0 && mf - mf == 0.0 && mu - mu == 0.0) ? 2 : 1;
    } else {
      // B = 12 max|u| + h^2 max|f|; S = 62 - ceil(log2 B)
      const double B = 12.0 * fmax(mh, mu) + a.hh * mf;
      int e = 0;
      if (B > 0.0) frexp(B, &e);
      S = 62 - e;
      if (S > 1022) S = 1022;
      if (S < -900) k.bad = 2;
    }
    FixedParams p;
    fx_conv(p, S, a.hh);
    k.S = S; k.Cu = p.Cu; k.Cg = p.Cg; k.H = p.H;
    k.rs = ldexp(1.0, -S) / a.hh;
    return k;
  }
  __device__ static __forceinline__ C in(T v, const K& k) { return fx_in(v, k.Cu); }
  __device__ static __forceinline__ C in_halo(T v, const K& k) { return in(v, k); }
  // R = G - (6 U_c - sum of the six neighbours' U), as a two's-complement word
  __device__ static __forceinline__ C residual(C c, C xm, C xp, C ym, C yp, C zm, C zp, T f, const K& k) {
    const uint64_t six = (c << 2) + (c << 1);
    const uint64_t D = six - (xm + xp + ym + yp + zm + zp);
    return static_cast<uint64_t>(fx_source(f, k.Cg, k.H)) - D;
  }
  __device__ static __forceinline__ C update(C, C, C, C, C, C, T, const K&) { return 0; }
  __device__ static __forceinline__ T out(C v, const K& k) {
    return k.bad ? __longlong_as_double(0x7ff8000000000000ll)
                 : __ll2double_rn(static_cast<long long>(v)) * k.rs;
  }
};

}  // namespace stencil
