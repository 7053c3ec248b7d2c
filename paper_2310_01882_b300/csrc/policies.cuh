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
  double nsw;                             // sweeps of the whole call (fixed-point bound)
  double lmin;                            // (smallest extent + 1) * h
  const unsigned long long* maxbits;      // [max|u|, max|f|] bit patterns (fixed point)
  uint32_t* status;                       // device status word
};

// binary64 storage and arithmetic: adds in the order of the definition,
// the source term fused (h*h*f + s), then a multiply by the rounded 1/6.
struct PolF64 {
  using T = double;
  using C = double;
  static constexpr int kElem = 8;
  static constexpr bool kFixed = false;
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
  struct K { float hh; };
  __device__ static __forceinline__ K make(const SweepArgs& a) { return K{static_cast<float>(a.hh)}; }
  __device__ static __forceinline__ C in(T v, const K&) { return v; }
  __device__ static __forceinline__ C in_halo(T v, const K& k) { return in(v, k); }
  __device__ static __forceinline__ T out(C v, const K&) { return v; }
  __device__ static __forceinline__ C update(C xm, C xp, C ym, C yp, C zm, C zp, T f, const K& k) {
    C s = xm + xp;
    s += ym;
    s += yp;
    s += zm;
    s += zp;
    return fmaf(k.hh, f, s) * (1.0f / 6.0f);
  }
};

// bfloat16 storage, binary32 arithmetic, round-to-nearest-even stores.
// Intermediate sweeps of a temporally blocked pass stay in binary32.
struct PolBF16 {
  using T = __nv_bfloat16;
  using C = float;
  static constexpr int kElem = 2;
  static constexpr bool kFixed = false;
  struct K { float hh; };
  __device__ static __forceinline__ K make(const SweepArgs& a) { return K{static_cast<float>(a.hh)}; }
  __device__ static __forceinline__ C in(T v, const K&) { return __bfloat162float(v); }
  __device__ static __forceinline__ C in_halo(T v, const K& k) { return in(v, k); }
  __device__ static __forceinline__ T out(C v, const K&) { return __float2bfloat16_rn(v); }
  __device__ static __forceinline__ C update(C xm, C xp, C ym, C yp, C zm, C zp, T f, const K& k) {
    C s = xm + xp;
    s += ym;
    s += yp;
    s += zm;
    s += zp;
    return fmaf(k.hh, __bfloat162float(f), s) * (1.0f / 6.0f);
  }
};

// binary64 storage, 64-bit fixed-point arithmetic (fixed.cuh).
struct PolFixed {
  using T = double;
  using C = uint64_t;
  static constexpr int kElem = 8;
  static constexpr bool kFixed = true;
  using K = FixedParams;
  __device__ static __forceinline__ K make(const SweepArgs& a) {
    K k = fx_params(__longlong_as_double(static_cast<long long>(a.maxbits[0])),
                    __longlong_as_double(static_cast<long long>(a.maxbits[1])), a.hh, a.nsw, a.lmin);
    if (k.bad && threadIdx.x == 0 && blockIdx.x == 0)
      atomicOr(a.status, k.bad == 1 ? kStatusNonFinite : kStatusRange);
    return k;
  }
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
// interior of the iterate buffers holds the biased integers U (fixed.cuh) and
// the work buffer holds the pre-scaled source G = round(h*h*f*2^S), both
// converted once per call.  Halo cells stay binary64 (the Dirichlet values
// are never rewritten); the kernel converts them as it loads them.
struct PolResident {
  using T = uint64_t;
  using C = uint64_t;
  static constexpr int kElem = 8;
  static constexpr bool kFixed = true;
  using K = FixedParams;
  __device__ static __forceinline__ K make(const SweepArgs& a) {
    return fx_params(__longlong_as_double(static_cast<long long>(a.maxbits[0])),
                     __longlong_as_double(static_cast<long long>(a.maxbits[1])), a.hh, a.nsw, a.lmin);
  }
  __device__ static __forceinline__ C in(T v, const K&) { return v; }
  __device__ static __forceinline__ C in_halo(T v, const K& k) {
    return fx_in(__longlong_as_double(static_cast<long long>(v)), k.Cu);
  }
  __device__ static __forceinline__ T out(C v, const K&) { return v; }
  __device__ static __forceinline__ C update(C xm, C xp, C ym, C yp, C zm, C zp, T g, const K&) {
    return fx_div6(xm + xp + ym + yp + zm + zp + g + 3ull);
  }
};

}  // namespace stencil
