// advect.cu -- Piacsek-Williams flux-form momentum advection (Section 4.1:
// the three stencils over u, v, w fused into one region, 63 operations per
// cell).
//
// B300 issues binary64 arithmetic at about 1/64 of its binary32 rate, so a
// binary64 evaluation of the 63 operations is bound by the FP64 pipe at a
// few percent of the HBM roofline.  The kernel therefore evaluates the
// tendencies in 64-bit integer fixed point, as the Jacobi sweep does:
//   * one scale S per call from max |u|, |v|, |w| (halos included):
//     X = round(x 2^S) with |X| <= 2^61, so every sum of two is exact;
//   * each product a (b + c) keeps the high 64 bits of its exact 128-bit
//     value (a truncation below 2^-56 max|x|^2), so equal fluxes cancel
//     exactly;
//   * the factors tcx, tcy, tzc1[k], tzc2[k] use one scale T from their
//     maximum (|C| <= 2^62; exact for the binary64 inputs in use), each
//     factor product again keeps its high 64 bits, the three terms are
//     summed in 64 bits and the sum is rounded to binary64 once.
// The error is at most about 2^-50 max|x|^2 max|C| per output, the order of
// the rounding error of a binary64 evaluation of the same formula.  When the fields'
// magnitudes differ by more than 2^8, or the factors' do, or a value is not
// finite, a single scale would cost the smaller field its precision, so the
// launch evaluates the formula in binary64 instead (the decision is taken
// on the device from the range reduction: the call stays asynchronous).
//
// Each CTA quantises a (32+2) x (8+2) x (4+2) halo tile of u, v, w into
// shared memory once; each thread then computes su, sv, sw for 4 cells
// along z from the tile.  48 algorithmic bytes per cell (three fields in,
// three out).  (Computing sw in binary64 on the otherwise idle FP64 pipe
// while su and sv use the integer pipe was measured slower, 3.85 against
// 3.72 ms at 512 x 512 x 256: 21 binary64 operations per cell keep the
// FP64 pipe busy for about 3 ms on their own.)
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace stencil {

namespace {

constexpr int kAdvBX = 32, kAdvBY = 8, kAdvZT = 4;
constexpr int kTX = kAdvBX + 2, kTY = kAdvBY + 2, kTZ = kAdvZT + 2;
constexpr int kTile = kTX * kTY * kTZ;
constexpr int kAdvSmem = 3 * kTile * 8;
constexpr unsigned long long kAbsMask = 0x7fffffffffffffffull;
constexpr unsigned long long kInfBits = 0x7ff0000000000000ull;

// Reduction of the magnitudes that fix the scales: r[0..2] = bits of
// max |u|, |v|, |w| over every cell (halos included), r[3] = bits of the
// largest |factor| (tcx, tcy, tzc1[], tzc2[]), r[4] = bits of the smallest
// nonzero |factor|.  Non-negative doubles order as their bit patterns.
__global__ void advect_range_kernel(const double* __restrict__ u, const double* __restrict__ v,
                                    const double* __restrict__ w, int64_t nx, int64_t ny, int64_t nz, int64_t sy,
                                    int64_t sz, const double* __restrict__ tzc1, const double* __restrict__ tzc2,
                                    double tcx, double tcy, unsigned long long* r) {
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
  if (blockIdx.x == 0 && threadIdx.y == 0) {
    unsigned long long cmax = 0, cmin = ~0ull;
    auto take = [&](double x) {
      const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x)) & kAbsMask;
      cmax = b > cmax ? b : cmax;
      if (b != 0) cmin = b < cmin ? b : cmin;
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
      const unsigned long long a = __shfl_xor_sync(0xffffffffu, cmax, o);
      const unsigned long long b = __shfl_xor_sync(0xffffffffu, cmin, o);
      cmax = a > cmax ? a : cmax;
      cmin = b < cmin ? b : cmin;
    }
    if (threadIdx.x == 0) {
      atomicMax(&r[3], cmax);
      atomicMin(&r[4], cmin);
    }
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
__device__ __forceinline__ AdvScales adv_scales(const unsigned long long* r) {
  AdvScales sc{0, 0, 0, false};
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
  sc.Q = 2 * sc.S + sc.T - 128;
  sc.fixed = true;
  return sc;
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

// floor(a (b + c) / 2^64): the high half of the exact product.
__device__ __forceinline__ long long prod(long long a, long long b, long long c) { return __mul64hi(a, b + c); }

// One flux difference a (b + c) - d (e + f) at scale 2^(2S - 64).
__device__ __forceinline__ long long flux(long long a, long long b, long long c, long long d, long long e,
                                          long long f) {
  return prod(a, b, c) - prod(d, e, f);
}

// The high half of c d for a horizontal factor c.  POW2: c = 2^m exactly
// (tcx, tcy powers of two, as 1/4 is), so the high half of c d is d shifted
// right by 64 - m, floor -- bit for bit what the multiply gives.
template <bool POW2>
__device__ __forceinline__ long long hfactor(long long c, int sh, long long d) {
  if constexpr (POW2) return d >> sh;
  else return __mul64hi(c, d);
}

// cx dx + cy dy + c1 p3 - c2 p4, each factor product's high half, as binary64.
template <bool POW2>
__device__ __forceinline__ double combine(long long cx, int shx, long long dx, long long cy, int shy, long long dy,
                                          long long c1, long long p3, long long c2, long long p4, int Q) {
  const long long s =
      hfactor<POW2>(cx, shx, dx) + hfactor<POW2>(cy, shy, dy) + __mul64hi(c1, p3) - __mul64hi(c2, p4);
  return fx64_to_double(s, Q);
}

// 64 - log2(c) for c a positive power of two (the shift of hfactor), else -1.
__device__ __forceinline__ int pow2_shift(long long c) {
  return (c > 0 && (c & (c - 1)) == 0) ? 64 - (63 - __clzll(c)) : -1;
}

template <bool POW2>
__global__ void __launch_bounds__(256, 4)
    advect_kernel(const double* __restrict__ u, const double* __restrict__ v, const double* __restrict__ w,
                  double* __restrict__ su, double* __restrict__ sv, double* __restrict__ sw,
                  const double* __restrict__ tzc1, const double* __restrict__ tzc2, double tcx, double tcy,
                  int64_t nx, int64_t ny, int64_t nz, int64_t sy, int64_t sz, int64_t osy, int64_t osz,
                  const unsigned long long* __restrict__ range) {
  extern __shared__ long long adv_tile[];
  __shared__ long long zfac[2 * kAdvZT];  // tzc1, tzc2 of the tile's planes at scale T
  const AdvScales sc = adv_scales(range);
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * kAdvBX;  // halo index of the tile's first cell
  const int64_t j0 = static_cast<int64_t>(blockIdx.y) * kAdvBY;
  const int64_t k0 = static_cast<int64_t>(blockIdx.z) * kAdvZT;
  const int64_t i = i0 + 1 + threadIdx.x, j = j0 + 1 + threadIdx.y;
  if (!sc.fixed) {
    if (i > nx || j > ny) return;
    for (int kk = 0; kk < kAdvZT; ++kk) {
      const int64_t k = k0 + 1 + kk;
      if (k > nz) break;
      const int64_t o = i + j * osy + k * osz;
      advect_cell_f64(u, v, w, i + j * sy + k * sz, sy, sz, tcx, tcy, tzc1[k - 1], tzc2[k - 1], su[o], sv[o],
                      sw[o]);
    }
    return;
  }
  long long* U = adv_tile;
  long long* V = adv_tile + kTile;
  long long* W = adv_tile + 2 * kTile;
  for (int t = threadIdx.y * kAdvBX + threadIdx.x; t < kTile; t += kAdvBX * kAdvBY) {
    const int xx = t % kTX, yy = (t / kTX) % kTY, zz = t / (kTX * kTY);
    const int64_t gi = i0 + xx, gj = j0 + yy, gk = k0 + zz;
    long long qu = 0, qv = 0, qw = 0;
    if (gi <= nx + 1 && gj <= ny + 1 && gk <= nz + 1) {
      const int64_t c = gi + gj * sy + gk * sz;
      qu = fx_quant(u[c], sc.S);
      qv = fx_quant(v[c], sc.S);
      qw = fx_quant(w[c], sc.S);
    }
    U[t] = qu;
    V[t] = qv;
    W[t] = qw;
  }
  {
    const int t = threadIdx.y * kAdvBX + threadIdx.x;
    if (t < 2 * kAdvZT) {
      const int64_t k = k0 + 1 + (t >> 1);
      zfac[t] = k <= nz ? fx_quant((t & 1) ? tzc2[k - 1] : tzc1[k - 1], sc.T) : 0;
    }
  }
  __syncthreads();
  if (i > nx || j > ny) return;
  const long long cx = fx_quant(tcx, sc.T), cy = fx_quant(tcy, sc.T);
  const int shx = pow2_shift(cx), shy = pow2_shift(cy);
  constexpr int DX = 1, DY = kTX, DZ = kTX * kTY;
  for (int kk = 0; kk < kAdvZT; ++kk) {
    const int64_t k = k0 + 1 + kk;
    if (k > nz) break;
    const long long c1 = zfac[2 * kk], c2 = zfac[2 * kk + 1];
    const int t = (kk + 1) * DZ + (threadIdx.y + 1) * DY + (threadIdx.x + 1);
    const long long u0 = U[t], v0 = V[t], w0 = W[t];
    const int64_t o = i + j * osy + k * osz;
    // su at (i+1/2, j, k)
    {
      const long long um = U[t - DX], up = U[t + DX];
      const long long dx = flux(um, u0, um, up, u0, up);
      const long long dy = flux(U[t - DY], V[t - DY], V[t - DY + DX], U[t + DY], v0, V[t + DX]);
      const long long p3 = prod(U[t - DZ], W[t - DZ], W[t - DZ + DX]);
      const long long p4 = prod(U[t + DZ], w0, W[t + DX]);
      su[o] = combine<POW2>(cx, shx, dx, cy, shy, dy, c1, p3, c2, p4, sc.Q);
    }
    // sv at (i, j+1/2, k)
    {
      const long long vm = V[t - DY], vp = V[t + DY];
      const long long dx = flux(V[t - DX], U[t - DX], U[t - DX + DY], V[t + DX], u0, U[t + DY]);
      const long long dy = flux(vm, v0, vm, vp, v0, vp);
      const long long p3 = prod(V[t - DZ], W[t - DZ], W[t - DZ + DY]);
      const long long p4 = prod(V[t + DZ], w0, W[t + DY]);
      sv[o] = combine<POW2>(cx, shx, dx, cy, shy, dy, c1, p3, c2, p4, sc.Q);
    }
    // sw at (i, j, k+1/2)
    {
      const long long wm = W[t - DZ], wp = W[t + DZ];
      const long long dx = flux(W[t - DX], U[t - DX], U[t - DX + DZ], W[t + DX], u0, U[t + DZ]);
      const long long dy = flux(W[t - DY], V[t - DY], V[t - DY + DZ], W[t + DY], v0, V[t + DZ]);
      const long long p3 = prod(wm, w0, wm);
      const long long p4 = prod(wp, w0, wp);
      sw[o] = combine<POW2>(cx, shx, dx, cy, shy, dy, c1, p3, c2, p4, sc.Q);
    }
  }
}

}  // namespace

int launch_advect(stencil_ctx* ctx, const Grid& u, const Grid& v, const Grid& w, const Grid& su,
                  const Grid& sv, const Grid& sw, const double* tzc1, const double* tzc2,
                  double tcx, double tcy, cudaStream_t st) {
  if (u.sy != v.sy || u.sy != w.sy || u.sz != v.sz || u.sz != w.sz)
    return set_error(STENCIL_ERR_ARG, "advect: u, v, w must share strides");
  if (su.sy != sv.sy || su.sy != sw.sy || su.sz != sv.sz || su.sz != sw.sz)
    return set_error(STENCIL_ERR_ARG, "advect: su, sv, sw must share strides");
  const int64_t gy = (u.ny + kAdvBY - 1) / kAdvBY, gz = (u.nz + kAdvZT - 1) / kAdvZT;
  if (gy > 65535 || gz > 65535) return set_error(STENCIL_ERR_ARG, "advect: grid too large");
  unsigned long long* range = reinterpret_cast<unsigned long long*>(ctx->scratch + kScratchAdvRange);
  int rc = check_cuda(cudaMemsetAsync(range, 0, 4 * sizeof(unsigned long long), st), "advect range init");
  if (!rc) rc = check_cuda(cudaMemsetAsync(range + 4, 0xff, sizeof(unsigned long long), st), "advect range init");
  if (rc) return rc;
  const int64_t rows = (u.ny + 2) * (u.nz + 2);
  const int rblocks = static_cast<int>(std::min<int64_t>((rows + 7) / 8, 8 * ctx->num_sms));
  advect_range_kernel<<<rblocks, dim3(32, 8), 0, st>>>(
      static_cast<const double*>(u.data), static_cast<const double*>(v.data), static_cast<const double*>(w.data),
      u.nx, u.ny, u.nz, u.sy, u.sz, tzc1, tzc2, tcx, tcy, range);
  rc = check_cuda(cudaGetLastError(), "advect range kernel");
  if (rc) return rc;
  // tcx and tcy positive powers of two (within the fixed-point range): their
  // factor products are shifts (the quantised factor is then exactly
  // 2^(m + T), see hfactor)
  auto pow2 = [](double c) {
    int e = 0;
    return c > 0.0 && std::frexp(c, &e) == 0.5 && e > -900 && e < 900;
  };
  const bool p2 = pow2(tcx) && pow2(tcy);
  auto kern = p2 ? advect_kernel<true> : advect_kernel<false>;
  rc = check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kAdvSmem),
                  "advect smem attribute");
  if (rc) return rc;
  const dim3 block(kAdvBX, kAdvBY);
  const dim3 grid(static_cast<unsigned>((u.nx + kAdvBX - 1) / kAdvBX), static_cast<unsigned>(gy),
                  static_cast<unsigned>(gz));
  kern<<<grid, block, kAdvSmem, st>>>(
      static_cast<const double*>(u.data), static_cast<const double*>(v.data),
      static_cast<const double*>(w.data), static_cast<double*>(su.data), static_cast<double*>(sv.data),
      static_cast<double*>(sw.data), tzc1, tzc2, tcx, tcy, u.nx, u.ny, u.nz, u.sy, u.sz, su.sy, su.sz, range);
  return check_cuda(cudaGetLastError(), "advect kernel");
}

}  // namespace stencil
