// apply.cu -- the general linear stencil apply (Section 2.2: a stencil.apply
// reads its input at constant offsets and yields one value per point of the
// output's bounds; here the body is a linear combination):
//   out(x) = sum_p c_p in(x + d_p),   |d_p| <= 3 per axis,
// over the interior points whose reads all lie in the field (halo
// included): with r = max |d|, indices r .. n + 1 - r per axis (the whole
// interior when the offsets stay in the one-cell halo).
//
// Two evaluations:
//  * coefficients that are integer multiples of one power of two, c_p =
//    k_p 2^E with |k_p| <= 2^20 (integer-weight stencils: Laplacians,
//    averages, finite differences with their denominators folded out):
//    64-bit fixed point.  The input is converted at one scale 2^-S per call
//    (S from max|in| and sum |k_p|, so no sum can overflow), sum k_p q_p is
//    exact and rounded to binary64 once, times 2^E.  Stars (the centre and
//    +-1..R along each axis: Laplacians of every order) run a z march that
//    keeps each thread's own column in registers (apply_star_march); other
//    offset sets a z march that keeps the 2R + 1 input planes the offsets
//    reach, with their x/y margins, in shared memory as fixed-point
//    integers; every loaded plane is written to two slots of a doubled
//    ring, so the planes z - R .. z + R always sit in consecutive slots and
//    each term's shared-memory offset is one constant, whatever the offsets
//    are.  Either way each input value is read from HBM and converted once.
//  * any other coefficients: binary64, each product rounded then added in
//    the listed order (no fused multiply-add): bitwise the definition; one
//    thread per point, neighbours through L1 (bound by the FP64 pipe).
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "fixed.cuh"
#include "internal.h"

namespace stencil {

namespace {

constexpr int kApBX = 32, kApBY = 8;

struct LinearTerms {
  int64_t off[kMaxLinearTerms];  // element offsets dx + dy sy + dz sz
  double c[kMaxLinearTerms];
  int n, r;
};

__global__ void __launch_bounds__(256)
    apply_linear_kernel(const double* __restrict__ in, double* __restrict__ out, int64_t nx, int64_t ny, int64_t nz,
                        int64_t sy, int64_t sz, int64_t osy, int64_t osz, const __grid_constant__ LinearTerms t) {
  const int64_t i = t.r + blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int64_t j = t.r + blockIdx.y * int64_t(blockDim.y) + threadIdx.y;
  if (i > nx + 1 - t.r || j > ny + 1 - t.r) return;
  for (int64_t k = t.r + blockIdx.z; k <= nz + 1 - t.r; k += gridDim.z) {
    const int64_t c = i + j * sy + k * sz;
    double acc = 0.0;
    for (int p = 0; p < t.n; ++p) acc = __dadd_rn(acc, __dmul_rn(t.c[p], in[c + t.off[p]]));
    out[i + j * osy + k * osz] = acc;
  }
}

// Terms of the fixed-point form: the shared-memory offset of each term
// (from the window's first slot), its integer weight, the power of two E.
struct FxTerms {
  int soff[kMaxLinearTerms];
  int k[kMaxLinearTerms];
  int n, r, E;
  double sumk;  // sum |k_p|
};

// max|in| over the field (halo included), as bits into *maxbits (zeroed first).
__global__ void apply_range_kernel(const double* __restrict__ in, int64_t nx, int64_t ny, int64_t nz, int64_t sy,
                                   int64_t sz, unsigned long long* maxbits) {
  const int64_t rows = (ny + 2) * (nz + 2);
  unsigned long long m = 0;
  for (int64_t row = blockIdx.x * int64_t(blockDim.y) + threadIdx.y; row < rows;
       row += int64_t(gridDim.x) * blockDim.y) {
    const int64_t k = row / (ny + 2), j = row - k * (ny + 2);
    for (int64_t i = threadIdx.x; i < nx + 2; i += blockDim.x) {
      const unsigned long long b =
          static_cast<unsigned long long>(__double_as_longlong(in[i + j * sy + k * sz])) & 0x7fffffffffffffffull;
      m = b > m ? b : m;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long a = __shfl_xor_sync(0xffffffffu, m, o);
    m = a > m ? a : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(maxbits, m);
}

// round(x 2^S) as a signed integer, halves away from zero, for |x| 2^S < 2^62
// (Cu = 1085 - S; zeros and subnormals give 0).
__device__ __forceinline__ int64_t fx_quant_signed(double x, int Cu) {
  const uint64_t b = static_cast<uint64_t>(__double_as_longlong(x));
  const int e = static_cast<int>((b >> 52) & 0x7ffu);
  const uint64_t m63 = (b << 11) | 0x8000000000000000ull;
  const uint64_t t = shr64(m63, static_cast<unsigned>(Cu - e));  // floor(2 |x| 2^S)
  return static_cast<int64_t>((t ^ fx_sign_mask(b)) + 1) >> 1;
}

// Compiled offset sets: the common shapes, offsets known at compile time so
// that every term's shared-memory offset is an immediate and its weight a
// constant-bank operand.  SHAPE 1: the star of radius R (the centre, then
// +-1..R along x, y, z); SHAPE 2: the 27-point box (R = 1).  SHAPE 0: any
// offsets (read from the launch parameters term by term).
template <int SHAPE, int R>
struct ApShape {
  static constexpr int N = SHAPE == 2 ? 27 : 1 + 6 * R;
  // offset of term q along x, y, z
  __host__ __device__ static constexpr int d(int q, int axis) {
    if (SHAPE == 2) return axis == 0 ? q % 3 - 1 : (axis == 1 ? (q / 3) % 3 - 1 : q / 9 - 1);
    if (q == 0) return 0;
    const int idx = q - 1, ax = idx / (2 * R), rem = idx % (2 * R);
    return ax != axis ? 0 : ((rem & 1) ? 1 : -1) * (rem / 2 + 1);
  }
};

// The z march of one CTA.  EXACT_EXP: every nonzero result's binary64
// exponent can be shifted by E - S without leaving the normal range (the
// scaling is then an integer add to the exponent field); otherwise ldexp.
template <int R, int SHAPE, bool EXACT_EXP>
__device__ __forceinline__ void apply_fx_march(const double* __restrict__ in, double* __restrict__ out, int64_t nx,
                                               int64_t ny, int64_t nz, int64_t sy, int64_t sz, int64_t osy,
                                               int64_t osz, const FxTerms& t, int Cu, int sh, bool bad, int zchunk,
                                               uint32_t& seen) {
  constexpr int WX = kApBX + 2 * R, WY = kApBY + 2 * R, PL = WX * WY, NP = 2 * R + 1;
  constexpr int NT = kApBX * kApBY, NL = (PL + NT - 1) / NT;
  extern __shared__ long long ap_win[];  // 2 NP slots of PL values
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kApBX + tx;
  const int64_t ox = t.r + static_cast<int64_t>(blockIdx.x) * kApBX;  // first output column of the tile
  const int64_t oy = t.r + static_cast<int64_t>(blockIdx.y) * kApBY;
  const int64_t zs = t.r + static_cast<int64_t>(blockIdx.z) * zchunk;
  const int64_t ze = min(zs + zchunk - 1, nz + 1 - t.r);
  const int64_t i = ox + tx, j = oy + ty;
  const bool owner = i <= nx + 1 - t.r && j <= ny + 1 - t.r;
  // the window cells this thread loads: their offset within a plane, and
  // whether they lie in the field (in x and y)
  int64_t goff[NL];
  bool gin[NL];
#pragma unroll
  for (int m = 0; m < NL; ++m) {
    const int c = tid + m * NT;
    const int cy = c / WX, cx = c - cy * WX;
    const int64_t gi = ox - R + cx, gj = oy - R + cy;
    gin[m] = c < PL && gi >= 0 && gi <= nx + 1 && gj >= 0 && gj <= ny + 1;
    goff[m] = gin[m] ? gi + gj * sy : 0;
  }
  int slot = static_cast<int>((((zs - R) % NP) + NP) % NP);  // ring slot of plane p
  const double* src = in + (zs - R) * sz;
  double* dst = out + i + j * osy + (zs - 2 * R) * osz;    // output plane p - R
  // software pipeline: the raw values of plane p are loaded while plane
  // p - 1 is computed, and converted into the ring at the top of step p
  double raw[NL];
  auto load = [&](int64_t p, const double* srcp) {
    const bool pin = p >= 0 && p <= nz + 1;
#pragma unroll
    for (int m = 0; m < NL; ++m) raw[m] = (pin && gin[m]) ? srcp[goff[m]] : 0.0;
  };
  load(zs - R, src);
  for (int64_t p = zs - R; p <= ze + R; ++p, src += sz, dst += osz) {
    // plane p into ring slots `slot` and `slot + NP`, so that the planes
    // z - R .. z + R are consecutive from the slot of z - R
#pragma unroll
    for (int m = 0; m < NL; ++m) {
      const int c = tid + m * NT;
      if (c < PL) {
        const long long q = fx_quant_signed(raw[m], Cu);
        seen = max(seen, static_cast<uint32_t>(__double2hiint(raw[m])) & 0x7fffffffu);
        ap_win[slot * PL + c] = q;
        ap_win[(slot + NP) * PL + c] = q;
      }
    }
    if (p < ze + R) load(p + 1, src + sz);
    __syncthreads();
    if (p - R >= zs && owner) {
      int b = slot - 2 * R;  // slot of plane (p - R) - R
      if (b < 0) b += NP;
      const long long* w = ap_win + b * PL + ty * WX + tx;
      long long acc = 0;
      if constexpr (SHAPE == 0) {
        for (int q = 0; q < t.n; ++q) acc += static_cast<long long>(t.k[q]) * w[t.soff[q]];
      } else {
        using Sh = ApShape<SHAPE, R>;
#pragma unroll
        for (int q = 0; q < Sh::N; ++q)
          acc += static_cast<long long>(t.k[q]) *
                 w[(R + Sh::d(q, 2)) * PL + (R + Sh::d(q, 1)) * WX + (R + Sh::d(q, 0))];
      }
      double v;
      if (bad) {
        v = __longlong_as_double(0x7ff8000000000000ll);
      } else if (acc == 0) {
        v = 0.0;
      } else if constexpr (EXACT_EXP) {
        v = __longlong_as_double(__double_as_longlong(__ll2double_rn(acc)) + (static_cast<long long>(sh) << 52));
      } else {
        v = ldexp(__ll2double_rn(acc), sh);
      }
      *dst = v;
    }
    __syncthreads();
    slot = slot + 1 == NP ? 0 : slot + 1;
  }
}

// Asynchronous 8-byte global -> shared copies (zero-filled when !valid),
// committed in groups; a thread waits only for its own copies.
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src), "r"(valid ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// The star of radius R (SHAPE 1), z march with the z terms in registers.
// A CTA of 32 x 8 threads owns a 32 x 16 column of outputs (two rows per
// thread, rows ty and ty + 8).  Input planes, with their x/y
// margin of R cells, stream into a ring of kApStarDepth raw planes in shared
// memory by asynchronous copies issued kApStarDepth - 1 planes ahead (each
// thread copies, then converts, the same cells, so only its own copies need
// waiting for).  Each plane is quantised once into a ring of R + 2 slots in
// pre-split form q = H 2^31 + L (0 <= L < 2^31, H signed 32-bit, one 64-bit
// word), and each thread keeps its own column's values of the 2R + 1 planes
// its z terms read in a register window (rotated by an unrolled loop, no
// moves).  Step p converts plane p, passes one CTA barrier, takes its own
// value of plane p into the window and computes output plane p - R: its z
// terms from the window, its x and y terms from that plane's slot.  The sum
// is two exact 64-bit dot products, sum k_p L_p and sum k_p H_p (one
// 32 x 32 -> 64-bit multiply-add per term each), recombined as
// (sum k H) 2^31 + sum k L.  The quantised slot written at step p + 1 held
// plane p - R - 1, last read before step p's barrier.  FASTQ: a thread's
// first cell of a plane is quantised by adding S to its exponent field and
// converting to the nearest integer on the FP64 pipe (valid for
// 0 <= S <= 1000), its other cells by fx_quant_signed in integer
// instructions (the two pipes share the work); both give round(x 2^S) up to
// the rounding of an exact half.
constexpr int kApStarDepth = 6;
constexpr int kApStarRows = 2;  // output rows per thread: the tile is 32 x 16
template <int R>
struct ApStar {
  static constexpr int ROWS = kApStarRows, TY = kApBY * ROWS;  // tile rows
  static constexpr int WX = kApBX + 2 * R, WY = TY + 2 * R, PL = WX * WY, NS = R + 2, NW = 2 * R + 1;
  static constexpr int NT = kApBX * kApBY, NL = (PL + NT - 1) / NT, D = kApStarDepth;
  static constexpr int kSmem = (NS + D) * PL * 8;
};

// d = a b + c with a, b signed 32-bit and c, d 64-bit (one wide multiply-add).
__device__ __forceinline__ long long madw(int a, int b, long long c) {
  long long d;
  asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long lds64(uint32_t a) {
  unsigned long long v;
  asm volatile("ld.shared.u64 %0, [%1];" : "=l"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ double lds64f(uint32_t a) {
  double v;
  asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void sts64(uint32_t a, unsigned long long v) {
  asm volatile("st.shared.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}

template <int R, bool FASTQ, bool EXACT_EXP, bool SYM>
__device__ __forceinline__ void apply_star_march(const double* __restrict__ in, double* __restrict__ out,
                                                 int64_t nx, int64_t ny, int64_t nz, int64_t sy, int64_t sz,
                                                 int64_t osy, int64_t osz, const FxTerms& t, int S, int Cu, int sh,
                                                 bool bad, int zchunk, uint32_t& seen) {
  using G = ApStar<R>;
  constexpr int WX = G::WX, PL = G::PL, NS = G::NS, NW = G::NW, NT = G::NT, NL = G::NL, D = G::D;
  constexpr uint32_t kPlaneBytes = PL * 8;
  using Sh = ApShape<1, R>;
  extern __shared__ long long ap_win[];  // NS slots of PL pre-split values, then D raw planes
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kApBX + tx;
  const int64_t ox = R + static_cast<int64_t>(blockIdx.x) * kApBX;  // first output column of the tile
  const int64_t oy = R + static_cast<int64_t>(blockIdx.y) * G::TY;
  const int64_t zs = R + static_cast<int64_t>(blockIdx.z) * zchunk;
  const int64_t ze = min(zs + zchunk - 1, nz + 1 - R);
  constexpr int ROWS = G::ROWS;
  const int64_t i = ox + tx;
  bool owner[ROWS];
#pragma unroll
  for (int r = 0; r < ROWS; ++r) owner[r] = i <= nx + 1 - R && oy + ty + r * kApBY <= ny + 1 - R;
  const int nplanes = static_cast<int>(ze - zs) + 1 + 2 * R;  // input planes zs - R .. ze + R
  // this thread's cells of every plane: source pointers (advanced a plane at
  // a time), validity, and shared-memory byte offsets
  const double* src[NL];
  bool gin[NL];
#pragma unroll
  for (int m = 0; m < NL; ++m) {
    const int c = tid + m * NT;
    const int cy = c / WX, cx = c - cy * WX;
    const int64_t gi = ox - R + cx, gj = oy - R + cy;
    gin[m] = c < PL && gi <= nx + 1 && gj <= ny + 1;  // gi, gj >= 0 always (ox, oy >= R)
    src[m] = in + (gin[m] ? gi + gj * sy + (zs - R) * sz : 0);
  }
  const uint32_t qbase = smem_addr(ap_win);               // quantised ring, slot 0
  const uint32_t rbase = qbase + NS * kPlaneBytes;         // raw ring, slot 0
  const uint32_t mine8 = static_cast<uint32_t>(tid) * 8;  // byte offset of cell tid in a plane
  const uint32_t own8 = static_cast<uint32_t>((ty + R) * WX + (tx + R)) * 8;  // row r: + r * 8 WX * 8
  const int sadd = S << 20;
  auto quant = [&](double x) -> long long {
    if constexpr (FASTQ) return __double2ll_rn(__hiloint2double(__double2hiint(x) + sadd, __double2loint(x)));
    else return fx_quant_signed(x, Cu);
  };
  // plane n (0-based from zs - R) into raw slot rslot (an empty group past the end)
  auto issue = [&](int n, uint32_t rslot) {
    if (n < nplanes) {
#pragma unroll
      for (int m = 0; m < NL; ++m) {
        if (m + 1 < NL || tid + m * NT < PL)
          cp_async8(rslot + mine8 + m * NT * 8, gin[m] ? src[m] : in, gin[m]);
        src[m] += sz;
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int d = 0; d < D - 1; ++d) issue(d, rbase + d * kPlaneBytes);
  int WL[ROWS][NW], WH[ROWS][NW];  // own columns: plane n's pre-split value in window slot n mod NW
  long long WQ[ROWS][NW];          // SYM: plane n's value q in window slot n mod NW
  double* dst = out + i + (oy + ty) * osy + zs * osz;  // row r: + r * 8 osy
  uint32_t qslot = qbase;                               // quantised slot of plane n
  uint32_t rslot = rbase;                               // raw slot of plane n
  uint32_t rnext = rbase + (D - 1) * kPlaneBytes;       // raw slot of plane n + D - 1
  const uint32_t qend = qbase + NS * kPlaneBytes, rend = rbase + D * kPlaneBytes;
  int n = 0;
  for (;;) {
#pragma unroll
    for (int rot = 0; rot < NW; ++rot) {
      if (n >= nplanes) return;
      issue(n + D - 1, rnext);  // into plane n - 1's raw slot (converted by this thread)
      cp_async_wait<D - 1>();   // plane n's copies (this thread's) have landed
#pragma unroll
      for (int m = 0; m < NL; ++m) {
        if (m + 1 < NL || tid + m * NT < PL) {
          // FASTQ: the first cell through the FP64 pipe's conversion, the
          // others in integer instructions (balances the two pipes)
          const double x = lds64f(rslot + mine8 + m * NT * 8);
          const long long q = (FASTQ && m == 0) ? quant(x) : fx_quant_signed(x, Cu);
          seen = max(seen, static_cast<uint32_t>(__double2hiint(x)) & 0x7fffffffu);
          if constexpr (SYM)
            sts64(qslot + mine8 + m * NT * 8, static_cast<unsigned long long>(q));
          else
            sts64(qslot + mine8 + m * NT * 8,
                  (static_cast<unsigned long long>(static_cast<unsigned>(static_cast<int>(q >> 31))) << 32) |
                      static_cast<unsigned>(q & 0x7fffffff));
        }
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        const unsigned long long v = lds64(qslot + own8 + r * kApBY * WX * 8);
        if constexpr (SYM) {
          WQ[r][rot] = static_cast<long long>(v);
        } else {
          WL[r][rot] = static_cast<int>(v);
          WH[r][rot] = static_cast<int>(v >> 32);
        }
      }
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
      if (n >= 2 * R && owner[r]) {
        // output plane zs + n - 2R: its window slot is rot - R, its ring slot R back
        const uint32_t ws = qslot >= qbase + R * kPlaneBytes ? qslot - R * kPlaneBytes
                                                             : qslot + (NS - R) * kPlaneBytes;
        long long acc;
        if constexpr (SYM) {
          // one weight per distance d: w_0 q + sum_d w_d (sum of the six
          // values at distance d).  Integer adds and multiplies wrap modulo
          // 2^64, so the result -- the same sum of k_p q_p, which fits in 64
          // bits -- is exact whatever the intermediate values.
          auto at = [&](int dx, int dy) -> long long {
            return static_cast<long long>(
                lds64(ws + own8 + static_cast<uint32_t>((r * kApBY * WX + dy * WX + dx) * 8)));
          };
          acc = static_cast<long long>(t.k[0]) * WQ[r][((rot - R) % NW + NW) % NW];
#pragma unroll
          for (int d = 1; d <= R; ++d) {
            const long long g = (at(-d, 0) + at(d, 0)) + (at(0, -d) + at(0, d)) +
                                (WQ[r][((rot - R - d) % NW + NW) % NW] + WQ[r][((rot - R + d) % NW + NW) % NW]);
            acc += static_cast<long long>(t.k[1 + 2 * (d - 1)]) * g;
          }
        } else {
          // two accumulators per half (terms alternate), so the multiply-add
          // chains are half as long
          long long aL[2] = {0, 0}, aH[2] = {0, 0};
#pragma unroll
          for (int q = 0; q < Sh::N; ++q) {
            const int dz = Sh::d(q, 2);
            int l, h;
            if (dz != 0 || q == 0) {
              const int wi = ((rot - R + dz) % NW + NW) % NW;
              l = WL[r][wi];
              h = WH[r][wi];
            } else {
              const unsigned long long v =
                  lds64(ws + own8 + static_cast<uint32_t>((r * kApBY * WX + Sh::d(q, 1) * WX + Sh::d(q, 0)) * 8));
              l = static_cast<int>(v);
              h = static_cast<int>(v >> 32);
            }
            aL[q & 1] = madw(t.k[q], l, aL[q & 1]);
            aH[q & 1] = madw(t.k[q], h, aH[q & 1]);
          }
          acc = (aH[0] + aH[1]) * (1ll << 31) + (aL[0] + aL[1]);
        }
        double vout;
        if (bad) {
          vout = __longlong_as_double(0x7ff8000000000000ll);
        } else if (acc == 0) {
          vout = 0.0;
        } else if constexpr (EXACT_EXP) {
          vout = __longlong_as_double(__double_as_longlong(__ll2double_rn(acc)) + (static_cast<long long>(sh) << 52));
        } else {
          vout = ldexp(__ll2double_rn(acc), sh);
        }
        dst[r * kApBY * osy] = vout;
      }
      }
      if (n >= 2 * R) dst += osz;
      qslot += kPlaneBytes;
      if (qslot == qend) qslot = qbase;
      rnext = rslot;
      rslot += kPlaneBytes;
      if (rslot == rend) rslot = rbase;
      ++n;
    }
  }
}

// Scale of a fixed-point apply (the same in every thread): sum |k_p|
// max|in| 2^S <= 2^61, so every partial sum stays below 2^62; max|in| is
// taken from its high word (rounded up), so a bound measured from high
// words gives the same scale.  bad: 1 for a non-finite input, 2 for a
// magnitude the exponent range cannot scale.
__device__ __forceinline__ int apply_scale(const unsigned long long* maxbits, double sumk, int* bad) {
  const double mx = __longlong_as_double(static_cast<long long>(maxbits[0] | 0xffffffffull));
  int S = 0;
  *bad = 0;
  if (!(mx <= 1.0e300)) {
    *bad = 1;
  } else {
    int e = 0;
    if (mx > 0.0) frexp(mx * sumk, &e);
    S = 61 - e;
    if (S > 1022) S = 1022;
    if (S < -900) *bad = 2;
  }
  return S;
}

// One pass of a fixed-point apply: the magnitudes it takes its scale from
// (`used`), where it records the magnitudes it reads (`seen`), the flag
// that makes it run (null: always) and the status word (null: the pass
// reports nothing; only a final pass does).
struct ApPass {
  const unsigned long long* used;
  unsigned long long* seen;
  const uint32_t* run_flag;
  uint32_t* status;
};

// Bound of the magnitudes a CTA read, published by one atomic per warp.
__device__ __forceinline__ void apply_publish(unsigned long long* dst, uint32_t seen) {
  const uint32_t m = __reduce_max_sync(0xffffffffu, seen);
  if ((threadIdx.x & 31) == 0) atomicMax(dst, (static_cast<unsigned long long>(m) << 32) | 0xffffffffull);
}

template <int R, int SHAPE>
__global__ void __launch_bounds__(kApBX * kApBY)
    apply_fx_kernel(const double* __restrict__ in, double* __restrict__ out, int64_t nx, int64_t ny, int64_t nz,
                    int64_t sy, int64_t sz, int64_t osy, int64_t osz, const __grid_constant__ FxTerms t,
                    const ApPass ps, int zchunk) {
  if (ps.run_flag && *ps.run_flag == 0u) return;  // uniform
  int bad = 0;
  const int S = apply_scale(ps.used, t.sumk, &bad);
  if (ps.status && bad && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 &&
      threadIdx.y == 0)
    atomicOr(ps.status, bad == 1 ? kStatusNonFinite : kStatusRange);
  const int sh = t.E - S;  // out = sum 2^sh
  uint32_t seen = 0;
  // |sum| in [1, 2^62): its exponent is 0..61, shifted stays normal when
  // -1022 <= sh and sh + 61 <= 1023
  if (sh >= -1022 && sh <= 962)
    apply_fx_march<R, SHAPE, true>(in, out, nx, ny, nz, sy, sz, osy, osz, t, 1085 - S, sh, bad != 0, zchunk, seen);
  else
    apply_fx_march<R, SHAPE, false>(in, out, nx, ny, nz, sy, sz, osy, osz, t, 1085 - S, sh, bad != 0, zchunk, seen);
  apply_publish(ps.seen, seen);
}

template <int R, bool SYM>
__global__ void __launch_bounds__(kApBX * kApBY, 3)
    apply_star_kernel(const double* __restrict__ in, double* __restrict__ out, int64_t nx, int64_t ny, int64_t nz,
                      int64_t sy, int64_t sz, int64_t osy, int64_t osz, const __grid_constant__ FxTerms t,
                      const ApPass ps, int zchunk) {
  if (ps.run_flag && *ps.run_flag == 0u) return;  // uniform
  int bad = 0;
  const int S = apply_scale(ps.used, t.sumk, &bad);
  if (ps.status && bad && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 &&
      threadIdx.y == 0)
    atomicOr(ps.status, bad == 1 ? kStatusNonFinite : kStatusRange);
  const int sh = t.E - S;  // out = sum 2^sh; the sum's exponent is 0..61
  const bool exact_exp = sh >= -1022 && sh <= 962;
  const bool fastq = S >= 0 && S <= 1000;
  uint32_t seen = 0;
  if (fastq && exact_exp)
    apply_star_march<R, true, true, SYM>(in, out, nx, ny, nz, sy, sz, osy, osz, t, S, 1085 - S, sh, bad != 0, zchunk,
                                    seen);
  else if (exact_exp)
    apply_star_march<R, false, true, SYM>(in, out, nx, ny, nz, sy, sz, osy, osz, t, S, 1085 - S, sh, bad != 0, zchunk,
                                     seen);
  else
    apply_star_march<R, false, false, SYM>(in, out, nx, ny, nz, sy, sz, osy, osz, t, S, 1085 - S, sh, bad != 0, zchunk,
                                      seen);
  apply_publish(ps.seen, seen);
}

// Accepts the scale the first pass used only if it is the scale of what it
// read; otherwise the second pass runs at the read magnitudes' scale.  The
// magnitudes read become the next call's guess.
__global__ void apply_check_kernel(const unsigned long long* used, const unsigned long long* __restrict__ seen,
                                   double sumk, unsigned long long* __restrict__ final_bits,
                                   uint32_t* __restrict__ redo, unsigned long long* guess) {
  int bg = 0, br = 0;
  const unsigned long long u0 = used[0], s0 = seen[0];
  const int sg = apply_scale(&u0, sumk, &bg), sr = apply_scale(&s0, sumk, &br);
  const bool ok = !bg && !br && sg == sr;
  final_bits[0] = ok ? u0 : s0;
  *redo = ok ? 0u : 1u;
  guess[0] = s0;
}

// c = k 2^e with k an odd integer (c != 0): the exact decomposition.
void odd_power(double c, long long* k, int* e) {
  int ex = 0;
  const double m = std::frexp(std::fabs(c), &ex);          // |c| = m 2^ex, m in [0.5, 1)
  long long M = static_cast<long long>(std::ldexp(m, 53));  // exact: 53-bit integer
  int tz = 0;
  while ((M & 1) == 0) {
    M >>= 1;
    ++tz;
  }
  *k = c < 0 ? -M : M;
  *e = ex - 53 + tz;
}

}  // namespace

int launch_apply_linear(stencil_ctx* ctx, const Grid& in, const Grid& out, const int32_t* offsets,
                        const double* coeffs, int npoints, cudaStream_t st) {
  int r = 1;
  for (int p = 0; p < 3 * npoints; ++p) r = std::max(r, std::abs(offsets[p]));
  // nothing to write when the bounds are empty
  if (in.nx + 2 - 2 * r < 1 || in.ny + 2 - 2 * r < 1 || in.nz + 2 - 2 * r < 1) return STENCIL_OK;
  // integer multiples of one power of two?
  bool fx = true;
  int E = 1 << 20;
  std::vector<long long> k0(npoints, 0);
  std::vector<int> e0(npoints, 0);
  for (int p = 0; p < npoints && fx; ++p) {
    if (!std::isfinite(coeffs[p])) fx = false;
    else if (coeffs[p] != 0.0) {
      odd_power(coeffs[p], &k0[p], &e0[p]);
      if (k0[p] > (1ll << 20) || k0[p] < -(1ll << 20)) fx = false;
      E = std::min(E, e0[p]);
    }
  }
  if (fx && E != (1 << 20)) {
    FxTerms t{};
    double sumk = 0.0;
    int n = 0;
    const int R = r;  // the window radius is the offsets' radius
    const int WX = kApBX + 2 * R, WY = kApBY + 2 * R, PL = WX * WY;
    // a compiled shape that holds every offset: the star of radius r (all
    // offsets on the axes) or, at r = 1, the 27-point box
    bool on_axes = true;
    for (int p = 0; p < npoints; ++p) {
      const int nz_axes = (offsets[3 * p] != 0) + (offsets[3 * p + 1] != 0) + (offsets[3 * p + 2] != 0);
      if (nz_axes > 1) on_axes = false;
    }
    const int shape = on_axes ? 1 : (r == 1 ? 2 : 0);
    const int nshape = shape == 2 ? 27 : 1 + 6 * r;
    auto shape_term = [&](int dx, int dy, int dz) {  // index of an offset in the compiled shape
      if (shape == 2) return (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
      if (dx == 0 && dy == 0 && dz == 0) return 0;
      const int ax = dx ? 0 : (dy ? 1 : 2), d = dx + dy + dz;
      return 1 + ax * 2 * r + 2 * (std::abs(d) - 1) + (d > 0);
    };
    for (int p = 0; p < npoints; ++p) {
      if (coeffs[p] == 0.0) continue;
      const int shift = e0[p] - E;
      if (shift > 20 || std::llabs(k0[p]) > ((1ll << 20) >> shift)) {  // |k_p| 2^shift > 2^20
        fx = false;
        break;
      }
      const int kp = static_cast<int>(k0[p] << shift);
      sumk += std::fabs(static_cast<double>(kp));
      const int dx = offsets[3 * p], dy = offsets[3 * p + 1], dz = offsets[3 * p + 2];
      if (shape) {  // the weights in the shape's order (repeated offsets add up: the sum is exact)
        t.k[shape_term(dx, dy, dz)] += kp;
      } else {
        t.k[n] = kp;
        t.soff[n] = (R + dz) * PL + (R + dy) * WX + (R + dx);
        ++n;
      }
    }
    for (int q = 0; shape && q < nshape; ++q)
      if (std::llabs(static_cast<long long>(t.k[q])) > (1ll << 20)) fx = false;  // summed repeats
    if (fx) {
      t.n = shape ? nshape : n;
      t.r = r;
      t.E = E;
      t.sumk = sumk > 0.0 ? sumk : 1.0;
      const int64_t ox = in.nx + 2 - 2 * r, oy = in.ny + 2 - 2 * r, oz = in.nz + 2 - 2 * r;  // output extents
      const int64_t tiles = ((ox + kApBX - 1) / kApBX) * ((oy + kApBY - 1) / kApBY);
      // the kernel and its launch shape: stars take the register-window
      // march (z chunks as long as still give every SM several CTAs: each
      // chunk re-reads 2R planes), other offset sets the shared-memory one
      // (about 8 CTAs per SM in total, each chunk at least 8 planes)
      void (*kern)(const double*, double*, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, FxTerms,
                   ApPass, int);
      dim3 grid;
      int smem = 0;
      int64_t zc = 0;
      if (shape == 1) {
        const int64_t sty = kApBY * kApStarRows;
        const int64_t stiles = ((ox + kApBX - 1) / kApBX) * ((oy + sty - 1) / sty);
        zc = 64;
        while (zc > 8 && stiles * ((oz + zc - 1) / zc) < int64_t(6) * ctx->num_sms) zc /= 2;
        zc = std::min<int64_t>(zc, oz);
        grid = dim3(static_cast<unsigned>((ox + kApBX - 1) / kApBX), static_cast<unsigned>((oy + sty - 1) / sty),
                    static_cast<unsigned>((oz + zc - 1) / zc));
        smem = R == 1 ? ApStar<1>::kSmem : (R == 2 ? ApStar<2>::kSmem : ApStar<3>::kSmem);
        // one weight per distance (every +-d offset on every axis alike, as
        // in the isotropic Laplacians): the neighbours at a distance are
        // summed first, one multiply per distance
        bool sym = true;
        for (int d = 1; d <= r; ++d)
          for (int q = 0; q < 6; ++q)
            if (t.k[1 + (q / 2) * 2 * r + 2 * (d - 1) + (q & 1)] != t.k[1 + 2 * (d - 1)]) sym = false;
        if (sym)
          kern = R == 1 ? apply_star_kernel<1, true> : (R == 2 ? apply_star_kernel<2, true> : apply_star_kernel<3, true>);
        else
          kern = R == 1 ? apply_star_kernel<1, false>
                        : (R == 2 ? apply_star_kernel<2, false> : apply_star_kernel<3, false>);
      } else {
        zc = std::max<int64_t>(8, (oz * tiles + 8 * ctx->num_sms - 1) / (8 * ctx->num_sms));
        zc = std::min<int64_t>(zc, oz);
        grid = dim3(static_cast<unsigned>((ox + kApBX - 1) / kApBX), static_cast<unsigned>((oy + kApBY - 1) / kApBY),
                    static_cast<unsigned>((oz + zc - 1) / zc));
        smem = 2 * (2 * R + 1) * PL * static_cast<int>(sizeof(long long));
        kern = shape == 2 ? apply_fx_kernel<1, 2>
                          : (R == 1 ? apply_fx_kernel<1, 0> : (R == 2 ? apply_fx_kernel<2, 0> : apply_fx_kernel<3, 0>));
      }
      if (grid.y > 65535 || grid.z > 65535) return set_error(STENCIL_ERR_ARG, "apply_linear: grid too large");
      int rc = check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                          "apply smem attribute");
      if (rc) return rc;
      auto launch = [&](const ApPass& ps) {
        kern<<<grid, dim3(kApBX, kApBY), smem, st>>>(static_cast<const double*>(in.data),
                                                      static_cast<double*>(out.data), in.nx, in.ny, in.nz, in.sy,
                                                      in.sz, out.sy, out.sz, t, ps, static_cast<int>(zc));
        return check_cuda(cudaGetLastError(), "apply_linear fixed-point kernel");
      };
      // The scale: the first call on a context measures max|in| with a range
      // pass; later calls take the previous call's magnitude as the guess.
      // The pass records the magnitude it reads; a one-thread check keeps
      // its output only if that gives the same scale, otherwise a second
      // pass (launched every call, returning at once when not needed)
      // recomputes at the scale of what was read -- the output is a function
      // of the input alone, and a call whose magnitude keeps the previous
      // scale reads its input once.
      unsigned char* sc = ctx->scratch;
      auto* guess = reinterpret_cast<unsigned long long*>(sc + kScratchApplyGuess);
      auto* seen = reinterpret_cast<unsigned long long*>(sc + kScratchApplySeen);
      auto* final_bits = reinterpret_cast<unsigned long long*>(sc + kScratchApplyFinal);
      auto* redo = reinterpret_cast<uint32_t*>(sc + kScratchApplyRedo);
      const unsigned long long* used = guess;
      if (!ctx->apply_guess) {
        unsigned long long* mb = reinterpret_cast<unsigned long long*>(sc + kScratchApplyRange);
        rc = check_cuda(cudaMemsetAsync(mb, 0, 8, st), "apply range init");
        if (rc) return rc;
        const int64_t rows = (in.ny + 2) * (in.nz + 2);
        const int rblocks = static_cast<int>(std::min<int64_t>((rows + 7) / 8, 8 * ctx->num_sms));
        apply_range_kernel<<<rblocks, dim3(32, 8), 0, st>>>(static_cast<const double*>(in.data), in.nx, in.ny,
                                                             in.nz, in.sy, in.sz, mb);
        rc = check_cuda(cudaGetLastError(), "apply range kernel");
        if (rc) return rc;
        used = mb;
      }
      rc = check_cuda(cudaMemsetAsync(seen, 0, 8, st), "apply magnitude init");
      if (rc) return rc;
      rc = launch(ApPass{used, seen, nullptr, nullptr});
      if (rc) return rc;
      apply_check_kernel<<<1, 1, 0, st>>>(used, seen, t.sumk, final_bits, redo, guess);
      rc = check_cuda(cudaGetLastError(), "apply check kernel");
      if (rc) return rc;
      rc = launch(ApPass{final_bits, seen, redo, reinterpret_cast<uint32_t*>(sc + kScratchStatus)});
      if (rc) return rc;
      ctx->apply_guess = 1;
      return STENCIL_OK;
    }
  }
  LinearTerms t;
  t.n = npoints;
  t.r = r;
  for (int p = 0; p < npoints; ++p) {
    t.off[p] = offsets[3 * p] + offsets[3 * p + 1] * in.sy + offsets[3 * p + 2] * in.sz;
    t.c[p] = coeffs[p];
  }
  for (int p = npoints; p < kMaxLinearTerms; ++p) {
    t.off[p] = 0;
    t.c[p] = 0.0;
  }
  const int64_t ox = in.nx + 2 - 2 * r, oy = in.ny + 2 - 2 * r, oz = in.nz + 2 - 2 * r;
  const dim3 block(32, 8);
  const dim3 grid(static_cast<unsigned>((ox + 31) / 32), static_cast<unsigned>((oy + 7) / 8),
                  static_cast<unsigned>(std::min<int64_t>(oz, 65535)));
  if (grid.y > 65535) return set_error(STENCIL_ERR_ARG, "apply_linear: ny too large");
  apply_linear_kernel<<<grid, block, 0, st>>>(static_cast<const double*>(in.data), static_cast<double*>(out.data),
                                              in.nx, in.ny, in.nz, in.sy, in.sz, out.sy, out.sz, t);
  return check_cuda(cudaGetLastError(), "apply_linear kernel");
}

}  // namespace stencil
