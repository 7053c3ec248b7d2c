// net.cu -- the learned warm start: a small 3D U-Net that maps the source f of
// a Poisson problem to a starting iterate u0, trained on (f, converged u)
// pairs, with its own BF16 tensor-core kernels (FP32 accumulation) for
// inference and training.  The paper has no learned component; this is the
// warm-start pattern layered on its Jacobi solver.
//
// Architecture (per-level channels C[0..L-1], L <= 4): per level two 3x3x3
// convolutions with ReLU; 2x2x2 average pooling between encoder levels;
// nearest 2x upsampling between decoder levels, whose first convolution adds
// the encoder feature of the same level before its ReLU; a 1x1x1 output layer
// and a fixed separable [1,2,1]/4 filter (it all but removes the checkerboard
// mode, which plain Jacobi damps as slowly as the smoothest one).
// Activations and gradients are bfloat16, channels-last [z][y][x][c]; weights
// are kept in FP32 (Adam) and mirrored to bfloat16 in two layouts: W[co][k]
// with k = tap*Cin + ci (forward) and Wt[ci][k'] with k' = (26-tap)*Cout + co
// (the input gradient is the forward convolution with flipped, transposed
// weights).  The convolutions and weight gradients are implicit GEMMs on the
// tcgen05 tensor cores (conv_tc.cuh) where the layer's channels and row
// length allow it, and on mma.sync m16n8k16 otherwise (the one-channel first
// layer, grids with rows shorter than 16 voxels).
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include <cuda_bf16.h>

#include "conv_tc.cuh"
#include "internal.h"

namespace stencil {
namespace net {

using bf16 = __nv_bfloat16;

constexpr int kMaxLevels = 4;

__host__ __device__ constexpr int kpad(int cin) { return (27 * cin + 15) / 16 * 16; }

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
  return static_cast<uint32_t>(__bfloat16_as_ushort(lo)) |
         (static_cast<uint32_t>(__bfloat16_as_ushort(hi)) << 16);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

struct Vox {
  int z, y, x;
  bool ok;
};

__device__ __forceinline__ Vox vox_of(int64_t v, int D, int H, int W) {
  Vox r;
  r.ok = v < static_cast<int64_t>(D) * H * W;
  const int64_t hw = static_cast<int64_t>(H) * W;
  r.z = static_cast<int>(v / hw);
  const int64_t rem = v - static_cast<int64_t>(r.z) * hw;
  r.y = static_cast<int>(rem / W);
  r.x = static_cast<int>(rem - static_cast<int64_t>(r.y) * W);
  return r;
}

// Index of the neighbour of p at tap (dz,dy,dx) = (tap/9-1, tap/3%3-1, tap%3-1),
// or -1 outside the grid (zero padding).
__device__ __forceinline__ int64_t nbr(const Vox& p, int tap, int D, int H, int W) {
  const int z = p.z + tap / 9 - 1, y = p.y + (tap / 3) % 3 - 1, x = p.x + tap % 3 - 1;
  if (!p.ok || tap >= 27 || z < 0 || z >= D || y < 0 || y >= H || x < 0 || x >= W) return -1;
  return (static_cast<int64_t>(z) * H + y) * W + x;
}

// Two consecutive K entries (k, k+1) of the implicit-GEMM A row of voxel p.
template <int CIN>
__device__ __forceinline__ uint32_t a_pair(const bf16* __restrict__ in, const Vox& p, int k, int D, int H,
                                           int W) {
  if (CIN >= 2) {
    const int tap = k / CIN, ci = k - (k / CIN) * CIN;
    const int64_t q = nbr(p, tap, D, H, W);
    return q < 0 ? 0u : *reinterpret_cast<const uint32_t*>(in + q * CIN + ci);
  } else {
    const int64_t q0 = nbr(p, k, D, H, W), q1 = nbr(p, k + 1, D, H, W);
    const bf16 z = __float2bfloat16_rn(0.0f);
    return pack2(q0 < 0 ? z : in[q0], q1 < 0 ? z : in[q1]);
  }
}

// out[v, co] = epilogue( bias[co] + sum_k A[v, k] W[co, k] ), 64 voxels per
// CTA, 16 per warp, all COUT channels per warp.  Epilogue: + skip (bf16),
// ReLU, store bf16 (out) and/or FP32 (out32).
template <int CIN, int COUT, bool RELU, bool SKIP>
__global__ void __launch_bounds__(128)
    conv3_fwd_kernel(const bf16* __restrict__ in, const bf16* __restrict__ Wk, const float* __restrict__ bias,
                     const bf16* __restrict__ skip, bf16* __restrict__ out, float* __restrict__ out32, int D, int H,
                     int W) {
  constexpr int KP = kpad(CIN);
  constexpr int NT = COUT / 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int64_t vb = static_cast<int64_t>(blockIdx.x) * 64 + warp * 16;
  const Vox p0 = vox_of(vb + g, D, H, W), p1 = vox_of(vb + g + 8, D, H, W);
  float acc[NT][4];
#pragma unroll
  for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
  for (int k0 = 0; k0 < KP; k0 += 16) {
    uint32_t a[4];
    a[0] = a_pair<CIN>(in, p0, k0 + 2 * t, D, H, W);
    a[1] = a_pair<CIN>(in, p1, k0 + 2 * t, D, H, W);
    a[2] = a_pair<CIN>(in, p0, k0 + 2 * t + 8, D, H, W);
    a[3] = a_pair<CIN>(in, p1, k0 + 2 * t + 8, D, H, W);
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const bf16* wr = Wk + static_cast<int64_t>(j * 8 + g) * KP + k0 + 2 * t;
      mma16816(acc[j], a, *reinterpret_cast<const uint32_t*>(wr), *reinterpret_cast<const uint32_t*>(wr + 8));
    }
  }
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const int co = j * 8 + 2 * t;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t v = vb + g + 8 * h;
      if (!(h ? p1.ok : p0.ok)) continue;
      float v0 = acc[j][2 * h] + bias[co], v1 = acc[j][2 * h + 1] + bias[co + 1];
      if (SKIP) {
        v0 += __bfloat162float(skip[v * COUT + co]);
        v1 += __bfloat162float(skip[v * COUT + co + 1]);
      }
      if (RELU) {
        v0 = fmaxf(v0, 0.0f);
        v1 = fmaxf(v1, 0.0f);
      }
      if (out) *reinterpret_cast<uint32_t*>(out + v * COUT + co) = pack2(__float2bfloat16_rn(v0), __float2bfloat16_rn(v1));
      if (out32) {
        out32[v * COUT + co] = v0;
        out32[v * COUT + co + 1] = v1;
      }
    }
  }
}

// Weight-gradient partials of one tap over one chunk of voxels:
//   P[chunk][co][tap*CIN + ci] = sum_{v in chunk} g[v, co] * in[v + tap, ci].
// GEMM with M = COUT, N = CIN, K = voxels; four warps split the chunk and
// their tiles are summed in warp order.
template <int CIN, int COUT>
__global__ void __launch_bounds__(128)
    conv3_wgrad_kernel(const bf16* __restrict__ in, const bf16* __restrict__ gr, float* __restrict__ part,
                       int D, int H, int W, int chunk) {
  constexpr int KP = kpad(CIN);
  constexpr int MT = COUT / 16;
  constexpr int NT = (CIN + 7) / 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int tap = blockIdx.y;
  const int64_t V = static_cast<int64_t>(D) * H * W;
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * chunk;
  const int64_t c1 = min(c0 + chunk, V);
  const int per_warp = (chunk + 3) / 4;
  const int64_t w0 = c0 + static_cast<int64_t>(warp) * per_warp;
  const int64_t w1 = min(w0 + per_warp, c1);
  float acc[MT][NT][4];
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0.0f;
  const bf16 zero = __float2bfloat16_rn(0.0f);
  for (int64_t vb = w0; vb < w1; vb += 16) {
    int64_t vv[4];
    vv[0] = vb + 2 * t; vv[1] = vv[0] + 1; vv[2] = vv[0] + 8; vv[3] = vv[0] + 9;
    int64_t q[4];
    bool ok[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      ok[e] = vv[e] < w1;
      const Vox p = vox_of(ok[e] ? vv[e] : 0, D, H, W);
      q[e] = ok[e] ? nbr(p, tap, D, H, W) : -1;
    }
    uint32_t a[MT][4];
#pragma unroll
    for (int i = 0; i < MT; ++i) {
      const int co = i * 16 + g;
      bf16 x[8];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        x[e] = ok[e] ? gr[vv[e] * COUT + co] : zero;
        x[4 + e] = ok[e] ? gr[vv[e] * COUT + co + 8] : zero;
      }
      a[i][0] = pack2(x[0], x[1]);   // (co, v0..v1)
      a[i][1] = pack2(x[4], x[5]);   // (co+8, v0..v1)
      a[i][2] = pack2(x[2], x[3]);   // (co, v0+8..)
      a[i][3] = pack2(x[6], x[7]);   // (co+8, v0+8..)
    }
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const int ci = j * 8 + g;
      bf16 y[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) y[e] = (q[e] >= 0 && ci < CIN) ? in[q[e] * CIN + ci] : zero;
      const uint32_t b0 = pack2(y[0], y[1]), b1 = pack2(y[2], y[3]);
#pragma unroll
      for (int i = 0; i < MT; ++i) mma16816(acc[i][j], a[i], b0, b1);
    }
  }
  // sum the four warps' tiles in warp order through shared memory
  __shared__ float red[COUT * NT * 8];
  for (int w = 0; w < 4; ++w) {
    if (warp == w) {
#pragma unroll
      for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int co = i * 16 + g + ((e & 2) ? 8 : 0);
            const int ci = j * 8 + 2 * t + (e & 1);
            const int idx = co * (NT * 8) + ci;
            red[idx] = (w == 0 ? 0.0f : red[idx]) + acc[i][j][e];
          }
    }
    __syncthreads();
  }
  float* P = part + static_cast<int64_t>(blockIdx.x) * COUT * KP;
  for (int idx = threadIdx.x; idx < COUT * NT * 8; idx += 128) {
    const int co = idx / (NT * 8), ci = idx - co * (NT * 8);
    if (ci >= CIN) continue;
    P[co * KP + tap * CIN + ci] = red[idx];
  }
}

// dW[co][k] += sum over chunks (in chunk order) of P[chunk][co][k], for
// k < kvalid = 27*CIN (P rows are kp long, dW rows kvalid long).
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, float* __restrict__ dW, int cout, int kp,
                                    int kvalid, int chunks) {
  const int64_t n = static_cast<int64_t>(cout) * kp;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t co = i / kp, k = i - co * kp;
    if (k >= kvalid) continue;
    float s = 0.0f;
    for (int c = 0; c < chunks; ++c) s += part[static_cast<int64_t>(c) * n + i];
    dW[co * kvalid + k] += s;
  }
}

// Per-channel sums over voxels of a channels-last bf16 tensor, for the bias
// gradients (GY = false: part[b][c] = sum_v x[v][c]) and the output layer's
// weight gradient (GY = true: part[b][c] = sum_v x[v][c] gy[v] for c < C and
// part[b][C] = sum_v gy[v]).  Block b covers voxels [b, b+1) * kSumChunk;
// its 256 threads are (voxel lane, channel pair), so one pass of the block
// reads 256 consecutive bf16 pairs; the lanes are then added in lane order
// (deterministic).  db[c] += sum over blocks in order (chan_sum_reduce).
constexpr int kSumChunk = 2048;

template <int C, bool GY>
__global__ void __launch_bounds__(256)
    chan_sum_kernel(const bf16* __restrict__ x, const float* __restrict__ gy, float* __restrict__ part, int64_t V) {
  constexpr int P = C / 2, LANES = 256 / P, OUT = GY ? C + 1 : C;
  __shared__ float red[3][256];
  const int cp = threadIdx.x % P, vl = threadIdx.x / P;
  const int64_t v0 = static_cast<int64_t>(blockIdx.x) * kSumChunk;
  const int64_t v1 = min(v0 + kSumChunk, V);
  float s0 = 0.0f, s1 = 0.0f, sg = 0.0f;
  for (int64_t v = v0 + vl; v < v1; v += LANES) {
    const __nv_bfloat162 b = reinterpret_cast<const __nv_bfloat162*>(x + v * C)[cp];
    if (GY) {
      const float g = gy[v];
      s0 += __low2float(b) * g;
      s1 += __high2float(b) * g;
      sg += g;
    } else {
      s0 += __low2float(b);
      s1 += __high2float(b);
    }
  }
  red[0][threadIdx.x] = s0;
  red[1][threadIdx.x] = s1;
  red[2][threadIdx.x] = sg;
  __syncthreads();
  if (threadIdx.x < P) {
    float t0 = 0.0f, t1 = 0.0f, tg = 0.0f;
    for (int l = 0; l < LANES; ++l) {
      t0 += red[0][l * P + threadIdx.x];
      t1 += red[1][l * P + threadIdx.x];
      tg += red[2][l * P + threadIdx.x];
    }
    float* o = part + static_cast<int64_t>(blockIdx.x) * OUT;
    o[2 * threadIdx.x] = t0;
    o[2 * threadIdx.x + 1] = t1;
    if (GY && threadIdx.x == 0) o[C] = tg;
  }
}

__global__ void chan_sum_reduce_kernel(const float* __restrict__ part, float* __restrict__ db, int C, int blocks) {
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    float s = 0.0f;
    for (int b = 0; b < blocks; ++b) s += part[static_cast<int64_t>(b) * C + c];
    db[c] += s;
  }
}

// The pooling, upsampling and ReLU-mask kernels move 8 channels (16 bytes)
// per thread; channel counts are multiples of 16.
__device__ __forceinline__ void load8(const bf16* p, float (&f)[8]) {
  const uint4 q = *reinterpret_cast<const uint4*>(p);
  const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    f[2 * i] = __uint_as_float(w[i] << 16);
    f[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}

__device__ __forceinline__ void store8(bf16* p, const float (&f)[8]) {
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) w[i] = pack2(__float2bfloat16_rn(f[2 * i]), __float2bfloat16_rn(f[2 * i + 1]));
  *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}

// 2x2x2 average pooling: coarse (D/2, H/2, W/2) from the fine grid.
__global__ void pool2_kernel(const bf16* __restrict__ in, bf16* __restrict__ out, int D, int H, int W, int C) {
  const uint32_t d = D / 2, h = H / 2, w = W / 2, G = C / 8;
  const uint32_t n = d * h * w * G;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t g = i % G, v = i / G;
    const uint32_t x = v % w, y = (v / w) % h, z = v / (w * h);
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          float f[8];
          load8(in + (((2 * z + dz) * static_cast<uint64_t>(H) + 2 * y + dy) * W + 2 * x + dx) * C + 8 * g, f);
#pragma unroll
          for (int k = 0; k < 8; ++k) s[k] += f[k];
        }
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] *= 0.125f;
    store8(out + static_cast<uint64_t>(v) * C + 8 * g, s);
  }
}

// Adjoint of pool2: every fine voxel gets g/8 of its block.
__global__ void pool2_bwd_kernel(const bf16* __restrict__ g, bf16* __restrict__ out, int D, int H, int W, int C) {
  const uint32_t G = C / 8;
  const uint32_t n = static_cast<uint32_t>(D) * H * W * G;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t c8 = i % G, v = i / G;
    const uint32_t x = v % W, y = (v / W) % H, z = v / (W * H);
    float f[8];
    load8(g + (((z / 2) * static_cast<uint64_t>(H / 2) + y / 2) * (W / 2) + x / 2) * C + 8 * c8, f);
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k] *= 0.125f;
    store8(out + static_cast<uint64_t>(v) * C + 8 * c8, f);
  }
}

// Nearest 2x upsampling: fine grid (D, H, W) from the coarse one.
__global__ void up2_kernel(const bf16* __restrict__ in, bf16* __restrict__ out, int D, int H, int W, int C) {
  const uint32_t G = C / 8;
  const uint32_t n = static_cast<uint32_t>(D) * H * W * G;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t c8 = i % G, v = i / G;
    const uint32_t x = v % W, y = (v / W) % H, z = v / (W * H);
    *reinterpret_cast<uint4*>(out + static_cast<uint64_t>(v) * C + 8 * c8) = *reinterpret_cast<const uint4*>(
        in + (((z / 2) * static_cast<uint64_t>(H / 2) + y / 2) * (W / 2) + x / 2) * C + 8 * c8);
  }
}

// Adjoint of up2: coarse voxel gets the sum of its 8 fine gradients.
__global__ void up2_bwd_kernel(const bf16* __restrict__ g, bf16* __restrict__ out, int d, int h, int w, int C) {
  const uint32_t H = 2 * h, W = 2 * w, G = C / 8;
  const uint32_t n = static_cast<uint32_t>(d) * h * w * G;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t c8 = i % G, v = i / G;
    const uint32_t x = v % w, y = (v / w) % h, z = v / (w * h);
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          float f[8];
          load8(g + (((2 * z + dz) * static_cast<uint64_t>(H) + 2 * y + dy) * W + 2 * x + dx) * C + 8 * c8, f);
#pragma unroll
          for (int k = 0; k < 8; ++k) s[k] += f[k];
        }
    store8(out + static_cast<uint64_t>(v) * C + 8 * c8, s);
  }
}

// g_out = (g + addend) * (act > 0), bf16 (addend may be null); n a multiple of 8.
__global__ void relu_bwd_kernel(const bf16* __restrict__ g, const bf16* __restrict__ addend,
                                const bf16* __restrict__ act, bf16* __restrict__ out, int64_t n) {
  for (int64_t i = 8 * (blockIdx.x * int64_t(blockDim.x) + threadIdx.x); i < n;
       i += 8 * int64_t(gridDim.x) * blockDim.x) {
    float v[8], a[8];
    load8(g + i, v);
    load8(act + i, a);
    if (addend) {
      float e[8];
      load8(addend + i, e);
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] += e[k];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = a[k] > 0.0f ? v[k] : 0.0f;
    store8(out + i, v);
  }
}

// The first layer (one input channel) is too thin for the tensor cores:
// 27 products per output channel.  Both kernels below use FP32 FMAs on the
// bf16 inputs and bf16 weights (exact products), one voxel per thread.
//
// Neighbour offsets of voxel (x, y, z) in tap order (9 dz + 3 dy + dx),
// with -1 for taps outside the grid.
__device__ __forceinline__ void first_layer_taps(const bf16* __restrict__ in, uint32_t v, int D, int H, int W,
                                                 float (&xv)[27]) {
  const uint32_t x = v % W, y = (v / W) % H, z = v / (W * H);
#pragma unroll
  for (int dz = 0; dz < 3; ++dz)
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
      const int zz = static_cast<int>(z) + dz - 1, yy = static_cast<int>(y) + dy - 1;
      const bool row_ok = zz >= 0 && zz < D && yy >= 0 && yy < H;
      const bf16* r = in + (static_cast<int64_t>(zz) * H + yy) * W;
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        const int xx = static_cast<int>(x) + dx - 1;
        xv[9 * dz + 3 * dy + dx] = (row_ok && xx >= 0 && xx < W) ? __bfloat162float(r[xx]) : 0.0f;
      }
    }
}

// out[v][co] = ReLU(b[co] + sum_tap x[v + tap] W[co][tap]), COUT channels.
template <int COUT>
__global__ void __launch_bounds__(256) conv1_fwd_kernel(const bf16* __restrict__ in, const bf16* __restrict__ Wf,
                                                        const float* __restrict__ bias, bf16* __restrict__ out,
                                                        int D, int H, int W) {
  constexpr int KP = kpad(1);
  __shared__ float ws[COUT][27];
  for (int i = threadIdx.x; i < COUT * 27; i += blockDim.x) ws[i / 27][i % 27] = __bfloat162float(Wf[(i / 27) * KP + i % 27]);
  __syncthreads();
  const uint32_t V = static_cast<uint32_t>(D) * H * W;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
    float xv[27];
    first_layer_taps(in, v, D, H, W, xv);
#pragma unroll 1
    for (int q = 0; q < COUT / 8; ++q) {
      float f[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int co = 8 * q + k;
        float a = 0.0f;
#pragma unroll
        for (int t = 0; t < 27; ++t) a = fmaf(xv[t], ws[co][t], a);
        f[k] = fmaxf(a + bias[co], 0.0f);
      }
      store8(out + static_cast<uint64_t>(v) * COUT + 8 * q, f);
    }
  }
}

// Weight-gradient partials of the first layer over chunks of voxels:
//   P[chunk][co][tap] = sum_{v in chunk} g[v][co] x[v + tap].
// 256 threads: warp w handles output channels 4 (w / 2) .. +3 for the
// voxels of lane slot (w % 2) * 32 + lane, stride 64; the 64 slots are then
// added in a fixed order (shuffle tree, then the two warps).
template <int COUT>
__global__ void __launch_bounds__(256) conv1_wgrad_kernel(const bf16* __restrict__ in, const bf16* __restrict__ g,
                                                          float* __restrict__ part, int D, int H, int W, int chunk) {
  static_assert(COUT == 16, "four channels per warp pair, eight warps");
  constexpr int KP = kpad(1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cg = warp >> 1, slot = (warp & 1) * 32 + lane;
  const uint32_t V = static_cast<uint32_t>(D) * H * W;
  const uint32_t c0 = blockIdx.x * static_cast<uint32_t>(chunk);
  const uint32_t c1 = min(c0 + static_cast<uint32_t>(chunk), V);
  float acc[4][27];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int t = 0; t < 27; ++t) acc[c][t] = 0.0f;
  for (uint32_t v = c0 + slot; v < c1; v += 64) {
    float xv[27];
    first_layer_taps(in, v, D, H, W, xv);
    const uint2 gq = *reinterpret_cast<const uint2*>(g + static_cast<uint64_t>(v) * COUT + 4 * cg);
    const float gv[4] = {__uint_as_float(gq.x << 16), __uint_as_float(gq.x & 0xffff0000u),
                         __uint_as_float(gq.y << 16), __uint_as_float(gq.y & 0xffff0000u)};
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int t = 0; t < 27; ++t) acc[c][t] = fmaf(gv[c], xv[t], acc[c][t]);
  }
  __shared__ float red[8][4][27];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int t = 0; t < 27; ++t) {
      float a = acc[c][t];
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) red[warp][c][t] = a;
    }
  __syncthreads();
  float* P = part + static_cast<int64_t>(blockIdx.x) * COUT * KP;
  for (int i = threadIdx.x; i < COUT * 27; i += blockDim.x) {
    const int co = i / 27, t = i % 27, w0 = 2 * (co / 4);
    P[co * KP + t] = red[w0][co % 4][t] + red[w0 + 1][co % 4][t];
  }
}

// Output layer: y[v] = b + sum_c h[v][c] w[c]  (FP32).
__global__ void out_fwd_kernel(const bf16* __restrict__ h, const float* __restrict__ w, const float* __restrict__ b,
                               float* __restrict__ y, int64_t V, int C) {
  for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < V; v += int64_t(gridDim.x) * blockDim.x) {
    float s = b[0];
    for (int c = 0; c < C; ++c) s = fmaf(__bfloat162float(h[v * C + c]), w[c], s);
    y[v] = s;
  }
}

// gy = 2 (y - t) / V and the loss partials per block.
__global__ void mse_bwd_kernel(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ gy,
                               float* __restrict__ loss_part, int64_t V, int chunk) {
  const int64_t v0 = static_cast<int64_t>(blockIdx.x) * chunk;
  const int64_t v1 = min(v0 + chunk, V);
  float s = 0.0f;
  for (int64_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
    const float d = y[v] - t[v];
    s = fmaf(d, d, s);
    gy[v] = 2.0f * d / static_cast<float>(V);
  }
  __shared__ float red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
}

// g_h[v][c] = gy[v] * w[c] (bf16): the gradient entering the last 3x3x3 layer.
__global__ void out_bwd_kernel(const float* __restrict__ gy, const float* __restrict__ w, bf16* __restrict__ gh,
                               int64_t V, int C) {
  for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < V; v += int64_t(gridDim.x) * blockDim.x)
    for (int c = 0; c < C; ++c) gh[v * C + c] = __float2bfloat16_rn(gy[v] * w[c]);
}

// The network's fixed last layer: the separable [1,2,1]/4 filter along each
// axis of an n^3 FP32 field, zero outside (27 taps, weights (a b c)/64 with
// a, b, c in {1, 2}).  Symmetric, so the backward pass applies it too.
__global__ void smooth121_kernel(const float* __restrict__ in, float* __restrict__ out, int n) {
  const int64_t V = static_cast<int64_t>(n) * n * n;
  for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < V; v += int64_t(gridDim.x) * blockDim.x) {
    const int x = static_cast<int>(v % n), y = static_cast<int>((v / n) % n), z = static_cast<int>(v / (int64_t(n) * n));
    float s = 0.0f;
    for (int dz = -1; dz <= 1; ++dz) {
      const int zz = z + dz;
      if (zz < 0 || zz >= n) continue;
      const float wz = dz == 0 ? 2.0f : 1.0f;
      for (int dy = -1; dy <= 1; ++dy) {
        const int yy = y + dy;
        if (yy < 0 || yy >= n) continue;
        const float wy = dy == 0 ? 2.0f : 1.0f;
        for (int dx = -1; dx <= 1; ++dx) {
          const int xx = x + dx;
          if (xx < 0 || xx >= n) continue;
          const float wx = dx == 0 ? 2.0f : 1.0f;
          s = fmaf(wz * wy * wx, in[(static_cast<int64_t>(zz) * n + yy) * n + xx], s);
        }
      }
    }
    out[v] = s * (1.0f / 64.0f);
  }
}

// Adam on the FP32 master parameters, then the bf16 mirrors in both layouts.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2, float gscale) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const float gr = grad[i] * gscale;
    const float mi = b1 * m[i] + (1.0f - b1) * gr;
    const float vi = b2 * v[i] + (1.0f - b2) * gr * gr;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// bf16 mirrors of a 3x3x3 layer: Wf[co][k] (k = tap*cin + ci, zero past 27 cin)
// and Wt[ci][k'] (k' = (26-tap)*cout + co) from the FP32 W[co][tap*cin+ci].
__global__ void mirror_kernel(const float* __restrict__ w, bf16* __restrict__ wf, bf16* __restrict__ wt, int cin,
                              int cout) {
  const int kpf = kpad(cin), kpt = kpad(cout);
  const int64_t nf = static_cast<int64_t>(cout) * kpf;
  const int64_t nt = static_cast<int64_t>(cin) * kpt;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < nf + nt; i += int64_t(gridDim.x) * blockDim.x) {
    if (i < nf) {
      const int co = static_cast<int>(i / kpf), k = static_cast<int>(i % kpf);
      wf[i] = __float2bfloat16_rn(k < 27 * cin ? w[static_cast<int64_t>(co) * 27 * cin + k] : 0.0f);
    } else if (wt) {
      const int64_t j = i - nf;
      const int ci = static_cast<int>(j / kpt), k = static_cast<int>(j % kpt);
      float val = 0.0f;
      if (k < 27 * cout) {
        const int tap = 26 - k / cout, co = k % cout;
        val = w[static_cast<int64_t>(co) * 27 * cin + tap * cin + ci];
      }
      wt[j] = __float2bfloat16_rn(val);
    }
  }
}

// x0 = bf16(f / s) on the interior of an F64 halo grid (channels-last, C=1),
// and u[interior] = y * scale (halo untouched).
__global__ void input_kernel(const double* __restrict__ f, int64_t sy, int64_t sz, int n,
                             const double* __restrict__ rms, bf16* __restrict__ x) {
  const int64_t V = static_cast<int64_t>(n) * n * n;
  const double inv = rms[0] > 0.0 ? 1.0 / rms[0] : 0.0;
  for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < V; v += int64_t(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(v % n), j = static_cast<int>((v / n) % n), k = static_cast<int>(v / (int64_t(n) * n));
    x[v] = __float2bfloat16_rn(static_cast<float>(f[(i + 1) + (j + 1) * sy + (k + 1) * sz] * inv));
  }
}

__global__ void output_kernel(const float* __restrict__ y, double* __restrict__ u, int64_t sy, int64_t sz, int n,
                              const double* __restrict__ rms, double s0) {
  const int64_t V = static_cast<int64_t>(n) * n * n;
  const double scale = rms[0] * s0;
  for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < V; v += int64_t(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(v % n), j = static_cast<int>((v / n) % n), k = static_cast<int>(v / (int64_t(n) * n));
    u[(i + 1) + (j + 1) * sy + (k + 1) * sz] = static_cast<double>(y[v]) * scale;
  }
}

// Normalised target t = u / scale (FP32, channels-last).
__global__ void target_kernel(const double* __restrict__ u, int64_t sy, int64_t sz, int n,
                              const double* __restrict__ rms, double s0, float* __restrict__ t) {
  const int64_t V = static_cast<int64_t>(n) * n * n;
  const double inv = rms[0] > 0.0 ? 1.0 / (rms[0] * s0) : 0.0;
  for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < V; v += int64_t(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(v % n), j = static_cast<int>((v / n) % n), k = static_cast<int>(v / (int64_t(n) * n));
    t[v] = static_cast<float>(u[(i + 1) + (j + 1) * sy + (k + 1) * sz] * inv);
  }
}

// Sum of squares of the interior of an F64 grid: per-block partials.
__global__ void sumsq_kernel(const double* __restrict__ f, int64_t sy, int64_t sz, int n, double* __restrict__ part) {
  const int64_t V = static_cast<int64_t>(n) * n * n;
  double s = 0.0;
  for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < V; v += int64_t(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(v % n), j = static_cast<int>((v / n) % n), k = static_cast<int>(v / (int64_t(n) * n));
    const double a = f[(i + 1) + (j + 1) * sy + (k + 1) * sz];
    s = fma(a, a, s);
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// rms = sqrt(sum of part[0..blocks) / V), in block order (one thread).
__global__ void rms_kernel(const double* __restrict__ part, int blocks, double V, double* __restrict__ rms) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < blocks; ++b) s += part[b];
  rms[0] = sqrt(s / V);
}

}  // namespace net
}  // namespace stencil

// ---------------------------------------------------------------------------
// Host side: the network object, its passes and the C ABI.
// ---------------------------------------------------------------------------
namespace stencil {
namespace net {
namespace {

// Launch helpers with the (cin, cout) pairs the U-Nets here use.
#define STENCIL_NET_PAIRS(X) \
  X(1, 16) X(1, 32) X(16, 16) X(16, 32) X(16, 64) X(32, 16) X(32, 32) X(32, 64) X(64, 16) X(64, 32) X(64, 64)

int blocks_for(int64_t n, int per = 256) {
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((n + per - 1) / per, 8192)));
}

// tcgen05 path: 128-voxel tiles of whole rows (W divides 128, 128/W rows of
// one plane), CIN and COUT in {16, 32, 64}.
bool tc_eligible(int cin, int cout, int D, int H, int W) {
  (void)D;
  if (cin < 16 || cout < 16) return false;
  if (W < 16 || W > 128 || 128 % W != 0) return false;
  const int hb = 128 / W;
  return H % hb == 0;
}

template <int CIN, int COUT>
int launch_conv_tc(bool relu, bool skip, const bf16* in, const bf16* w, const float* bias, const bf16* sk, bf16* out,
                   int D, int H, int W, uint32_t* status, cudaStream_t st) {
  constexpr int S = 4;
  using Cfg = TcCfg<CIN, COUT, S>;
  TcParams p;
  const CUtensorMapSwizzle swz = CIN == 16 ? CU_TENSOR_MAP_SWIZZLE_32B
                                 : CIN == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                                             : CU_TENSOR_MAP_SWIZZLE_128B;
  const uint64_t dims_in[4] = {static_cast<uint64_t>(CIN), static_cast<uint64_t>(W), static_cast<uint64_t>(H),
                               static_cast<uint64_t>(D)};
  const uint64_t str_in[3] = {static_cast<uint64_t>(CIN) * 2, static_cast<uint64_t>(W) * CIN * 2,
                              static_cast<uint64_t>(H) * W * CIN * 2};
  const uint32_t box_in[4] = {static_cast<uint32_t>(CIN), static_cast<uint32_t>(W), static_cast<uint32_t>(128 / W), 1};
  int rc = encode_tiled(&p.tm_in, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(in), dims_in, str_in, box_in,
                        swz);
  if (rc) return rc;
  const uint64_t dims_w[2] = {static_cast<uint64_t>(27 * CIN), static_cast<uint64_t>(COUT)};
  const uint64_t str_w[1] = {static_cast<uint64_t>(kpad(CIN)) * 2};
  const uint32_t box_w[2] = {static_cast<uint32_t>(CIN), static_cast<uint32_t>(COUT)};
  rc = encode_tiled(&p.tm_w, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(w), dims_w, str_w, box_w, swz);
  if (rc) return rc;
  p.bias = bias;
  p.skip = sk;
  p.out = out;
  p.D = D; p.H = H; p.W = W; p.HB = 128 / W; p.ZB = 1;
  p.status = status;
  const int64_t V = static_cast<int64_t>(D) * H * W;
  const int grid = static_cast<int>(V / 128);
  auto go = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return check_cuda(e, "conv tc attribute");
    kern<<<grid, 128, Cfg::SMEM, st>>>(p);
    return check_cuda(cudaGetLastError(), "conv tc launch");
  };
  if (relu && skip) return go(conv3_tc_kernel<CIN, COUT, S, true, true>);
  if (relu) return go(conv3_tc_kernel<CIN, COUT, S, true, false>);
  return go(conv3_tc_kernel<CIN, COUT, S, false, false>);
}

// The row kernel (grids with 128-voxel rows).  Returns STENCIL_OK, an error,
// or 1 when its tensor maps cannot be encoded (the caller then uses
// conv3_tc_kernel).
template <int CIN, int COUT>
int launch_conv_row(bool relu, bool skip, const bf16* in, const bf16* w, const float* bias, const bf16* sk,
                    bf16* out, int D, int H, int num_sms, uint32_t* status, cudaStream_t st) {
  using Cfg = RowCfg<CIN, COUT>;
  RowParams p;
  const uint64_t dims_in[5] = {8, static_cast<uint64_t>(CIN / 8), 128, static_cast<uint64_t>(H),
                               static_cast<uint64_t>(D)};
  const uint64_t str_in[4] = {16, static_cast<uint64_t>(CIN) * 2, 128ull * CIN * 2,
                              static_cast<uint64_t>(H) * 128 * CIN * 2};
  const uint32_t box_in[5] = {8, 1, static_cast<uint32_t>(Cfg::BOXW), 3, 1};
  if (encode_tiled(&p.tm_in, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16*>(in), dims_in, str_in, box_in,
                   CU_TENSOR_MAP_SWIZZLE_NONE))
    return 1;
  const uint64_t dims_w[3] = {8, static_cast<uint64_t>(COUT), static_cast<uint64_t>(Cfg::KG)};
  const uint64_t str_w[2] = {static_cast<uint64_t>(kpad(CIN)) * 2, 16};
  const uint32_t box_w[3] = {8, static_cast<uint32_t>(COUT), static_cast<uint32_t>(Cfg::KG)};
  if (encode_tiled(&p.tm_w, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16*>(w), dims_w, str_w, box_w,
                   CU_TENSOR_MAP_SWIZZLE_NONE))
    return 1;
  p.bias = bias;
  p.skip = sk;
  p.out = out;
  p.D = D;
  p.H = H;
  p.status = status;
  auto go = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return check_cuda(e, "conv row attribute");
    // two CTAs per SM: shared memory allows it for 16 input channels, and
    // the CTAs never wait on one another (extra ones simply run later)
    const int grid = std::max(1, std::min(D * H, 2 * num_sms));
    kern<<<grid, 192, Cfg::SMEM, st>>>(p);
    return check_cuda(cudaGetLastError(), "conv row launch");
  };
  if (relu && skip) return go(conv3_row_tc_kernel<CIN, COUT, true, true>);
  if (relu) return go(conv3_row_tc_kernel<CIN, COUT, true, false>);
  return go(conv3_row_tc_kernel<CIN, COUT, false, false>);
}

// tc_status: device status word of the tcgen05 path's bounded waits, or null
// to use the mma.sync kernel for every layer.
int launch_conv(int cin, int cout, bool relu, bool skip, const bf16* in, const bf16* w, const float* bias,
                const bf16* sk, bf16* out, int D, int H, int W, uint32_t* tc_status, int num_sms, cudaStream_t st) {
  const int64_t V = static_cast<int64_t>(D) * H * W;
  // 16 input channels: the row kernel (at 32 its two row stages need 150 KB
  // of shared memory, one CTA per SM, and the tile kernel is faster)
  if (tc_status && W == 128 && cin == 16 && (cout == 16 || cout == 32)) {
    int rc = 1;
    if (cout == 16) rc = launch_conv_row<16, 16>(relu, skip, in, w, bias, sk, out, D, H, num_sms, tc_status, st);
    else rc = launch_conv_row<16, 32>(relu, skip, in, w, bias, sk, out, D, H, num_sms, tc_status, st);
    if (rc != 1) return rc;
  }
  if (tc_status && tc_eligible(cin, cout, D, H, W)) {
#define X(CI, CO) \
    if (cin == CI && cout == CO) return launch_conv_tc<CI, CO>(relu, skip, in, w, bias, sk, out, D, H, W, tc_status, st);
    X(16, 16) X(16, 32) X(16, 64) X(32, 16) X(32, 32) X(32, 64) X(64, 16) X(64, 32) X(64, 64)
#undef X
  }
  if (cin == 1 && (cout == 16 || cout == 32 || cout == 64) && relu && !skip) {
    const int g1 = static_cast<int>(std::min<int64_t>((V + 255) / 256, 16 * num_sms));
    if (cout == 16) conv1_fwd_kernel<16><<<g1, 256, 0, st>>>(in, w, bias, out, D, H, W);
    else if (cout == 32) conv1_fwd_kernel<32><<<g1, 256, 0, st>>>(in, w, bias, out, D, H, W);
    else conv1_fwd_kernel<64><<<g1, 256, 0, st>>>(in, w, bias, out, D, H, W);
    return check_cuda(cudaGetLastError(), "first-layer conv");
  }
  const int grid = static_cast<int>((V + 63) / 64);
#define X(CI, CO)                                                                                           \
  if (cin == CI && cout == CO) {                                                                           \
    if (relu && skip)                                                                                      \
      conv3_fwd_kernel<CI, CO, true, true><<<grid, 128, 0, st>>>(in, w, bias, sk, out, nullptr, D, H, W);  \
    else if (relu)                                                                                         \
      conv3_fwd_kernel<CI, CO, true, false><<<grid, 128, 0, st>>>(in, w, bias, sk, out, nullptr, D, H, W); \
    else                                                                                                   \
      conv3_fwd_kernel<CI, CO, false, false><<<grid, 128, 0, st>>>(in, w, bias, sk, out, nullptr, D, H, W); \
    return check_cuda(cudaGetLastError(), "conv3 fwd");                                                    \
  }
  STENCIL_NET_PAIRS(X)
#undef X
  return set_error(STENCIL_ERR_ARG, "wsnet: no convolution kernel for %d -> %d channels", cin, cout);
}

constexpr int kWgradChunk = 8192;

template <int CIN, int COUT>
int launch_wgrad_tc(const bf16* in, const bf16* g, float* part, int chunks, int D, int H, int W, uint32_t* status,
                    cudaStream_t st) {
  using Cfg = WgCfg<CIN, COUT>;
  WgParams p;
  auto swz = [](int c) {
    return c == 16 ? CU_TENSOR_MAP_SWIZZLE_32B : c == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
  };
  const int hb = 128 / W;
  const uint64_t dims_in[4] = {static_cast<uint64_t>(CIN), static_cast<uint64_t>(W), static_cast<uint64_t>(H),
                               static_cast<uint64_t>(D)};
  const uint64_t str_in[3] = {static_cast<uint64_t>(CIN) * 2, static_cast<uint64_t>(W) * CIN * 2,
                              static_cast<uint64_t>(H) * W * CIN * 2};
  const uint32_t box_in[4] = {static_cast<uint32_t>(CIN), static_cast<uint32_t>(W), static_cast<uint32_t>(hb), 1};
  int rc = encode_tiled(&p.tm_in, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(in), dims_in, str_in, box_in,
                        swz(CIN));
  if (rc) return rc;
  const uint64_t dims_g[4] = {static_cast<uint64_t>(COUT), static_cast<uint64_t>(W), static_cast<uint64_t>(H),
                              static_cast<uint64_t>(D)};
  const uint64_t str_g[3] = {static_cast<uint64_t>(COUT) * 2, static_cast<uint64_t>(W) * COUT * 2,
                             static_cast<uint64_t>(H) * W * COUT * 2};
  const uint32_t box_g[4] = {static_cast<uint32_t>(COUT), static_cast<uint32_t>(W), static_cast<uint32_t>(hb), 1};
  rc = encode_tiled(&p.tm_g, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(g), dims_g, str_g, box_g,
                    swz(COUT));
  if (rc) return rc;
  p.part = part;
  p.kp = kpad(CIN);
  p.D = D; p.H = H; p.W = W; p.HB = hb;
  const int64_t V = static_cast<int64_t>(D) * H * W;
  p.tiles = static_cast<int>(V / 128);
  p.chunk_tiles = kWgradChunk / 128;
  p.status = status;
  const dim3 grid(chunks, (27 + Cfg::TG - 1) / Cfg::TG);
  auto kern = wgrad_tc_kernel<CIN, COUT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return check_cuda(e, "wgrad tc attribute");
  kern<<<grid, 128, Cfg::SMEM, st>>>(p);
  return check_cuda(cudaGetLastError(), "wgrad tc launch");
}

// tc_status: as for launch_conv (null: the mma.sync kernel).
int launch_wgrad(int cin, int cout, const bf16* in, const bf16* g, float* part, float* dW, int D, int H, int W,
                 uint32_t* tc_status, cudaStream_t st) {
  const int64_t V = static_cast<int64_t>(D) * H * W;
  const int chunks = static_cast<int>((V + kWgradChunk - 1) / kWgradChunk);
  if (cin == 1 && cout == 16) {
    conv1_wgrad_kernel<16><<<chunks, 256, 0, st>>>(in, g, part, D, H, W, kWgradChunk);
    int rc = check_cuda(cudaGetLastError(), "first-layer wgrad");
    if (rc) return rc;
    wgrad_reduce_kernel<<<blocks_for(int64_t(cout) * kpad(cin)), 256, 0, st>>>(part, dW, cout, kpad(cin), 27 * cin,
                                                                                 chunks);
    return check_cuda(cudaGetLastError(), "wgrad reduce");
  }
  if (tc_status && tc_eligible(cin, cout, D, H, W)) {
    int rc = STENCIL_ERR_ARG;
#define X(CI, CO) \
    if (cin == CI && cout == CO) rc = launch_wgrad_tc<CI, CO>(in, g, part, chunks, D, H, W, tc_status, st);
    X(16, 16) X(16, 32) X(16, 64) X(32, 16) X(32, 32) X(32, 64) X(64, 16) X(64, 32) X(64, 64)
#undef X
    if (rc) return rc == STENCIL_ERR_ARG ? set_error(rc, "wsnet: no tensor-core weight gradient for %d -> %d",
                                                     cin, cout)
                                         : rc;
    wgrad_reduce_kernel<<<blocks_for(int64_t(cout) * kpad(cin)), 256, 0, st>>>(part, dW, cout, kpad(cin), 27 * cin,
                                                                                 chunks);
    return check_cuda(cudaGetLastError(), "wgrad reduce");
  }
  const dim3 grid(chunks, 27);
#define X(CI, CO)                                                                                   \
  if (cin == CI && cout == CO) {                                                                   \
    conv3_wgrad_kernel<CI, CO><<<grid, 128, 0, st>>>(in, g, part, D, H, W, kWgradChunk);           \
    int rc = check_cuda(cudaGetLastError(), "conv3 wgrad");                                         \
    if (rc) return rc;                                                                              \
    wgrad_reduce_kernel<<<blocks_for(int64_t(CO) * kpad(CI)), 256, 0, st>>>(part, dW, CO, kpad(CI), \
                                                                             27 * CI, chunks);      \
    return check_cuda(cudaGetLastError(), "wgrad reduce");                                          \
  }
  STENCIL_NET_PAIRS(X)
#undef X
  return set_error(STENCIL_ERR_ARG, "wsnet: no weight-gradient kernel for %d -> %d channels", cin, cout);
}

uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Standard normal deviates by the Box-Muller transform of splitmix64 uniforms.
double normal(uint64_t& s) {
  const double u1 = (static_cast<double>(splitmix64(s) >> 11) + 0.5) / 9007199254740992.0;
  const double u2 = (static_cast<double>(splitmix64(s) >> 11) + 0.5) / 9007199254740992.0;
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

}  // namespace

struct Layer {
  int cin, cout, level;
  int64_t woff, boff;  // offsets into the FP32 parameter vector
  bf16* wf;            // [cout][kpad(cin)]
  bf16* wt;            // [cin][kpad(cout)]
};

}  // namespace net
}  // namespace stencil

// Output scale: u0 = net(f / rms f) * rms(f) * kOutScale.  1/(3 pi^2) is the
// solution of the lowest sine mode per unit of its source, so the network's
// output is of order one.
static const double kOutScale = 1.0 / (3.0 * 9.869604401089358);

struct wsnet {
  int device;
  int L;
  int C[stencil::net::kMaxLevels];
  int n;  // interior extent of the grids it maps
  std::vector<stencil::net::Layer> layers;
  int64_t nparams;
  int64_t out_w, out_b;
  float *p, *g, *m, *v;  // device FP32: parameters, gradients, Adam moments
  stencil::net::bf16* wbuf;
  int64_t wbuf_elems;
  float* zero_bias;
  int64_t V[stencil::net::kMaxLevels];
  int dim[stencil::net::kMaxLevels];
  stencil::net::bf16 *x0, *a[4], *b[4], *pl[4], *u[4], *da[4], *db[4], *gA[4], *gB[4], *gs[4];
  float *y, *yraw, *t, *gy, *gyf, *part, *misc;
  double *rms_part, *rms;
  uint32_t* status;  // device status word (bounded waits of the tensor-core kernels)
  int use_tc;        // 1: tcgen05 convolutions where eligible, 0: mma.sync everywhere
  int num_sms;
  int64_t part_elems;
  int step;
  std::vector<void*> allocs;
};

namespace stencil {
namespace net {
namespace {

int dalloc(wsnet* w, void** p, size_t bytes) {
  int rc = check_cuda(cudaMalloc(p, std::max<size_t>(bytes, 256)), "wsnet cudaMalloc");
  if (!rc) {
    w->allocs.push_back(*p);
    rc = check_cuda(cudaMemset(*p, 0, std::max<size_t>(bytes, 256)), "wsnet cudaMemset");
  }
  return rc;
}

template <class T>
int dalloc_t(wsnet* w, T** p, size_t count) {
  void* q = nullptr;
  int rc = dalloc(w, &q, count * sizeof(T));
  *p = static_cast<T*>(q);
  return rc;
}

int mirror(wsnet* w, cudaStream_t st) {
  for (const Layer& ly : w->layers) {
    const int64_t n = static_cast<int64_t>(ly.cout) * kpad(ly.cin) + static_cast<int64_t>(ly.cin) * kpad(ly.cout);
    mirror_kernel<<<blocks_for(n), 256, 0, st>>>(w->p + ly.woff, ly.wf, ly.wt, ly.cin, ly.cout);
  }
  return check_cuda(cudaGetLastError(), "wsnet mirror");
}

int forward(wsnet* w, cudaStream_t st) {
  const int L = w->L;
  int li = 0;
  for (int l = 0; l < L; ++l) {
    const int d = w->dim[l];
    const bf16* in = w->x0;
    if (l > 0) {
      pool2_kernel<<<blocks_for(w->V[l] * w->C[l - 1] / 8), 256, 0, st>>>(w->b[l - 1], w->pl[l], 2 * d, 2 * d, 2 * d,
                                                                      w->C[l - 1]);
      in = w->pl[l];
    }
    const Layer& la = w->layers[li++];
    uint32_t* tcs = w->use_tc ? w->status : nullptr;
    int rc = launch_conv(la.cin, la.cout, true, false, in, la.wf, w->p + la.boff, nullptr, w->a[l], d, d, d, tcs,
                         w->num_sms, st);
    if (rc) return rc;
    const Layer& lb = w->layers[li++];
    rc = launch_conv(lb.cin, lb.cout, true, false, w->a[l], lb.wf, w->p + lb.boff, nullptr, w->b[l], d, d, d, tcs,
                     w->num_sms, st);
    if (rc) return rc;
  }
  const bf16* h = w->b[L - 1];
  for (int l = L - 2; l >= 0; --l) {
    const int d = w->dim[l];
    up2_kernel<<<blocks_for(w->V[l] * w->C[l + 1] / 8), 256, 0, st>>>(h, w->u[l], d, d, d, w->C[l + 1]);
    const Layer& la = w->layers[li++];
    uint32_t* tcs = w->use_tc ? w->status : nullptr;
    int rc = launch_conv(la.cin, la.cout, true, true, w->u[l], la.wf, w->p + la.boff, w->b[l], w->da[l], d, d, d, tcs,
                         w->num_sms, st);
    if (rc) return rc;
    const Layer& lb = w->layers[li++];
    rc = launch_conv(lb.cin, lb.cout, true, false, w->da[l], lb.wf, w->p + lb.boff, nullptr, w->db[l], d, d, d, tcs,
                     w->num_sms, st);
    if (rc) return rc;
    h = w->db[l];
  }
  const bf16* last = L > 1 ? w->db[0] : w->b[0];
  out_fwd_kernel<<<blocks_for(w->V[0]), 256, 0, st>>>(last, w->p + w->out_w, w->p + w->out_b, w->yraw, w->V[0],
                                                       w->C[0]);
  smooth121_kernel<<<blocks_for(w->V[0]), 256, 0, st>>>(w->yraw, w->y, w->n);
  return check_cuda(cudaGetLastError(), "wsnet forward");
}

// Accumulates dLoss/dtheta into w->g for the current y, t; loss partials in
// w->misc (one per block of kLossChunk voxels).
constexpr int kLossChunk = 16384;

int bias_grad(wsnet* w, const bf16* g, int64_t V, int C, float* db, cudaStream_t st) {
  const int blocks = static_cast<int>((V + kSumChunk - 1) / kSumChunk);
  if (C == 16) chan_sum_kernel<16, false><<<blocks, 256, 0, st>>>(g, nullptr, w->part, V);
  else if (C == 32) chan_sum_kernel<32, false><<<blocks, 256, 0, st>>>(g, nullptr, w->part, V);
  else if (C == 64) chan_sum_kernel<64, false><<<blocks, 256, 0, st>>>(g, nullptr, w->part, V);
  else return set_error(STENCIL_ERR_ARG, "wsnet: no bias-gradient kernel for %d channels", C);
  chan_sum_reduce_kernel<<<1, 64, 0, st>>>(w->part, db, C, blocks);
  return check_cuda(cudaGetLastError(), "bias grad");
}

int conv_backward(wsnet* w, const Layer& ly, const bf16* in, const bf16* g, bf16* gin, int d, cudaStream_t st) {
  const int64_t V = static_cast<int64_t>(d) * d * d;
  int rc = launch_wgrad(ly.cin, ly.cout, in, g, w->part, w->g + ly.woff, d, d, d, w->use_tc ? w->status : nullptr,
                        st);
  if (!rc) rc = bias_grad(w, g, V, ly.cout, w->g + ly.boff, st);
  if (!rc && gin)
    rc = launch_conv(ly.cout, ly.cin, false, false, g, ly.wt, w->zero_bias, nullptr, gin, d, d, d,
                     w->use_tc ? w->status : nullptr, w->num_sms, st);
  return rc;
}

int backward(wsnet* w, cudaStream_t st) {
  const int L = w->L;
  const int64_t V0 = w->V[0];
  const bf16* last = L > 1 ? w->db[0] : w->b[0];
  const int lblocks = static_cast<int>((V0 + kLossChunk - 1) / kLossChunk);
  mse_bwd_kernel<<<lblocks, 256, 0, st>>>(w->y, w->t, w->gy, w->misc, V0, kLossChunk);
  smooth121_kernel<<<blocks_for(V0), 256, 0, st>>>(w->gy, w->gyf, w->n);
  out_bwd_kernel<<<blocks_for(V0), 256, 0, st>>>(w->gyf, w->p + w->out_w, w->gA[0], V0, w->C[0]);
  const int oblocks = static_cast<int>((V0 + kSumChunk - 1) / kSumChunk);
  const int C0 = w->C[0];
  if (C0 == 16) chan_sum_kernel<16, true><<<oblocks, 256, 0, st>>>(last, w->gyf, w->part, V0);
  else if (C0 == 32) chan_sum_kernel<32, true><<<oblocks, 256, 0, st>>>(last, w->gyf, w->part, V0);
  else chan_sum_kernel<64, true><<<oblocks, 256, 0, st>>>(last, w->gyf, w->part, V0);
  chan_sum_reduce_kernel<<<1, 64, 0, st>>>(w->part, w->g + w->out_w, C0 + 1, oblocks);
  int rc = check_cuda(cudaGetLastError(), "output layer backward");
  if (rc) return rc;
  int li = static_cast<int>(w->layers.size()) - 1;  // layers in reverse forward order
  for (int l = 0; l <= L - 2; ++l) {
    const int d = w->dim[l];
    const int64_t V = w->V[l];
    const Layer& lb = w->layers[li--];
    const Layer& la = w->layers[li--];
    relu_bwd_kernel<<<blocks_for(V * lb.cout / 8), 256, 0, st>>>(w->gA[l], nullptr, w->db[l], w->gB[l], V * lb.cout);
    rc = conv_backward(w, lb, w->da[l], w->gB[l], w->gA[l], d, st);
    if (rc) return rc;
    relu_bwd_kernel<<<blocks_for(V * la.cout / 8), 256, 0, st>>>(w->gA[l], nullptr, w->da[l], w->gs[l], V * la.cout);
    rc = conv_backward(w, la, w->u[l], w->gs[l], w->gB[l], d, st);
    if (rc) return rc;
    up2_bwd_kernel<<<blocks_for(w->V[l + 1] * la.cin / 8), 256, 0, st>>>(w->gB[l], w->gA[l + 1], w->dim[l + 1],
                                                                     w->dim[l + 1], w->dim[l + 1], la.cin);
  }
  for (int l = L - 1; l >= 0; --l) {
    const int d = w->dim[l];
    const int64_t V = w->V[l];
    const Layer& lb = w->layers[li--];
    const Layer& la = w->layers[li--];
    relu_bwd_kernel<<<blocks_for(V * lb.cout / 8), 256, 0, st>>>(w->gA[l], l <= L - 2 ? w->gs[l] : nullptr, w->b[l],
                                                             w->gB[l], V * lb.cout);
    rc = conv_backward(w, lb, w->a[l], w->gB[l], w->gA[l], d, st);
    if (rc) return rc;
    relu_bwd_kernel<<<blocks_for(V * la.cout / 8), 256, 0, st>>>(w->gA[l], nullptr, w->a[l], w->gB[l], V * la.cout);
    rc = conv_backward(w, la, l > 0 ? w->pl[l] : w->x0, w->gB[l], l > 0 ? w->gA[l] : nullptr, d, st);
    if (rc) return rc;
    if (l > 0)
      pool2_bwd_kernel<<<blocks_for(w->V[l - 1] * la.cin / 8), 256, 0, st>>>(w->gA[l], w->gA[l - 1], 2 * d, 2 * d,
                                                                         2 * d, la.cin);
  }
  return check_cuda(cudaGetLastError(), "wsnet backward");
}

int check_grid(const wsnet* w, const stencil_grid* g, const char* name, Grid* out) {
  int rc = validate_grid(g, name, out, false);
  if (rc) return rc;
  if (out->dtype != STENCIL_F64) return set_error(STENCIL_ERR_DTYPE, "wsnet: %s must be F64", name);
  if (out->nx != w->n || out->ny != w->n || out->nz != w->n)
    return set_error(STENCIL_ERR_ARG, "wsnet: %s must be %d^3 (the size the net was created for)", name, w->n);
  return STENCIL_OK;
}

// rms of f's interior into w->rms, then the normalised input x0.
int load_input(wsnet* w, const Grid& f, cudaStream_t st) {
  const int blocks = 256;
  sumsq_kernel<<<blocks, 256, 0, st>>>(static_cast<const double*>(f.data), f.sy, f.sz, w->n, w->rms_part);
  rms_kernel<<<1, 32, 0, st>>>(w->rms_part, blocks, static_cast<double>(w->V[0]), w->rms);
  input_kernel<<<blocks_for(w->V[0]), 256, 0, st>>>(static_cast<const double*>(f.data), f.sy, f.sz, w->n, w->rms,
                                                    w->x0);
  return check_cuda(cudaGetLastError(), "wsnet input");
}

struct DevGuard {
  int prev = -1;
  int rc = STENCIL_OK;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) rc = check_cuda(cudaSetDevice(dev), "cudaSetDevice");
  }
  ~DevGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace
}  // namespace net
}  // namespace stencil

using namespace stencil;
using namespace stencil::net;

extern "C" int wsnet_create(int device, int32_t levels, const int32_t* channels, int32_t n, uint64_t seed,
                            wsnet** out) {
  if (!out || !channels || levels < 1 || levels > kMaxLevels || n < 1)
    return set_error(STENCIL_ERR_ARG, "wsnet_create: bad arguments");
  *out = nullptr;
  if (n % (1 << (levels - 1)) != 0)
    return set_error(STENCIL_ERR_ARG, "wsnet_create: n must be a multiple of 2^(levels-1)");
  for (int l = 0; l < levels; ++l)
    if (channels[l] != 16 && channels[l] != 32 && channels[l] != 64)
      return set_error(STENCIL_ERR_ARG, "wsnet_create: channels must be 16, 32 or 64");
  DevGuard dg(device);
  if (dg.rc) return dg.rc;
  wsnet* w = new (std::nothrow) wsnet();
  if (!w) return set_error(STENCIL_ERR_ARG, "wsnet_create: out of host memory");
  w->device = device;
  w->L = levels;
  w->n = n;
  w->num_sms = 148;
  cudaDeviceGetAttribute(&w->num_sms, cudaDevAttrMultiProcessorCount, device);
  for (int l = 0; l < levels; ++l) {
    w->C[l] = channels[l];
    w->dim[l] = n >> l;
    w->V[l] = static_cast<int64_t>(w->dim[l]) * w->dim[l] * w->dim[l];
  }
  // parameter layout: per layer W[cout][27*cin] then b[cout]; then out.w, out.b
  int64_t off = 0, welems = 0;
  auto add = [&](int cin, int cout, int level) {
    Layer ly;
    ly.cin = cin; ly.cout = cout; ly.level = level;
    ly.woff = off; off += static_cast<int64_t>(cout) * 27 * cin;
    ly.boff = off; off += cout;
    ly.wf = ly.wt = nullptr;
    welems += static_cast<int64_t>(cout) * kpad(cin) + static_cast<int64_t>(cin) * kpad(cout);
    w->layers.push_back(ly);
  };
  for (int l = 0; l < levels; ++l) {
    add(l == 0 ? 1 : channels[l - 1], channels[l], l);
    add(channels[l], channels[l], l);
  }
  for (int l = levels - 2; l >= 0; --l) {
    add(channels[l + 1], channels[l], l);
    add(channels[l], channels[l], l);
  }
  w->out_w = off; off += channels[0];
  w->out_b = off; off += 1;
  w->nparams = off;
  int rc = STENCIL_OK;
  auto A = [&](auto** p, size_t count) { if (!rc) rc = dalloc_t(w, p, count); };
  A(&w->p, off); A(&w->g, off); A(&w->m, off); A(&w->v, off);
  A(&w->wbuf, static_cast<size_t>(welems));
  A(&w->zero_bias, 64);
  A(&w->x0, static_cast<size_t>(w->V[0]));
  int64_t part = 0;
  for (int l = 0; l < levels; ++l) {
    const size_t V = static_cast<size_t>(w->V[l]);
    A(&w->a[l], V * channels[l]);
    A(&w->b[l], V * channels[l]);
    if (l > 0) A(&w->pl[l], V * channels[l - 1]);
    if (l <= levels - 2) {
      A(&w->u[l], V * channels[l + 1]);
      A(&w->da[l], V * channels[l]);
      A(&w->db[l], V * channels[l]);
      A(&w->gs[l], V * channels[l]);
    }
    A(&w->gA[l], V * 64);
    A(&w->gB[l], V * 64);
  }
  for (const Layer& ly : w->layers) {
    const int64_t chunks = (w->V[ly.level] + kWgradChunk - 1) / kWgradChunk;
    part = std::max(part, chunks * ly.cout * kpad(ly.cin));
  }
  part = std::max<int64_t>(part, (w->V[0] / kSumChunk + 2) * 65);
  w->part_elems = part;
  A(&w->part, static_cast<size_t>(part));
  A(&w->y, static_cast<size_t>(w->V[0]));
  A(&w->yraw, static_cast<size_t>(w->V[0]));
  A(&w->gyf, static_cast<size_t>(w->V[0]));
  A(&w->t, static_cast<size_t>(w->V[0]));
  A(&w->gy, static_cast<size_t>(w->V[0]));
  A(&w->misc, static_cast<size_t>(w->V[0] / kLossChunk + 16));
  A(&w->rms_part, 256);
  A(&w->rms, 4);
  A(&w->status, 4);
  w->use_tc = 1;
  if (rc) {
    wsnet_destroy(w);
    return rc;
  }
  int64_t wo = 0;
  for (Layer& ly : w->layers) {
    ly.wf = w->wbuf + wo;
    wo += static_cast<int64_t>(ly.cout) * kpad(ly.cin);
    ly.wt = w->wbuf + wo;
    wo += static_cast<int64_t>(ly.cin) * kpad(ly.cout);
  }
  // He-normal weights (std sqrt(2 / (27 cin))), zero biases; output layer
  // std sqrt(1 / C0).
  std::vector<float> hp(static_cast<size_t>(off), 0.0f);
  uint64_t s = seed;
  for (const Layer& ly : w->layers) {
    const double sd = sqrt(2.0 / (27.0 * ly.cin));
    for (int64_t i = 0; i < static_cast<int64_t>(ly.cout) * 27 * ly.cin; ++i)
      hp[ly.woff + i] = static_cast<float>(normal(s) * sd);
  }
  for (int c = 0; c < channels[0]; ++c) hp[w->out_w + c] = static_cast<float>(normal(s) * sqrt(1.0 / channels[0]));
  rc = check_cuda(cudaMemcpy(w->p, hp.data(), sizeof(float) * off, cudaMemcpyHostToDevice), "wsnet init");
  if (!rc) rc = mirror(w, nullptr);
  if (!rc) rc = check_cuda(cudaDeviceSynchronize(), "wsnet init sync");
  if (rc) {
    wsnet_destroy(w);
    return rc;
  }
  *out = w;
  return STENCIL_OK;
}

extern "C" int wsnet_destroy(wsnet* w) {
  if (!w) return STENCIL_OK;
  DevGuard dg(w->device);
  cudaDeviceSynchronize();
  for (void* p : w->allocs) cudaFree(p);
  delete w;
  return STENCIL_OK;
}

extern "C" int wsnet_num_params(const wsnet* w, int64_t* count) {
  if (!w || !count) return set_error(STENCIL_ERR_ARG, "wsnet_num_params: null argument");
  *count = w->nparams;
  return STENCIL_OK;
}

extern "C" int wsnet_get_params(wsnet* w, float* host, int64_t count) {
  if (!w || !host || count != w->nparams) return set_error(STENCIL_ERR_ARG, "wsnet_get_params: bad arguments");
  DevGuard dg(w->device);
  return check_cuda(cudaMemcpy(host, w->p, sizeof(float) * count, cudaMemcpyDeviceToHost), "wsnet_get_params");
}

extern "C" int wsnet_set_params(wsnet* w, const float* host, int64_t count) {
  if (!w || !host || count != w->nparams) return set_error(STENCIL_ERR_ARG, "wsnet_set_params: bad arguments");
  DevGuard dg(w->device);
  int rc = check_cuda(cudaMemcpy(w->p, host, sizeof(float) * count, cudaMemcpyHostToDevice), "wsnet_set_params");
  if (!rc) rc = mirror(w, nullptr);
  if (!rc) rc = check_cuda(cudaDeviceSynchronize(), "wsnet_set_params sync");
  return rc;
}

// File layout of wsnet_save / wsnet_load (little endian): 8 bytes magic,
// int32 levels, int32 channels[levels], int32 n, int64 parameter count,
// the FP32 parameters in wsnet_get_params order; with the magic "WSNET02"
// (what wsnet_save writes) the optimiser state follows: int64 Adam step
// count, then the FP32 first and second moments in the same order.  Files
// with the magic "WSNET01" hold the parameters only; loading one starts the
// optimiser afresh (zero moments, step 0).
static const char kWsMagic1[8] = {'W', 'S', 'N', 'E', 'T', '0', '1', 0};
static const char kWsMagic2[8] = {'W', 'S', 'N', 'E', 'T', '0', '2', 0};

extern "C" int wsnet_save(wsnet* w, const char* path) {
  if (!w || !path) return set_error(STENCIL_ERR_ARG, "wsnet_save: bad arguments");
  const size_t np = static_cast<size_t>(w->nparams);
  std::vector<float> host(3 * np);
  int rc = wsnet_get_params(w, host.data(), w->nparams);
  if (rc) return rc;
  DevGuard dg(w->device);
  rc = check_cuda(cudaMemcpy(host.data() + np, w->m, sizeof(float) * np, cudaMemcpyDeviceToHost), "wsnet_save m");
  if (!rc) rc = check_cuda(cudaMemcpy(host.data() + 2 * np, w->v, sizeof(float) * np, cudaMemcpyDeviceToHost),
                           "wsnet_save v");
  if (rc) return rc;
  FILE* fp = fopen(path, "wb");
  if (!fp) return set_error(STENCIL_ERR_ARG, "wsnet_save: cannot open %s", path);
  const int32_t hdr[2] = {w->L, w->n};
  bool ok = fwrite(kWsMagic2, 1, 8, fp) == 8 && fwrite(&hdr[0], 4, 1, fp) == 1;
  for (int l = 0; l < w->L && ok; ++l) {
    const int32_t c = w->C[l];
    ok = fwrite(&c, 4, 1, fp) == 1;
  }
  const int64_t cnt = w->nparams;
  const int64_t step = w->step;
  ok = ok && fwrite(&hdr[1], 4, 1, fp) == 1 && fwrite(&cnt, 8, 1, fp) == 1 &&
       fwrite(host.data(), sizeof(float), np, fp) == np && fwrite(&step, 8, 1, fp) == 1 &&
       fwrite(host.data() + np, sizeof(float), 2 * np, fp) == 2 * np;
  ok = (fclose(fp) == 0) && ok;
  return ok ? STENCIL_OK : set_error(STENCIL_ERR_ARG, "wsnet_save: write to %s failed", path);
}

extern "C" int wsnet_load(wsnet* w, const char* path) {
  if (!w || !path) return set_error(STENCIL_ERR_ARG, "wsnet_load: bad arguments");
  FILE* fp = fopen(path, "rb");
  if (!fp) return set_error(STENCIL_ERR_ARG, "wsnet_load: cannot open %s", path);
  char magic[8];
  int32_t L = 0, n = 0;
  int64_t cnt = 0, step = 0;
  bool ok = fread(magic, 1, 8, fp) == 8;
  const bool v1 = ok && memcmp(magic, kWsMagic1, 8) == 0;
  const bool v2 = ok && memcmp(magic, kWsMagic2, 8) == 0;
  ok = (v1 || v2) && fread(&L, 4, 1, fp) == 1 && L == w->L;
  for (int l = 0; l < L && ok; ++l) {
    int32_t c = 0;
    ok = fread(&c, 4, 1, fp) == 1 && c == w->C[l];
  }
  ok = ok && fread(&n, 4, 1, fp) == 1 && n == w->n && fread(&cnt, 8, 1, fp) == 1 && cnt == w->nparams;
  const size_t np = static_cast<size_t>(w->nparams);
  std::vector<float> host;
  if (ok) {
    host.assign(3 * np, 0.0f);  // parameters, then the moments (zero for a parameters-only file)
    ok = fread(host.data(), sizeof(float), np, fp) == np;
    if (ok && v2)
      ok = fread(&step, 8, 1, fp) == 1 && step >= 0 && fread(host.data() + np, sizeof(float), 2 * np, fp) == 2 * np;
  }
  fclose(fp);
  if (!ok) return set_error(STENCIL_ERR_ARG, "wsnet_load: %s is not a file of a net of this configuration", path);
  int rc = wsnet_set_params(w, host.data(), cnt);
  if (rc) return rc;
  DevGuard dg(w->device);
  rc = check_cuda(cudaMemcpy(w->m, host.data() + np, sizeof(float) * np, cudaMemcpyHostToDevice), "wsnet_load m");
  if (!rc) rc = check_cuda(cudaMemcpy(w->v, host.data() + 2 * np, sizeof(float) * np, cudaMemcpyHostToDevice),
                           "wsnet_load v");
  if (!rc) w->step = step;
  return rc;
}

extern "C" int wsnet_infer(wsnet* w, const stencil_grid* f, const stencil_grid* u, void* stream) {
  if (!w) return set_error(STENCIL_ERR_ARG, "wsnet_infer: null net");
  Grid gf, gu;
  int rc = check_grid(w, f, "f", &gf);
  if (!rc) rc = check_grid(w, u, "u", &gu);
  if (rc) return rc;
  DevGuard dg(w->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  rc = load_input(w, gf, st);
  if (!rc) rc = forward(w, st);
  if (rc) return rc;
  output_kernel<<<blocks_for(w->V[0]), 256, 0, st>>>(w->y, static_cast<double*>(gu.data), gu.sy, gu.sz, w->n, w->rms,
                                                     kOutScale);
  return check_cuda(cudaGetLastError(), "wsnet output");
}

extern "C" int wsnet_train_step(wsnet* w, const stencil_grid* f, const stencil_grid* u, int32_t count, float lr,
                                double* loss, void* stream) {
  if (!w || !f || !u || count < 1) return set_error(STENCIL_ERR_ARG, "wsnet_train_step: bad arguments");
  DevGuard dg(w->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = check_cuda(cudaMemsetAsync(w->g, 0, sizeof(float) * w->nparams, st), "zero grads");
  if (rc) return rc;
  const int lblocks = static_cast<int>((w->V[0] + kLossChunk - 1) / kLossChunk);
  double total = 0.0;
  std::vector<float> lp(static_cast<size_t>(lblocks));
  for (int s = 0; s < count; ++s) {
    Grid gf, gu;
    rc = check_grid(w, &f[s], "f", &gf);
    if (!rc) rc = check_grid(w, &u[s], "u", &gu);
    if (!rc) rc = load_input(w, gf, st);
    if (rc) return rc;
    target_kernel<<<blocks_for(w->V[0]), 256, 0, st>>>(static_cast<const double*>(gu.data), gu.sy, gu.sz, w->n,
                                                       w->rms, kOutScale, w->t);
    rc = forward(w, st);
    if (!rc) rc = backward(w, st);
    if (!rc) rc = check_cuda(cudaMemcpyAsync(lp.data(), w->misc, sizeof(float) * lblocks, cudaMemcpyDeviceToHost, st),
                             "loss read");
    if (!rc) rc = check_cuda(cudaStreamSynchronize(st), "train sync");
    if (rc) return rc;
    double sl = 0.0;
    for (float x : lp) sl += x;
    total += sl / static_cast<double>(w->V[0]);
  }
  w->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, static_cast<float>(w->step));
  const float c2 = 1.0f - powf(b2, static_cast<float>(w->step));
  adam_kernel<<<blocks_for(w->nparams), 256, 0, st>>>(w->p, w->g, w->m, w->v, w->nparams, lr, b1, b2, 1e-8f, c1, c2,
                                                      1.0f / static_cast<float>(count));
  rc = check_cuda(cudaGetLastError(), "adam");
  if (!rc) rc = mirror(w, st);
  if (rc) return rc;
  if (loss) *loss = total / count;
  return STENCIL_OK;
}

// Test hook: for a normalised input x and target t (device FP32 arrays of
// n^3 values, channels-last), run forward and backward once from zeroed
// gradients; y (device, optional) receives the output, grads (host,
// optional) the parameter gradients, *loss the mean squared error.
extern "C" int wsnet_loss_grad(wsnet* w, const float* x, const float* t, float* y, float* grads, double* loss,
                               void* stream) {
  if (!w || !x || !t) return set_error(STENCIL_ERR_ARG, "wsnet_loss_grad: null argument");
  DevGuard dg(w->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<float> hx(static_cast<size_t>(w->V[0]));
  int rc = check_cuda(cudaMemcpyAsync(hx.data(), x, sizeof(float) * w->V[0], cudaMemcpyDeviceToHost, st), "x read");
  if (!rc) rc = check_cuda(cudaStreamSynchronize(st), "sync");
  if (rc) return rc;
  std::vector<bf16> hb(hx.size());
  for (size_t i = 0; i < hx.size(); ++i) hb[i] = __float2bfloat16_rn(hx[i]);
  rc = check_cuda(cudaMemcpyAsync(w->x0, hb.data(), sizeof(bf16) * hb.size(), cudaMemcpyHostToDevice, st), "x load");
  if (!rc) rc = check_cuda(cudaMemcpyAsync(w->t, t, sizeof(float) * w->V[0], cudaMemcpyDeviceToDevice, st), "t load");
  if (!rc) rc = check_cuda(cudaMemsetAsync(w->g, 0, sizeof(float) * w->nparams, st), "zero grads");
  if (!rc) rc = forward(w, st);
  if (!rc) rc = backward(w, st);
  if (rc) return rc;
  if (y) rc = check_cuda(cudaMemcpyAsync(y, w->y, sizeof(float) * w->V[0], cudaMemcpyDeviceToDevice, st), "y copy");
  const int lblocks = static_cast<int>((w->V[0] + kLossChunk - 1) / kLossChunk);
  std::vector<float> lp(static_cast<size_t>(lblocks));
  if (!rc) rc = check_cuda(cudaMemcpyAsync(lp.data(), w->misc, sizeof(float) * lblocks, cudaMemcpyDeviceToHost, st),
                           "loss read");
  if (!rc && grads)
    rc = check_cuda(cudaMemcpyAsync(grads, w->g, sizeof(float) * w->nparams, cudaMemcpyDeviceToHost, st), "grads");
  if (!rc) rc = check_cuda(cudaStreamSynchronize(st), "sync");
  if (rc) return rc;
  double sl = 0.0;
  for (float v : lp) sl += v;
  if (loss) *loss = sl / static_cast<double>(w->V[0]);
  return STENCIL_OK;
}

// Choose the convolution kernels: 1 (default) = tcgen05 for eligible layers,
// 0 = mma.sync for every layer.
extern "C" int wsnet_use_tcgen05(wsnet* w, int32_t enable) {
  if (!w) return set_error(STENCIL_ERR_ARG, "wsnet_use_tcgen05: null net");
  w->use_tc = enable ? 1 : 0;
  return STENCIL_OK;
}

// Read and clear the net's device status (bounded waits of its kernels).
extern "C" int wsnet_status(wsnet* w, void* stream) {
  if (!w) return set_error(STENCIL_ERR_ARG, "wsnet_status: null net");
  DevGuard dg(w->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t bits = 0;
  int rc = check_cuda(cudaMemcpyAsync(&bits, w->status, 4, cudaMemcpyDeviceToHost, st), "status read");
  if (!rc) rc = check_cuda(cudaStreamSynchronize(st), "sync");
  if (!rc) rc = check_cuda(cudaMemsetAsync(w->status, 0, 4, st), "status clear");
  if (!rc) rc = check_cuda(cudaStreamSynchronize(st), "sync");
  if (rc) return rc;
  if (bits & kStatusTimeout) return set_error(STENCIL_ERR_TIMEOUT, "a bounded device wait expired");
  return STENCIL_OK;
}
