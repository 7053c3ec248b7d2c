// conv_tc.cuh -- 3x3x3 convolution as an implicit GEMM on the 5th-generation
// tensor cores (tcgen05, sm_100 family): M = 128 output voxels, N = COUT,
// K = 27 taps x CIN channels.
//
// One CTA (4 warps) computes 128 consecutive voxels x COUT channels:
//   * warp 0 lane 0 streams, per tap, the A tile (the 128 voxels' neighbours
//     at that tap, CIN channels each: one box of the channels-last activation
//     tensor, zero-filled outside the grid) and the B tile (the tap's
//     COUT x CIN weights) with TMA into a ring of S stages, 128/64/32-byte
//     swizzled to match the MMA operand layout (K-major);
//   * warp 1 lane 0 issues tcgen05.mma (M=128, N=COUT, K=16, BF16 in, FP32
//     accumulate in tensor memory) for each 16-channel chunk of each tap and
//     releases the stage with tcgen05.commit;
//   * after the last tap all 4 warps read the accumulator rows (one voxel per
//     thread) with tcgen05.ld and apply bias, skip, ReLU, and store bf16.
// Every wait is bounded; on expiry the status is set, the kernel still waits
// (bounded) for outstanding MMAs, frees its tensor memory and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"

namespace stencil {
namespace net {

template <int CIN>
struct TcSwz {
  static constexpr int ROW = CIN * 2;  // bytes per K-major row (one voxel or one output channel)
  // smem descriptor layout codes: 6 = 32B, 4 = 64B, 2 = 128B swizzle
  static constexpr uint64_t LAYOUT = ROW == 32 ? 6 : (ROW == 64 ? 4 : 2);
  static constexpr int ATOM = 8 * ROW;  // bytes of one 8-row swizzle atom (the stride between row groups)
};

template <int CIN, int COUT, int S>
struct TcCfg {
  static constexpr int ABYTES = 128 * CIN * 2;
  static constexpr int BBYTES = COUT * CIN * 2;
  static constexpr int STAGE = ((ABYTES + BBYTES) + 1023) / 1024 * 1024;
  static constexpr int SMEM = 1024 /*align*/ + S * STAGE + 256 /*barriers, tmem slot*/;
  static constexpr int TMEM_COLS = COUT < 32 ? 32 : COUT;
};

__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t addr, uint64_t layout, uint32_t sbo_bytes) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((addr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>(1u) << 16;                          // leading byte offset (unused for these swizzles)
  d |= static_cast<uint64_t>((sbo_bytes >> 4) & 0x3FFFu) << 32;  // stride byte offset: 8-row groups
  d |= static_cast<uint64_t>(1u) << 46;                          // descriptor version
  d |= layout << 61;
  return d;
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

struct TcParams {
  CUtensorMap tm_in;   // activations [D][H][W][CIN] as (CIN, W, H, D), box (CIN, W, HB, ZB)
  CUtensorMap tm_w;    // weights [COUT][27*CIN] as (27*CIN, COUT), box (CIN, COUT)
  const float* bias;
  const __nv_bfloat16* skip;
  __nv_bfloat16* out;
  int D, H, W, HB, ZB;  // tile = ZB planes x HB rows x W voxels = 128
  uint32_t* status;
};

template <int CIN, int COUT, int S, bool RELU, bool SKIP>
__global__ void __launch_bounds__(128, 1) conv3_tc_kernel(const __grid_constant__ TcParams p) {
  using Cfg = TcCfg<CIN, COUT, S>;
  using Sw = TcSwz<CIN>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* ring = base;
  unsigned char* tail = base + S * Cfg::STAGE;
  const uint32_t bar_full = smem_addr(tail);
  const uint32_t bar_empty = bar_full + 8 * S;
  const uint32_t bar_acc = bar_empty + 8 * S;
  volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(tail + 8 * (2 * S + 1));
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(bar_full + 8 * s, 1);
      mbar_init(bar_empty + 8 * s, 1);
    }
    mbar_init(bar_acc, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(const_cast<uint32_t*>(tmem_slot))),
                 "r"(Cfg::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  // tile origin: 128 consecutive voxels = ZB planes x HB rows x W
  const int64_t v0 = static_cast<int64_t>(blockIdx.x) * 128;
  const int z0 = static_cast<int>(v0 / (static_cast<int64_t>(p.H) * p.W));
  const int y0 = static_cast<int>((v0 / p.W) % p.H);
  constexpr int KC = CIN / 16;  // MMAs per tap
  bool ok = true;
  if (warp == 0 && lane == 0) {
    // producer
    prefetch_tensormap(&p.tm_in);
    prefetch_tensormap(&p.tm_w);
    int issued = 0;
    for (int tap = 0; tap < 27; ++tap) {
      const int s = tap % S;
      const uint32_t par = (tap / S) & 1u;
      if (!mbar_wait_bounded(bar_empty + 8 * s, par ^ 1u, p.status)) { ok = false; abort_flag = 1; break; }
      const uint32_t a = smem_addr(ring + s * Cfg::STAGE);
      mbar_arrive_expect_tx(bar_full + 8 * s, Cfg::ABYTES + Cfg::BBYTES);
      tma_load_4d(a, &p.tm_in, 0, tap % 3 - 1, y0 + (tap / 3) % 3 - 1, z0 + tap / 9 - 1, bar_full + 8 * s);
      tma_load_2d(a + Cfg::ABYTES, &p.tm_w, tap * CIN, 0, bar_full + 8 * s);
      issued = tap + 1;
    }
    // no copy may still be landing in shared memory when the CTA exits: wait
    // (bounded) for the last load issued to every stage
    for (int s = 0; s < S && s < issued; ++s) {
      const int last = s + (issued - 1 - s) / S * S;
      mbar_wait_bounded(bar_full + 8 * s, (last / S) & 1u, p.status);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t idesc = tc_idesc(128, COUT);
    for (int tap = 0; tap < 27; ++tap) {
      const int s = tap % S;
      const uint32_t par = (tap / S) & 1u;
      if (*reinterpret_cast<volatile int*>(&abort_flag) ||
          !mbar_wait_bounded(bar_full + 8 * s, par, p.status)) {
        ok = false;
        abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a = smem_addr(ring + s * Cfg::STAGE);
      const uint32_t b = a + Cfg::ABYTES;
#pragma unroll
      for (int kc = 0; kc < KC; ++kc) {
        const uint64_t ad = tc_smem_desc(a + 32 * kc, Sw::LAYOUT, Sw::ATOM);
        const uint64_t bd = tc_smem_desc(b + 32 * kc, Sw::LAYOUT, Sw::ATOM);
        const uint32_t acc = (tap > 0 || kc > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       bar_empty + 8 * s)
                   : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_acc)
                 : "memory");
  }
  __syncwarp();
  // epilogue: every thread owns one accumulator row (one voxel)
  const bool acc_ok = mbar_wait_bounded(bar_acc, 0, p.status);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // warp-uniform decision: tcgen05.ld is a warp-wide (.sync.aligned) load
  if (__all_sync(0xffffffffu, acc_ok && !*reinterpret_cast<volatile int*>(&abort_flag))) {
    const int row = warp * 32 + lane;
    const int64_t v = v0 + row;
    float vals[COUT];
#pragma unroll
    for (int c0 = 0; c0 < COUT; c0 += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j) vals[c0 + j] = __uint_as_float(r[j]);
    }
    uint32_t packed[COUT / 2];
#pragma unroll
    for (int c = 0; c < COUT; c += 2) {
      float a0 = vals[c] + p.bias[c], a1 = vals[c + 1] + p.bias[c + 1];
      if (SKIP) {
        a0 += __bfloat162float(p.skip[v * COUT + c]);
        a1 += __bfloat162float(p.skip[v * COUT + c + 1]);
      }
      if (RELU) {
        a0 = fmaxf(a0, 0.0f);
        a1 = fmaxf(a1, 0.0f);
      }
      const __nv_bfloat162 h2 = __floats2bfloat162_rn(a0, a1);
      packed[c / 2] = *reinterpret_cast<const uint32_t*>(&h2);
    }
    uint4* dst = reinterpret_cast<uint4*>(p.out + v * COUT);
#pragma unroll
    for (int q = 0; q < COUT / 8; ++q)
      dst[q] = make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
  }
  // bar_acc completing means every issued MMA has finished; free the
  // tensor memory once all warps are past their loads
  (void)ok;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// Weight gradient on the tensor cores.  For one chunk of 128-voxel tiles and
// one group of TG = 128 / CIN taps:
//   D[(tap, ci)][co] = sum over the chunk's voxels v of x[v + off(tap)][ci] g[v][co]
// i.e. M = 128 rows (TG taps x CIN channels), N = COUT, K = voxels.  Both
// operands are used as TMA lands them, MN-major: a tap's box is [v][ci]
// (the M values of one voxel contiguous, one swizzle atom wide) and the
// gradient box is [v][co].  The TG tap boxes of a stage sit TAP_BYTES apart
// (the descriptor's leading byte offset between M atoms); 8-voxel row groups
// are 8 rows apart (its stride byte offset).  The chunk's partial sums go to
// part[chunk][co][tap*CIN + ci], the layout the fixed-order chunk reduction
// reads.
template <int CIN, int COUT>
struct WgCfg {
  static constexpr int TG = 128 / CIN;
  static constexpr int TAP_BYTES = 128 * CIN * 2;
  static constexpr int ABYTES = TG * TAP_BYTES;  // 32 KB
  static constexpr int BBYTES = 128 * COUT * 2;
  static constexpr int S = 3;
  static constexpr int STAGE = ABYTES + BBYTES;  // a multiple of 1024
  static constexpr int SMEM = 1024 + S * STAGE + 256;
  static constexpr int TMEM_COLS = COUT < 32 ? 32 : COUT;
  static constexpr uint64_t LAYOUT_A = TcSwz<CIN>::LAYOUT;
  static constexpr uint64_t LAYOUT_B = TcSwz<COUT>::LAYOUT;
};

struct WgParams {
  CUtensorMap tm_in;  // activations (CIN, W, H, D), box (CIN, W, HB, 1)
  CUtensorMap tm_g;   // output gradient (COUT, W, H, D), box (COUT, W, HB, 1)
  float* part;        // [chunk][COUT][kp]
  int kp;
  int D, H, W, HB;
  int tiles;          // 128-voxel tiles in the grid
  int chunk_tiles;    // tiles per chunk (K steps of one CTA)
  uint32_t* status;
};

// smem descriptor with both offsets given (MN-major operands).
__device__ __forceinline__ uint64_t tc_smem_desc2(uint32_t addr, uint64_t layout, uint32_t lbo_bytes,
                                                  uint32_t sbo_bytes) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((addr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>((lbo_bytes >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo_bytes >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1u) << 46;
  d |= layout << 61;
  return d;
}

// kind::f16 instruction descriptor with A and B MN-major (transposed).
__host__ __device__ constexpr uint32_t tc_idesc_mn(int M, int N) {
  return tc_idesc(M, N) | (1u << 15) | (1u << 16);
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(128, 1) wgrad_tc_kernel(const __grid_constant__ WgParams p) {
  using Cfg = WgCfg<CIN, COUT>;
  constexpr int S = Cfg::S;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* ring = base;
  unsigned char* tail = base + S * Cfg::STAGE;
  const uint32_t bar_full = smem_addr(tail);
  const uint32_t bar_empty = bar_full + 8 * S;
  const uint32_t bar_acc = bar_empty + 8 * S;
  volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(tail + 8 * (2 * S + 1));
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tap0 = blockIdx.y * Cfg::TG;
  const int ntap = min(Cfg::TG, 27 - tap0);
  const int t_begin = blockIdx.x * p.chunk_tiles;
  const int nk = min(p.chunk_tiles, p.tiles - t_begin);
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(bar_full + 8 * s, 1);
      mbar_init(bar_empty + 8 * s, 1);
    }
    mbar_init(bar_acc, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(const_cast<uint32_t*>(tmem_slot))),
                 "r"(Cfg::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const int64_t HW = static_cast<int64_t>(p.H) * p.W;
  if (warp == 0 && lane == 0) {
    prefetch_tensormap(&p.tm_in);
    prefetch_tensormap(&p.tm_g);
    int issued = 0;
    for (int k = 0; k < nk; ++k) {
      const int s = k % S;
      const uint32_t par = (k / S) & 1u;
      if (!mbar_wait_bounded(bar_empty + 8 * s, par ^ 1u, p.status)) { abort_flag = 1; break; }
      const int64_t v0 = static_cast<int64_t>(t_begin + k) * 128;
      const int z0 = static_cast<int>(v0 / HW);
      const int y0 = static_cast<int>((v0 / p.W) % p.H);
      const uint32_t a = smem_addr(ring + s * Cfg::STAGE);
      mbar_arrive_expect_tx(bar_full + 8 * s, ntap * Cfg::TAP_BYTES + Cfg::BBYTES);
      for (int j = 0; j < ntap; ++j) {
        const int tap = tap0 + j;
        tma_load_4d(a + j * Cfg::TAP_BYTES, &p.tm_in, 0, tap % 3 - 1, y0 + (tap / 3) % 3 - 1, z0 + tap / 9 - 1,
                    bar_full + 8 * s);
      }
      tma_load_4d(a + Cfg::ABYTES, &p.tm_g, 0, 0, y0, z0, bar_full + 8 * s);
      issued = k + 1;
    }
    // no copy may still be landing in shared memory when the CTA exits
    for (int s = 0; s < S && s < issued; ++s) {
      const int last = s + (issued - 1 - s) / S * S;
      mbar_wait_bounded(bar_full + 8 * s, (last / S) & 1u, p.status);
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = tc_idesc_mn(128, COUT);
    for (int k = 0; k < nk; ++k) {
      const int s = k % S;
      const uint32_t par = (k / S) & 1u;
      if (*reinterpret_cast<volatile int*>(&abort_flag) || !mbar_wait_bounded(bar_full + 8 * s, par, p.status)) {
        abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a = smem_addr(ring + s * Cfg::STAGE);
      const uint32_t b = a + Cfg::ABYTES;
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {  // 16 voxels per MMA
        const uint64_t ad = tc_smem_desc2(a + kk * 16 * CIN * 2, Cfg::LAYOUT_A, Cfg::TAP_BYTES, 8 * CIN * 2);
        const uint64_t bd = tc_smem_desc2(b + kk * 16 * COUT * 2, Cfg::LAYOUT_B, 16, 8 * COUT * 2);
        const uint32_t acc = (k > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       bar_empty + 8 * s)
                   : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_acc)
                 : "memory");
  }
  __syncwarp();
  const bool acc_ok = mbar_wait_bounded(bar_acc, 0, p.status);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (__all_sync(0xffffffffu, acc_ok && !*reinterpret_cast<volatile int*>(&abort_flag))) {
    const int m = warp * 32 + lane;  // row (tap0 + m / CIN, m % CIN)
    const bool valid = m < ntap * CIN;
    float* dst = p.part + static_cast<int64_t>(blockIdx.x) * COUT * p.kp + tap0 * CIN + m;
#pragma unroll
    for (int c0 = 0; c0 < COUT; c0 += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (valid) {
#pragma unroll
        for (int j = 0; j < 16; ++j) dst[static_cast<int64_t>(c0 + j) * p.kp] = __uint_as_float(r[j]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// Convolution of grids whose rows are 128 voxels long, one output row
// (M = 128 voxels) per tile, persistent CTAs.  Instead of one TMA box per
// tap, a CTA loads for each row the three planes' halo boxes (3 rows x 130
// voxels, one per 8-channel group) once and forms the 27 taps' A operands as
// shifted views of them: a tap (dz, dy, dx) starts (dy * 130 + dx) voxels
// into plane dz's box.  The operands use the unswizzled K-major layout
// (8-voxel x 16-byte core matrices, contiguous since a box row is one
// voxel's 8 channels), so any voxel offset is a valid start; the two
// 8-channel halves of a 16-channel MMA chunk are one box apart (the
// descriptor's leading byte offset).  The weights, [k/8][co][8] with
// k = tap*CIN + ci, are loaded once per CTA with one TMA box.
// Warp roles: 0 = TMA producer (double-buffered row boxes), 1 = MMA issuer
// (two accumulators in tensor memory, so a row's MMAs overlap the previous
// row's epilogue), 2..5 = epilogue (bias, skip, ReLU, bf16 store).
template <int CIN, int COUT>
struct RowCfg {
  static constexpr int G = CIN / 8;              // 8-channel groups
  static constexpr int BOXW = 130;               // voxels per box row (x = -1 .. 128)
  static constexpr int BOX_TX = 8 * BOXW * 3 * 2;  // bytes TMA writes per box
  static constexpr int BOX = (BOX_TX + 127) / 128 * 128;
  static constexpr int ASTAGE = 3 * G * BOX;     // one row's boxes (3 planes x G groups)
  static constexpr int KG = 27 * G;              // 8-wide k groups of the weights
  static constexpr int BBYTES = 16 * COUT * KG;
  static constexpr int BOFF = 2 * ASTAGE;        // weights after the two row stages
  static constexpr int SMEM = 1024 + BOFF + (BBYTES + 127) / 128 * 128 + 256;
  static constexpr int ACC_COLS = COUT < 32 ? 32 : COUT;
  static constexpr int TMEM_COLS = 2 * ACC_COLS;
};

struct RowParams {
  CUtensorMap tm_in;  // activations as (8, G, W, H, D), box (8, 1, 130, 3, 1), no swizzle
  CUtensorMap tm_w;   // weights as (8, COUT, KG), box (8, COUT, KG), no swizzle
  const float* bias;
  const __nv_bfloat16* skip;
  __nv_bfloat16* out;
  int D, H;
  uint32_t* status;
};

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            int c4, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d_net(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                                uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

template <int CIN, int COUT, bool RELU, bool SKIP>
__global__ void __launch_bounds__(192, 1) conv3_row_tc_kernel(const __grid_constant__ RowParams p) {
  using Cfg = RowCfg<CIN, COUT>;
  constexpr int G = Cfg::G;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* tail = base + Cfg::BOFF + (Cfg::BBYTES + 127) / 128 * 128;
  const uint32_t bar_a_full = smem_addr(tail);  // [2]
  const uint32_t bar_a_empty = bar_a_full + 16;  // [2]
  const uint32_t bar_acc_full = bar_a_empty + 16;  // [2]
  const uint32_t bar_acc_empty = bar_acc_full + 16;  // [2]
  const uint32_t bar_w = bar_acc_empty + 16;
  volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(tail + 128);
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rows = p.D * p.H;
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(bar_a_full + 8 * s, 1);
      mbar_init(bar_a_empty + 8 * s, 1);
      mbar_init(bar_acc_full + 8 * s, 1);
      mbar_init(bar_acc_empty + 8 * s, 4);
    }
    mbar_init(bar_w, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(const_cast<uint32_t*>(tmem_slot))),
                 "r"(Cfg::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t a_base = smem_addr(base);
  const uint32_t b_base = a_base + Cfg::BOFF;
  if (warp == 0) {
    if (lane == 0) {
      prefetch_tensormap(&p.tm_in);
      prefetch_tensormap(&p.tm_w);
      mbar_arrive_expect_tx(bar_w, Cfg::BBYTES);
      tma_load_3d_net(b_base, &p.tm_w, 0, 0, 0, bar_w);
      int i = 0;
      for (int r = blockIdx.x; r < rows; r += gridDim.x, ++i) {
        const int s = i & 1;
        if (!mbar_wait_bounded(bar_a_empty + 8 * s, ((i >> 1) & 1) ^ 1u, p.status)) { abort_flag = 1; break; }
        const int z0 = r / p.H, y0 = r - z0 * p.H;
        mbar_arrive_expect_tx(bar_a_full + 8 * s, 3 * G * Cfg::BOX_TX);
        for (int dz = 0; dz < 3; ++dz)
          for (int g = 0; g < G; ++g)
            tma_load_5d(a_base + s * Cfg::ASTAGE + (dz * G + g) * Cfg::BOX, &p.tm_in, 0, g, -1, y0 - 1,
                        z0 + dz - 1, bar_a_full + 8 * s);
      }
      // no copy may still be landing in shared memory when the CTA exits
      for (int q = i > 2 ? i - 2 : 0; q < i; ++q) mbar_wait_bounded(bar_a_full + 8 * (q & 1), (q >> 1) & 1, p.status);
      mbar_wait_bounded(bar_w, 0, p.status);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc_idesc(128, COUT);
      bool ok = mbar_wait_bounded(bar_w, 0, p.status);
      int i = 0;
      for (int r = blockIdx.x; ok && r < rows; r += gridDim.x, ++i) {
        const int s = i & 1, acc = i & 1;
        if (*reinterpret_cast<volatile int*>(&abort_flag) ||
            !mbar_wait_bounded(bar_a_full + 8 * s, (i >> 1) & 1, p.status) ||
            !mbar_wait_bounded(bar_acc_empty + 8 * acc, ((i >> 1) & 1) ^ 1u, p.status)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + acc * Cfg::ACC_COLS;
        const uint32_t a_row = a_base + s * Cfg::ASTAGE;
        for (int tap = 0; tap < 27; ++tap) {
          const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
#pragma unroll
          for (int kc = 0; kc < CIN / 16; ++kc) {
            const uint32_t a = a_row + (dz * G + 2 * kc) * Cfg::BOX + (dy * Cfg::BOXW + dx) * 16;
            const uint32_t b = b_base + (tap * G + 2 * kc) * (COUT * 16);
            const uint64_t ad = tc_smem_desc2(a, 0, Cfg::BOX, 128);
            const uint64_t bd = tc_smem_desc2(b, 0, COUT * 16, 128);
            const uint32_t en = (tap > 0 || kc > 0) ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                "l"(ad), "l"(bd), "r"(idesc), "r"(en)
                : "memory");
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         bar_a_empty + 8 * s)
                     : "memory");
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         bar_acc_full + 8 * acc)
                     : "memory");
      }
      if (!ok) abort_flag = 1;
    }
  } else {
    // epilogue warps 2..5: warp w reads tensor-memory lanes 32 (w % 4) ...
    const int quarter = warp & 3;
    const int x = quarter * 32 + lane;  // output voxel in the row
    int i = 0;
    for (int r = blockIdx.x; r < rows; r += gridDim.x, ++i) {
      const int acc = i & 1;
      const bool ready = mbar_wait_bounded(bar_acc_full + 8 * acc, (i >> 1) & 1, p.status);
      if (!__all_sync(0xffffffffu, ready)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int64_t v = static_cast<int64_t>(r) * 128 + x;
      float vals[COUT];
#pragma unroll
      for (int c0 = 0; c0 < COUT; c0 += 16) {
        uint32_t q[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]),
              "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]), "=r"(q[15])
            : "r"(tmem + (static_cast<uint32_t>(quarter * 32) << 16) + acc * Cfg::ACC_COLS + c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) vals[c0 + j] = __uint_as_float(q[j]);
      }
      // the accumulator may be reused once every epilogue warp has read it
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_acc_empty + 8 * acc);
      uint32_t packed[COUT / 2];
#pragma unroll
      for (int c = 0; c < COUT; c += 2) {
        float a0 = vals[c] + p.bias[c], a1 = vals[c + 1] + p.bias[c + 1];
        if (SKIP) {
          a0 += __bfloat162float(p.skip[v * COUT + c]);
          a1 += __bfloat162float(p.skip[v * COUT + c + 1]);
        }
        if (RELU) {
          a0 = fmaxf(a0, 0.0f);
          a1 = fmaxf(a1, 0.0f);
        }
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(a0, a1);
        packed[c / 2] = *reinterpret_cast<const uint32_t*>(&h2);
      }
      uint4* dst = reinterpret_cast<uint4*>(p.out + v * COUT);
#pragma unroll
      for (int q = 0; q < COUT / 8; ++q)
        dst[q] = make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::TMEM_COLS)
                 : "memory");
  }
}

}  // namespace net
}  // namespace stencil
