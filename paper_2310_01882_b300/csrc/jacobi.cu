// jacobi.cu -- the 7-point Jacobi sweep (Section 4.1's relaxation in the
// Poisson form, applied out of place as a stencil apply is, Section 2.2),
// with temporal blocking: T sweeps per pass over HBM.
//
// One kernel template, jacobi_tb<Policy, T, R, WY, S>, for every storage /
// arithmetic policy (policies.cuh).  A persistent CTA owns a tile of the xy
// plane and marches through a chunk of z planes (2.5D blocking).  A producer
// warp streams each z plane of u and f, with the halo the T sweeps need,
// into a ring of S shared-memory stages by TMA tile loads.  Each consumer
// warp owns 32 x-columns and R rows of the tile and keeps everything else in
// registers:
//   * lane l converts its column of each staged u plane once (rows -T..R+T-1);
//   * x neighbours come from lanes l-1, l+1 by warp shuffle, y neighbours
//     from the lane's own rows, z neighbours from the registers of the
//     previous and next planes (three planes per sweep stage, rotated by a
//     three-way unrolled loop, so no register moves);
//   * sweep stage t (1..T) updates plane p - t when raw plane p arrives, on
//     lanes t..31-t and rows -(T-t)..R-1+(T-t), from stage t-1's planes; its
//     source term is read from the staged f plane, which is held until the
//     last stage has used it;
//   * cells that are not interior (the Dirichlet halo) keep their value
//     through every stage, so the T sweeps equal T separate sweeps exactly.
// Lanes T..31-T of stage T write the result: a tile is (32-2T) x (R*WY).
// No CTA barrier and no shared-memory exchange between warps.
#include <stdlib.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "policies.cuh"

namespace stencil {

struct SweepGeom {
  int64_t nx, ny, nz, sy, sz;
  int tiles_x, tiles_y, zc;  // zc: planes per z chunk
  int bxo, byo;              // output tile extents
  int64_t items;             // tiles_x * tiles_y * z chunks
};

struct Item {
  int xo, yo;  // halo index of the tile's first output column / row
  int zs, ze;  // output planes [zs, ze]
};

__device__ __forceinline__ Item decode_item(const SweepGeom& g, int64_t item) {
  Item t;
  const int64_t txy = static_cast<int64_t>(g.tiles_x) * g.tiles_y;
  const int zci = static_cast<int>(item / txy);
  const int64_t r = item - static_cast<int64_t>(zci) * txy;
  const int ty = static_cast<int>(r / g.tiles_x);
  const int tx = static_cast<int>(r - static_cast<int64_t>(ty) * g.tiles_x);
  t.xo = 1 + tx * g.bxo;
  t.yo = 1 + ty * g.byo;
  t.zs = zci * g.zc + 1;
  t.ze = min(t.zs + g.zc - 1, static_cast<int>(g.nz));
  return t;
}

template <class Pol, int T_, int R_, int WY_, int S_, int MINB_>
struct TbCfg {
  static constexpr int T = T_, R = R_, WY = WY_, S = S_, MINB = MINB_;
  static constexpr int A = 16 / Pol::kElem;      // TMA x granule in elements
  static constexpr int BOXW = 32 + A;            // staged columns (any 0 <= off < A)
  static constexpr int BXO = 32 - 2 * T;         // output columns per tile
  static constexpr int BYO = R * WY;             // output rows per tile
  static constexpr int NROW = R + 2 * T;         // rows a warp converts per plane
  static constexpr int UROWS = BYO + 2 * T;
  static constexpr int FROWS = BYO + 2 * T - 2;
  static constexpr int UBYTES = BOXW * UROWS * Pol::kElem;
  static constexpr int FBYTES = BOXW * FROWS * Pol::kElem;
  static constexpr int UB = (UBYTES + 127) / 128 * 128;
  static constexpr int FB = (FBYTES + 127) / 128 * 128;
  static constexpr int STAGE = UB + FB;
  static constexpr int RING = S * STAGE;
  static constexpr int CONSUMERS = 32 * WY;
  static constexpr int THREADS = CONSUMERS + 32;
  static constexpr int SMEM = 128 + RING + 128;
  static_assert(S >= T + 2, "each warp holds T+1 staged planes");
  static_assert(NROW <= 32, "row mask");
};

__device__ __forceinline__ int align_down(int x, int a) { return x >= 0 ? x - x % a : -((-x + a - 1) / a) * a; }

// Producer (lane 0 of the last warp): for every item of this CTA, the u
// boxes of planes zs-T .. ze+T and the f boxes of the same planes.
template <class Cfg>
__device__ __forceinline__ void produce(const CUtensorMap* tm_u, const CUtensorMap* tm_f,
                                        const SweepGeom& g, uint32_t bar_full, uint32_t bar_empty,
                                        uint32_t ring, uint32_t* status, volatile int* abort_flag) {
  constexpr int S = Cfg::S, T = Cfg::T;
  prefetch_tensormap(tm_u);
  prefetch_tensormap(tm_f);
  uint32_t it = 0;
  for (int64_t item = blockIdx.x; item < g.items; item += gridDim.x) {
    const Item t = decode_item(g, item);
    const int xa = align_down(t.xo - T, Cfg::A);
    for (int p = t.zs - T; p <= t.ze + T; ++p, ++it) {
      const uint32_t s = it % S;
      if (*abort_flag || !mbar_wait_bounded(bar_empty + 8 * s, ((it / S) & 1u) ^ 1u, status)) {
        *abort_flag = 1;
        goto drain;
      }
      mbar_arrive_expect_tx(bar_full + 8 * s, Cfg::UBYTES + Cfg::FBYTES);
      tma_load_3d(ring + s * Cfg::STAGE, tm_u, xa, t.yo - T, p, bar_full + 8 * s);
      tma_load_3d(ring + s * Cfg::STAGE + Cfg::UB, tm_f, xa, t.yo - T + 1, p, bar_full + 8 * s);
    }
  }
drain:
  // Do not leave the CTA with copies in flight into its shared memory.
  for (uint32_t q = (it > S ? it - S : 0); q < it; ++q)
    if (!mbar_wait_bounded(bar_full + 8 * (q % S), (q / S) & 1u, status)) break;
}

// Register state of one consumer lane.
template <class Pol, class Cfg>
struct LaneState {
  using C = typename Pol::C;
  C W[Cfg::T][3][Cfg::NROW];  // stage t's three planes (stage 0 = converted input)
};

// One z step with the three plane slots rotated by ROT: raw plane p (sequence
// number seq) has arrived in stage slot `slot`.
template <class Pol, class Cfg, int ROT>
__device__ __forceinline__ void tb_step(LaneState<Pol, Cfg>& st, const typename Pol::K& k,
                                        const unsigned char* ring, int slot, uint32_t seq, int j,
                                        int p, int row0, int lane, int off, bool xin, uint32_t ymask,
                                        typename Pol::T* orow0, int64_t sy, int64_t sz, int nz) {
  using T = typename Pol::T;
  using C = typename Pol::C;
  constexpr int TT = Cfg::T, S = Cfg::S;
  constexpr int OLD = (0 + ROT) % 3, MID = (1 + ROT) % 3, NEW = (2 + ROT) % 3;
  {
    const T* U = reinterpret_cast<const T*>(ring + slot * Cfg::STAGE);
    const bool zin_p = (p >= 1 && p <= nz);
#pragma unroll
    for (int q = 0; q < Cfg::NROW; ++q) st.W[0][NEW][q] = Pol::in(U[(row0 + q) * Cfg::BOXW + off + lane], k);
    // Cells outside the interior (Dirichlet halo, or beyond the grid) may be
    // stored in a different form (PolResident keeps them binary64); only
    // warps that touch one take this branch.
    const uint32_t halo_rows = (xin && zin_p) ? ~ymask : 0xffffffffu;
    if (__any_sync(0xffffffffu, (halo_rows & ((1u << Cfg::NROW) - 1u)) != 0u)) {
#pragma unroll
      for (int q = 0; q < Cfg::NROW; ++q)
        if ((halo_rows >> q) & 1u) st.W[0][NEW][q] = Pol::in_halo(U[(row0 + q) * Cfg::BOXW + off + lane], k);
    }
  }
#pragma unroll
  for (int t = 1; t <= TT; ++t) {
    if (j < 2 * t) break;  // stage t has no complete input yet
    const int q = p - t;   // plane this stage updates
    const bool zin = (q >= 1 && q <= nz);
    const T* F = reinterpret_cast<const T*>(ring + ((seq - t) % S) * Cfg::STAGE + Cfg::UB);
    constexpr int dummy = 0;
    (void)dummy;
    const int nr = Cfg::R + 2 * (TT - t);  // rows this stage updates
#pragma unroll
    for (int rr = 0; rr < Cfg::R + 2 * (TT - 1); ++rr) {
      if (rr >= nr) break;
      const C c = st.W[t - 1][MID][rr + 1];
      const C xm = __shfl_up_sync(0xffffffffu, c, 1);
      const C xp = __shfl_down_sync(0xffffffffu, c, 1);
      const int w = rr - (TT - t);  // warp row, -T..R+T-1
      const bool in = xin && zin && ((ymask >> (w + TT)) & 1u);
      C v = c;
      if (in) {
        const T fv = F[(row0 + rr + t - 1) * Cfg::BOXW + off + lane];
        v = Pol::update(xm, xp, st.W[t - 1][MID][rr], st.W[t - 1][MID][rr + 2],
                        st.W[t - 1][OLD][rr + 1], st.W[t - 1][NEW][rr + 1], fv, k);
      }
      if (t < TT) {
        st.W[t][NEW][rr] = v;
      } else if (in && lane >= TT && lane < 32 - TT) {
        orow0[static_cast<int64_t>(q) * sz + rr * sy] = Pol::out(v, k);
      }
    }
  }
}

template <class Pol, class Cfg>
__global__ void __launch_bounds__(Cfg::THREADS, Cfg::MINB)
    jacobi_tb(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_f,
              typename Pol::T* __restrict__ out, const SweepGeom g, const SweepArgs args) {
  constexpr int S = Cfg::S, TT = Cfg::T, WY = Cfg::WY;
  extern __shared__ unsigned char smem_raw[];
  __shared__ int abort_flag;
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const uint32_t bar_full = smem_addr(base);
  const uint32_t bar_empty = bar_full + 8 * S;
  unsigned char* ring = base + 128;
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(bar_full + 8 * s, 1);
      mbar_init(bar_empty + 8 * s, WY);
    }
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  const int warp = tid >> 5;
  const int lane = tid & 31;
  if (warp == WY) {
    if (lane == 0)
      produce<Cfg>(&tm_u, &tm_f, g, bar_full, bar_empty, smem_addr(ring), args.status, &abort_flag);
    return;
  }
  const typename Pol::K k = Pol::make(args);
  const int row0 = warp * Cfg::R;
  LaneState<Pol, Cfg> st;
  uint32_t it = 0;
  for (int64_t item = blockIdx.x; item < g.items; item += gridDim.x) {
    const Item t = decode_item(g, item);
    const int xa = align_down(t.xo - TT, Cfg::A);
    const int off = t.xo - TT - xa;
    const int64_t x = t.xo - TT + lane;  // halo index of this lane's column
    const bool xin = (x >= 1 && x <= g.nx);
    uint32_t ymask = 0;                  // bit w+T: warp row w is interior
#pragma unroll
    for (int w = -TT; w < Cfg::R + TT; ++w) {
      const int64_t y = t.yo + row0 + w;
      ymask |= (y >= 1 && y <= g.ny) ? (1u << (w + TT)) : 0u;
    }
    typename Pol::T* orow0 = out + x + (t.yo + row0) * g.sy;
    const int steps = (t.ze - t.zs + 1) + 2 * TT;
    const uint32_t seq0 = it;
    int j = 0;
    auto wait = [&](int jj) -> int {
      const uint32_t seq = seq0 + jj;
      const uint32_t s = seq % S;
      if (!mbar_wait_bounded(bar_full + 8 * s, (seq / S) & 1u, args.status)) {
        abort_flag = 1;
        return -1;
      }
      return static_cast<int>(s);
    };
    auto release = [&](uint32_t seq) {
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_empty + 8 * (seq % S));
    };
    for (;;) {
#define STENCIL_TB_STEP(ROT)                                                                    \
  {                                                                                             \
    const int slot = wait(j);                                                                   \
    if (slot < 0) return;                                                                       \
    tb_step<Pol, Cfg, ROT>(st, k, ring, slot, seq0 + j, j, t.zs - TT + j, row0, lane, off, xin, \
                           ymask, orow0, g.sy, g.sz, static_cast<int>(g.nz));                   \
    if (j >= TT) release(seq0 + j - TT);                                                        \
    if (++j >= steps) break;                                                                    \
  }
      STENCIL_TB_STEP(0)
      STENCIL_TB_STEP(1)
      STENCIL_TB_STEP(2)
#undef STENCIL_TB_STEP
    }
    for (int q = steps - TT; q < steps; ++q)
      if (q >= 0) release(seq0 + q);
    it = seq0 + steps;
  }
}

// max|u| over every cell (halo included) and max|f| over the interior, as
// the bit patterns of non-negative doubles (their integer order is their
// numeric order; NaN sorts above Inf, so a NaN anywhere is seen).
__global__ void range_kernel(const double* __restrict__ u, const double* __restrict__ f,
                             int64_t nx, int64_t ny, int64_t nz, int64_t usy, int64_t usz,
                             int64_t fsy, int64_t fsz, unsigned long long* maxbits) {
  const int64_t rows = (ny + 2) * (nz + 2);
  unsigned long long mu = 0, mf = 0;
  for (int64_t row = blockIdx.x * int64_t(blockDim.y) + threadIdx.y; row < rows;
       row += int64_t(gridDim.x) * blockDim.y) {
    const int64_t k = row / (ny + 2);
    const int64_t j = row - k * (ny + 2);
    const bool inner = (j >= 1 && j <= ny && k >= 1 && k <= nz);
    for (int64_t i = threadIdx.x; i < nx + 2; i += blockDim.x) {
      const unsigned long long bu =
          static_cast<unsigned long long>(__double_as_longlong(u[i + j * usy + k * usz])) &
          0x7fffffffffffffffull;
      mu = bu > mu ? bu : mu;
      if (inner && i >= 1 && i <= nx) {
        const unsigned long long bf =
            static_cast<unsigned long long>(__double_as_longlong(f[i + j * fsy + k * fsz])) &
            0x7fffffffffffffffull;
        mf = bf > mf ? bf : mf;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long a = __shfl_xor_sync(0xffffffffu, mu, o);
    const unsigned long long b = __shfl_xor_sync(0xffffffffu, mf, o);
    mu = a > mu ? a : mu;
    mf = b > mf ? b : mf;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&maxbits[0], mu);
    atomicMax(&maxbits[1], mf);
  }
}

// Copy the halo cells of src into dst (same extents).
template <class T>
__global__ void halo_copy_kernel(const T* __restrict__ src, T* __restrict__ dst, int64_t nx,
                                 int64_t ny, int64_t nz, int64_t ssy, int64_t ssz, int64_t dsy,
                                 int64_t dsz) {
  const int64_t X = nx + 2, Y = ny + 2;
  const int64_t nzf = 2 * X * Y;          // planes k = 0, nz+1
  const int64_t nyf = 2 * X * nz;         // rows j = 0, ny+1 of interior planes
  const int64_t nxf = 2 * ny * nz;        // columns i = 0, nx+1 of interior rows
  const int64_t total = nzf + nyf + nxf;
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < total;
       q += int64_t(gridDim.x) * blockDim.x) {
    int64_t i, j, k;
    if (q < nzf) {
      const int64_t side = q / (X * Y), r = q - side * X * Y;
      k = side ? nz + 1 : 0; j = r / X; i = r - j * X;
    } else if (q < nzf + nyf) {
      const int64_t r0 = q - nzf, side = r0 / (X * nz), r = r0 - side * X * nz;
      j = side ? ny + 1 : 0; k = 1 + r / X; i = r - (k - 1) * X;
    } else {
      const int64_t r0 = q - nzf - nyf, side = r0 / (ny * nz), r = r0 - side * ny * nz;
      i = side ? nx + 1 : 0; k = 1 + r / ny; j = 1 + r - (k - 1) * ny;
    }
    dst[i + j * dsy + k * dsz] = src[i + j * ssy + k * ssz];
  }
}

// Copy the interior cells of src into dst.
template <class T>
__global__ void interior_copy_kernel(const T* __restrict__ src, T* __restrict__ dst, int64_t nx,
                                     int64_t ny, int64_t nz, int64_t ssy, int64_t ssz,
                                     int64_t dsy, int64_t dsz) {
  const int64_t rows = ny * nz;
  for (int64_t row = blockIdx.x * int64_t(blockDim.y) + threadIdx.y; row < rows;
       row += int64_t(gridDim.x) * blockDim.y) {
    const int64_t k = 1 + row / ny;
    const int64_t j = 1 + row - (k - 1) * ny;
    for (int64_t i = 1 + threadIdx.x; i <= nx; i += blockDim.x)
      dst[i + j * dsy + k * dsz] = src[i + j * ssy + k * ssz];
  }
}

// Resident fixed point: convert the interior of u (in place) to the biased
// integers U and the interior of f to G = round(h*h*f*2^S) in work.
__global__ void fx_pack_kernel(double* __restrict__ u, const double* __restrict__ f,
                               unsigned long long* __restrict__ work, int64_t nx, int64_t ny,
                               int64_t nz, int64_t usy, int64_t usz, int64_t fsy, int64_t fsz,
                               int64_t wsy, int64_t wsz, SweepArgs a) {
  const FixedParams k = PolResident::make(a);
  const int64_t rows = ny * nz;
  for (int64_t row = blockIdx.x * int64_t(blockDim.y) + threadIdx.y; row < rows;
       row += int64_t(gridDim.x) * blockDim.y) {
    const int64_t kz = 1 + row / ny;
    const int64_t j = 1 + row - (kz - 1) * ny;
    double* ur = u + j * usy + kz * usz;
    const double* fr = f + j * fsy + kz * fsz;
    unsigned long long* wr = work + j * wsy + kz * wsz;
    for (int64_t i = 1 + threadIdx.x; i <= nx; i += blockDim.x) {
      ur[i] = __longlong_as_double(static_cast<long long>(fx_in(ur[i], k.Cu)));
      wr[i] = static_cast<unsigned long long>(fx_source(fr[i], k.Cg, k.H));
    }
  }
}

// Back to binary64: the interior of src (U) into the interior of u.
__global__ void fx_unpack_kernel(const unsigned long long* __restrict__ src, double* __restrict__ u,
                                 int64_t nx, int64_t ny, int64_t nz, int64_t ssy, int64_t ssz,
                                 int64_t usy, int64_t usz, SweepArgs a) {
  const FixedParams k = PolResident::make(a);
  if (k.bad && threadIdx.x == 0 && threadIdx.y == 0 && blockIdx.x == 0)
    atomicOr(a.status, k.bad == 1 ? kStatusNonFinite : kStatusRange);
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  const int64_t rows = ny * nz;
  for (int64_t row = blockIdx.x * int64_t(blockDim.y) + threadIdx.y; row < rows;
       row += int64_t(gridDim.x) * blockDim.y) {
    const int64_t kz = 1 + row / ny;
    const int64_t j = 1 + row - (kz - 1) * ny;
    const unsigned long long* sr = src + j * ssy + kz * ssz;
    double* ur = u + j * usy + kz * usz;
    for (int64_t i = 1 + threadIdx.x; i <= nx; i += blockDim.x) ur[i] = k.bad ? nan : fx_out(sr[i], k.S);
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

template <class Cfg>
SweepGeom make_geom(const Grid& u, int zc) {
  SweepGeom g;
  g.nx = u.nx; g.ny = u.ny; g.nz = u.nz; g.sy = u.sy; g.sz = u.sz;
  g.bxo = Cfg::BXO;
  g.byo = Cfg::BYO;
  g.tiles_x = static_cast<int>((u.nx + Cfg::BXO - 1) / Cfg::BXO);
  g.tiles_y = static_cast<int>((u.ny + Cfg::BYO - 1) / Cfg::BYO);
  g.zc = zc;
  const int64_t zch = (u.nz + zc - 1) / zc;
  g.items = static_cast<int64_t>(g.tiles_x) * g.tiles_y * zch;
  return g;
}

// z chunk length: the longest (fewest re-read planes, 2T per chunk) that
// still gives every resident CTA about four items for load balance.
int pick_zc(int64_t tiles_xy, int64_t nz, int slots, int T) {
  int zc = 256;
  while (zc > 4 * T + 4 && tiles_xy * ((nz + zc - 1) / zc) < 4 * static_cast<int64_t>(slots)) zc /= 2;
  return static_cast<int>(std::min<int64_t>(zc, nz));
}

template <class K>
int grid_for(K kernel, int threads, int smem, int64_t items, int num_sms, int* grid, int* per_sm_out) {
  int per_sm = 0;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return check_cuda(e, "cudaFuncSetAttribute");
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return check_cuda(e, "cudaFuncSetAttribute(carveout)");
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  if (e != cudaSuccess) return check_cuda(e, "occupancy");
  if (per_sm < 1) return set_error(STENCIL_ERR_CUDA, "sweep kernel cannot be resident");
  *grid = static_cast<int>(std::min<int64_t>(items, static_cast<int64_t>(per_sm) * num_sms));
  if (per_sm_out) *per_sm_out = per_sm;
  return STENCIL_OK;
}

template <class Pol, class Cfg>
int run_tb(stencil_ctx* ctx, const Grid& in, const Grid& out, const Grid& f, const SweepArgs& a,
           cudaStream_t st) {
  auto kern = jacobi_tb<Pol, Cfg>;
  CUtensorMap tu, tf;
  int rc = make_tensor_map(&tu, in, Cfg::BOXW, Cfg::UROWS);
  if (rc) return rc;
  rc = make_tensor_map(&tf, f, Cfg::BOXW, Cfg::FROWS);
  if (rc) return rc;
  int grid = 0, per_sm = 0;
  const int64_t txy = ((in.nx + Cfg::BXO - 1) / Cfg::BXO) * ((in.ny + Cfg::BYO - 1) / Cfg::BYO);
  rc = grid_for(kern, Cfg::THREADS, Cfg::SMEM, txy * in.nz, ctx->num_sms, &grid, &per_sm);
  if (rc) return rc;
  const int zc = pick_zc(txy, in.nz, per_sm * ctx->num_sms, Cfg::T);
  const SweepGeom g = make_geom<Cfg>(in, zc);
  grid = static_cast<int>(std::min<int64_t>(g.items, static_cast<int64_t>(per_sm) * ctx->num_sms));
  kern<<<grid, Cfg::THREADS, Cfg::SMEM, st>>>(tu, tf, static_cast<typename Pol::T*>(out.data), g, a);
  return check_cuda(cudaGetLastError(), "jacobi_tb launch");
}

// Compiled tile shapes: (policy, sweeps per pass T, rows per warp R, warps
// WY, stages S, CTAs per SM the register budget targets).
using FixT1 = TbCfg<PolFixed, 1, 8, 4, 4, 3>;
using ResT1 = TbCfg<PolResident, 1, 8, 4, 4, 3>;
using ResT2 = TbCfg<PolResident, 2, 4, 4, 5, 2>;
using F64T1 = TbCfg<PolF64, 1, 8, 4, 4, 3>;
using F32T1 = TbCfg<PolF32, 1, 8, 8, 4, 2>;
using F32T2 = TbCfg<PolF32, 2, 8, 4, 5, 1>;
using F32T4 = TbCfg<PolF32, 4, 4, 4, 7, 1>;
using B16T1 = TbCfg<PolBF16, 1, 8, 8, 4, 2>;
using B16T2 = TbCfg<PolBF16, 2, 8, 4, 5, 1>;
using B16T4 = TbCfg<PolBF16, 4, 4, 4, 7, 1>;

// One pass of T sweeps from `in` to `out`.
int run_pass(stencil_ctx* ctx, int dtype, bool fixed, int T, const Grid& in, const Grid& out,
             const Grid& f, const SweepArgs& a, cudaStream_t st) {
  if (dtype == kDtypeU64) {
    if (T >= 2) return run_tb<PolResident, ResT2>(ctx, in, out, f, a, st);
    return run_tb<PolResident, ResT1>(ctx, in, out, f, a, st);
  }
  if (dtype == STENCIL_F64) {
    if (!fixed) return run_tb<PolF64, F64T1>(ctx, in, out, f, a, st);
    return run_tb<PolFixed, FixT1>(ctx, in, out, f, a, st);
  }
  if (dtype == STENCIL_F32) {
    if (T >= 4) return run_tb<PolF32, F32T4>(ctx, in, out, f, a, st);
    if (T >= 2) return run_tb<PolF32, F32T2>(ctx, in, out, f, a, st);
    return run_tb<PolF32, F32T1>(ctx, in, out, f, a, st);
  }
  if (T >= 4) return run_tb<PolBF16, B16T4>(ctx, in, out, f, a, st);
  if (T >= 2) return run_tb<PolBF16, B16T2>(ctx, in, out, f, a, st);
  return run_tb<PolBF16, B16T1>(ctx, in, out, f, a, st);
}

// Sweeps per pass the library picks when the caller passes 0.
int default_spp(int dtype, bool fixed) {
  (void)fixed;
  if (dtype == STENCIL_F64 || dtype == kDtypeU64) return 1;
  return 4;
}

// Largest compiled T not above `want` for this policy.
int supported_t(int dtype, bool fixed, int want) {
  if (dtype == kDtypeU64) return want >= 2 ? 2 : 1;
  if (dtype == STENCIL_F64) return 1;
  (void)fixed;
  return want >= 4 ? 4 : (want >= 2 ? 2 : 1);
}

template <class T>
int copy_halo(const Grid& src, const Grid& dst, cudaStream_t st) {
  const int64_t total = 2 * (src.nx + 2) * (src.ny + 2) + 2 * (src.nx + 2) * src.nz + 2 * src.ny * src.nz;
  const int blocks = static_cast<int>(std::min<int64_t>((total + 255) / 256, 4096));
  halo_copy_kernel<T><<<blocks, 256, 0, st>>>(static_cast<const T*>(src.data), static_cast<T*>(dst.data),
                                              src.nx, src.ny, src.nz, src.sy, src.sz, dst.sy, dst.sz);
  return check_cuda(cudaGetLastError(), "halo copy");
}

template <class T>
int copy_interior(const Grid& src, const Grid& dst, cudaStream_t st) {
  const int64_t rows = src.ny * src.nz;
  const int blocks = static_cast<int>(std::min<int64_t>((rows + 7) / 8, 8192));
  interior_copy_kernel<T><<<blocks, dim3(64, 8), 0, st>>>(
      static_cast<const T*>(src.data), static_cast<T*>(dst.data), src.nx, src.ny, src.nz, src.sy,
      src.sz, dst.sy, dst.sz);
  return check_cuda(cudaGetLastError(), "interior copy");
}

int copy_halo_any(const Grid& src, const Grid& dst, cudaStream_t st) {
  if (src.elem == 8) return copy_halo<double>(src, dst, st);
  if (src.elem == 4) return copy_halo<float>(src, dst, st);
  return copy_halo<unsigned short>(src, dst, st);
}

int copy_interior_any(const Grid& src, const Grid& dst, cudaStream_t st) {
  if (src.elem == 8) return copy_interior<double>(src, dst, st);
  if (src.elem == 4) return copy_interior<float>(src, dst, st);
  return copy_interior<unsigned short>(src, dst, st);
}

}  // namespace

int launch_jacobi(stencil_ctx* ctx, const Grid& u, const Grid& ut, const Grid& f, const Grid* work,
                  double h, int64_t nsweeps, int spp, int flags, cudaStream_t st) {
  if (nsweeps == 0) return STENCIL_OK;
  const bool fixed = (u.dtype == STENCIL_F64) && (flags != STENCIL_SWEEP_FP64_NATIVE);
  const bool resident = fixed && work != nullptr && nsweeps >= kResidentMinSweeps;
  int rc = copy_halo_any(u, ut, st);
  if (rc) return rc;
  SweepArgs a;
  a.hh = h * h;
  a.nsw = static_cast<double>(nsweeps);
  a.lmin = static_cast<double>(std::min(std::min(u.nx, u.ny), u.nz) + 1) * h;
  a.maxbits = reinterpret_cast<const unsigned long long*>(ctx->scratch + kScratchMaxU);
  a.status = reinterpret_cast<uint32_t*>(ctx->scratch + kScratchStatus);
  if (fixed) {
    rc = check_cuda(cudaMemsetAsync(ctx->scratch + kScratchMaxU, 0, 16, st), "memset range");
    if (rc) return rc;
    const int64_t rows = (u.ny + 2) * (u.nz + 2);
    const int blocks = static_cast<int>(std::min<int64_t>((rows + 7) / 8, 8 * ctx->num_sms));
    range_kernel<<<blocks, dim3(32, 8), 0, st>>>(
        static_cast<const double*>(u.data), static_cast<const double*>(f.data), u.nx, u.ny, u.nz,
        u.sy, u.sz, f.sy, f.sz, reinterpret_cast<unsigned long long*>(ctx->scratch + kScratchMaxU));
    rc = check_cuda(cudaGetLastError(), "range kernel");
    if (rc) return rc;
  }
  const int64_t rows = u.ny * u.nz;
  const int cblocks = static_cast<int>(std::min<int64_t>((rows + 7) / 8, 16 * ctx->num_sms));
  Grid ui = u, ti = ut, fi = f;
  if (resident) {
    fx_pack_kernel<<<cblocks, dim3(32, 8), 0, st>>>(
        static_cast<double*>(u.data), static_cast<const double*>(f.data),
        static_cast<unsigned long long*>(work->data), u.nx, u.ny, u.nz, u.sy, u.sz, f.sy, f.sz,
        work->sy, work->sz, a);
    rc = check_cuda(cudaGetLastError(), "pack kernel");
    if (rc) return rc;
    ui.dtype = ti.dtype = kDtypeU64;
    fi = *work;
    fi.dtype = kDtypeU64;
  }
  const int want = spp > 0 ? spp : default_spp(resident ? kDtypeU64 : u.dtype, fixed);
  const Grid* a_in = &ui;
  const Grid* b_out = &ti;
  int64_t left = nsweeps;
  while (left > 0) {
    const int T = supported_t(ui.dtype, fixed, static_cast<int>(std::min<int64_t>(left, want)));
    rc = run_pass(ctx, ui.dtype, fixed, T, *a_in, *b_out, fi, a, st);
    if (rc) return rc;
    std::swap(a_in, b_out);
    left -= T;
  }
  if (resident) {
    fx_unpack_kernel<<<cblocks, dim3(32, 8), 0, st>>>(
        static_cast<const unsigned long long*>(a_in->data), static_cast<double*>(u.data), u.nx, u.ny,
        u.nz, a_in->sy, a_in->sz, u.sy, u.sz, a);
    return check_cuda(cudaGetLastError(), "unpack kernel");
  }
  if (a_in != &ui) rc = copy_interior_any(*a_in, u, st);
  return rc;
}

}  // namespace stencil
