// sweep_kernel.cuh -- the 7-point Jacobi sweep kernel template (Section 4.1's
// relaxation in the Poisson form, applied out of place as a stencil apply is,
// Section 2.2), with temporal blocking: T sweeps per pass over HBM.  Its
// red-black Gauss-Seidel sibling is sweep_rb_kernel.cuh.
//
// jacobi_tb<Policy, Cfg, Src>: one kernel for every storage / arithmetic
// policy (policies.cuh) and every work source: a single grid (SrcGrid) or a
// table of independent instances (SrcBatch, batch.cu).  Persistent CTAs
// stride over work items, each an (xy tile, z chunk) of one grid, and march
// through the chunk's z planes (2.5D blocking).  A producer warp streams each
// z plane of u and f, with the halo the T sweeps need, into a ring of S
// shared-memory stages by TMA tile loads.  Each consumer warp owns 32
// x-columns and R rows of the tile and keeps everything else in registers:
//   * lane l converts its column of each staged u plane once (rows -T..R+T-1);
//   * x neighbours come from lanes l-1, l+1 by warp shuffle, y neighbours
//     from the lane's own rows, z neighbours from the registers of the
//     previous and next planes (three planes per sweep stage, rotated by a
//     three-way unrolled loop, so no register moves);
//   * sweep stage t (1..T) updates plane p - t when raw plane p arrives, on
//     its valid lanes (below) and rows -(T-t)..R-1+(T-t), from stage t-1's
//     planes; its source term is read from the staged f plane, which is
//     held until the last stage has used it;
//   * cells that are not interior (the Dirichlet halo) keep their value
//     through every stage, so the T sweeps equal T separate sweeps exactly.
// With EDGE (the default at one sweep per pass), stage 1 reads the x
// neighbours that fall outside the warp (left of lane 0, right of lane 31)
// from the staged raw plane instead of shuffling them, so it is valid on
// all 32 lanes and stage t on lanes t-1..32-t: lanes T-1..32-T of stage T
// write the result, a tile is (34-2T) x (R*WY) (32 columns at one sweep per
// pass).  Without EDGE stage t is valid on lanes t..31-t and a tile is
// (32-2T) x (R*WY).
// No CTA barrier and no shared-memory exchange between warps.
#pragma once

#include "common.cuh"
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

// EDGE is the default at one sweep per pass only: with two sweeps per pass
// it gains two output columns per tile but stages a wider box (40 instead of
// 36 FP32 columns), and measured slower on a 512^3 grid and on the batch.
// XSMEM (one sweep per pass, policies whose halo cells convert as interior
// ones): both x neighbours are read from the staged plane instead of
// shuffled, so no lane is special.
template <class Pol, int T_, int R_, int WY_, int S_, int MINB_, bool EDGE_ = (T_ == 1), bool XSMEM_ = false>
struct TbCfg {
  static constexpr int T = T_, R = R_, WY = WY_, S = S_, MINB = MINB_;
  static constexpr bool RB = false;
  static constexpr bool EDGE = EDGE_;
  static constexpr bool XSMEM = XSMEM_;
  static_assert(!XSMEM || (T == 1 && EDGE && !Pol::kFixed), "staged x neighbours: one-sweep float policies");
  static constexpr int A = 16 / Pol::kElem;      // TMA x granule in elements
  // Staged columns from xo - T rounded down to the TMA granule: the 32 lanes
  // (+ A - 1 for an unaligned start), or, with EDGE, the 34 columns
  // lane 0 - 1 .. lane 31 + 1 (+ A - 1; at one sweep per pass tiles start
  // at xo = 1 + 32 k, so xo - 1 is always aligned).
  static constexpr int BOXW = !EDGE ? 32 + A : (T == 1 ? (34 + A - 1) / A * A : (33 + A + A - 1) / A * A);
  static constexpr int BXO = EDGE ? 34 - 2 * T : 32 - 2 * T;  // output columns per tile
  static constexpr int XL = EDGE ? T - 1 : T;    // lane l holds column xo - XL + l
  static constexpr int COL0 = T - XL;            // staged column of lane 0 (after off)
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

// What a work item needs: its tile and chunk, its grid's geometry, the tensor
// maps of the input and source, the output pointer and the policy constants.
template <class Pol>
struct ItemView {
  Item t;
  int64_t nx, ny, nz, sy, sz;
  int64_t osy, osz;  // strides of the output grid
  const CUtensorMap* tm_u;
  const CUtensorMap* tm_f;
  typename Pol::T* out;
  typename Pol::K k;
};

// Parameters of a single-grid launch (passed as a __grid_constant__ so the
// tensor maps can be addressed in parameter space).
template <class Pol>
struct SingleParams {
  CUtensorMap tm_u;
  CUtensorMap tm_f;
  CUtensorMap tm_f64;  // resident fixed point: the binary64 source (read by fpath passes)
  typename Pol::T* out;
  int64_t osy, osz;    // strides of the output grid
  SweepGeom g;
  SweepArgs a;
};

template <class Pol>
struct SrcGrid {
  using Params = SingleParams<Pol>;
  const Params* p;
  typename Pol::K k;
  bool f64src = false;  // resident fixed point: this pass loads the binary64 source
  __device__ __forceinline__ SrcGrid(const Params* pp, bool need_k) : p(pp) {
    if (need_k) k = Pol::make(pp->a);
    if constexpr (Pol::kResident) {
      const int prev = (pp->a.pass + 2) % 3;
      f64src = pp->a.fxgscale[prev] != pp->a.fxscale[prev];
    }
  }
  __device__ __forceinline__ int64_t items() const { return p->g.items; }
  __device__ __forceinline__ uint32_t* status() const { return p->a.status; }
  // Fixed point: publish this pass's scale (block 0), and combine the
  // magnitude keys of what a warp wrote.
  __device__ __forceinline__ void fx_begin() const {
    if constexpr (Pol::kTrack) Pol::publish(p->a, k);
  }
  __device__ __forceinline__ void fx_end(uint32_t key) const {
    if constexpr (Pol::kTrack) fx_track_commit(p->a, key);
  }
  // Residual: this CTA's sums of R^2 (exact) and f^2, over its consumer
  // warps in warp order, into partial slot blockIdx.x (block 0 also stores
  // the CTA count).  Every consumer warp calls it.
  __device__ __forceinline__ void resid_end(typename Pol::Track& trk, int warp, int nwarps) const {
    if constexpr (Pol::kResidual) {
      __shared__ unsigned long long wsum[4 * 32];
      __syncwarp();
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long a0 = __shfl_xor_sync(0xffffffffu, trk.s0, o);
        const unsigned long long a1 = __shfl_xor_sync(0xffffffffu, trk.s1, o);
        const unsigned long long a2 = __shfl_xor_sync(0xffffffffu, trk.s2, o);
        const double af = __shfl_xor_sync(0xffffffffu, trk.ff, o);
        trk.merge(a0, a1, a2, af);
      }
      if (p->a.seen) {  // bounds of the magnitudes this warp read (the next call's scale guess)
        const uint32_t mu = __reduce_max_sync(0xffffffffu, trk.mu);
        const uint32_t mf = __reduce_max_sync(0xffffffffu, trk.mf);
        if ((threadIdx.x & 31) == 0) {
          atomicMax(p->a.seen, (static_cast<unsigned long long>(mu) << 32) | 0xffffffffull);
          atomicMax(p->a.seen + 1, (static_cast<unsigned long long>(mf) << 32) | 0xffffffffull);
        }
      }
      if ((threadIdx.x & 31) == 0) {
        wsum[4 * warp] = trk.s0;
        wsum[4 * warp + 1] = trk.s1;
        wsum[4 * warp + 2] = trk.s2;
        wsum[4 * warp + 3] = static_cast<unsigned long long>(__double_as_longlong(trk.ff));
      }
      named_barrier(1, 32 * nwarps);
      if (threadIdx.x == 0) {
        typename Pol::Track t;
        for (int w = 0; w < nwarps; ++w)
          t.merge(wsum[4 * w], wsum[4 * w + 1], wsum[4 * w + 2],
                  __longlong_as_double(static_cast<long long>(wsum[4 * w + 3])));
        unsigned long long* out = p->a.rpart + 4 + 4 * static_cast<int64_t>(blockIdx.x);
        out[0] = t.s0;
        out[1] = t.s1;
        out[2] = t.s2;
        out[3] = static_cast<unsigned long long>(__double_as_longlong(t.ff));
        if (blockIdx.x == 0) p->a.rpart[0] = gridDim.x;
      }
    }
  }
  // Resident fixed point, an fpath pass: store the source of cell (x, y, z).
  __device__ __forceinline__ void store_source(int64_t x, int64_t y, int64_t z, unsigned long long g) const {
    const SweepArgs& a = p->a;
    a.gdst[x + y * a.gsy + z * a.gsz] = g;
  }
  __device__ __forceinline__ bool view(int64_t item, ItemView<Pol>& v) const {
    v.t = decode_item(p->g, item);
    v.nx = p->g.nx; v.ny = p->g.ny; v.nz = p->g.nz; v.sy = p->g.sy; v.sz = p->g.sz;
    v.osy = p->osy; v.osz = p->osz;
    v.tm_u = &p->tm_u;
    v.tm_f = f64src ? &p->tm_f64 : &p->tm_f;
    v.out = p->out;
    v.k = k;
    return true;
  }
};

// Producer (lane 0 of the last warp): for every item of this CTA, the u
// boxes of planes zs-T .. ze+T and the f boxes of the same planes.
template <class Pol, class Cfg, class Src>
__device__ __forceinline__ void produce(const Src& src, uint32_t bar_full, uint32_t bar_empty,
                                        uint32_t ring, volatile int* abort_flag) {
  constexpr int S = Cfg::S, T = Cfg::T;
  uint32_t it = 0;
  uint32_t* status = src.status();
  for (int64_t item = blockIdx.x; item < src.items(); item += gridDim.x) {
    ItemView<Pol> v;
    if (!src.view(item, v)) continue;
    prefetch_tensormap(v.tm_u);
    prefetch_tensormap(v.tm_f);
    const Item& t = v.t;
    const int xa = align_down(t.xo - T, Cfg::A);
    for (int p = t.zs - T; p <= t.ze + T; ++p, ++it) {
      const uint32_t s = it % S;
      if (*abort_flag || !mbar_wait_bounded(bar_empty + 8 * s, ((it / S) & 1u) ^ 1u, status)) {
        *abort_flag = 1;
        goto drain;
      }
      mbar_arrive_expect_tx(bar_full + 8 * s, Cfg::UBYTES + Cfg::FBYTES);
      tma_load_3d(ring + s * Cfg::STAGE, v.tm_u, xa, t.yo - T, p, bar_full + 8 * s);
      tma_load_3d(ring + s * Cfg::STAGE + Cfg::UB, v.tm_f, xa, t.yo - T + 1, p, bar_full + 8 * s);
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
// number seq) has arrived in stage slot `slot`.  RS (resident fixed point,
// rare passes): the pass writes its output at a new scale (k.dshift: each
// written value is shifted) and/or its ring holds the binary64 source
// (k.fpath: converted at the computing scale as it is used, and stored in
// the work grid for the cells this lane writes).
template <class Pol, class Cfg, class Src, int ROT, bool RS>
__device__ __forceinline__ void tb_step(LaneState<Pol, Cfg>& st, const typename Pol::K& k,
                                        const unsigned char* ring, int slot, uint32_t seq, int j,
                                        int p, int row0, int lane, int off, bool xin, uint32_t ymask,
                                        bool edge_halo, bool any_edge_halo, typename Pol::T* orow0,
                                        int64_t sy, int64_t sz, int nz, const Src& src, int64_t x,
                                        int64_t y0, typename Pol::Track& trk) {
  using T = typename Pol::T;
  using C = typename Pol::C;
  constexpr int TT = Cfg::T, S = Cfg::S;
  constexpr int OLD = (0 + ROT) % 3, MID = (1 + ROT) % 3, NEW = (2 + ROT) % 3;
  {
    const T* U = reinterpret_cast<const T*>(ring + slot * Cfg::STAGE);
    const bool zin_p = (p >= 1 && p <= nz);
#pragma unroll
    for (int q = 0; q < Cfg::NROW; ++q) {
      const T uv = U[(row0 + q) * Cfg::BOXW + off + Cfg::COL0 + lane];
      st.W[0][NEW][q] = Pol::in(uv, k);
      if constexpr (Pol::kResidual) trk.see_u(uv);
    }
    // Cells outside the interior (Dirichlet halo, or beyond the grid) may be
    // stored in a different form (PolResident keeps them binary64); only
    // warps that touch one take this branch.
    const uint32_t halo_rows = (xin && zin_p) ? ~ymask : 0xffffffffu;
    if (__any_sync(0xffffffffu, (halo_rows & ((1u << Cfg::NROW) - 1u)) != 0u)) {
#pragma unroll
      for (int q = 0; q < Cfg::NROW; ++q)
        if ((halo_rows >> q) & 1u)
          st.W[0][NEW][q] = Pol::in_halo(U[(row0 + q) * Cfg::BOXW + off + Cfg::COL0 + lane], k);
    }
  }
#pragma unroll
  for (int t = 1; t <= TT; ++t) {
    if (j < 2 * t) break;  // stage t has no complete input yet
    const int q = p - t;   // plane this stage updates
    const bool zin = (q >= 1 && q <= nz);
    const T* F = reinterpret_cast<const T*>(ring + ((seq - t) % S) * Cfg::STAGE + Cfg::UB);
    const int nr = Cfg::R + 2 * (TT - t);  // rows this stage updates
#pragma unroll
    for (int rr = 0; rr < Cfg::R + 2 * (TT - 1); ++rr) {
      if (rr >= nr) break;
      const C c = st.W[t - 1][MID][rr + 1];
      C xm, xp;
      if constexpr (Cfg::XSMEM) {
        // both x neighbours from the staged middle plane (held until this
        // step ends)
        const T* Um = reinterpret_cast<const T*>(ring + ((seq - 1) % S) * Cfg::STAGE);
        const int e0 = (row0 + rr + 1) * Cfg::BOXW + off + Cfg::COL0 + lane;
        xm = Pol::in(Um[e0 - 1], k);
        xp = Pol::in(Um[e0 + 1], k);
      } else {
      xm = __shfl_up_sync(0xffffffffu, c, 1);
      xp = __shfl_down_sync(0xffffffffu, c, 1);
      if (Cfg::EDGE && t == 1) {
        // Lane 0's left and lane 31's right neighbour, from the staged plane
        // of stage 0's middle plane (held until this step ends); the other
        // lanes read an in-range cell they do not use.  Its y and z are the
        // updated cell's, so it is a halo cell only at x = 0 or x = nx + 1.
        const T* Um = reinterpret_cast<const T*>(ring + ((seq - 1) % S) * Cfg::STAGE);
        const T e = Um[(row0 + rr + 1) * Cfg::BOXW + off + (lane == 0 ? 0 : 33)];
        C ec = Pol::in(e, k);
        if constexpr (Pol::kResidual) {
          if (lane == 0 || lane == 31) trk.see_u(e);
        }
        if (any_edge_halo && edge_halo) ec = Pol::in_halo(e, k);
        if (lane == 0) xm = ec;
        if (lane == 31) xp = ec;
      }
      }
      const int w = rr - (TT - t);  // warp row, -T..R+T-1
      const bool in = xin && zin && ((ymask >> (w + TT)) & 1u);
      C v = c;
      T fv{};
      if (in) {
        fv = F[(row0 + rr + t - 1) * Cfg::BOXW + off + Cfg::COL0 + lane];
        if constexpr (RS) {
          if (k.fpath) fv = Pol::source_at(fv, k);
        }
        if constexpr (Pol::kResidual) {
          v = Pol::residual(c, xm, xp, st.W[t - 1][MID][rr], st.W[t - 1][MID][rr + 2], st.W[t - 1][OLD][rr + 1],
                            st.W[t - 1][NEW][rr + 1], fv, k);
        } else {
          v = Pol::update(xm, xp, st.W[t - 1][MID][rr], st.W[t - 1][MID][rr + 2],
                          st.W[t - 1][OLD][rr + 1], st.W[t - 1][NEW][rr + 1], fv, k);
        }
      }
      if (t < TT) {
        st.W[t][NEW][rr] = v;
      } else if (in && lane >= Cfg::XL && lane < 32 - Cfg::XL) {
        if constexpr (Pol::kResidual) {
          trk.add(v, fv);
          if (k.write) orow0[static_cast<int64_t>(q) * sz + rr * sy] = Pol::out(v, k);
        } else {
          T o = Pol::out(v, k);
          if constexpr (RS) {
            if (k.dshift) o = Pol::rescale(o, k);
            if (k.fpath) src.store_source(x, y0 + rr, q, fv);
          }
          orow0[static_cast<int64_t>(q) * sz + rr * sy] = o;
          trk.add(o);
        }
      }
    }
  }
}

// The work items of one consumer warp; false if a bounded wait expired.
template <class Pol, class Cfg, class Src, bool RS>
__device__ __forceinline__ bool tb_consume(const Src& src, const unsigned char* ring, uint32_t bar_full,
                                           uint32_t bar_empty, volatile int* abort_flag, int warp, int lane,
                                           typename Pol::Track& trk) {
  constexpr int S = Cfg::S, TT = Cfg::T;
  uint32_t* status = src.status();
  const int row0 = warp * Cfg::R;
  LaneState<Pol, Cfg> st;
  uint32_t it = 0;
  for (int64_t item = blockIdx.x; item < src.items(); item += gridDim.x) {
    ItemView<Pol> v;
    if (!src.view(item, v)) continue;
    const Item& t = v.t;
    const int xa = align_down(t.xo - TT, Cfg::A);
    const int off = t.xo - TT - xa;
    const int64_t x = t.xo - Cfg::XL + lane;  // halo index of this lane's column
    const bool xin = (x >= 1 && x <= v.nx);
    // EDGE: is the neighbour this lane reads from the staged plane (lane 0:
    // x - 1, lane 31: x + 1) a Dirichlet halo cell?
    const bool edge_halo = lane == 0 ? (x - 1 < 1) : (x + 1 > v.nx);
    const bool any_edge_halo = __any_sync(0xffffffffu, (lane == 0 || lane == 31) && edge_halo);
    uint32_t ymask = 0;                  // bit w+T: warp row w is interior
#pragma unroll
    for (int w = -TT; w < Cfg::R + TT; ++w) {
      const int64_t y = t.yo + row0 + w;
      ymask |= (y >= 1 && y <= v.ny) ? (1u << (w + TT)) : 0u;
    }
    typename Pol::T* orow0 = v.out + x + (t.yo + row0) * v.osy;
    const int steps = (t.ze - t.zs + 1) + 2 * TT;
    const uint32_t seq0 = it;
    int j = 0;
    auto wait = [&](int jj) -> int {
      const uint32_t seq = seq0 + jj;
      const uint32_t s = seq % S;
      if (!mbar_wait_bounded(bar_full + 8 * s, (seq / S) & 1u, status)) {
        *abort_flag = 1;
        return -1;
      }
      return static_cast<int>(s);
    };
    auto release = [&](uint32_t seq) {
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_empty + 8 * (seq % S));
    };
    for (;;) {
#define STENCIL_TB_STEP(ROT)                                                                       \
  {                                                                                                \
    const int slot = wait(j);                                                                      \
    if (slot < 0) return false;                                                                    \
    tb_step<Pol, Cfg, Src, ROT, RS>(st, v.k, ring, slot, seq0 + j, j, t.zs - TT + j, row0, lane,   \
                                    off, xin, ymask, edge_halo, any_edge_halo, orow0, v.osy, v.osz,\
                                    static_cast<int>(v.nz), src, x, t.yo + row0, trk);             \
    if (j >= TT) release(seq0 + j - TT);                                                           \
    if (++j >= steps) break;                                                                       \
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
  return true;
}

template <class Pol, class Cfg, class Src>
__global__ void __launch_bounds__(Cfg::THREADS, Cfg::MINB)
    jacobi_tb(const __grid_constant__ typename Src::Params params) {
  constexpr int S = Cfg::S, WY = Cfg::WY;
  extern __shared__ unsigned char smem_raw[];
  __shared__ int abort_flag;
  if constexpr (Pol::kResidual) {  // a conditional pass (uniform: every thread reads the same word)
    if (params.a.run_flag && *params.a.run_flag == 0u) return;
  }
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
    if (lane == 0) {
      const Src src(&params, false);
      produce<Pol, Cfg, Src>(src, bar_full, bar_empty, smem_addr(ring), &abort_flag);
    }
    return;
  }
  const Src src(&params, true);
  src.fx_begin();
  typename Pol::Track trk;
  bool ok;
  if constexpr (Pol::kResident) {
    // the rare passes that change the scale, or that follow such a pass, run
    // their own instantiation, so the common one carries none of that code
    ok = Pol::needs_rescale(src.k)
             ? tb_consume<Pol, Cfg, Src, true>(src, ring, bar_full, bar_empty, &abort_flag, warp, lane, trk)
             : tb_consume<Pol, Cfg, Src, false>(src, ring, bar_full, bar_empty, &abort_flag, warp, lane, trk);
  } else {
    ok = tb_consume<Pol, Cfg, Src, false>(src, ring, bar_full, bar_empty, &abort_flag, warp, lane, trk);
  }
  if constexpr (Pol::kResidual) {
    src.resid_end(trk, warp, WY);  // every consumer warp takes part (a failed wait is in the status)
  } else {
    if (ok) src.fx_end(trk.key());
  }
}

}  // namespace stencil
