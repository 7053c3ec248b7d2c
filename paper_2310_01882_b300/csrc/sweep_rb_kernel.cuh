// sweep_rb_kernel.cuh -- red-black Gauss-Seidel sweeps with two x-columns
// per lane, so that each colour stage computes only the points of its
// colour.
//
// With jacobi_tb's one column per lane the colours alternate along x, so
// every warp instruction of a colour stage would cover both colours and
// throw half of the arithmetic away.  Here lane l of a consumer warp owns
// columns 2l and 2l+1 of a 64-column tile (a tile is (64 - 2T) x (R * WY)
// outputs).  Along any row exactly one of the two has a given colour, and
// which one is the same for every lane of the warp (the lanes' first
// columns share their parity).  The registers hold values by colour, not
// by column: stage t keeps, for three planes and its rows, the one value
// per row of the colour it computed (stage 0: the raw values of the colour
// stage 1 does not update).  Stage t (1..T) computes colour (t-1) mod 2 on
// plane p - t when raw plane p arrives:
//   * the updated cell's x neighbours are the lane's own value of the other
//     colour in that row (its other column) and the same register of lane
//     l-1 or l+1 (one shuffle, warp-uniform direction);
//   * y and z neighbours are the lane's stage t-1 registers of the adjacent
//     rows and planes, as in jacobi_tb;
//   * a cell that is not interior keeps its staged value (the Dirichlet
//     halo; still staged, since a warp holds T+1 planes).
// The last stage writes both colours of its plane.  T stages make T/2
// red-black sweeps per pass.  The producer, the stage ring, the bounded
// waits and the work sources are those of jacobi_tb (sweep_kernel.cuh).
#pragma once

#include "sweep_kernel.cuh"

namespace stencil {

template <class Pol, int T_, int R_, int WY_, int S_, int MINB_>
struct RbCfg {
  static constexpr int T = T_, R = R_, WY = WY_, S = S_, MINB = MINB_;
  static constexpr bool RB = true;
  static constexpr bool WIDE = true;
  static constexpr int A = 16 / Pol::kElem;      // TMA x granule in elements
  static constexpr int BOXW = 64 + A;            // staged columns (any 0 <= off < A)
  static constexpr int BXO = 64 - 2 * T;         // output columns per tile
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
  static_assert(T % 2 == 0, "a red-black pass holds whole sweeps");
};

template <class Pol, class Cfg>
struct RbLaneState {
  using C = typename Pol::C;
  C W[Cfg::T][3][Cfg::NROW];  // stage t's values of its colour: three planes, its rows
};

// RS: the pass writes the resident fixed point at a new scale (see tb_step).
template <class Pol, class Cfg, class Src, int ROT, bool RS>
__device__ __forceinline__ void rb_step(RbLaneState<Pol, Cfg>& st, const typename Pol::K& k,
                                        const unsigned char* ring, int slot, uint32_t seq, int j, int p, int row0,
                                        int lane, int off, bool xin0, bool xin1, uint32_t ymask, int pb,
                                        typename Pol::T* orow0, int64_t sy, int64_t sz, int nz,
                                        const Src& src, int64_t x, int64_t y0, typename Pol::Track& trk) {
  using T = typename Pol::T;
  using C = typename Pol::C;
  constexpr int TT = Cfg::T, S = Cfg::S;
  constexpr int OLD = (0 + ROT) % 3, MID = (1 + ROT) % 3, NEW = (2 + ROT) % 3;
  // Cell (column i of the lane, warp row w, plane q) is red iff
  // pb + i + w + q is even; colour c (0 red, 1 black) of row w of plane q
  // sits in column (pb + w + q + c) & 1.
  {
    // stage 0: plane p's cells of colour 1 (black), rows -T .. R+T-1
    const T* U = reinterpret_cast<const T*>(ring + slot * Cfg::STAGE);
    const bool zin_p = (p >= 1 && p <= nz);
    bool halo = false;
#pragma unroll
    for (int q = 0; q < Cfg::NROW; ++q) {
      const int ic = (pb + q - TT + p + 1) & 1;
      st.W[0][NEW][q] = Pol::in(U[(row0 + q) * Cfg::BOXW + off + 2 * lane + ic], k);
      halo |= !((ic ? xin1 : xin0) && zin_p && ((ymask >> q) & 1u));
    }
    if (__any_sync(0xffffffffu, halo)) {
#pragma unroll
      for (int q = 0; q < Cfg::NROW; ++q) {
        const int ic = (pb + q - TT + p + 1) & 1;
        if (!((ic ? xin1 : xin0) && zin_p && ((ymask >> q) & 1u)))
          st.W[0][NEW][q] = Pol::in_halo(U[(row0 + q) * Cfg::BOXW + off + 2 * lane + ic], k);
      }
    }
  }
#pragma unroll
  for (int t = 1; t <= TT; ++t) {
    if (j < 2 * t) break;  // stage t has no complete input yet
    const int q = p - t;   // plane this stage updates
    const bool zin = (q >= 1 && q <= nz);
    const T* F = reinterpret_cast<const T*>(ring + ((seq - t) % S) * Cfg::STAGE + Cfg::UB);
    const T* Uq = reinterpret_cast<const T*>(ring + ((seq - t) % S) * Cfg::STAGE);
    const int nr = Cfg::R + 2 * (TT - t);
#pragma unroll
    for (int rr = 0; rr < Cfg::R + 2 * (TT - 1); ++rr) {
      if (rr >= nr) break;
      const int w = rr - (TT - t);  // warp row, -T..R+T-1
      const int ic = (pb + w + q + ((t - 1) & 1)) & 1;  // column of this stage's colour
      const bool yzin = zin && ((ymask >> (w + TT)) & 1u);
      const bool in = yzin && (ic ? xin1 : xin0);
      // the other colour in this row: own column 1 - ic, and the facing
      // column of lane l-1 (ic = 0) or lane l+1 (ic = 1)
      const C own = st.W[t - 1][MID][rr + 1];
      const C other = __shfl_sync(0xffffffffu, own, (lane + (ic ? 1 : 31)) & 31);
      C v;
      if (in) {
        // Every policy's update starts with xm + xp, and addition is
        // commutative, so the two x neighbours go in without a select.
        T fv = F[(row0 + rr + t - 1) * Cfg::BOXW + off + 2 * lane + ic];
        if constexpr (RS) {
          // fpath: the source converted here; stored once, by the tile that
          // owns the cell, at the stage that updates it
          if (k.fpath) {
            fv = Pol::source_at(fv, k);
            if (w >= 0 && w < Cfg::R && 2 * lane >= TT && 2 * lane + 1 < 64 - TT)
              src.store_source(x + ic, y0 + w, q, fv);
          }
        }
        v = Pol::update(other, own, st.W[t - 1][MID][rr], st.W[t - 1][MID][rr + 2], st.W[t - 1][OLD][rr + 1],
                        st.W[t - 1][NEW][rr + 1], fv, k);
      } else {
        v = Pol::in_halo(Uq[(row0 + w + TT) * Cfg::BOXW + off + 2 * lane + ic], k);
      }
      if (t < TT) {
        st.W[t][NEW][rr] = v;
      } else if (yzin && 2 * lane >= TT && 2 * lane + 1 < 64 - TT) {
        // both colours of plane q are final: this stage's and stage T-1's
        typename Pol::T* o = orow0 + static_cast<int64_t>(q) * sz + rr * sy;
        // both outputs' magnitudes in one step; a cell that is not interior
        // keeps its staged value, which the other output's stands in for
        T ov = Pol::out(v, k);
        T oo = Pol::out(own, k);
        if constexpr (RS) {
          if (k.dshift) {
            ov = Pol::rescale(ov, k);
            oo = Pol::rescale(oo, k);
          }
        }
        const bool wo = ic ? xin0 : xin1;
        if (in) o[ic] = ov;
        if (wo) o[ic ^ 1] = oo;
        if (in || wo) trk.add2(in ? ov : oo, wo ? oo : ov);

      }
    }
  }
}

// The work items of one consumer warp; false if a bounded wait expired.
template <class Pol, class Cfg, class Src, bool RS>
__device__ __forceinline__ bool rb_consume(const Src& src, const unsigned char* ring, uint32_t bar_full,
                                           uint32_t bar_empty, volatile int* abort_flag, int warp, int lane,
                                           typename Pol::Track& trk) {
  constexpr int S = Cfg::S, TT = Cfg::T;
  uint32_t* status = src.status();
  const int row0 = warp * Cfg::R;
  RbLaneState<Pol, Cfg> st;
  uint32_t it = 0;
  for (int64_t item = blockIdx.x; item < src.items(); item += gridDim.x) {
    ItemView<Pol> v;
    if (!src.view(item, v)) continue;
    const Item& t = v.t;
    const int xa = align_down(t.xo - TT, Cfg::A);
    const int off = t.xo - TT - xa;
    const int64_t x = t.xo - TT + 2 * lane;  // halo index of this lane's first column
    const bool xin0 = x >= 1 && x <= v.nx, xin1 = x + 1 >= 1 && x + 1 <= v.nx;
    uint32_t ymask = 0;                      // bit w+T: warp row w is interior
#pragma unroll
    for (int w = -TT; w < Cfg::R + TT; ++w) {
      const int64_t y = t.yo + row0 + w;
      ymask |= (y >= 1 && y <= v.ny) ? (1u << (w + TT)) : 0u;
    }
    typename Pol::T* orow0 = v.out + x + (t.yo + row0) * v.osy;
    const int pb = static_cast<int>((t.xo - TT + t.yo + row0) & 1);
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
#define STENCIL_RB_STEP(ROT)                                                                         \
  {                                                                                                  \
    const int slot = wait(j);                                                                        \
    if (slot < 0) return false;                                                                      \
    rb_step<Pol, Cfg, Src, ROT, RS>(st, v.k, ring, slot, seq0 + j, j, t.zs - TT + j, row0, lane, off,  \
                                    xin0, xin1, ymask, pb, orow0, v.osy, v.osz, static_cast<int>(v.nz),\
                                    src, x, t.yo + row0, trk);                                         \
    if (j >= TT) release(seq0 + j - TT);                                                             \
    if (++j >= steps) break;                                                                         \
  }
      STENCIL_RB_STEP(0)
      STENCIL_RB_STEP(1)
      STENCIL_RB_STEP(2)
#undef STENCIL_RB_STEP
    }
    for (int q = steps - TT; q < steps; ++q)
      if (q >= 0) release(seq0 + q);
    it = seq0 + steps;
  }
  return true;
}

template <class Pol, class Cfg, class Src>
__global__ void __launch_bounds__(Cfg::THREADS, Cfg::MINB)
    redblack_tb(const __grid_constant__ typename Src::Params params) {
  constexpr int S = Cfg::S, WY = Cfg::WY;
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
    ok = Pol::needs_rescale(src.k)
             ? rb_consume<Pol, Cfg, Src, true>(src, ring, bar_full, bar_empty, &abort_flag, warp, lane, trk)
             : rb_consume<Pol, Cfg, Src, false>(src, ring, bar_full, bar_empty, &abort_flag, warp, lane, trk);
  } else {
    ok = rb_consume<Pol, Cfg, Src, false>(src, ring, bar_full, bar_empty, &abort_flag, warp, lane, trk);
  }
  if (ok) src.fx_end(trk.key());
}

// The kernel a configuration runs: redblack_tb for RbCfg, jacobi_tb for
// TbCfg.
template <class Cfg, class = void>
struct IsWide {
  static constexpr bool value = false;
};
template <class Cfg>
struct IsWide<Cfg, decltype(void(Cfg::WIDE))> {
  static constexpr bool value = Cfg::WIDE;
};

template <class Pol, class Cfg, class Src>
constexpr auto sweep_kernel_for() {
  if constexpr (IsWide<Cfg>::value) return &redblack_tb<Pol, Cfg, Src>;
  else return &jacobi_tb<Pol, Cfg, Src>;
}

}  // namespace stencil
