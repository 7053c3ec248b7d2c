// sweep_rb_kernel.cuh -- red-black Gauss-Seidel sweeps with two x-columns
// per lane, so that each colour stage computes only the points of its
// colour.
//
// With jacobi_tb's one column per lane the colours alternate along x, so
// every warp instruction of a colour stage would cover both colours and
// throw half of the arithmetic away.  Here lane l of a consumer warp owns
// columns 2l and 2l+1 of a 64-column
// tile (a tile is (64 - 2T) x (R * WY) outputs).  Along any row exactly one
// of the two has the stage's colour, so each lane updates one point per row
// and carries the other over:
//   * the updated column phi = (colour + x0 + y + z) mod 2, x0 the parity of
//     the lane's first column (the same for every lane);
//   * its x neighbours are the lane's other column and the facing column of
//     lane l-1 (phi = 0) or lane l+1 (phi = 1): one shuffle up of column 1
//     and one shuffle down of column 0 per row serve both cases;
//   * y and z neighbours are the lane's own registers (rows, rotating
//     planes), as in jacobi_tb.
// Stage t (1..T) handles colour (t-1) mod 2 on plane p - t when raw plane p
// arrives; T stages make T/2 red-black sweeps per pass.  The producer, the
// stage ring, the bounded waits and the work sources are those of
// jacobi_tb (sweep_kernel.cuh).
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
  C W[Cfg::T][3][Cfg::NROW][2];  // stage t's three planes, two columns
};

template <class Pol, class Cfg, int ROT>
__device__ __forceinline__ void rb_step(RbLaneState<Pol, Cfg>& st, const typename Pol::K& k,
                                        const unsigned char* ring, int slot, uint32_t seq, int j, int p, int row0,
                                        int lane, int off, bool xin0, bool xin1, uint32_t ymask, int pb,
                                        typename Pol::T* orow0, int64_t sy, int64_t sz, int nz) {
  using T = typename Pol::T;
  using C = typename Pol::C;
  constexpr int TT = Cfg::T, S = Cfg::S;
  constexpr int OLD = (0 + ROT) % 3, MID = (1 + ROT) % 3, NEW = (2 + ROT) % 3;
  {
    const T* U = reinterpret_cast<const T*>(ring + slot * Cfg::STAGE);
    const bool zin_p = (p >= 1 && p <= nz);
#pragma unroll
    for (int q = 0; q < Cfg::NROW; ++q) {
      const T* row = U + (row0 + q) * Cfg::BOXW + off + 2 * lane;
      st.W[0][NEW][q][0] = Pol::in(row[0], k);
      st.W[0][NEW][q][1] = Pol::in(row[1], k);
    }
    const uint32_t rows_mask = (1u << Cfg::NROW) - 1u;
    const uint32_t halo0 = (xin0 && zin_p) ? ~ymask : 0xffffffffu;
    const uint32_t halo1 = (xin1 && zin_p) ? ~ymask : 0xffffffffu;
    if (__any_sync(0xffffffffu, ((halo0 | halo1) & rows_mask) != 0u)) {
#pragma unroll
      for (int q = 0; q < Cfg::NROW; ++q) {
        const T* row = U + (row0 + q) * Cfg::BOXW + off + 2 * lane;
        if ((halo0 >> q) & 1u) st.W[0][NEW][q][0] = Pol::in_halo(row[0], k);
        if ((halo1 >> q) & 1u) st.W[0][NEW][q][1] = Pol::in_halo(row[1], k);
      }
    }
  }
#pragma unroll
  for (int t = 1; t <= TT; ++t) {
    if (j < 2 * t) break;  // stage t has no complete input yet
    const int q = p - t;   // plane this stage updates
    const bool zin = (q >= 1 && q <= nz);
    const T* F = reinterpret_cast<const T*>(ring + ((seq - t) % S) * Cfg::STAGE + Cfg::UB);
    const int nr = Cfg::R + 2 * (TT - t);
#pragma unroll
    for (int rr = 0; rr < Cfg::R + 2 * (TT - 1); ++rr) {
      if (rr >= nr) break;
      const C c0 = st.W[t - 1][MID][rr + 1][0];
      const C c1 = st.W[t - 1][MID][rr + 1][1];
      const C left = __shfl_up_sync(0xffffffffu, c1, 1);    // lane l-1, column 1
      const C right = __shfl_down_sync(0xffffffffu, c0, 1); // lane l+1, column 0
      const int w = rr - (TT - t);                           // warp row, -T..R+T-1
      const bool yzin = zin && ((ymask >> (w + TT)) & 1u);
      const int phi = ((t - 1) + pb + w + q) & 1;            // the column of this stage's colour
      const bool in = yzin && (phi ? xin1 : xin0);
      C v = phi ? c1 : c0;
      if (in) {
        const C xm = phi ? c0 : left;
        const C xp = phi ? right : c1;
        const C ym = phi ? st.W[t - 1][MID][rr][1] : st.W[t - 1][MID][rr][0];
        const C yp = phi ? st.W[t - 1][MID][rr + 2][1] : st.W[t - 1][MID][rr + 2][0];
        const C zm = phi ? st.W[t - 1][OLD][rr + 1][1] : st.W[t - 1][OLD][rr + 1][0];
        const C zp = phi ? st.W[t - 1][NEW][rr + 1][1] : st.W[t - 1][NEW][rr + 1][0];
        const T fv = F[(row0 + rr + t - 1) * Cfg::BOXW + off + 2 * lane + phi];
        v = Pol::update(xm, xp, ym, yp, zm, zp, fv, k);
      }
      const C n0 = phi ? c0 : v;
      const C n1 = phi ? v : c1;
      if (t < TT) {
        st.W[t][NEW][rr][0] = n0;
        st.W[t][NEW][rr][1] = n1;
      } else if (yzin) {
        typename Pol::T* o = orow0 + static_cast<int64_t>(q) * sz + rr * sy;
        // columns TT .. 63-TT of the lane pair space hold final values
        if (xin0 && 2 * lane >= TT && 2 * lane < 64 - TT) o[0] = Pol::out(n0, k);
        if (xin1 && 2 * lane + 1 >= TT && 2 * lane + 1 < 64 - TT) o[1] = Pol::out(n1, k);
      }
    }
  }
}

template <class Pol, class Cfg, class Src>
__global__ void __launch_bounds__(Cfg::THREADS, Cfg::MINB)
    redblack_tb(const __grid_constant__ typename Src::Params params) {
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
    if (lane == 0) {
      const Src src(&params, false);
      produce<Pol, Cfg, Src>(src, bar_full, bar_empty, smem_addr(ring), &abort_flag);
    }
    return;
  }
  const Src src(&params, true);
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
    typename Pol::T* orow0 = v.out + x + (t.yo + row0) * v.sy;
    const int pb = static_cast<int>((t.xo - TT + t.yo + row0) & 1);
    const int steps = (t.ze - t.zs + 1) + 2 * TT;
    const uint32_t seq0 = it;
    int j = 0;
    auto wait = [&](int jj) -> int {
      const uint32_t seq = seq0 + jj;
      const uint32_t s = seq % S;
      if (!mbar_wait_bounded(bar_full + 8 * s, (seq / S) & 1u, status)) {
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
#define STENCIL_RB_STEP(ROT)                                                                       \
  {                                                                                                \
    const int slot = wait(j);                                                                      \
    if (slot < 0) return;                                                                          \
    rb_step<Pol, Cfg, ROT>(st, v.k, ring, slot, seq0 + j, j, t.zs - TT + j, row0, lane, off, xin0, \
                           xin1, ymask, pb, orow0, v.sy, v.sz, static_cast<int>(v.nz));            \
    if (j >= TT) release(seq0 + j - TT);                                                           \
    if (++j >= steps) break;                                                                       \
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
