// batch.cu -- stencil_batch_solve: many independent Poisson instances solved
// in lockstep by mixed-precision iterative refinement.
//
// One refinement cycle for every active instance:
//   1. batch_resid_kernel<0>: r = f - A u in binary64 (the operations of
//      stencil_residual, bitwise), per-item partial sums of r^2 and f^2;
//      for binary32 inner storage also r rounded into the source buffer and
//      the correction e zeroed;
//   2. batch_check_kernel: per instance, the norms in item order, the
//      convergence / budget / stall decisions, BF16 -> F32 escalation;
//   3. (bfloat16 runs) batch_resid_kernel<1>: r again, rounded, e zeroed,
//      for the bfloat16 instances and those that escalated this cycle;
//   4. sweeps_per_cycle Jacobi (or red-black Gauss-Seidel) sweeps of
//      A e = r_lo: each pass is one persistent launch of jacobi_tb over the
//      tiles of all active instances (a device table of per-instance TMA
//      descriptors, SrcBatch);
//   5. batch_update_kernel: u += e in binary64.
// The cycle is captured once as a CUDA graph and replayed; after each replay
// the host reads the number of instances still active.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "sweep_rb_kernel.cuh"

namespace stencil {

namespace {

constexpr int kRowsPerItem = 32;  // interior (y, z) rows per residual item

struct InstState {
  int32_t active;  // 1 while the instance iterates
  int32_t dtype;   // inner storage: STENCIL_F32 or STENCIL_BF16
  int32_t cycles;  // corrections applied
  int32_t code;    // outcome (STENCIL_OK / _NOT_CONVERGED / _NONFINITE)
  int64_t sweeps;
  double rel;      // last relative residual
  double prev;     // relative residual of the previous cycle
  int32_t escalated;  // set when this cycle switched BF16 -> F32 storage
  int32_t pad;
};

// Inner-storage index: 0 = F32, 1 = BF16.
__host__ __device__ __forceinline__ int dix(int dtype) { return dtype == STENCIL_BF16 ? 1 : 0; }

struct alignas(64) InstDesc {
  CUtensorMap tm_e[2][2];  // [storage][ping, pong]: the correction as sweep input
  CUtensorMap tm_r[2];     // [storage]: the rounded residual, the sweep source
  SweepGeom g[2];          // [storage]: tile geometry of the chosen configuration
  double* u;
  const double* f;
  void* e[2];              // ping, pong buffers (shared by both storage layouts)
  void* r;
  int64_t nx, ny, nz, usy, usz, fsy, fsz;
  int64_t esy[2], esz[2];  // [storage] element strides of e and r
  int64_t ebytes;          // bytes of each of e[0], e[1], r
  double h, hh;
};

struct BatchTables {
  const InstDesc* desc;
  InstState* state;
  const int64_t* rbase;    // n+1 prefix sums of residual items
  double* partials;        // 2 per residual item
  unsigned long long* n_active;
  int n;
};

__device__ __forceinline__ int find_instance(const int64_t* base, int n, int64_t item) {
  int lo = 0, hi = n;  // base[lo] <= item < base[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (base[mid] <= item) lo = mid; else hi = mid;
  }
  return lo;
}

// Work source of the inner sweeps: the tiles of every active instance whose
// inner storage is DT.
template <class Pol, int DT>
struct SrcBatch {
  struct Params {
    const InstDesc* desc;
    const InstState* state;
    const int64_t* base;  // n+1 prefix sums of sweep items (storage DT)
    int n;
    int parity;           // 0: e ping -> pong, 1: pong -> ping
    uint32_t* status;
  };
  const Params* p;
  __device__ __forceinline__ SrcBatch(const Params* pp, bool) : p(pp) {}
  __device__ __forceinline__ int64_t items() const { return p->base[p->n]; }
  __device__ __forceinline__ uint32_t* status() const { return p->status; }
  __device__ __forceinline__ void fx_begin() const {}
  __device__ __forceinline__ void fx_end(uint32_t) const {}
  __device__ __forceinline__ bool view(int64_t item, ItemView<Pol>& v) const {
    const int i = find_instance(p->base, p->n, item);
    const InstState& s = p->state[i];
    if (!s.active || dix(s.dtype) != DT) return false;
    const InstDesc& d = p->desc[i];
    const SweepGeom& g = d.g[DT];
    v.t = decode_item(g, item - p->base[i]);
    v.nx = g.nx; v.ny = g.ny; v.nz = g.nz; v.sy = g.sy; v.sz = g.sz;
    v.osy = g.sy; v.osz = g.sz;
    v.tm_u = &d.tm_e[DT][p->parity];
    v.tm_f = &d.tm_r[DT];
    v.out = static_cast<typename Pol::T*>(d.e[p->parity ^ 1]);
    v.k.hh = static_cast<float>(d.hh);
    return true;
  }
};

// MODE 0: per-item partial sums of r^2 and f^2; for the instances whose inner
// storage is already binary32 (it can only change from bfloat16), also r
// rounded to binary32 into the source buffer and the interior of e (ping)
// zeroed, so r is computed once per cycle for them.  MODE 1 (after the
// check): the same rounding and zeroing for the bfloat16 instances and for
// those that switched to binary32 this cycle.  r is rounded binary64 ->
// binary32 -> bfloat16, each to nearest even.
template <int MODE>
__global__ void __launch_bounds__(256) batch_resid_kernel(BatchTables tb) {
  const int64_t total = tb.rbase[tb.n];
  __shared__ double wr[8], wf[8];
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
    const int i = find_instance(tb.rbase, tb.n, item);
    const InstState& s = tb.state[i];
    if (!s.active) continue;
    const bool write = MODE == 0 ? (s.dtype == STENCIL_F32) : (s.dtype == STENCIL_BF16 || s.escalated != 0);
    if (MODE == 1 && !write) continue;
    const InstDesc& d = tb.desc[i];
    const int64_t rows = d.ny * d.nz;
    const int64_t r0 = (item - tb.rbase[i]) * kRowsPerItem;
    const int64_t r1 = min(r0 + kRowsPerItem, rows);
    const double hh = d.hh;
    const int di = dix(s.dtype);
    double rr = 0.0, ff = 0.0;
    for (int64_t row = r0 + threadIdx.y; row < r1; row += 8) {
      const int64_t k = 1 + row / d.ny;
      const int64_t j = 1 + row - (k - 1) * d.ny;
      const double* uc = d.u + j * d.usy + k * d.usz;
      const double* fc = d.f + j * d.fsy + k * d.fsz;
      for (int64_t x = 1 + threadIdx.x; x <= d.nx; x += 32) {
        double sm = __dadd_rn(uc[x - 1], uc[x + 1]);
        sm = __dadd_rn(sm, uc[x - d.usy]);
        sm = __dadd_rn(sm, uc[x + d.usy]);
        sm = __dadd_rn(sm, uc[x - d.usz]);
        sm = __dadd_rn(sm, uc[x + d.usz]);
        const double au = __ddiv_rn(__dsub_rn(__dmul_rn(6.0, uc[x]), sm), hh);
        const double fv = fc[x];
        const double res = __dsub_rn(fv, au);
        if (MODE == 0) {
          rr = fma(res, res, rr);
          ff = fma(fv, fv, ff);
        }
        if (write) {
          const int64_t o = x + j * d.esy[di] + k * d.esz[di];
          const float r32 = __double2float_rn(res);
          if (di == 0) {
            static_cast<float*>(d.r)[o] = r32;
            static_cast<float*>(d.e[0])[o] = 0.0f;
          } else {
            static_cast<__nv_bfloat16*>(d.r)[o] = __float2bfloat16_rn(r32);
            static_cast<__nv_bfloat16*>(d.e[0])[o] = __float2bfloat16_rn(0.0f);
          }
        }
      }
    }
    if (MODE == 0) {
      for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_xor_sync(0xffffffffu, rr, o);
        ff += __shfl_xor_sync(0xffffffffu, ff, o);
      }
      if (threadIdx.x == 0) {
        wr[threadIdx.y] = rr;
        wf[threadIdx.y] = ff;
      }
      __syncthreads();
      if (threadIdx.x == 0 && threadIdx.y == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < 8; ++w) {
          a += wr[w];
          b += wf[w];
        }
        tb.partials[2 * item] = a;
        tb.partials[2 * item + 1] = b;
      }
      __syncthreads();
    }
  }
}

struct CheckArgs {
  double rtol, stall_ratio;
  int64_t max_sweeps;
  int sweeps_per_cycle;
};

__global__ void batch_check_kernel(BatchTables tb, CheckArgs ca) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= tb.n) return;
  InstState& s = tb.state[i];
  if (!s.active) return;
  double rr = 0.0, ff = 0.0;
  for (int64_t q = tb.rbase[i]; q < tb.rbase[i + 1]; ++q) {
    rr += tb.partials[2 * q];
    ff += tb.partials[2 * q + 1];
  }
  const double nr = sqrt(rr), nf = sqrt(ff);
  const double rel = nf > 0.0 ? nr / nf : nr;
  s.rel = rel;
  int go = 1;
  if (!isfinite(rel)) {
    s.code = STENCIL_ERR_NONFINITE;
    go = 0;
  } else if (rel <= ca.rtol) {
    s.code = STENCIL_OK;
    go = 0;
  } else if (s.sweeps >= ca.max_sweeps) {
    s.code = STENCIL_ERR_NOT_CONVERGED;
    go = 0;
  } else if (s.cycles > 0 && rel > ca.stall_ratio * s.prev) {
    if (s.dtype == STENCIL_BF16) {
      s.dtype = STENCIL_F32;
      s.escalated = 1;
    } else {
      s.code = STENCIL_ERR_NOT_CONVERGED;
      go = 0;
    }
  }
  if (go) {
    s.prev = rel;
    s.cycles += 1;
    s.sweeps += ca.sweeps_per_cycle;
    atomicAdd(tb.n_active, 1ull);
  } else {
    s.active = 0;
  }
}

// After a BF16 -> F32 escalation the inner buffers are read in the F32
// layout, whose halo cells held BF16 interior values: zero the three buffers
// of every instance that escalated this cycle.
__global__ void __launch_bounds__(256) batch_rezero_kernel(BatchTables tb) {
  for (int i = 0; i < tb.n; ++i) {
    InstState& s = tb.state[i];
    if (!s.escalated) continue;
    const InstDesc& d = tb.desc[i];
    const int64_t words = d.ebytes / 16;
    for (int b = 0; b < 3; ++b) {
      uint4* p = static_cast<uint4*>(b == 0 ? d.e[0] : (b == 1 ? d.e[1] : d.r));
      for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < words;
           q += int64_t(gridDim.x) * blockDim.x)
        p[q] = make_uint4(0u, 0u, 0u, 0u);
    }
  }
}

// Clears the escalation flags once the buffers are zeroed (single thread).
__global__ void batch_clear_flags_kernel(BatchTables tb) {
  for (int i = threadIdx.x; i < tb.n; i += blockDim.x) tb.state[i].escalated = 0;
}

// u += e (the correction in buffer `which`) on the interior, binary64.
__global__ void __launch_bounds__(256) batch_update_kernel(BatchTables tb, int which) {
  const int64_t total = tb.rbase[tb.n];
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
    const int i = find_instance(tb.rbase, tb.n, item);
    const InstState& s = tb.state[i];
    if (!s.active) continue;
    const InstDesc& d = tb.desc[i];
    const int di = dix(s.dtype);
    const int64_t rows = d.ny * d.nz;
    const int64_t r0 = (item - tb.rbase[i]) * kRowsPerItem;
    const int64_t r1 = min(r0 + kRowsPerItem, rows);
    for (int64_t row = r0 + threadIdx.y; row < r1; row += 8) {
      const int64_t k = 1 + row / d.ny;
      const int64_t j = 1 + row - (k - 1) * d.ny;
      double* uc = d.u + j * d.usy + k * d.usz;
      const int64_t eo = j * d.esy[di] + k * d.esz[di];
      for (int64_t x = 1 + threadIdx.x; x <= d.nx; x += 32) {
        const double e = di == 0 ? static_cast<double>(static_cast<const float*>(d.e[which])[eo + x])
                                 : static_cast<double>(__bfloat162float(
                                       static_cast<const __nv_bfloat16*>(d.e[which])[eo + x]));
        uc[x] = uc[x] + e;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int64_t sy_for(int64_t nx, int elem) {
  const int64_t g = 16 / elem;
  return (nx + 2 + g - 1) / g * g;
}

// Bytes of one inner buffer (e ping, e pong or r): room for the F32 layout
// and the BF16 layout of the same grid.
size_t inner_buffer_bytes(int64_t nx, int64_t ny, int64_t nz) {
  const size_t f32 = static_cast<size_t>(sy_for(nx, 4)) * (ny + 2) * (nz + 2) * 4;
  const size_t b16 = static_cast<size_t>(sy_for(nx, 2)) * (ny + 2) * (nz + 2) * 2;
  return align_up(std::max(f32, b16), 256);
}

struct Layout {
  size_t desc, state, rbase, sbase, partials, nactive, buffers, total;
  int64_t ritems;
  std::vector<size_t> inst_off;  // offset of instance i's three inner buffers
};

Layout plan(const stencil_problem* probs, int n) {
  Layout L;
  size_t off = 0;
  L.desc = off; off = align_up(off + sizeof(InstDesc) * n, 256);
  L.state = off; off = align_up(off + sizeof(InstState) * n, 256);
  L.rbase = off; off = align_up(off + sizeof(int64_t) * (n + 1), 256);
  L.sbase = off; off = align_up(off + sizeof(int64_t) * 2 * (n + 1), 256);
  L.ritems = 0;
  for (int i = 0; i < n; ++i)
    L.ritems += (probs[i].u.ny * probs[i].u.nz + kRowsPerItem - 1) / kRowsPerItem;
  L.partials = off; off = align_up(off + sizeof(double) * 2 * L.ritems, 256);
  L.nactive = off; off = align_up(off + 256, 256);
  L.buffers = off;
  L.inst_off.resize(n);
  for (int i = 0; i < n; ++i) {
    L.inst_off[i] = off;
    off += 3 * inner_buffer_bytes(probs[i].u.nx, probs[i].u.ny, probs[i].u.nz);
  }
  L.total = off;
  return L;
}

// Compiled configurations of the inner sweep per storage type: (T, R, WY,
// S, CTAs per SM).  The autotuner times each and keeps the fastest per
// sweep.  Red-black passes (RbCfg) hold one sweep per two colour stages.
template <class... Cs>
struct CfgList {};
template <class P>
using BatchCfgs = CfgList<TbCfg<P, 1, 8, 4, 4, 3>, TbCfg<P, 1, 8, 8, 4, 2>, TbCfg<P, 1, 4, 8, 6, 3>,
                          TbCfg<P, 1, 4, 4, 5, 6>, TbCfg<P, 1, 4, 16, 5, 1>, TbCfg<P, 1, 2, 16, 5, 2>,
                          TbCfg<P, 2, 4, 4, 5, 2>, TbCfg<P, 2, 8, 4, 5, 1>, TbCfg<P, 2, 4, 8, 6, 2>,
                          TbCfg<P, 2, 8, 4, 5, 3>, TbCfg<P, 2, 4, 4, 5, 4>>;
template <class P>
using BatchCfgsRB = CfgList<RbCfg<P, 2, 4, 4, 5, 4>, RbCfg<P, 2, 4, 4, 4, 4>, RbCfg<P, 2, 8, 4, 4, 2>,
                            RbCfg<P, 2, 4, 8, 6, 1>, RbCfg<P, 4, 4, 4, 6, 2>>;
template <class... Cs>
constexpr int list_size(CfgList<Cs...>) {
  return static_cast<int>(sizeof...(Cs));
}
static_assert(list_size(BatchCfgs<PolF32>{}) == list_size(BatchCfgs<PolBF16>{}), "same shapes per storage");
int num_cfg(bool rb) { return rb ? list_size(BatchCfgsRB<PolF32>{}) : list_size(BatchCfgs<PolF32>{}); }

// Calls f(Cfg{}) for the c-th configuration of the list.
template <class F, class... Cs>
void with_cfg(int c, CfgList<Cs...>, F&& f) {
  int i = 0;
  ((i++ == c ? (f(Cs{}), 0) : 0), ...);
}

// Calls f(Cfg{}) for configuration c of storage di (0 = F32, 1 = BF16).
template <class F>
void with_batch_cfg(int di, bool rb, int c, F&& f) {
  if (di == 0) {
    if (rb) with_cfg(c, BatchCfgsRB<PolF32>{}, f);
    else with_cfg(c, BatchCfgs<PolF32>{}, f);
  } else {
    if (rb) with_cfg(c, BatchCfgsRB<PolBF16>{}, f);
    else with_cfg(c, BatchCfgs<PolBF16>{}, f);
  }
}

struct CfgInfo {
  int T;  // sweeps per pass
  int BXO, BYO, BOXW, UROWS, FROWS, THREADS, SMEM;
};

CfgInfo cfg_info(int di, bool rb, int c) {
  CfgInfo out{};
  with_batch_cfg(di, rb, c, [&](auto cfg) {
    using C = decltype(cfg);
    out = CfgInfo{C::RB ? C::T / 2 : C::T, C::BXO, C::BYO, C::BOXW, C::UROWS, C::FROWS, C::THREADS, C::SMEM};
  });
  return out;
}

template <class Pol, class Cfg, int DT>
int launch_pass_cfg(const typename SrcBatch<Pol, DT>::Params& prm, int num_sms, cudaStream_t st) {
  auto kern = sweep_kernel_for<Pol, Cfg, SrcBatch<Pol, DT>>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
  if (e != cudaSuccess) return check_cuda(e, "cudaFuncSetAttribute");
  e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return check_cuda(e, "cudaFuncSetAttribute(carveout)");
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Cfg::THREADS, Cfg::SMEM);
  if (e != cudaSuccess) return check_cuda(e, "occupancy");
  if (per_sm < 1) return set_error(STENCIL_ERR_CUDA, "batch sweep kernel cannot be resident");
  kern<<<per_sm * num_sms, Cfg::THREADS, Cfg::SMEM, st>>>(prm);
  return check_cuda(cudaGetLastError(), "batch sweep launch");
}

int launch_pass(int di, bool rb, int c, const InstDesc* desc, const InstState* state, const int64_t* base, int n,
                int parity, uint32_t* status, int num_sms, cudaStream_t st) {
  int rc = 1;  // not a status: set when the configuration index matches
  if (di == 0) {
    typename SrcBatch<PolF32, 0>::Params p{desc, state, base, n, parity, status};
    auto go = [&](auto cfg) { rc = launch_pass_cfg<PolF32, decltype(cfg), 0>(p, num_sms, st); };
    if (rb) with_cfg(c, BatchCfgsRB<PolF32>{}, go);
    else with_cfg(c, BatchCfgs<PolF32>{}, go);
  } else {
    typename SrcBatch<PolBF16, 1>::Params p{desc, state, base, n, parity, status};
    auto go = [&](auto cfg) { rc = launch_pass_cfg<PolBF16, decltype(cfg), 1>(p, num_sms, st); };
    if (rb) with_cfg(c, BatchCfgsRB<PolBF16>{}, go);
    else with_cfg(c, BatchCfgs<PolBF16>{}, go);
  }
  return rc == 1 ? set_error(STENCIL_ERR_ARG, "batch: no sweep configuration %d", c) : rc;
}

// Geometry and tensor maps of instance i for storage di under configuration
// c, with z chunks of zc planes.
int describe(InstDesc& d, int di, const CfgInfo& ci, int elem, int zc) {
  Grid e0, e1, r;
  for (Grid* g : {&e0, &e1, &r}) {
    g->nx = d.nx; g->ny = d.ny; g->nz = d.nz;
    g->sy = d.esy[di]; g->sz = d.esz[di];
    g->dtype = di == 0 ? STENCIL_F32 : STENCIL_BF16;
    g->elem = elem;
  }
  e0.data = d.e[0];
  e1.data = d.e[1];
  r.data = d.r;
  int rc = make_tensor_map(&d.tm_e[di][0], e0, ci.BOXW, ci.UROWS);
  if (!rc) rc = make_tensor_map(&d.tm_e[di][1], e1, ci.BOXW, ci.UROWS);
  if (!rc) rc = make_tensor_map(&d.tm_r[di], r, ci.BOXW, ci.FROWS);
  if (rc) return rc;
  SweepGeom& g = d.g[di];
  g.nx = d.nx; g.ny = d.ny; g.nz = d.nz; g.sy = d.esy[di]; g.sz = d.esz[di];
  g.bxo = ci.BXO;
  g.byo = ci.BYO;
  g.tiles_x = static_cast<int>((d.nx + ci.BXO - 1) / ci.BXO);
  g.tiles_y = static_cast<int>((d.ny + ci.BYO - 1) / ci.BYO);
  g.zc = static_cast<int>(std::min<int64_t>(d.nz, zc));
  g.items = static_cast<int64_t>(g.tiles_x) * g.tiles_y * ((d.nz + g.zc - 1) / g.zc);
  return STENCIL_OK;
}

struct Solver {
  stencil_ctx* ctx;
  int n;
  cudaStream_t st;
  unsigned char* ws;
  Layout L;
  std::vector<InstDesc> desc;
  std::vector<int64_t> sbase;  // 2 x (n+1)
  int cfg[2] = {0, 0};
  bool rb = false;             // red-black Gauss-Seidel inner sweeps

  InstDesc* d_desc() const { return reinterpret_cast<InstDesc*>(ws + L.desc); }
  InstState* d_state() const { return reinterpret_cast<InstState*>(ws + L.state); }
  int64_t* d_rbase() const { return reinterpret_cast<int64_t*>(ws + L.rbase); }
  int64_t* d_sbase(int di) const { return reinterpret_cast<int64_t*>(ws + L.sbase) + di * (n + 1); }
  BatchTables tables() const {
    return BatchTables{d_desc(), d_state(), d_rbase(), reinterpret_cast<double*>(ws + L.partials),
                       reinterpret_cast<unsigned long long*>(ws + L.nactive), n};
  }
  uint32_t* status() const { return reinterpret_cast<uint32_t*>(ctx->scratch + kScratchStatus); }

  // Build tensor maps, geometry and item tables for configuration c of
  // storage di and upload them.
  int configure(int di, int c) {
    const CfgInfo ci = cfg_info(di, rb, c);
    const int elem = di == 0 ? 4 : 2;
    // z chunk: the longest (fewest re-read planes) that still gives the
    // resident CTAs (about 3 per SM) four items each over the whole batch.
    int zc = 64;
    for (; zc > 8; zc /= 2) {
      int64_t items = 0;
      for (int i = 0; i < n; ++i)
        items += ((desc[i].nx + ci.BXO - 1) / ci.BXO) * ((desc[i].ny + ci.BYO - 1) / ci.BYO) *
                 ((desc[i].nz + zc - 1) / zc);
      if (items >= 12 * static_cast<int64_t>(ctx->num_sms)) break;
    }
    int64_t acc = 0;
    for (int i = 0; i < n; ++i) {
      int rc = describe(desc[i], di, ci, elem, zc);
      if (rc) return rc;
      sbase[di * (n + 1) + i] = acc;
      acc += desc[i].g[di].items;
    }
    sbase[di * (n + 1) + n] = acc;
    cfg[di] = c;
    int rc = check_cuda(cudaMemcpyAsync(d_desc(), desc.data(), sizeof(InstDesc) * n, cudaMemcpyHostToDevice, st),
                        "upload descriptors");
    if (rc) return rc;
    return check_cuda(cudaMemcpyAsync(d_sbase(di), sbase.data() + di * (n + 1), sizeof(int64_t) * (n + 1),
                                      cudaMemcpyHostToDevice, st),
                      "upload item table");
  }

  int pass(int di, int parity) {
    return launch_pass(di, rb, cfg[di], d_desc(), d_state(), d_sbase(di), n, parity, status(), ctx->num_sms, st);
  }
};

int resid_blocks(const Layout& L, int num_sms) {
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(L.ritems, 16 * num_sms)));
}

}  // namespace

}  // namespace stencil

using namespace stencil;

extern "C" int stencil_batch_workspace_size(const stencil_problem* probs, int32_t n, size_t* bytes) {
  if (!probs || n < 1 || !bytes) return set_error(STENCIL_ERR_ARG, "batch_workspace_size: bad arguments");
  for (int i = 0; i < n; ++i) {
    Grid g;
    int rc = validate_grid(&probs[i].u, "u", &g, false);
    if (rc) return rc;
  }
  *bytes = plan(probs, n).total;
  return STENCIL_OK;
}

extern "C" int stencil_batch_solve(stencil_ctx* ctx, const stencil_problem* probs, int32_t n,
                                   const stencil_batch_opts* opts, void* workspace,
                                   size_t workspace_bytes, stencil_result* results, void* stream) {
  if (!ctx || !probs || n < 1 || !opts || !results)
    return set_error(STENCIL_ERR_ARG, "batch_solve: null argument or n < 1");
  if (opts->inner_dtype != STENCIL_F32 && opts->inner_dtype != STENCIL_BF16)
    return set_error(STENCIL_ERR_DTYPE, "batch_solve: inner_dtype must be F32 or BF16");
  if (!(opts->rtol >= 0.0)) return set_error(STENCIL_ERR_ARG, "batch_solve: rtol must be >= 0");
  if (opts->sweeps_per_cycle < 0 || opts->sweeps_per_pass < 0 || opts->sweeps_per_pass > 8 ||
      opts->max_sweeps < 0 || opts->smoother < 0 || opts->smoother > 1)
    return set_error(STENCIL_ERR_ARG, "batch_solve: bad options");
  for (int i = 0; i < n; ++i) {
    Grid gu, gf;
    int rc = validate_grid(&probs[i].u, "u", &gu, false);
    if (!rc) rc = validate_grid(&probs[i].f, "f", &gf, false);
    if (rc) return rc;
    if ((rc = same_extents(gu, gf, "u", "f"))) return rc;
    if (gu.dtype != STENCIL_F64 || gf.dtype != STENCIL_F64)
      return set_error(STENCIL_ERR_DTYPE, "batch_solve: u and f must be F64 (instance %d)", i);
    if (!(probs[i].h > 0.0) || !(probs[i].h < 1e150))
      return set_error(STENCIL_ERR_ARG, "batch_solve: bad h (instance %d)", i);
  }
  const Layout L = plan(probs, n);
  if (!workspace || workspace_bytes < L.total)
    return set_error(STENCIL_ERR_ARG, "batch_solve: workspace of %zu bytes needed", L.total);
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
    return set_error(STENCIL_ERR_ALIGN, "batch_solve: workspace must be 256-byte aligned");
  int prev_dev = -1;
  cudaGetDevice(&prev_dev);
  if (prev_dev != ctx->device) {
    int rc = check_cuda(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (rc) return rc;
  }
  struct Restore {
    int dev;
    ~Restore() { if (dev >= 0) cudaSetDevice(dev); }
  } restore{prev_dev != ctx->device ? prev_dev : -1};

  const int m0 = opts->sweeps_per_cycle > 0 ? opts->sweeps_per_cycle : 100;
  const double stall = opts->stall_ratio > 0.0 ? opts->stall_ratio : 0.9999;
  const int64_t max_sweeps = opts->max_sweeps > 0 ? opts->max_sweeps : 10000000;

  // All work runs on the context's private stream (a capture cannot be made
  // on the legacy default stream), ordered after the caller's stream.
  {
    int rc0 = check_cuda(cudaEventRecord(ctx->solve_event, static_cast<cudaStream_t>(stream)), "event record");
    if (!rc0) rc0 = check_cuda(cudaStreamWaitEvent(ctx->solve_stream, ctx->solve_event, 0), "stream wait");
    if (rc0) return rc0;
  }
  Solver S;
  S.ctx = ctx;
  S.n = n;
  S.rb = opts->smoother == 1;
  S.st = ctx->solve_stream;
  S.ws = static_cast<unsigned char*>(workspace);
  S.L = L;
  S.desc.assign(n, InstDesc());
  S.sbase.assign(2 * (n + 1), 0);
  std::vector<int64_t> rbase(n + 1, 0);
  std::vector<InstState> state(n);
  for (int i = 0; i < n; ++i) {
    InstDesc& d = S.desc[i];
    memset(&d, 0, sizeof(d));
    const stencil_grid& u = probs[i].u;
    const stencil_grid& f = probs[i].f;
    d.u = static_cast<double*>(u.data);
    d.f = static_cast<const double*>(f.data);
    d.nx = u.nx; d.ny = u.ny; d.nz = u.nz;
    d.usy = u.sy; d.usz = u.sz; d.fsy = f.sy; d.fsz = f.sz;
    d.h = probs[i].h;
    d.hh = probs[i].h * probs[i].h;
    const size_t bb = inner_buffer_bytes(u.nx, u.ny, u.nz);
    unsigned char* b = S.ws + L.inst_off[i];
    d.e[0] = b;
    d.e[1] = b + bb;
    d.r = b + 2 * bb;
    d.ebytes = static_cast<int64_t>(bb);
    for (int di = 0; di < 2; ++di) {
      const int elem = di == 0 ? 4 : 2;
      d.esy[di] = sy_for(u.nx, elem);
      d.esz[di] = d.esy[di] * (u.ny + 2);
    }
    rbase[i + 1] = rbase[i] + (u.ny * u.nz + kRowsPerItem - 1) / kRowsPerItem;
    InstState& s = state[i];
    memset(&s, 0, sizeof(s));
    s.active = 1;
    s.dtype = opts->inner_dtype;
    s.prev = INFINITY;
    s.rel = INFINITY;
  }
  cudaStream_t st = S.st;
  int rc = check_cuda(cudaMemsetAsync(S.ws + L.buffers, 0, L.total - L.buffers, st), "zero inner buffers");
  if (!rc) rc = check_cuda(cudaMemcpyAsync(S.ws + L.rbase, rbase.data(), sizeof(int64_t) * (n + 1),
                                           cudaMemcpyHostToDevice, st), "upload residual items");
  if (!rc) rc = check_cuda(cudaMemcpyAsync(S.ws + L.state, state.data(), sizeof(InstState) * n,
                                           cudaMemcpyHostToDevice, st), "upload states");
  if (rc) return rc;

  // Autotune: per inner storage in use (F32 always: BF16 instances may
  // escalate to it), time one pass of every compiled configuration over the
  // whole batch and keep the fastest per sweep (for BF16 Jacobi passes, the
  // fastest of two sweeps or more).
  const bool use_bf16 = opts->inner_dtype == STENCIL_BF16;
  int Tsel[2] = {1, 1};
  for (int di = 0; di < (use_bf16 ? 2 : 1); ++di) {
    int best = -1;
    float best_t = 1e30f;
    for (int c = 0; c < num_cfg(S.rb); ++c) {
      const CfgInfo ci = cfg_info(di, S.rb, c);
      if (opts->sweeps_per_pass > 0 && ci.T != std::min(opts->sweeps_per_pass, 2)) continue;
      // bfloat16 storage rounds the iterate once per pass: one-sweep passes
      // round every sweep and cost more sweeps to the tolerance than they
      // save per sweep, so the library's choice for it is a longer pass.
      if (di == 1 && !S.rb && opts->sweeps_per_pass <= 0 && ci.T < 2) continue;
      rc = S.configure(di, c);
      if (rc) return rc;
      // for timing, every instance counts as storage di
      std::vector<InstState> tstate(state);
      for (auto& s : tstate) s.dtype = di == 0 ? STENCIL_F32 : STENCIL_BF16;
      rc = check_cuda(cudaMemcpyAsync(S.ws + L.state, tstate.data(), sizeof(InstState) * n, cudaMemcpyHostToDevice, st),
                      "upload tuning states");
      if (rc) return rc;
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      rc = S.pass(di, 0);  // warm-up
      cudaEventRecord(e0, st);
      if (!rc) rc = S.pass(di, 1);
      if (!rc) rc = S.pass(di, 0);
      cudaEventRecord(e1, st);
      if (!rc) rc = check_cuda(cudaEventSynchronize(e1), "tuning sync");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (rc) return rc;
      const float per_sweep = ms / (2.0f * ci.T);
      if (per_sweep < best_t) {
        best_t = per_sweep;
        best = c;
      }
    }
    if (best < 0) best = 0;
    rc = S.configure(di, best);
    if (rc) return rc;
    Tsel[di] = cfg_info(di, S.rb, best).T;
  }
  rc = check_cuda(cudaMemcpyAsync(S.ws + L.state, state.data(), sizeof(InstState) * n, cudaMemcpyHostToDevice, st),
                  "upload states");
  if (!rc) rc = check_cuda(cudaMemsetAsync(S.ws + L.buffers, 0, L.total - L.buffers, st), "zero inner buffers");
  if (rc) return rc;
  // Sweeps per cycle: a multiple of twice every pass length, so every storage
  // ends the cycle with the correction in the ping buffer.
  const int Tl = std::max(Tsel[0], use_bf16 ? Tsel[1] : 1);
  const int m = (m0 + 2 * Tl - 1) / (2 * Tl) * (2 * Tl);
  const int passes0 = m / Tsel[0];
  const int passes1 = m / Tsel[1];
  const int final_buf = 0;

  // Capture one cycle as a graph.
  const BatchTables tb = S.tables();
  const CheckArgs ca{opts->rtol, stall, max_sweeps, m};
  const int rblocks = resid_blocks(L, ctx->num_sms);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  rc = check_cuda(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
  if (rc) return rc;
  int crc = check_cuda(cudaMemsetAsync(tb.n_active, 0, sizeof(unsigned long long), st), "memset");
  if (!crc) {
    batch_resid_kernel<0><<<rblocks, dim3(32, 8), 0, st>>>(tb);
    batch_check_kernel<<<(n + 127) / 128, 128, 0, st>>>(tb, ca);
    if (use_bf16) {
      batch_rezero_kernel<<<4 * ctx->num_sms, 256, 0, st>>>(tb);
      batch_resid_kernel<1><<<rblocks, dim3(32, 8), 0, st>>>(tb);
      batch_clear_flags_kernel<<<1, 256, 0, st>>>(tb);
    }
    for (int di = 0; di < (use_bf16 ? 2 : 1) && !crc; ++di) {
      const int passes = di == 0 ? passes0 : passes1;
      for (int p = 0; p < passes && !crc; ++p) crc = S.pass(di, p & 1);
    }
    if (!crc) {
      batch_update_kernel<<<rblocks, dim3(32, 8), 0, st>>>(tb, final_buf);
      crc = check_cuda(cudaGetLastError(), "cycle kernels");
    }
    if (!crc)
      crc = check_cuda(cudaMemcpyAsync(ctx->host_word, tb.n_active, sizeof(unsigned long long),
                                       cudaMemcpyDeviceToHost, st), "read active count");
  }
  rc = check_cuda(cudaStreamEndCapture(st, &graph), "end capture");
  if (crc || rc) {
    if (graph) cudaGraphDestroy(graph);
    return crc ? crc : rc;
  }
  rc = check_cuda(cudaGraphInstantiate(&exec, graph, 0), "graph instantiate");
  cudaGraphDestroy(graph);
  if (rc) return rc;
  const int64_t max_cycles = max_sweeps / m + 2;
  for (int64_t c = 0; c <= max_cycles; ++c) {
    rc = check_cuda(cudaGraphLaunch(exec, st), "graph launch");
    if (!rc) rc = check_cuda(cudaStreamSynchronize(st), "cycle sync");
    if (rc) break;
    if (*ctx->host_word == 0) break;
  }
  cudaGraphExecDestroy(exec);
  if (rc) return rc;
  rc = check_cuda(cudaMemcpyAsync(state.data(), S.ws + L.state, sizeof(InstState) * n, cudaMemcpyDeviceToHost, st),
                  "read states");
  if (!rc) rc = check_cuda(cudaStreamSynchronize(st), "final sync");
  if (rc) return rc;
  for (int i = 0; i < n; ++i) {
    results[i].sweeps = state[i].sweeps;
    results[i].cycles = state[i].cycles;
    results[i].status = state[i].active ? STENCIL_ERR_NOT_CONVERGED : state[i].code;
    results[i].rel_residual = state[i].rel;
    results[i].final_dtype = state[i].dtype;
    results[i].reserved = 0;
  }
  return STENCIL_OK;
}
