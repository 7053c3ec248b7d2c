// sweep_launch.cuh -- host-side launch of one configuration of the sweep
// kernel (sweep_kernel.cuh) over a single grid; included by the files that
// instantiate the compiled configurations (sweep_f64.cu, sweep_f32.cu,
// sweep_bf16.cu).
#pragma once

#include <algorithm>

#include "internal.h"
#include "sweep_rb_kernel.cuh"

namespace stencil {
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
  auto kern = sweep_kernel_for<Pol, Cfg, SrcGrid<Pol>>();
  SingleParams<Pol> prm;
  int rc = make_tensor_map(&prm.tm_u, in, Cfg::BOXW, Cfg::UROWS);
  if (rc) return rc;
  rc = make_tensor_map(&prm.tm_f, f, Cfg::BOXW, Cfg::FROWS);
  if (rc) return rc;
  if (a.fsrc64) {  // resident fixed point: the caller's binary64 source, same box
    Grid f64 = f;
    f64.data = const_cast<double*>(a.fsrc64);
    f64.sy = a.fsy;
    f64.sz = a.fsz;
    f64.dtype = STENCIL_F64;
    rc = make_tensor_map(&prm.tm_f64, f64, Cfg::BOXW, Cfg::FROWS);
    if (rc) return rc;
  } else {
    prm.tm_f64 = prm.tm_f;
  }
  int grid = 0, per_sm = 0;
  const int64_t txy = ((in.nx + Cfg::BXO - 1) / Cfg::BXO) * ((in.ny + Cfg::BYO - 1) / Cfg::BYO);
  rc = grid_for(kern, Cfg::THREADS, Cfg::SMEM, txy * in.nz, ctx->num_sms, &grid, &per_sm);
  if (rc) return rc;
  const int zc = pick_zc(txy, in.nz, per_sm * ctx->num_sms, Cfg::T);
  prm.g = make_geom<Cfg>(in, zc);
  prm.out = static_cast<typename Pol::T*>(out.data);
  prm.osy = out.sy;
  prm.osz = out.sz;
  prm.a = a;
  grid = static_cast<int>(std::min<int64_t>(prm.g.items, static_cast<int64_t>(per_sm) * ctx->num_sms));
  if constexpr (Pol::kResidual) grid = std::min(grid, kMaxResidFxCtas);  // one partial-sum slot per CTA
  kern<<<grid, Cfg::THREADS, Cfg::SMEM, st>>>(prm);
  return check_cuda(cudaGetLastError(), "jacobi_tb launch");
}

}  // namespace

// The registry entry of configuration Cfg of policy Pol.
template <class Pol, class Cfg>
SweepVariant variant() {
  return SweepVariant{Cfg::T, Cfg::R, Cfg::WY, Cfg::S, Cfg::MINB, &run_tb<Pol, Cfg>};
}

}  // namespace stencil
