// advect.cu -- Piacsek-Williams flux-form momentum advection (Section 4.1:
// the three stencils over u, v, w fused into one region, 63 operations per
// cell), binary64.
//
// One thread per interior cell computes su, sv and sw together, so every
// neighbour value is loaded once per cell from L1 and the three outputs
// leave in one pass (48 algorithmic bytes per cell: three fields in, three
// out).  On B300 this kernel is bound by the binary64 pipe, not by HBM.
#include "common.cuh"
#include "internal.h"

namespace stencil {

__global__ void __launch_bounds__(256)
    advect_kernel(const double* __restrict__ u, const double* __restrict__ v,
                  const double* __restrict__ w, double* __restrict__ su, double* __restrict__ sv,
                  double* __restrict__ sw, const double* __restrict__ tzc1,
                  const double* __restrict__ tzc2, double tcx, double tcy, int64_t nx, int64_t ny,
                  int64_t nz, int64_t sy, int64_t sz, int64_t osy, int64_t osz) {
  const int64_t i = 1 + blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int64_t j = 1 + blockIdx.y * int64_t(blockDim.y) + threadIdx.y;
  if (i > nx || j > ny) return;
  for (int64_t k = 1 + blockIdx.z; k <= nz; k += gridDim.z) {
    const int64_t c = i + j * sy + k * sz;
    const double c1 = tzc1[k - 1], c2 = tzc2[k - 1];
    const double u0 = u[c], v0 = v[c], w0 = w[c];
    // u component at (i+1/2, j, k)
    const double um = u[c - 1], up = u[c + 1];
    double tx = tcx * (um * (u0 + um) - up * (u0 + up));
    double ty = tcy * (u[c - sy] * (v[c - sy] + v[c - sy + 1]) - u[c + sy] * (v0 + v[c + 1]));
    double tz = c1 * u[c - sz] * (w[c - sz] + w[c - sz + 1]) - c2 * u[c + sz] * (w0 + w[c + 1]);
    const int64_t o = i + j * osy + k * osz;
    su[o] = tx + ty + tz;
    // v component at (i, j+1/2, k)
    const double vm = v[c - sy], vp = v[c + sy];
    tx = tcx * (v[c - 1] * (u[c - 1] + u[c - 1 + sy]) - v[c + 1] * (u0 + u[c + sy]));
    ty = tcy * (vm * (v0 + vm) - vp * (v0 + vp));
    tz = c1 * v[c - sz] * (w[c - sz] + w[c - sz + sy]) - c2 * v[c + sz] * (w0 + w[c + sy]);
    sv[o] = tx + ty + tz;
    // w component at (i, j, k+1/2)
    const double wm = w[c - sz], wp = w[c + sz];
    tx = tcx * (w[c - 1] * (u[c - 1] + u[c - 1 + sz]) - w[c + 1] * (u0 + u[c + sz]));
    ty = tcy * (w[c - sy] * (v[c - sy] + v[c - sy + sz]) - w[c + sy] * (v0 + v[c + sz]));
    tz = c1 * wm * (w0 + wm) - c2 * wp * (w0 + wp);
    sw[o] = tx + ty + tz;
  }
}

int launch_advect(stencil_ctx* ctx, const Grid& u, const Grid& v, const Grid& w, const Grid& su,
                  const Grid& sv, const Grid& sw, const double* tzc1, const double* tzc2,
                  double tcx, double tcy, cudaStream_t st) {
  (void)ctx;
  if (u.sy != v.sy || u.sy != w.sy || u.sz != v.sz || u.sz != w.sz)
    return set_error(STENCIL_ERR_ARG, "advect: u, v, w must share strides");
  if (su.sy != sv.sy || su.sy != sw.sy || su.sz != sv.sz || su.sz != sw.sz)
    return set_error(STENCIL_ERR_ARG, "advect: su, sv, sw must share strides");
  const dim3 block(32, 8);
  const int64_t gz = u.nz < 65535 ? u.nz : 65535;
  const dim3 grid(static_cast<unsigned>((u.nx + 31) / 32), static_cast<unsigned>((u.ny + 7) / 8),
                  static_cast<unsigned>(gz));
  if (grid.y > 65535) return set_error(STENCIL_ERR_ARG, "advect: ny too large");
  advect_kernel<<<grid, block, 0, st>>>(
      static_cast<const double*>(u.data), static_cast<const double*>(v.data),
      static_cast<const double*>(w.data), static_cast<double*>(su.data), static_cast<double*>(sv.data),
      static_cast<double*>(sw.data), tzc1, tzc2, tcx, tcy, u.nx, u.ny, u.nz, u.sy, u.sz, su.sy, su.sz);
  return check_cuda(cudaGetLastError(), "advect kernel");
}

}  // namespace stencil
