// residual.cu -- r = f - A u for the 7-point operator, in binary64, with
// deterministic norms.
//
// Each point is evaluated with the same IEEE operations, in the same order,
// as the definition (neighbour sum left to right, (6u - s)/h^2 with a true
// division, f - Au) and no fused multiply-add, so every r value is bitwise
// the definition's.  Near convergence r is a small difference of large
// terms; any reordering there changes r by far more than its last bit.
// The two squared norms are summed per thread in a fixed order, combined
// per block by a fixed shuffle tree, written to per-block partials in ctx
// scratch, and summed in block order by a single-block kernel, so the norms
// are reproducible bit for bit from run to run.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace stencil {

constexpr int kResWarps = 8;

__global__ void __launch_bounds__(32 * kResWarps)
    residual_kernel(const double* __restrict__ u, const double* __restrict__ f, double* __restrict__ r,
                    int64_t nx, int64_t ny, int64_t nz, int64_t usy, int64_t usz, int64_t fsy,
                    int64_t fsz, int64_t rsy, int64_t rsz, double hh, double* __restrict__ partials) {
  const int64_t rows = ny * nz;
  double rr = 0.0, ff = 0.0;
  for (int64_t row = blockIdx.x * int64_t(kResWarps) + threadIdx.y; row < rows;
       row += int64_t(gridDim.x) * kResWarps) {
    const int64_t k = 1 + row / ny;
    const int64_t j = 1 + row - (k - 1) * ny;
    const double* uc = u + j * usy + k * usz;
    const double* fc = f + j * fsy + k * fsz;
    for (int64_t i = 1 + threadIdx.x; i <= nx; i += 32) {
      double s = __dadd_rn(uc[i - 1], uc[i + 1]);
      s = __dadd_rn(s, uc[i - usy]);
      s = __dadd_rn(s, uc[i + usy]);
      s = __dadd_rn(s, uc[i - usz]);
      s = __dadd_rn(s, uc[i + usz]);
      const double au = __ddiv_rn(__dsub_rn(__dmul_rn(6.0, uc[i]), s), hh);
      const double fv = fc[i];
      const double res = __dsub_rn(fv, au);
      if (r) r[i + j * rsy + k * rsz] = res;
      rr = fma(res, res, rr);
      ff = fma(fv, fv, ff);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    rr += __shfl_xor_sync(0xffffffffu, rr, o);
    ff += __shfl_xor_sync(0xffffffffu, ff, o);
  }
  __shared__ double wr[kResWarps], wf[kResWarps];
  if (threadIdx.x == 0) {
    wr[threadIdx.y] = rr;
    wf[threadIdx.y] = ff;
  }
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kResWarps; ++w) {
      a += wr[w];
      b += wf[w];
    }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
}

__global__ void __launch_bounds__(256)
    residual_finish_kernel(const double* __restrict__ partials, int nblocks, double* norms) {
  __shared__ double sr[256], sf[256];
  double a = 0.0, b = 0.0;
  for (int q = threadIdx.x; q < nblocks; q += 256) {
    a += partials[2 * q];
    b += partials[2 * q + 1];
  }
  sr[threadIdx.x] = a;
  sf[threadIdx.x] = b;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sr[threadIdx.x] += sr[threadIdx.x + w];
      sf[threadIdx.x] += sf[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    norms[0] = sqrt(sr[0]);
    norms[1] = sqrt(sf[0]);
  }
}

// Number of residual blocks for a grid: a function of the extents only, so
// that the reduction tree (and hence the result) does not depend on anything
// but the input.
int residual_blocks(int64_t ny, int64_t nz) {
  const int64_t rows = ny * nz;
  return static_cast<int>(std::min<int64_t>((rows + kResWarps - 1) / kResWarps, kMaxPartials));
}

int launch_residual_with(double* partials, const Grid& u, const Grid& f, double h, const Grid* r,
                         double* norms_dev, cudaStream_t st) {
  const int blocks = residual_blocks(u.ny, u.nz);
  residual_kernel<<<blocks, dim3(32, kResWarps), 0, st>>>(
      static_cast<const double*>(u.data), static_cast<const double*>(f.data),
      r ? static_cast<double*>(r->data) : nullptr, u.nx, u.ny, u.nz, u.sy, u.sz, f.sy, f.sz,
      r ? r->sy : 0, r ? r->sz : 0, h * h, partials);
  int rc = check_cuda(cudaGetLastError(), "residual kernel");
  if (rc) return rc;
  residual_finish_kernel<<<1, 256, 0, st>>>(partials, blocks, norms_dev);
  return check_cuda(cudaGetLastError(), "residual finish kernel");
}

int launch_residual(stencil_ctx* ctx, const Grid& u, const Grid& f, double h, const Grid* r,
                    double* norms_dev, cudaStream_t st) {
  return launch_residual_with(reinterpret_cast<double*>(ctx->scratch + kScratchPartials), u, f, h,
                              r, norms_dev, st);
}

}  // namespace stencil
