// jacobi.cu -- host side of stencil_jacobi_sweep: per-call conversions
// (fixed-point scale, pack/unpack), halo copies, and the choice of kernel
// configuration for each pass (sweep_kernel.cuh holds the kernel).
#include <stdlib.h>

#include <algorithm>

#include "internal.h"
#include "sweep_kernel.cuh"

namespace stencil {

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
  auto kern = jacobi_tb<Pol, Cfg, SrcGrid<Pol>>;
  SingleParams<Pol> prm;
  int rc = make_tensor_map(&prm.tm_u, in, Cfg::BOXW, Cfg::UROWS);
  if (rc) return rc;
  rc = make_tensor_map(&prm.tm_f, f, Cfg::BOXW, Cfg::FROWS);
  if (rc) return rc;
  int grid = 0, per_sm = 0;
  const int64_t txy = ((in.nx + Cfg::BXO - 1) / Cfg::BXO) * ((in.ny + Cfg::BYO - 1) / Cfg::BYO);
  rc = grid_for(kern, Cfg::THREADS, Cfg::SMEM, txy * in.nz, ctx->num_sms, &grid, &per_sm);
  if (rc) return rc;
  const int zc = pick_zc(txy, in.nz, per_sm * ctx->num_sms, Cfg::T);
  prm.g = make_geom<Cfg>(in, zc);
  prm.out = static_cast<typename Pol::T*>(out.data);
  prm.a = a;
  grid = static_cast<int>(std::min<int64_t>(prm.g.items, static_cast<int64_t>(per_sm) * ctx->num_sms));
  kern<<<grid, Cfg::THREADS, Cfg::SMEM, st>>>(prm);
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
