// jacobi.cu -- host side of stencil_jacobi_sweep: per-call conversions
// (fixed-point scale, pack/unpack), halo copies, and the choice of kernel
// configuration for each pass (sweep_kernel.cuh holds the kernel).
#include <stdlib.h>

#include <algorithm>
#include <string>

#include <stdio.h>
#include <string.h>

#include "internal.h"
#include "sweep_kernel.cuh"

namespace stencil {

// max|u| over the halo cells, max|f| and max|u| over the interior, as the
// bit patterns of non-negative doubles (their integer order is their
// numeric order; NaN sorts above Inf, so a NaN anywhere is seen).
__global__ void range_kernel(const double* __restrict__ u, const double* __restrict__ f,
                             int64_t nx, int64_t ny, int64_t nz, int64_t usy, int64_t usz,
                             int64_t fsy, int64_t fsz, unsigned long long* maxbits) {
  const int64_t rows = (ny + 2) * (nz + 2);
  unsigned long long mh = 0, mf = 0, mu = 0;
  for (int64_t row = blockIdx.x * int64_t(blockDim.y) + threadIdx.y; row < rows;
       row += int64_t(gridDim.x) * blockDim.y) {
    const int64_t k = row / (ny + 2);
    const int64_t j = row - k * (ny + 2);
    const bool inner = (j >= 1 && j <= ny && k >= 1 && k <= nz);
    for (int64_t i = threadIdx.x; i < nx + 2; i += blockDim.x) {
      const unsigned long long bu =
          static_cast<unsigned long long>(__double_as_longlong(u[i + j * usy + k * usz])) &
          0x7fffffffffffffffull;
      if (inner && i >= 1 && i <= nx) {
        const unsigned long long bf =
            static_cast<unsigned long long>(__double_as_longlong(f[i + j * fsy + k * fsz])) &
            0x7fffffffffffffffull;
        mf = bf > mf ? bf : mf;
        mu = bu > mu ? bu : mu;
      } else {
        mh = bu > mh ? bu : mh;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long a = __shfl_xor_sync(0xffffffffu, mh, o);
    const unsigned long long b = __shfl_xor_sync(0xffffffffu, mf, o);
    const unsigned long long c = __shfl_xor_sync(0xffffffffu, mu, o);
    mh = a > mh ? a : mh;
    mf = b > mf ? b : mf;
    mu = c > mu ? c : mu;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&maxbits[0], mh);
    atomicMax(&maxbits[1], mf);
    atomicMax(&maxbits[2], mu);
  }
}

// Slot 0 of the fixed-point state, read by pass 1: the scale the first pass
// would choose from the caller's u (RESIDENT: the scale the interior is packed
// at) and the magnitude key of u's interior, so that pass 1 normally keeps
// that scale.  One thread.
template <bool RESIDENT>
__global__ void fx_init_kernel(SweepArgs a) {
  const double mu = bits_as_double(a.maxbits[2]);
  const double mh = bits_as_double(a.maxbits[0]);
  const double mf = bits_as_double(a.maxbits[1]);
  int bad = 0;
  int S = 0;
  if (!(mu <= 1.0e300) || !(mh <= 1.0e300) || !(mf <= 1.0e300)) {
    bad = (mu - mu == 0.0 && mh - mh == 0.0 && mf - mf == 0.0) ? 2 : 1;
  } else {
    const double hmf = a.hh * mf;
    S = fx_scale_for(6.0 * (fmax(mu, mh) + static_cast<double>(a.stages) * hmf / 6.0) + hmf, &bad);
  }
  uint32_t key;
  if (RESIDENT) {  // largest |q| of the packed interior is below (key + 1) 2^32
    key = bad ? 0u : static_cast<uint32_t>(ldexp(mu, S - 32));
  } else {         // high word of max|u| over the interior
    key = static_cast<uint32_t>(a.maxbits[2] >> 32);
  }
  a.fxmag[0] = key;
  a.fxmag[1] = 0u;
  a.fxscale[0] = bad ? kFxBadScale + bad : S;
  if (RESIDENT) a.fxgscale[0] = S;  // the set-up packs the source at S
  if (bad) atomicOr(a.status, bad == 1 ? kStatusNonFinite : kStatusRange);
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
// integers U, and the interior of f to G = round(h*h*f*2^S) in work, both at
// the scale S of slot 0.
__global__ void fx_pack_kernel(double* __restrict__ u, const double* __restrict__ f,
                               unsigned long long* __restrict__ work, int64_t nx, int64_t ny,
                               int64_t nz, int64_t usy, int64_t usz, int64_t fsy, int64_t fsz,
                               int64_t wsy, int64_t wsz, SweepArgs a) {
  const int S0 = a.fxscale[0];
  if (S0 >= kFxBadScale) return;  // reported by the set-up; the result will be NaN
  FixedParams k;
  fx_conv(k, S0, a.hh);
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

// Back to binary64: the interior of src (U, at the scale the last pass,
// a.pass, published) into the interior of u; NaN if the call failed.
__global__ void fx_unpack_kernel(const unsigned long long* __restrict__ src, double* __restrict__ u,
                                 int64_t nx, int64_t ny, int64_t nz, int64_t ssy, int64_t ssz,
                                 int64_t usy, int64_t usz, SweepArgs a) {
  const int S = a.fxscale[a.pass % 3];
  const bool bad = S >= kFxBadScale;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  const int64_t rows = ny * nz;
  for (int64_t row = blockIdx.x * int64_t(blockDim.y) + threadIdx.y; row < rows;
       row += int64_t(gridDim.x) * blockDim.y) {
    const int64_t kz = 1 + row / ny;
    const int64_t j = 1 + row - (kz - 1) * ny;
    const unsigned long long* sr = src + j * ssy + kz * ssz;
    double* ur = u + j * usy + kz * usz;
    for (int64_t i = 1 + threadIdx.x; i <= nx; i += blockDim.x) ur[i] = bad ? nan : fx_out(sr[i], S);
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

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

int policy_of(int dtype, bool fixed, bool resident) {
  if (dtype == STENCIL_F64) return resident ? kPolResident : (fixed ? kPolFixed : kPolF64);
  return dtype == STENCIL_F32 ? kPolF32 : kPolBF16;
}

// Largest pass length with compiled configurations, not above `want`.
int supported_t(int policy, int want) {
  for (int T = std::min(want, kMaxPass); T > 1; --T) {
    const SweepVariant* v;
    if (sweep_variants(policy, T, &v) > 0) return T;
  }
  return 1;
}

int run_pass(stencil_ctx* ctx, int policy, int T, const Grid& in, const Grid& out, const Grid& f,
             const SweepArgs& a, cudaStream_t st) {
  const SweepVariant* vs;
  const int nv = sweep_variants(policy, T, &vs);
  if (nv < 1) return set_error(STENCIL_ERR_ARG, "no compiled sweep configuration for T=%d", T);
  int c = ctx->sweep_choice[policy][T];
  if (c < 0 || c >= nv) c = 0;
  return vs[c].fn(ctx, in, out, f, a, st);
}

}  // namespace

int sweep_variants(int policy, int T, const SweepVariant** out) {
  if (policy == kPolF32) return sweep_variants_f32(T, out);
  if (policy == kPolBF16) return sweep_variants_bf16(T, out);
  return sweep_variants_f64(policy, T, out);
}

namespace {

// Per-call set-up shared by the sweep and its autotuner: u_tmp's halo, the
// fixed-point range, and (resident) the packed iterate and source.
struct Prepared {
  int policy;
  Grid ui, ti, fi;
  SweepArgs a;
};

int prepare(stencil_ctx* ctx, const Grid& u, const Grid& ut, const Grid& f, const Grid* work, double h,
            int64_t nsweeps, int first_stages, int flags, bool pack, cudaStream_t st, Prepared* P) {
  const bool fixed = (u.dtype == STENCIL_F64) && (flags != STENCIL_SWEEP_FP64_NATIVE);
  const bool resident = fixed && work != nullptr && nsweeps >= kResidentMinSweeps;
  P->policy = policy_of(u.dtype, fixed, resident);
  int rc = copy_halo_any(u, ut, st);
  if (rc) return rc;
  SweepArgs& a = P->a;
  a.hh = h * h;
  a.maxbits = reinterpret_cast<const unsigned long long*>(ctx->scratch + kScratchRange);
  a.status = reinterpret_cast<uint32_t*>(ctx->scratch + kScratchStatus);
  a.fxmag = reinterpret_cast<uint32_t*>(ctx->scratch + kScratchFxMag);
  a.fxscale = reinterpret_cast<int32_t*>(ctx->scratch + kScratchFxScale);
  a.pass = 1;
  a.stages = first_stages;
  a.fsrc64 = resident ? static_cast<const double*>(f.data) : nullptr;
  a.fsy = f.sy;
  a.fsz = f.sz;
  a.fxgscale = resident ? reinterpret_cast<int32_t*>(ctx->scratch + kScratchFxGScale) : nullptr;
  a.gdst = resident ? static_cast<unsigned long long*>(work->data) : nullptr;
  a.gsy = resident ? work->sy : 0;
  a.gsz = resident ? work->sz : 0;
  if (fixed) {
    rc = check_cuda(cudaMemsetAsync(ctx->scratch + kScratchRange, 0, 24, st), "memset range");
    if (rc) return rc;
    const int64_t rows = (u.ny + 2) * (u.nz + 2);
    const int blocks = static_cast<int>(std::min<int64_t>((rows + 7) / 8, 8 * ctx->num_sms));
    range_kernel<<<blocks, dim3(32, 8), 0, st>>>(
        static_cast<const double*>(u.data), static_cast<const double*>(f.data), u.nx, u.ny, u.nz,
        u.sy, u.sz, f.sy, f.sz, reinterpret_cast<unsigned long long*>(ctx->scratch + kScratchRange));
    rc = check_cuda(cudaGetLastError(), "range kernel");
    if (rc) return rc;
    if (resident) fx_init_kernel<true><<<1, 1, 0, st>>>(a);
    else fx_init_kernel<false><<<1, 1, 0, st>>>(a);
    rc = check_cuda(cudaGetLastError(), "fixed-point set-up kernel");
    if (rc) return rc;
  }
  P->ui = u;
  P->ti = ut;
  P->fi = f;
  if (resident) {
    if (pack) {
      const int64_t rows = u.ny * u.nz;
      const int cblocks = static_cast<int>(std::min<int64_t>((rows + 7) / 8, 16 * ctx->num_sms));
      fx_pack_kernel<<<cblocks, dim3(32, 8), 0, st>>>(
          static_cast<double*>(u.data), static_cast<const double*>(f.data),
          static_cast<unsigned long long*>(work->data), u.nx, u.ny, u.nz, u.sy, u.sz, f.sy, f.sz, work->sy,
          work->sz, a);
      rc = check_cuda(cudaGetLastError(), "pack kernel");
      if (rc) return rc;
    }
    P->ui.dtype = P->ti.dtype = kDtypeU64;
    P->fi = *work;
    P->fi.dtype = kDtypeU64;
  }
  return STENCIL_OK;
}

}  // namespace

namespace {

// After the last pass: the iterate is in `last` (u's buffer or u_tmp's);
// bring it back into u (the resident policy unpacks the fixed point).
int finish(stencil_ctx* ctx, const Prepared& P, const Grid& u, const Grid& last, bool in_tmp, int passes,
           cudaStream_t st) {
  if (P.policy == kPolResident) {
    SweepArgs a = P.a;
    a.pass = passes;
    const int64_t rows = u.ny * u.nz;
    const int cblocks = static_cast<int>(std::min<int64_t>((rows + 7) / 8, 16 * ctx->num_sms));
    fx_unpack_kernel<<<cblocks, dim3(32, 8), 0, st>>>(
        static_cast<const unsigned long long*>(last.data), static_cast<double*>(u.data), u.nx, u.ny, u.nz,
        last.sy, last.sz, u.sy, u.sz, a);
    return check_cuda(cudaGetLastError(), "unpack kernel");
  }
  return in_tmp ? copy_interior_any(last, u, st) : STENCIL_OK;
}

}  // namespace

namespace {

// The four-neighbour average of the paper's running example (Section 2.2,
// Listing 1) on every z plane, binary64 in the order of the definition
// (two neighbours along x, then y-1, then y+1, times 0.25; no fused
// multiply-add), one thread per point; neighbours come through L1.
__global__ void __launch_bounds__(256)
    average2d_kernel(const double* __restrict__ in, double* __restrict__ out, int64_t nx, int64_t ny, int64_t nz,
                     int64_t sy, int64_t sz) {
  const int64_t i = 1 + blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int64_t j = 1 + blockIdx.y * int64_t(blockDim.y) + threadIdx.y;
  if (i > nx || j > ny) return;
  for (int64_t k = 1 + blockIdx.z; k <= nz; k += gridDim.z) {
    const int64_t c = i + j * sy + k * sz;
    double s = __dadd_rn(in[c - 1], in[c + 1]);
    s = __dadd_rn(s, in[c - sy]);
    s = __dadd_rn(s, in[c + sy]);
    out[c] = __dmul_rn(s, 0.25);
  }
}

}  // namespace

int launch_average2d(stencil_ctx* ctx, const Grid& u, const Grid& ut, int64_t nsweeps, cudaStream_t st) {
  (void)ctx;
  if (nsweeps == 0) return STENCIL_OK;
  int rc = copy_halo_any(u, ut, st);
  if (rc) return rc;
  const dim3 block(32, 8);
  const dim3 grid(static_cast<unsigned>((u.nx + 31) / 32), static_cast<unsigned>((u.ny + 7) / 8),
                  static_cast<unsigned>(std::min<int64_t>(u.nz, 65535)));
  if (grid.y > 65535) return set_error(STENCIL_ERR_ARG, "average2d: ny too large");
  const Grid* a = &u;
  const Grid* b = &ut;
  for (int64_t s = 0; s < nsweeps; ++s) {
    average2d_kernel<<<grid, block, 0, st>>>(static_cast<const double*>(a->data), static_cast<double*>(b->data),
                                             u.nx, u.ny, u.nz, u.sy, u.sz);
    rc = check_cuda(cudaGetLastError(), "average2d kernel");
    if (rc) return rc;
    std::swap(a, b);
  }
  return a != &u ? copy_interior_any(*a, u, st) : STENCIL_OK;
}

int launch_jacobi(stencil_ctx* ctx, const Grid& u, const Grid& ut, const Grid& f, const Grid* work,
                  double h, int64_t nsweeps, int spp, int flags, cudaStream_t st) {
  if (nsweeps == 0) return STENCIL_OK;
  const int policy = policy_of(u.dtype, u.dtype == STENCIL_F64 && flags != STENCIL_SWEEP_FP64_NATIVE,
                               u.dtype == STENCIL_F64 && flags != STENCIL_SWEEP_FP64_NATIVE && work != nullptr &&
                                   nsweeps >= kResidentMinSweeps);
  const int want = spp > 0 ? spp : ctx->best_pass[policy];
  const int T1 = supported_t(policy, static_cast<int>(std::min<int64_t>(nsweeps, want)));
  Prepared P;
  int rc = prepare(ctx, u, ut, f, work, h, nsweeps, T1, flags, true, st, &P);
  if (rc) return rc;
  const Grid* a_in = &P.ui;
  const Grid* b_out = &P.ti;
  int64_t left = nsweeps;
  int pass = 0;
  while (left > 0) {
    const int T = supported_t(P.policy, static_cast<int>(std::min<int64_t>(left, want)));
    P.a.pass = ++pass;
    P.a.stages = T;
    rc = run_pass(ctx, P.policy, T, *a_in, *b_out, P.fi, P.a, st);
    if (rc) return rc;
    std::swap(a_in, b_out);
    left -= T;
  }
  return finish(ctx, P, u, *a_in, a_in != &P.ui, pass, st);
}

// nsweeps red-black Gauss-Seidel sweeps: passes of T = 2 x (sweeps per
// pass) colour stages through the same kernel.  The fixed-point bound holds
// as for Jacobi with 2 nsweeps half sweeps (each half sweep is an average
// of neighbours plus h^2 f / 6, monotone in its inputs).
int launch_redblack(stencil_ctx* ctx, const Grid& u, const Grid& ut, const Grid& f, const Grid* work,
                    double h, int64_t nsweeps, int spp, int flags, cudaStream_t st) {
  if (nsweeps == 0) return STENCIL_OK;
  const int want = spp > 0 ? spp : 1;
  Prepared P;
  int rc = prepare(ctx, u, ut, f, work, h, 2 * nsweeps, 2 * static_cast<int>(std::min<int64_t>(nsweeps, want)),
                   flags, true, st, &P);
  if (rc) return rc;
  const Grid* a_in = &P.ui;
  const Grid* b_out = &P.ti;
  int64_t left = nsweeps;
  int pass = 0;
  while (left > 0) {
    int T = 2 * static_cast<int>(std::min<int64_t>(left, want));
    const SweepVariant* vs = nullptr;
    int nv = 0;
    for (; T >= 2; T -= 2)
      if ((nv = sweep_variants_rb(P.policy, T, &vs)) > 0) break;
    if (nv < 1) return set_error(STENCIL_ERR_ARG, "no compiled red-black configuration");
    const int c = ctx->rb_choice[P.policy][T];
    P.a.pass = ++pass;
    P.a.stages = T;
    rc = vs[c < nv ? c : 0].fn(ctx, *a_in, *b_out, P.fi, P.a, st);
    if (rc) return rc;
    std::swap(a_in, b_out);
    left -= T / 2;
  }
  return finish(ctx, P, u, *a_in, a_in != &P.ui, pass, st);
}

int autotune_sweep(stencil_ctx* ctx, const Grid& u, const Grid& ut, const Grid& f, const Grid* work, double h,
                   int flags, char* report, size_t report_len, cudaStream_t st) {
  // Trial passes read u and write u_tmp only (u's contents are never
  // changed; the resident policy's trials read u's binary64 interior as if
  // it were packed, which costs the same).
  Prepared P;
  int rc = prepare(ctx, u, ut, f, work, h, 1000, 1, flags, false, st, &P);
  if (rc) return rc;
  std::string rep;
  char line[256];
  cudaEvent_t e0, e1;
  rc = check_cuda(cudaEventCreate(&e0), "event");
  if (!rc) rc = check_cuda(cudaEventCreate(&e1), "event");
  if (rc) return rc;
  double best_rate = 1e300;
  int best_T = 1;
  for (int T = 1; T <= kMaxPass && !rc; ++T) {
    const SweepVariant* vs;
    const int nv = sweep_variants(P.policy, T, &vs);
    if (nv < 1) continue;
    int best = 0;
    float best_ms = 1e30f;
    for (int c = 0; c < nv && !rc; ++c) {
      const int reps = 4;
      rc = vs[c].fn(ctx, P.ui, P.ti, P.fi, P.a, st);  // warm-up
      if (!rc) rc = check_cuda(cudaEventRecord(e0, st), "event record");
      for (int r = 0; r < reps && !rc; ++r) rc = vs[c].fn(ctx, P.ui, P.ti, P.fi, P.a, st);
      if (!rc) rc = check_cuda(cudaEventRecord(e1, st), "event record");
      if (!rc) rc = check_cuda(cudaEventSynchronize(e1), "event sync");
      float ms = 0.0f;
      if (!rc) cudaEventElapsedTime(&ms, e0, e1);
      const float per_sweep = ms / (reps * T);
      snprintf(line, sizeof(line), "policy %d T=%d R=%d WY=%d S=%d minb=%d: %.4f ms/sweep\n", P.policy, T,
               vs[c].R, vs[c].WY, vs[c].S, vs[c].minb, per_sweep);
      rep += line;
      if (per_sweep < best_ms) {
        best_ms = per_sweep;
        best = c;
      }
    }
    ctx->sweep_choice[P.policy][T] = best;
    if (best_ms < best_rate) {
      best_rate = best_ms;
      best_T = T;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  ctx->best_pass[P.policy] = best_T;
  snprintf(line, sizeof(line), "chosen: T=%d\n", best_T);
  rep += line;
  if (report && report_len > 0) {
    strncpy(report, rep.c_str(), report_len - 1);
    report[report_len - 1] = 0;
  }
  return STENCIL_OK;
}

}  // namespace stencil
