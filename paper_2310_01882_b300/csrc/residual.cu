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
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "sweep_kernel.cuh"

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

// ---------------------------------------------------------------------------
// Fixed-point residual (PolResid, policies.cuh): the caller's u and f staged
// by TMA through one pass of the sweep kernel, R = round(h^2 r 2^S) per
// point, its squared norm summed exactly per CTA (192-bit integers), f's in
// binary64.  The scale S follows from the magnitudes of the u and f values
// the pass reads (their high words).  The first call on a context measures
// a bound with a range pass; later calls take the previous call's
// magnitudes as the guess.  The pass records the magnitudes it actually
// read, and a one-thread check accepts the scale it used only if it is the
// scale of those magnitudes; otherwise a second pass, launched
// unconditionally but returning at once unless the check asked for it,
// recomputes everything at that scale.  So the result is a function of the
// input alone (whatever ran before on the context), computed at the scale
// the input fixes, and a call whose magnitudes keep the previous call's
// scale reads u and f once.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int resid_scale_of(const unsigned long long* m, double hh) {
  SweepArgs a{};
  a.hh = hh;
  a.maxbits = m;
  const PolResid::K k = PolResid::make(a);
  return k.bad ? 100000 : k.S;  // any failure: no guess is accepted
}

__global__ void resid_check_kernel(const unsigned long long* __restrict__ guess,
                                   const unsigned long long* __restrict__ seen, double hh,
                                   unsigned long long* __restrict__ final_bits, uint32_t* __restrict__ redo) {
  const int sg = resid_scale_of(guess, hh);
  const unsigned long long m[3] = {seen[0], seen[1], seen[0]};
  const int sr = resid_scale_of(m, hh);
  const bool ok = sg < 100000 && sg == sr;
  for (int i = 0; i < 3; ++i) final_bits[i] = ok ? guess[i] : m[i];
  *redo = ok ? 0u : 1u;
}

// Sums the CTA partials: the 192-bit integer sums exactly (in any order),
// f's binary64 sums per thread in a fixed order and then by a fixed tree;
// stores the norms and the magnitudes read as the next call's guess.
__global__ void __launch_bounds__(256)
    resid_fx_finish_kernel(const unsigned long long* __restrict__ rpart, SweepArgs a, double* __restrict__ norms,
                           const unsigned long long* __restrict__ seen, unsigned long long* __restrict__ guess) {
  __shared__ unsigned long long ws[3][256];
  __shared__ double wf[256];
  const PolResid::K k = PolResid::make(a);
  const int n = static_cast<int>(rpart[0]);
  PolResid::Track t;
  for (int b = threadIdx.x; b < n; b += 256) {
    const unsigned long long* p = rpart + 4 + 4 * b;
    t.merge(p[0], p[1], p[2], __longlong_as_double(static_cast<long long>(p[3])));
  }
  ws[0][threadIdx.x] = t.s0;
  ws[1][threadIdx.x] = t.s1;
  ws[2][threadIdx.x] = t.s2;
  wf[threadIdx.x] = t.ff;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      t.merge(ws[0][threadIdx.x + w], ws[1][threadIdx.x + w], ws[2][threadIdx.x + w], wf[threadIdx.x + w]);
      ws[0][threadIdx.x] = t.s0;
      ws[1][threadIdx.x] = t.s1;
      ws[2][threadIdx.x] = t.s2;
      wf[threadIdx.x] = t.ff;
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  if (seen) {
    guess[0] = seen[0];
    guess[1] = seen[1];
    guess[2] = seen[2];
  }
  if (k.bad) {
    atomicOr(a.status, k.bad == 1 ? kStatusNonFinite : kStatusRange);
    norms[0] = norms[1] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  // s = s2 2^128 + s1 2^64 + s0 (a few roundings), ||r|| = sqrt(s) 2^-S / h^2
  const double s = fma(static_cast<double>(t.s2), 0x1p128, fma(static_cast<double>(t.s1), 0x1p64,
                                                               static_cast<double>(t.s0)));
  norms[0] = ldexp(sqrt(s), -k.S) / a.hh;
  norms[1] = sqrt(t.ff);
}

namespace {

bool tma_aligned(const Grid& g) {
  return (reinterpret_cast<uintptr_t>(g.data) & 15) == 0 && ((g.sy * g.elem) & 15) == 0 &&
         ((g.sz * g.elem) & 15) == 0 && g.nz + 2 < (1ll << 31) && g.sz * g.elem < (1ll << 40);
}

}  // namespace

int launch_residual(stencil_ctx* ctx, const Grid& u, const Grid& f, double h, const Grid* r,
                    double* norms_dev, cudaStream_t st) {
  // Grids a TMA descriptor cannot address (unaligned rows) take the
  // binary64 kernel, which evaluates the definition in its written order.
  if (!tma_aligned(u) || !tma_aligned(f))
    return launch_residual_with(reinterpret_cast<double*>(ctx->scratch + kScratchPartials), u, f, h,
                                r, norms_dev, st);
  unsigned long long* guess = reinterpret_cast<unsigned long long*>(ctx->scratch + kScratchResidGuess);
  unsigned long long* seen = reinterpret_cast<unsigned long long*>(ctx->scratch + kScratchResidMeas);
  unsigned long long* final_bits = reinterpret_cast<unsigned long long*>(ctx->scratch + kScratchResidFinal);
  uint32_t* redo = reinterpret_cast<uint32_t*>(ctx->scratch + kScratchResidRedo);
  int rc = check_cuda(cudaMemsetAsync(seen, 0, 24, st), "residual magnitude init");
  if (rc) return rc;
  SweepArgs a{};
  a.hh = h * h;
  a.status = reinterpret_cast<uint32_t*>(ctx->scratch + kScratchStatus);
  a.write_r = r != nullptr;
  a.rpart = reinterpret_cast<unsigned long long*>(ctx->scratch + kScratchResidFx);
  a.seen = seen;
  const SweepVariant* vs;
  const int nv = sweep_variants_resid(&vs);
  const int c = (ctx->resid_choice >= 0 && ctx->resid_choice < nv) ? ctx->resid_choice : 0;
  const unsigned long long* used = guess;  // magnitudes the first pass takes its scale from
  if (!ctx->resid_guess) {
    // first call on this context: a bound from a range pass
    unsigned long long* range = reinterpret_cast<unsigned long long*>(ctx->scratch + kScratchRange);
    rc = check_cuda(cudaMemsetAsync(range, 0, 24, st), "residual range init");
    if (rc) return rc;
    const int64_t rows = (u.ny + 2) * (u.nz + 2);
    const int blocks = static_cast<int>(std::min<int64_t>((rows + 7) / 8, 8 * ctx->num_sms));
    range_kernel<<<blocks, dim3(32, 8), 0, st>>>(static_cast<const double*>(u.data),
                                                 static_cast<const double*>(f.data), u.nx, u.ny, u.nz, u.sy, u.sz,
                                                 f.sy, f.sz, range);
    rc = check_cuda(cudaGetLastError(), "residual range kernel");
    if (rc) return rc;
    used = range;
  }
  a.maxbits = used;
  rc = vs[c].fn(ctx, u, r ? *r : u, f, a, st);  // without r nothing is written
  if (rc) return rc;
  resid_check_kernel<<<1, 1, 0, st>>>(used, seen, a.hh, final_bits, redo);
  rc = check_cuda(cudaGetLastError(), "residual check kernel");
  if (rc) return rc;
  a.maxbits = final_bits;
  a.run_flag = redo;  // the same pass again, at the scale of what was read, only if that differs
  rc = vs[c].fn(ctx, u, r ? *r : u, f, a, st);
  if (rc) return rc;
  a.run_flag = nullptr;
  resid_fx_finish_kernel<<<1, 256, 0, st>>>(a.rpart, a, norms_dev, seen, guess);
  rc = check_cuda(cudaGetLastError(), "residual finish kernel");
  if (rc) return rc;
  ctx->resid_guess = 1;
  return STENCIL_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free residual (stencil_residual_noalloc).
//
// For callers that may not allocate device memory themselves and cannot hold
// a stencil_ctx (whose creation allocates): the per-block partial sums live
// in a fixed array compiled into this library, so the call allocates
// nothing.  The array is shared by every call on a device, so calls that
// overlap on that device race; every call overwrites all the partial sums
// it reads, so nothing needs clearing between calls.
// ---------------------------------------------------------------------------
constexpr int kNoAllocMaxPartials = 8192;   // partial-sum pairs the array holds (128 KiB)
constexpr int kNoAllocRowsPerBlock = 64;    // interior (y, z) rows per block
constexpr int64_t kNoAllocMaxRows = static_cast<int64_t>(kNoAllocMaxPartials) * kNoAllocRowsPerBlock;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[2 * kNoAllocMaxPartials];

// Device address of g_noalloc_partials in the CUDA context current on the
// calling thread.  The address belongs to one context (and one load of this
// library's module into it): it is looked up with the device current on the
// first call in each context and kept per device together with that
// context's unique id, so a new context on the device -- after
// cudaDeviceReset, or one the caller created with the driver API -- gets its
// own lookup instead of a stale address.  The first call in a context
// belongs before any stream capture on the device.
static std::mutex g_noalloc_mutex;
static double* g_noalloc_ptr[kNoAllocMaxDevices] = {};
static unsigned long long g_noalloc_ctx[kNoAllocMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Unique id of the context current on this thread (0 if there is none).
static int current_ctx_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(p);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(p);
  });
  if (!get_current || !get_id) return set_error(STENCIL_ERR_CUDA, "residual_noalloc: context query unavailable");
  CUcontext c = nullptr;
  if (get_current(&c) != CUDA_SUCCESS) return set_error(STENCIL_ERR_CUDA, "residual_noalloc: cuCtxGetCurrent failed");
  *id = 0;
  if (c && get_id(c, id) != CUDA_SUCCESS) return set_error(STENCIL_ERR_CUDA, "residual_noalloc: cuCtxGetId failed");
  return STENCIL_OK;
}

static int noalloc_scratch(int device, double** out) {
  if (device < 0 || device >= kNoAllocMaxDevices)
    return set_error(STENCIL_ERR_ARG, "residual_noalloc: device %d out of range", device);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  unsigned long long id = 0;
  int rc = current_ctx_id(&id);
  if (rc) return rc;
  if (!g_noalloc_ptr[device] || id == 0 || id != g_noalloc_ctx[device]) {
    void* p = nullptr;
    rc = check_cuda(cudaGetSymbolAddress(&p, g_noalloc_partials), "residual_noalloc: cudaGetSymbolAddress");
    if (rc) return rc;
    rc = current_ctx_id(&id);  // the lookup makes the device's primary context current if none was
    if (rc) return rc;
    g_noalloc_ptr[device] = static_cast<double*>(p);
    g_noalloc_ctx[device] = id;
  }
  *out = g_noalloc_ptr[device];
  return STENCIL_OK;
}

}  // namespace stencil

extern "C" int stencil_residual_noalloc(const stencil_grid* u, const stencil_grid* f, double h,
                                        const stencil_grid* r, double* norms_dev, void* stream) {
  using namespace stencil;
  Grid gu, gf, gr;
  int rc = validate_grid(u, "u", &gu, false);
  if (!rc) rc = validate_grid(f, "f", &gf, false);
  if (!rc && r) rc = validate_grid(r, "r", &gr, false);
  if (rc) return rc;
  if ((rc = same_extents(gu, gf, "u", "f"))) return rc;
  if (r && (rc = same_extents(gu, gr, "u", "r"))) return rc;
  if (gu.dtype != STENCIL_F64 || gf.dtype != STENCIL_F64 || (r && gr.dtype != STENCIL_F64))
    return set_error(STENCIL_ERR_DTYPE, "residual_noalloc: u, f and r must be F64");
  if (r && (gr.data == gu.data || gr.data == gf.data))
    return set_error(STENCIL_ERR_ARG, "residual_noalloc: r aliases %s (r is written while u and f are read)",
                     gr.data == gu.data ? "u" : "f");
  if (!norms_dev) return set_error(STENCIL_ERR_ARG, "residual_noalloc: null norms pointer");
  if (!(h > 0.0) || !(h < 1.0e150))
    return set_error(STENCIL_ERR_ARG, "residual_noalloc: h must be positive and finite");
  const int64_t rows = gu.ny * gu.nz;
  if (rows > kNoAllocMaxRows)
    return set_error(STENCIL_ERR_ARG,
                     "residual_noalloc: ny*nz = %lld exceeds %lld, the most its built-in scratch "
                     "(%d partial sums) covers; use stencil_residual with a context",
                     (long long)rows, (long long)kNoAllocMaxRows, kNoAllocMaxPartials);
  int device = -1;
  rc = check_cuda(cudaGetDevice(&device), "residual_noalloc: cudaGetDevice");
  if (rc) return rc;
  double* partials = nullptr;
  rc = noalloc_scratch(device, &partials);
  if (rc) return rc;
  const int blocks = static_cast<int>((rows + kNoAllocRowsPerBlock - 1) / kNoAllocRowsPerBlock);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  residual_kernel<<<blocks, dim3(32, kResWarps), 0, st>>>(
      static_cast<const double*>(gu.data), static_cast<const double*>(gf.data),
      r ? static_cast<double*>(gr.data) : nullptr, gu.nx, gu.ny, gu.nz, gu.sy, gu.sz, gf.sy, gf.sz,
      r ? gr.sy : 0, r ? gr.sz : 0, h * h, partials);
  rc = check_cuda(cudaGetLastError(), "residual_noalloc kernel");
  if (rc) return rc;
  residual_finish_kernel<<<1, 256, 0, st>>>(partials, blocks, norms_dev);
  return check_cuda(cudaGetLastError(), "residual_noalloc finish kernel");
}
