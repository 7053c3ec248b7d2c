// api.cu -- the C ABI (include/stencil.h): contexts, argument validation,
// error reporting and TMA descriptors.  No compute happens here; every entry
// point validates on the host, then enqueues kernels on the caller's stream.
#include <cudaTypedefs.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "internal.h"

namespace stencil {

static thread_local char g_last_error[512] = "no error";

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return code;
}

int check_cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return STENCIL_OK;
  return set_error(STENCIL_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

static int elem_size(int dtype) {
  switch (dtype) {
    case STENCIL_F64: return 8;
    case STENCIL_F32: return 4;
    case STENCIL_BF16: return 2;
    default: return 0;
  }
}

int validate_grid(const stencil_grid* g, const char* name, Grid* out, bool need_tma) {
  if (!g) return set_error(STENCIL_ERR_ARG, "%s: null grid descriptor", name);
  const int e = elem_size(g->dtype);
  if (!e) return set_error(STENCIL_ERR_DTYPE, "%s: unknown dtype %d", name, g->dtype);
  if (!g->data) return set_error(STENCIL_ERR_ARG, "%s: null data pointer", name);
  if (g->nx < 1 || g->ny < 1 || g->nz < 1)
    return set_error(STENCIL_ERR_ARG, "%s: extents must be >= 1 (got %lld x %lld x %lld)", name,
                     (long long)g->nx, (long long)g->ny, (long long)g->nz);
  if (g->nx > (1 << 30) || g->ny > (1 << 30) || g->nz > (1 << 30))
    return set_error(STENCIL_ERR_ARG, "%s: extent too large", name);
  if (g->sy < g->nx + 2 || g->sz < g->sy * (g->ny + 2))
    return set_error(STENCIL_ERR_ARG, "%s: strides too small (sy=%lld sz=%lld)", name,
                     (long long)g->sy, (long long)g->sz);
  if (g->reserved != 0) return set_error(STENCIL_ERR_ARG, "%s: reserved field must be 0", name);
  if (need_tma) {
    if ((reinterpret_cast<uintptr_t>(g->data) & 15) != 0)
      return set_error(STENCIL_ERR_ALIGN, "%s: data must be 16-byte aligned", name);
    if (((g->sy * e) & 15) != 0 || ((g->sz * e) & 15) != 0)
      return set_error(STENCIL_ERR_ALIGN, "%s: sy and sz must be multiples of 16 bytes", name);
    if (g->nz + 2 > (1ll << 31) || g->sz * e >= (1ll << 40))
      return set_error(STENCIL_ERR_ARG, "%s: grid too large for a tensor map", name);
  }
  out->data = g->data;
  out->nx = g->nx; out->ny = g->ny; out->nz = g->nz;
  out->sy = g->sy; out->sz = g->sz;
  out->dtype = g->dtype;
  out->elem = e;
  return STENCIL_OK;
}

int same_extents(const Grid& a, const Grid& b, const char* an, const char* bn) {
  if (a.nx != b.nx || a.ny != b.ny || a.nz != b.nz)
    return set_error(STENCIL_ERR_ARG, "%s and %s have different extents", an, bn);
  return STENCIL_OK;
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

int make_tensor_map(CUtensorMap* map, const Grid& g, int box_x, int box_y) {
  auto fn = encode_fn();
  if (!fn) return set_error(STENCIL_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  CUtensorMapDataType dt = g.dtype == STENCIL_F64   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                           : g.dtype == STENCIL_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                           : g.dtype == kDtypeU64   ? CU_TENSOR_MAP_DATA_TYPE_UINT64
                                                    : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const cuuint64_t dims[3] = {(cuuint64_t)(g.nx + 2), (cuuint64_t)(g.ny + 2), (cuuint64_t)(g.nz + 2)};
  const cuuint64_t strides[2] = {(cuuint64_t)(g.sy * g.elem), (cuuint64_t)(g.sz * g.elem)};
  const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, dt, 3, g.data, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return set_error(STENCIL_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return STENCIL_OK;
}

int encode_tiled(CUtensorMap* map, CUtensorMapDataType dt, int rank, void* ptr, const uint64_t* dims,
                 const uint64_t* strides, const uint32_t* box, CUtensorMapSwizzle swz) {
  auto fn = encode_fn();
  if (!fn) return set_error(STENCIL_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  cuuint64_t d[5], st[4];
  cuuint32_t b[5], e[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    b[i] = box[i];
    e[i] = 1;
    if (i + 1 < rank) st[i] = strides[i];
  }
  CUresult r = fn(map, dt, rank, ptr, d, st, b, e, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(STENCIL_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return STENCIL_OK;
}

// Make ctx's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  int rc = STENCIL_OK;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) rc = check_cuda(cudaSetDevice(dev), "cudaSetDevice");
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace stencil

using namespace stencil;

extern "C" {

const char* stencil_version(void) { return "b300-stencil 0.1 (sm_103a)"; }

const char* stencil_last_error(void) { return g_last_error; }

int stencil_ctx_create(int device, stencil_ctx** out) {
  if (!out) return set_error(STENCIL_ERR_ARG, "ctx_create: null out pointer");
  *out = nullptr;
  int n = 0;
  int rc = check_cuda(cudaGetDeviceCount(&n), "cudaGetDeviceCount");
  if (rc) return rc;
  if (device < 0 || device >= n) return set_error(STENCIL_ERR_ARG, "ctx_create: bad device %d", device);
  DeviceGuard dg(device);
  if (dg.rc) return dg.rc;
  cudaDeviceProp prop;
  rc = check_cuda(cudaGetDeviceProperties(&prop, device), "cudaGetDeviceProperties");
  if (rc) return rc;
  if (prop.major < 10)
    return set_error(STENCIL_ERR_CUDA, "device %d is sm_%d%d; this library is built for sm_103a",
                     device, prop.major, prop.minor);
  stencil_ctx* c = new (std::nothrow) stencil_ctx();
  if (!c) return set_error(STENCIL_ERR_ARG, "ctx_create: out of host memory");
  c->device = device;
  c->num_sms = prop.multiProcessorCount;
  for (int p = 0; p < kNumPolicies; ++p) {
    for (int t = 0; t <= kMaxPass; ++t) c->sweep_choice[p][t] = c->rb_choice[p][t] = 0;
    c->best_pass[p] = (p == kPolF32 || p == kPolBF16) ? 4 : 1;
  }
  c->scratch_bytes = kScratchBytes;
  void* p = nullptr;
  rc = check_cuda(cudaMalloc(&p, c->scratch_bytes), "cudaMalloc(ctx scratch)");
  if (rc) { delete c; return rc; }
  c->scratch = static_cast<unsigned char*>(p);
  rc = check_cuda(cudaMemset(p, 0, c->scratch_bytes), "cudaMemset(ctx scratch)");
  if (rc) { cudaFree(p); delete c; return rc; }
  void* hw = nullptr;
  rc = check_cuda(cudaHostAlloc(&hw, 64, cudaHostAllocDefault), "cudaHostAlloc(ctx host word)");
  if (rc) { cudaFree(p); delete c; return rc; }
  c->host_word = static_cast<unsigned long long*>(hw);
  rc = check_cuda(cudaStreamCreateWithFlags(&c->solve_stream, cudaStreamNonBlocking), "cudaStreamCreate");
  if (!rc) rc = check_cuda(cudaEventCreateWithFlags(&c->solve_event, cudaEventDisableTiming), "cudaEventCreate");
  if (rc) { cudaFreeHost(hw); cudaFree(p); delete c; return rc; }
  *out = c;
  return STENCIL_OK;
}

int stencil_ctx_destroy(stencil_ctx* ctx) {
  if (!ctx) return STENCIL_OK;
  DeviceGuard dg(ctx->device);
  int rc = check_cuda(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
  expr_cache_free(ctx);
  cudaFree(ctx->scratch);
  cudaFreeHost(ctx->host_word);
  cudaEventDestroy(ctx->solve_event);
  cudaStreamDestroy(ctx->solve_stream);
  delete ctx;
  return rc;
}

int stencil_ctx_status(stencil_ctx* ctx, void* stream) {
  if (!ctx) return set_error(STENCIL_ERR_ARG, "ctx_status: null ctx");
  DeviceGuard dg(ctx->device);
  if (dg.rc) return dg.rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t bits = 0;
  int rc = check_cuda(cudaMemcpyAsync(&bits, ctx->scratch + kScratchStatus, 4, cudaMemcpyDeviceToHost, st),
                      "status read");
  if (rc) return rc;
  rc = check_cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  if (rc) return rc;
  rc = check_cuda(cudaMemsetAsync(ctx->scratch + kScratchStatus, 0, 4, st), "status clear");
  if (rc) return rc;
  rc = check_cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  if (rc) return rc;
  if (bits & kStatusTimeout) return set_error(STENCIL_ERR_TIMEOUT, "a bounded device wait expired");
  if (bits & kStatusNonFinite)
    return set_error(STENCIL_ERR_NONFINITE, "non-finite input to a fixed-point sweep");
  if (bits & kStatusRange) return set_error(STENCIL_ERR_RANGE, "input beyond the fixed-point range");
  return STENCIL_OK;
}

}  // extern "C"

namespace {

// Validation shared by the Jacobi and red-black sweep entry points.
int sweep_call(const char* name, bool redblack, stencil_ctx* ctx, const stencil_grid* u, const stencil_grid* u_tmp,
               const stencil_grid* f, const stencil_grid* work, double h, int64_t nsweeps, int32_t sweeps_per_pass,
               int32_t flags, void* stream) {
  if (!ctx) return set_error(STENCIL_ERR_ARG, "%s: null ctx", name);
  Grid gu, gt, gf, gw;
  int rc = validate_grid(u, "u", &gu, true);
  if (!rc) rc = validate_grid(u_tmp, "u_tmp", &gt, true);
  if (!rc) rc = validate_grid(f, "f", &gf, true);
  if (!rc && work) rc = validate_grid(work, "work", &gw, true);
  if (rc) return rc;
  if ((rc = same_extents(gu, gt, "u", "u_tmp")) || (rc = same_extents(gu, gf, "u", "f"))) return rc;
  if (work && (rc = same_extents(gu, gw, "u", "work"))) return rc;
  if (gu.dtype != gt.dtype || gu.dtype != gf.dtype)
    return set_error(STENCIL_ERR_DTYPE, "%s: u, u_tmp and f must share one dtype", name);
  if (work && gw.dtype != STENCIL_F64) return set_error(STENCIL_ERR_DTYPE, "%s: work must be F64", name);
  if (gu.data == gt.data || gu.data == gf.data || gt.data == gf.data ||
      (work && (gw.data == gu.data || gw.data == gt.data || gw.data == gf.data)))
    return set_error(STENCIL_ERR_ARG, "%s: u, u_tmp, f and work must be distinct buffers", name);
  if (nsweeps < 0) return set_error(STENCIL_ERR_ARG, "%s: nsweeps < 0", name);
  const int max_pass = redblack ? 4 : 8;
  if (sweeps_per_pass < 0 || sweeps_per_pass > max_pass)
    return set_error(STENCIL_ERR_ARG, "%s: sweeps_per_pass must be 0..%d", name, max_pass);
  if (flags < STENCIL_SWEEP_AUTO || flags > STENCIL_SWEEP_FP64_FIXED)
    return set_error(STENCIL_ERR_ARG, "%s: unknown flags %d", name, flags);
  if (!(h > 0.0) || !(h < 1.0e150)) return set_error(STENCIL_ERR_ARG, "%s: h must be positive and finite", name);
  DeviceGuard dg(ctx->device);
  if (dg.rc) return dg.rc;
  const bool use_work = work && gu.dtype == STENCIL_F64;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (redblack)
    return launch_redblack(ctx, gu, gt, gf, use_work ? &gw : nullptr, h, nsweeps, sweeps_per_pass, flags, st);
  return launch_jacobi(ctx, gu, gt, gf, use_work ? &gw : nullptr, h, nsweeps, sweeps_per_pass, flags, st);
}

}  // namespace

extern "C" {

int stencil_jacobi_sweep(stencil_ctx* ctx, const stencil_grid* u, const stencil_grid* u_tmp,
                         const stencil_grid* f, const stencil_grid* work, double h, int64_t nsweeps,
                         int32_t sweeps_per_pass, int32_t flags, void* stream) {
  return sweep_call("jacobi_sweep", false, ctx, u, u_tmp, f, work, h, nsweeps, sweeps_per_pass, flags, stream);
}

int stencil_apply_linear(stencil_ctx* ctx, const stencil_grid* in, const stencil_grid* out, const int32_t* offsets,
                         const double* coeffs, int32_t npoints, void* stream) {
  if (!ctx) return set_error(STENCIL_ERR_ARG, "apply_linear: null ctx");
  Grid gi, go;
  int rc = validate_grid(in, "in", &gi, false);
  if (!rc) rc = validate_grid(out, "out", &go, false);
  if (rc) return rc;
  if ((rc = same_extents(gi, go, "in", "out"))) return rc;
  if (gi.dtype != STENCIL_F64 || go.dtype != STENCIL_F64)
    return set_error(STENCIL_ERR_DTYPE, "apply_linear: in and out must be F64");
  if (gi.data == go.data) return set_error(STENCIL_ERR_ARG, "apply_linear: in and out must be distinct (out of place)");
  if (npoints < 1 || npoints > kMaxLinearTerms || !offsets || !coeffs)
    return set_error(STENCIL_ERR_ARG, "apply_linear: need 1..%d terms", kMaxLinearTerms);
  for (int p = 0; p < 3 * npoints; ++p)
    if (offsets[p] < -kMaxApplyRadius || offsets[p] > kMaxApplyRadius)
      return set_error(STENCIL_ERR_ARG, "apply_linear: offsets must lie in -%d..%d", kMaxApplyRadius,
                       kMaxApplyRadius);
  DeviceGuard dg(ctx->device);
  if (dg.rc) return dg.rc;
  return launch_apply_linear(ctx, gi, go, offsets, coeffs, npoints, static_cast<cudaStream_t>(stream));
}

int stencil_apply_expr(stencil_ctx* ctx, const stencil_grid* const* inputs, int32_t ninputs,
                       const stencil_grid* out, const char* expr, void* stream) {
  if (!ctx) return set_error(STENCIL_ERR_ARG, "apply_expr: null ctx");
  if (!inputs || ninputs < 1 || ninputs > 8) return set_error(STENCIL_ERR_ARG, "apply_expr: need 1..8 inputs");
  Grid gi[8], go;
  int rc = validate_grid(out, "out", &go, false);
  if (rc) return rc;
  if (go.dtype != STENCIL_F64) return set_error(STENCIL_ERR_DTYPE, "apply_expr: out must be F64");
  for (int q = 0; q < ninputs; ++q) {
    if ((rc = validate_grid(inputs[q], "input", &gi[q], false))) return rc;
    if ((rc = same_extents(gi[q], go, "input", "out"))) return rc;
    if (gi[q].dtype != STENCIL_F64) return set_error(STENCIL_ERR_DTYPE, "apply_expr: inputs must be F64");
    if (gi[q].data == go.data) return set_error(STENCIL_ERR_ARG, "apply_expr: out aliases input %d", q);
  }
  DeviceGuard dg(ctx->device);
  if (dg.rc) return dg.rc;
  return launch_apply_expr(ctx, gi, ninputs, go, expr, static_cast<cudaStream_t>(stream));
}

int stencil_expr_source(const char* expr, int32_t ninputs, char* buf, size_t len, int32_t* radius) {
  std::string src;
  int r = 1;
  const int rc = expr_source(expr, ninputs, &src, &r);
  if (rc) return rc;
  if (radius) *radius = r;
  if (buf && len > 0) {
    const size_t n = std::min(len - 1, src.size());
    memcpy(buf, src.data(), n);
    buf[n] = '\0';
  }
  return STENCIL_OK;
}

int stencil_average2d(stencil_ctx* ctx, const stencil_grid* u, const stencil_grid* u_tmp, int64_t nsweeps,
                      void* stream) {
  if (!ctx) return set_error(STENCIL_ERR_ARG, "average2d: null ctx");
  Grid gu, gt;
  int rc = validate_grid(u, "u", &gu, false);
  if (!rc) rc = validate_grid(u_tmp, "u_tmp", &gt, false);
  if (rc) return rc;
  if ((rc = same_extents(gu, gt, "u", "u_tmp"))) return rc;
  if (gu.dtype != STENCIL_F64 || gt.dtype != STENCIL_F64)
    return set_error(STENCIL_ERR_DTYPE, "average2d: u and u_tmp must be F64");
  if (gu.data == gt.data) return set_error(STENCIL_ERR_ARG, "average2d: u and u_tmp must be distinct buffers");
  if (gu.sy != gt.sy || gu.sz != gt.sz) return set_error(STENCIL_ERR_ARG, "average2d: u and u_tmp must share strides");
  if (nsweeps < 0) return set_error(STENCIL_ERR_ARG, "average2d: nsweeps < 0");
  DeviceGuard dg(ctx->device);
  if (dg.rc) return dg.rc;
  return launch_average2d(ctx, gu, gt, nsweeps, static_cast<cudaStream_t>(stream));
}

int stencil_redblack_sweep(stencil_ctx* ctx, const stencil_grid* u, const stencil_grid* u_tmp,
                           const stencil_grid* f, const stencil_grid* work, double h, int64_t nsweeps,
                           int32_t sweeps_per_pass, int32_t flags, void* stream) {
  return sweep_call("redblack_sweep", true, ctx, u, u_tmp, f, work, h, nsweeps, sweeps_per_pass, flags, stream);
}

static int policy_for(int32_t dtype, int32_t flags, int32_t with_work, int* policy) {
  if (dtype == STENCIL_F64) {
    if (flags == STENCIL_SWEEP_FP64_NATIVE) *policy = kPolF64;
    else *policy = with_work ? kPolResident : kPolFixed;
  } else if (dtype == STENCIL_F32) {
    *policy = kPolF32;
  } else if (dtype == STENCIL_BF16) {
    *policy = kPolBF16;
  } else {
    return set_error(STENCIL_ERR_DTYPE, "unknown dtype %d", dtype);
  }
  return STENCIL_OK;
}

int stencil_sweep_config_count(int32_t dtype, int32_t flags, int32_t with_work, int32_t T, int32_t* count) {
  if (!count) return set_error(STENCIL_ERR_ARG, "sweep_config_count: null count");
  int policy = 0;
  int rc = policy_for(dtype, flags, with_work, &policy);
  if (rc) return rc;
  const SweepVariant* v;
  *count = (T >= 1 && T <= kMaxPass) ? sweep_variants(policy, T, &v) : 0;
  return STENCIL_OK;
}

int stencil_sweep_config_select(stencil_ctx* ctx, int32_t dtype, int32_t flags, int32_t with_work, int32_t T,
                                int32_t index) {
  if (!ctx) return set_error(STENCIL_ERR_ARG, "sweep_config_select: null ctx");
  int policy = 0;
  int rc = policy_for(dtype, flags, with_work, &policy);
  if (rc) return rc;
  const SweepVariant* v;
  const int n = (T >= 1 && T <= kMaxPass) ? sweep_variants(policy, T, &v) : 0;
  if (index < 0 || index >= n)
    return set_error(STENCIL_ERR_ARG, "sweep_config_select: index %d out of range (%d configurations)", index, n);
  ctx->sweep_choice[policy][T] = index;
  return STENCIL_OK;
}

int stencil_redblack_config_count(int32_t dtype, int32_t flags, int32_t with_work, int32_t sweeps_per_pass,
                                  int32_t* count) {
  if (!count) return set_error(STENCIL_ERR_ARG, "redblack_config_count: null count");
  int policy = 0;
  int rc = policy_for(dtype, flags, with_work, &policy);
  if (rc) return rc;
  const SweepVariant* v;
  *count = (sweeps_per_pass >= 1 && 2 * sweeps_per_pass <= kMaxPass)
               ? sweep_variants_rb(policy, 2 * sweeps_per_pass, &v)
               : 0;
  return STENCIL_OK;
}

int stencil_residual_config_count(int32_t* count) {
  if (!count) return set_error(STENCIL_ERR_ARG, "residual_config_count: null count");
  const SweepVariant* v;
  *count = sweep_variants_resid(&v);
  return STENCIL_OK;
}

int stencil_residual_config_select(stencil_ctx* ctx, int32_t index) {
  if (!ctx) return set_error(STENCIL_ERR_ARG, "residual_config_select: null ctx");
  const SweepVariant* v;
  const int n = sweep_variants_resid(&v);
  if (index < 0 || index >= n)
    return set_error(STENCIL_ERR_ARG, "residual_config_select: index %d out of range (%d configurations)", index, n);
  ctx->resid_choice = index;
  return STENCIL_OK;
}

int stencil_advect_config_count(int32_t* count) {
  if (!count) return set_error(STENCIL_ERR_ARG, "advect_config_count: null count");
  *count = advect_config_count();
  return STENCIL_OK;
}

int stencil_advect_config_select(stencil_ctx* ctx, int32_t index) {
  if (!ctx) return set_error(STENCIL_ERR_ARG, "advect_config_select: null ctx");
  const int n = advect_config_count();
  if (index < 0 || index >= n)
    return set_error(STENCIL_ERR_ARG, "advect_config_select: index %d out of range (%d configurations)", index, n);
  ctx->advect_choice = index;
  return STENCIL_OK;
}

int stencil_redblack_config_select(stencil_ctx* ctx, int32_t dtype, int32_t flags, int32_t with_work,
                                   int32_t sweeps_per_pass, int32_t index) {
  if (!ctx) return set_error(STENCIL_ERR_ARG, "redblack_config_select: null ctx");
  int policy = 0;
  int rc = policy_for(dtype, flags, with_work, &policy);
  if (rc) return rc;
  const SweepVariant* v;
  const int T = 2 * sweeps_per_pass;
  const int n = (sweeps_per_pass >= 1 && T <= kMaxPass) ? sweep_variants_rb(policy, T, &v) : 0;
  if (index < 0 || index >= n)
    return set_error(STENCIL_ERR_ARG, "redblack_config_select: index %d out of range (%d configurations)", index,
                     n);
  ctx->rb_choice[policy][T] = index;
  return STENCIL_OK;
}

int stencil_autotune_sweep(stencil_ctx* ctx, const stencil_grid* u, const stencil_grid* u_tmp,
                           const stencil_grid* f, const stencil_grid* work, double h, int32_t flags, char* report,
                           size_t report_len, void* stream) {
  if (!ctx) return set_error(STENCIL_ERR_ARG, "autotune_sweep: null ctx");
  Grid gu, gt, gf, gw;
  int rc = validate_grid(u, "u", &gu, true);
  if (!rc) rc = validate_grid(u_tmp, "u_tmp", &gt, true);
  if (!rc) rc = validate_grid(f, "f", &gf, true);
  if (!rc && work) rc = validate_grid(work, "work", &gw, true);
  if (rc) return rc;
  if ((rc = same_extents(gu, gt, "u", "u_tmp")) || (rc = same_extents(gu, gf, "u", "f"))) return rc;
  if (work && (rc = same_extents(gu, gw, "u", "work"))) return rc;
  if (gu.dtype != gt.dtype || gu.dtype != gf.dtype || (work && gw.dtype != STENCIL_F64))
    return set_error(STENCIL_ERR_DTYPE, "autotune_sweep: dtype mismatch");
  if (gu.data == gt.data || gu.data == gf.data || gt.data == gf.data)
    return set_error(STENCIL_ERR_ARG, "autotune_sweep: u, u_tmp and f must be distinct buffers");
  if (flags < STENCIL_SWEEP_AUTO || flags > STENCIL_SWEEP_FP64_FIXED)
    return set_error(STENCIL_ERR_ARG, "autotune_sweep: unknown flags %d", flags);
  if (!(h > 0.0) || !(h < 1.0e150)) return set_error(STENCIL_ERR_ARG, "autotune_sweep: bad h");
  DeviceGuard dg(ctx->device);
  if (dg.rc) return dg.rc;
  const bool use_work = work && gu.dtype == STENCIL_F64;
  return autotune_sweep(ctx, gu, gt, gf, use_work ? &gw : nullptr, h, flags, report, report_len,
                        static_cast<cudaStream_t>(stream));
}

int stencil_residual(stencil_ctx* ctx, const stencil_grid* u, const stencil_grid* f, double h,
                     const stencil_grid* r, double* norms_dev, void* stream) {
  if (!ctx) return set_error(STENCIL_ERR_ARG, "residual: null ctx");
  Grid gu, gf, gr;
  int rc = validate_grid(u, "u", &gu, false);
  if (!rc) rc = validate_grid(f, "f", &gf, false);
  if (!rc && r) rc = validate_grid(r, "r", &gr, false);
  if (rc) return rc;
  if ((rc = same_extents(gu, gf, "u", "f"))) return rc;
  if (r && (rc = same_extents(gu, gr, "u", "r"))) return rc;
  if (gu.dtype != STENCIL_F64 || gf.dtype != STENCIL_F64 || (r && gr.dtype != STENCIL_F64))
    return set_error(STENCIL_ERR_DTYPE, "residual: u, f and r must be F64");
  if (r && (gr.data == gu.data || gr.data == gf.data))
    return set_error(STENCIL_ERR_ARG, "residual: r aliases %s (r is written while u and f are read)",
                     gr.data == gu.data ? "u" : "f");
  if (!norms_dev) return set_error(STENCIL_ERR_ARG, "residual: null norms pointer");
  if (!(h > 0.0) || !(h < 1.0e150)) return set_error(STENCIL_ERR_ARG, "residual: h must be positive and finite");
  DeviceGuard dg(ctx->device);
  if (dg.rc) return dg.rc;
  return launch_residual(ctx, gu, gf, h, r ? &gr : nullptr, norms_dev,
                         static_cast<cudaStream_t>(stream));
}

int stencil_advect_uvw(stencil_ctx* ctx, const stencil_grid* u, const stencil_grid* v,
                       const stencil_grid* w, const stencil_grid* su, const stencil_grid* sv,
                       const stencil_grid* sw, const double* tzc1, const double* tzc2, double tcx,
                       double tcy, void* stream) {
  if (!ctx) return set_error(STENCIL_ERR_ARG, "advect: null ctx");
  Grid g[6];
  const stencil_grid* in[6] = {u, v, w, su, sv, sw};
  const char* names[6] = {"u", "v", "w", "su", "sv", "sw"};
  for (int i = 0; i < 6; ++i) {
    int rc = validate_grid(in[i], names[i], &g[i], false);
    if (rc) return rc;
    if (g[i].dtype != STENCIL_F64) return set_error(STENCIL_ERR_DTYPE, "advect: %s must be F64", names[i]);
    if (i && (rc = same_extents(g[0], g[i], names[0], names[i]))) return rc;
  }
  for (int i = 3; i < 6; ++i)
    for (int j = 0; j < 6; ++j)
      if (i != j && g[i].data == g[j].data)
        return set_error(STENCIL_ERR_ARG, "advect: output %s aliases %s", names[i], names[j]);
  if (!tzc1 || !tzc2) return set_error(STENCIL_ERR_ARG, "advect: null tzc pointer");
  DeviceGuard dg(ctx->device);
  if (dg.rc) return dg.rc;
  return launch_advect(ctx, g[0], g[1], g[2], g[3], g[4], g[5], tzc1, tzc2, tcx, tcy,
                       static_cast<cudaStream_t>(stream));
}

}  // extern "C"
