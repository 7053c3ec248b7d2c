// internal.h -- host-side declarations shared by the library's .cu files.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/stencil.h"

namespace stencil {
struct ExprCache;  // generated stencil.apply kernels of a context (apply_expr.cu)
// Sweep policies (storage / arithmetic) and the registry of compiled
// configurations of the sweep kernel, indexed by policy and pass length T.
enum SweepPolicy { kPolResident = 0, kPolFixed = 1, kPolF64 = 2, kPolF32 = 3, kPolBF16 = 4, kNumPolicies = 5 };
constexpr int kMaxPass = 8;
}  // namespace stencil

struct stencil_ctx {
  int device;
  int num_sms;
  // autotuned choice per policy: configuration index per pass length, and
  // the pass length used when the caller asks for the library's choice
  int sweep_choice[stencil::kNumPolicies][stencil::kMaxPass + 1];
  int best_pass[stencil::kNumPolicies];
  // red-black configuration index per policy and colour stages per pass
  int rb_choice[stencil::kNumPolicies][stencil::kMaxPass + 1];
  int resid_choice;  // fixed-point residual configuration index
  int advect_choice; // advection tile configuration index
  int resid_guess;   // a residual ran on this ctx: its magnitudes are the next call's scale guess
  int apply_guess;   // the same for the fixed-point linear apply
  int advect_guess;  // the same for the fixed-point advection
  int advect_pos;    // which of the three advection magnitude records this call fills
  stencil::ExprCache* expr_cache;  // kernels generated by stencil_apply_expr (null until the first)
  unsigned char* scratch;  // device memory owned by the ctx
  size_t scratch_bytes;
  unsigned long long* host_word;  // pinned host word (batch solve progress)
  cudaStream_t solve_stream;      // private stream the batch solve captures and replays on
  cudaEvent_t solve_event;
};

namespace stencil {

// Device status bits (ctx scratch word), read back by stencil_ctx_status.
constexpr uint32_t kStatusTimeout = 1u;
constexpr uint32_t kStatusNonFinite = 2u;
constexpr uint32_t kStatusRange = 4u;

// Layout of the ctx scratch block (device memory).
constexpr size_t kScratchStatus = 0;      // uint32 status bits
constexpr size_t kScratchAdvRange = 32;   // 5 x uint64: an advection magnitude record (advect.cu), first call
constexpr size_t kScratchRange = 176;     // 3 x uint64 bits: max|u| halo, max|f|, max|u| interior
constexpr size_t kScratchFxMag = 208;     // 4 x uint32: fixed-point magnitude keys (ring of 3)
constexpr size_t kScratchFxScale = 224;   // 4 x int32: fixed-point scales (ring of 3)
constexpr size_t kScratchFxGScale = 240;  // 4 x int32: scale of the stored source (ring of 3)
constexpr size_t kScratchApplyRange = 80; // uint64 bits of max|in| (linear apply, fixed point)
// fixed-point residual: magnitudes (3 x uint64 bits, the layout of
// kScratchRange) of the previous call (the next call's scale guess), of what
// this call's pass read, and of the scale the final pass used; then the
// flag that makes the second pass run (uint32)
constexpr size_t kScratchResidGuess = 88;
constexpr size_t kScratchResidMeas = 112;
constexpr size_t kScratchResidFinal = 136;
constexpr size_t kScratchResidRedo = 160;
constexpr size_t kScratchPartials = 256;  // residual partial sums
constexpr int kMaxPartials = 2048;        // blocks of the residual kernel
// fixed-point residual: CTA count, then 4 words per CTA (up to 2047 CTAs)
constexpr size_t kScratchResidFx = kScratchPartials + sizeof(double) * 2 * kMaxPartials;
constexpr int kMaxResidFxCtas = 2047;
// scale guesses of the fixed-point apply and advection: for each, the
// previous call's magnitudes (bits), those this call's pass read, those
// the final pass used, and the flag that makes the second pass run
constexpr size_t kScratchGuess = kScratchResidFx + 32 * (kMaxResidFxCtas + 1);
constexpr size_t kScratchApplyGuess = kScratchGuess;        // 1 x uint64 each: max|in|
constexpr size_t kScratchApplySeen = kScratchGuess + 8;
constexpr size_t kScratchApplyFinal = kScratchGuess + 16;
constexpr size_t kScratchApplyRedo = kScratchGuess + 24;    // uint32
// advection: three magnitude records of 5 x uint64 (the kScratchAdvRange
// layout) in rotation: the previous call's, this call's, the next call's
constexpr size_t kScratchAdvRec = kScratchGuess + 32;
constexpr size_t kScratchBytes = kScratchGuess + 152;

// Internal dtype code: biased 64-bit fixed-point iterate (never in the ABI).
constexpr int kDtypeU64 = 100;
// Below this many sweeps the resident fixed-point path costs more (one
// conversion pass each way) than converting in every pass.
constexpr int64_t kResidentMinSweeps = 4;

// Validated view of a stencil_grid.
struct Grid {
  void* data;
  int64_t nx, ny, nz, sy, sz;
  int dtype;
  int elem;
};

// Returns STENCIL_OK or an error code (and sets the thread's last error).
int set_error(int code, const char* fmt, ...);
int check_cuda(cudaError_t e, const char* what);
int validate_grid(const stencil_grid* g, const char* name, Grid* out, bool need_tma);
int same_extents(const Grid& a, const Grid& b, const char* an, const char* bn);

// TMA descriptor of a 3D halo grid with box (bx, by, 1).
int make_tensor_map(CUtensorMap* map, const Grid& g, int box_x, int box_y);
// General tiled TMA descriptor (rank <= 5; strides in bytes for dims 1..).
int encode_tiled(CUtensorMap* map, CUtensorMapDataType dt, int rank, void* ptr, const uint64_t* dims,
                 const uint64_t* strides, const uint32_t* box, CUtensorMapSwizzle swz);

struct SweepArgs;
using PassFn = int (*)(stencil_ctx* ctx, const Grid& in, const Grid& out, const Grid& f, const SweepArgs& a,
                       cudaStream_t st);
struct SweepVariant {
  int T, R, WY, S, minb;  // sweeps per pass, rows per warp, warps, stages, CTAs per SM
  PassFn fn;
};
// Compiled configurations for (policy, T); returns their count (0 if none).
int sweep_variants(int policy, int T, const SweepVariant** out);
int sweep_variants_f64(int policy, int T, const SweepVariant** out);
int sweep_variants_f32(int T, const SweepVariant** out);
int sweep_variants_bf16(int T, const SweepVariant** out);
// Red-black Gauss-Seidel configurations (T stages = T/2 sweeps per pass).
int sweep_variants_rb(int policy, int T, const SweepVariant** out);
// Fixed-point residual configurations (one pass of the sweep kernel).
int sweep_variants_resid(const SweepVariant** out);

#ifdef __CUDACC__
// max|u| over the halo, max|f| and max|u| over the interior, as bit patterns
// into maxbits[0..2] (jacobi.cu); maxbits must be zeroed first.
__global__ void range_kernel(const double* __restrict__ u, const double* __restrict__ f, int64_t nx, int64_t ny,
                             int64_t nz, int64_t usy, int64_t usz, int64_t fsy, int64_t fsz,
                             unsigned long long* maxbits);
#endif

// Kernel launchers (jacobi.cu, residual.cu, advect.cu).
int launch_jacobi(stencil_ctx* ctx, const Grid& u, const Grid& ut, const Grid& f, const Grid* work,
                  double h, int64_t nsweeps, int spp, int flags, cudaStream_t st);
int launch_average2d(stencil_ctx* ctx, const Grid& u, const Grid& ut, int64_t nsweeps, cudaStream_t st);
constexpr int kMaxLinearTerms = 64;
constexpr int kMaxApplyRadius = 3;
int launch_apply_linear(stencil_ctx* ctx, const Grid& in, const Grid& out, const int32_t* offsets,
                        const double* coeffs, int npoints, cudaStream_t st);
int launch_redblack(stencil_ctx* ctx, const Grid& u, const Grid& ut, const Grid& f, const Grid* work,
                    double h, int64_t nsweeps, int spp, int flags, cudaStream_t st);
int autotune_sweep(stencil_ctx* ctx, const Grid& u, const Grid& ut, const Grid& f, const Grid* work, double h,
                   int flags, char* report, size_t report_len, cudaStream_t st);
int launch_residual(stencil_ctx* ctx, const Grid& u, const Grid& f, double h, const Grid* r,
                    double* norms_dev, cudaStream_t st);
int launch_advect(stencil_ctx* ctx, const Grid& u, const Grid& v, const Grid& w, const Grid& su,
                  const Grid& sv, const Grid& sw, const double* tzc1, const double* tzc2,
                  double tcx, double tcy, cudaStream_t st);
int advect_config_count();
// General stencil.apply from an expression (apply_expr.cu).
int expr_source(const char* expr, int ninputs, std::string* src, int* radius);
int launch_apply_expr(stencil_ctx* ctx, const Grid* in, int ninputs, const Grid& out, const char* expr,
                      cudaStream_t st);
void expr_cache_free(stencil_ctx* ctx);

}  // namespace stencil
