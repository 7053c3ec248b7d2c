/*
 * stencil.h -- C ABI of the B300 stencil library (libstencil.so).
 *
 * The library applies the two stencil kernels measured in arXiv 2310.01882
 * (Brown et al., SC-W 2023) over 3D structured grids on one GPU:
 *   - the 7-point relaxation sweep (Section 4.1, "Gauss Seidel" benchmark:
 *     each cell becomes the average of its six orthogonal neighbours), in
 *     the Poisson form with a source term, applied out of place (Jacobi) as
 *     a stencil apply is (Section 2.2);
 *   - the Piacsek-Williams flux-form advection of u, v, w (Section 4.1,
 *     three stencils fused into one region, 63 operations per cell);
 * plus the FP64 residual that decides convergence.
 *
 * Conventions (Section 2.2: first index fastest, offsets relative to the
 * cell; Section 3: data crosses the boundary as raw pointers, and, with the
 * optimised data approach of Section 4.3, stays resident on the device):
 *   - A field is a stencil_grid: interior extents nx, ny, nz >= 1 and a
 *     one-cell halo, stored x fastest.  `data` is a DEVICE pointer to the
 *     halo cell (0,0,0); cell (i,j,k), 0 <= i <= nx+1 etc., is at
 *     data + i + j*sy + k*sz (element strides, x stride 1).
 *   - Interior cells are 1..n per axis; index 0 and n+1 are the halo, which
 *     holds the boundary values (Dirichlet values for the Poisson routines,
 *     caller-filled periodic/zero values for advection).
 *   - Alignment: `data` must be 16-byte aligned and sy*elem, sz*elem must be
 *     multiples of 16 bytes (the tiles are staged by the tensor-memory
 *     accelerator); sy >= nx+2, sz >= sy*(ny+2).  Violations return
 *     STENCIL_ERR_ALIGN or STENCIL_ERR_ARG and launch nothing.
 *   - Ownership: the caller owns every grid and stream.  The library never
 *     allocates, frees or copies caller memory to the host.  Scratch memory
 *     belongs to the stencil_ctx (allocated in stencil_ctx_create).
 *   - Asynchrony: every compute call only enqueues work on `stream` (a
 *     cudaStream_t; NULL = the legacy default stream) and returns.  Errors
 *     detected on the host are returned immediately; errors detected on the
 *     device (a bounded wait that expired, a non-finite input to a
 *     fixed-point sweep) are recorded in the ctx and returned by
 *     stencil_ctx_status().
 *   - Thread safety: one ctx per host thread (or external locking).  Calls
 *     through the same ctx that overlap on the GPU (different streams) race
 *     on its scratch memory.
 *   - Errors: 0 on success, a negative STENCIL_ERR_* code otherwise;
 *     stencil_last_error() describes the last error of the calling thread.
 *     Nothing crosses the ABI as an exception, nothing prints or exits.
 */
#ifndef STENCIL_H_
#define STENCIL_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define STENCIL_API __attribute__((visibility("default")))
#else
#define STENCIL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define STENCIL_OK 0
#define STENCIL_ERR_ARG (-1)           /* bad argument or descriptor */
#define STENCIL_ERR_ALIGN (-2)         /* pointer or stride alignment */
#define STENCIL_ERR_DTYPE (-3)         /* unsupported dtype combination */
#define STENCIL_ERR_CUDA (-4)          /* a CUDA runtime/driver call failed */
#define STENCIL_ERR_TIMEOUT (-5)       /* a bounded device wait expired */
#define STENCIL_ERR_NONFINITE (-6)     /* NaN/Inf input where not allowed */
#define STENCIL_ERR_NOT_CONVERGED (-7) /* tolerance not reached */
#define STENCIL_ERR_RANGE (-8)         /* values beyond the fixed-point range */

typedef enum {
  STENCIL_F64 = 0,  /* IEEE binary64 */
  STENCIL_F32 = 1,  /* IEEE binary32 */
  STENCIL_BF16 = 2  /* bfloat16 storage (upper half of a binary32) */
} stencil_dtype;

typedef struct {
  void* data;             /* device pointer to halo cell (0,0,0) */
  int64_t nx, ny, nz;     /* interior extents (>= 1) */
  int64_t sy, sz;         /* element strides of y and z */
  int32_t dtype;          /* stencil_dtype */
  int32_t reserved;       /* must be 0 */
} stencil_grid;

typedef struct stencil_ctx stencil_ctx;

/* Library version string (static storage). */
STENCIL_API const char* stencil_version(void);

/* Description of the calling thread's last error (static/thread storage). */
STENCIL_API const char* stencil_last_error(void);

/*
 * Create a context bound to CUDA device `device`: allocates the scratch
 * memory the routines below use (a few KB of reduction space on the device
 * and one pinned host word).  *out
 * receives the handle.  Not to be called while a stream capture is active.
 */
STENCIL_API int stencil_ctx_create(int device, stencil_ctx** out);

/* Release a context and its scratch memory (synchronises the device). */
STENCIL_API int stencil_ctx_destroy(stencil_ctx* ctx);

/*
 * Read and clear the device-side status of ctx: synchronises `stream`, then
 * returns STENCIL_OK, STENCIL_ERR_TIMEOUT (a bounded wait inside a kernel
 * expired; the kernel stopped early and its outputs are incomplete) or
 * STENCIL_ERR_NONFINITE (a fixed-point sweep saw NaN/Inf input and wrote
 * NaN to its output interior).
 */
STENCIL_API int stencil_ctx_status(stencil_ctx* ctx, void* stream);

/* Sweep arithmetic for F64 grids (the `flags` argument below). */
#define STENCIL_SWEEP_AUTO 0         /* library's choice (FIXED for F64) */
#define STENCIL_SWEEP_FP64_NATIVE 1  /* binary64 adds/multiplies */
#define STENCIL_SWEEP_FP64_FIXED 2   /* exact 64-bit fixed-point integers */

/*
 * stencil_jacobi_sweep -- nsweeps Jacobi sweeps of the 7-point Poisson
 * relaxation (Section 4.1; Section 2.2 for the out-of-place apply):
 *     u'[i,j,k] = (u[i-1,j,k] + u[i+1,j,k] + u[i,j-1,k] + u[i,j+1,k]
 *                 + u[i,j,k-1] + u[i,j,k+1] + h*h*f[i,j,k]) / 6
 * on the interior; the halo of u is the Dirichlet boundary and is never
 * changed.  With f = 0 this is exactly the paper's Laplace average.
 *
 *   u        in/out: the iterate; the result of the last sweep ends in u.
 *            (While the call runs its interior may hold other encodings.)
 *   u_tmp    scratch grid of the same extents and dtype (its halo is
 *            overwritten with u's halo; its interior is clobbered).
 *   f        source, same extents and dtype as u.
 *   work     NULL, or an F64 scratch grid of the same extents (interior
 *            clobbered).  With it, F64 fixed-point sweeps convert u and f
 *            once per call instead of once per pass (faster for nsweeps of
 *            4 or more).  Ignored for F32/BF16 and FP64_NATIVE.
 *   h        grid spacing (the coefficient is h*h).
 *   nsweeps  >= 0 sweeps (0 is a no-op).
 *   sweeps_per_pass  sweeps fused into one pass over HBM (temporal
 *            blocking; 0 = library's choice; 1..8; the library uses the
 *            largest compiled pass length not above it).
 *   flags    STENCIL_SWEEP_* (F64 only; ignored for F32/BF16).
 *
 * dtype F64: binary64 storage.  FP64_NATIVE computes each sweep in binary64
 * (adds in the order written, h*h*f fused, then a multiply by 1/6).
 * FP64_FIXED (the default) computes in 64-bit fixed point with a scale
 * 2^-S chosen for every pass from a bound M on the values that pass can
 * produce: the largest value the previous pass wrote (max|u| for the
 * first), the Dirichlet values, plus the source's share over the pass
 * (h*h*max|f|/6 per sweep); S = 58 - ceil(log2(6M + h*h*max|f|)), so no sum
 * can overflow.  Sums are exact and each update is rounded once to the
 * nearest 2^-S: at most 2^-54 (M + h*h*max|f|/6) per update, the order of
 * one binary64 rounding of the six-neighbour sum, and since a sweep does not
 * amplify errors in the max norm, n sweeps add at most n such errors.  The
 * resolution follows the iterate, so a solution far below its initial
 * bound (zero start with an oscillating or point source) keeps the same
 * relative accuracy.  Values are rounded to binary64 once per pass (without
 * `work`) or once per call (with `work`).  FIXED needs finite inputs with
 * |values| < 2^900 (otherwise the interior is set to NaN and the ctx status
 * reports STENCIL_ERR_NONFINITE or STENCIL_ERR_RANGE).
 * dtype F32: binary32 storage and arithmetic.  dtype BF16: bfloat16
 * storage, binary32 arithmetic; each pass rounds to bfloat16 once
 * (round-to-nearest-even), intermediate sweeps of a pass stay binary32.
 */
STENCIL_API int stencil_jacobi_sweep(stencil_ctx* ctx, const stencil_grid* u,
                         const stencil_grid* u_tmp, const stencil_grid* f,
                         const stencil_grid* work, double h, int64_t nsweeps,
                         int32_t sweeps_per_pass, int32_t flags, void* stream);

/*
 * stencil_apply_linear -- a general linear stencil apply (Section 2.2: a
 * stencil.apply reads its input at constant offsets and yields one value
 * per point of the output's bounds; here the body is a linear combination):
 *   out(x, y, z) = sum_{p < npoints} coeffs[p] * in(x + dx_p, y + dy_p, z + dz_p)
 * on the output's bounds: the interior points whose reads all lie in the
 * field, halo included -- with r = max |offset|, indices r .. n + 1 - r
 * per axis (the whole interior when every offset is within one cell).
 * Nothing else of out is written.
 *   Coefficients that are all integer multiples of one power of two,
 *   coeffs[p] = k_p 2^E with |k_p| <= 2^20 (integer-weight stencils such as
 *   Laplacians, or averages with weight 1/4): computed in 64-bit fixed
 *   point, the input converted at one scale 2^-S per call (S from max|in|
 *   and sum |k_p|), sum k_p q_p exact and rounded to binary64 once, so the
 *   result is within 2^-61 sum|coeffs| max|in| of the exact sum (exactly it
 *   for inputs on the 2^-S grid, e.g. integer-valued ones).  max|in| is
 *   that of the values read (high word, rounded up): the first call on a
 *   ctx measures it with a range pass, later calls take the previous
 *   call's and check on the device that the values read give the same
 *   scale, repeating the pass when not, so the result depends on the input
 *   alone.  Any other
 *   coefficients: each product rounded, then added in the listed order
 *   (binary64, no fused multiply-add): bitwise that order's result.
 *   in, out   F64 grids of equal extents, distinct (out of place).
 *   offsets   HOST array of 3 * npoints int32 (dx, dy, dz), each in -3..3;
 *             coeffs: HOST array of npoints doubles; 1 <= npoints <= 64.
 *             Both are copied into the launch.
 * Asynchronous on `stream`; STENCIL_ERR_ARG / _DTYPE on bad arguments; a
 * non-finite input to the fixed-point form gives NaN and the ctx status
 * reports STENCIL_ERR_NONFINITE.
 */
STENCIL_API int stencil_apply_linear(stencil_ctx* ctx, const stencil_grid* in, const stencil_grid* out,
                                     const int32_t* offsets, const double* coeffs, int32_t npoints,
                                     void* stream);

/*
 * stencil_apply_expr -- the general stencil.apply (Section 2.2: an apply
 * reads its inputs at constant offsets and yields one value per point of
 * its output's bounds; its body may be any arithmetic, as in the
 * Piacsek-Williams products of Section 4.1):
 *   out(x) = expr, at every point x with r <= index <= n + 1 - r on each
 *   axis, r = max(1, largest |offset|) (as stencil_apply_linear).
 * expr is a NUL-terminated expression over the inputs:
 *   aN(dx,dy,dz)   input N (0 <= N < ninputs) at offset (dx, dy, dz),
 *                  each offset an integer in -3..3;
 *   numbers        decimal literals (e.g. 0.25, 6, 1e-3);
 *   + - * /        left-associative, * and / binding tighter; unary minus;
 *   ( )            grouping.
 * Evaluated in binary64, every operation rounded on its own (no fused
 * multiply-add) in the order the expression's tree gives, so the result is
 * bitwise that of evaluating the same expression in IEEE binary64.  The
 * library translates the expression into a CUDA C kernel, compiles it for
 * the device at run time with the CUDA run-time compiler (NVRTC, loaded on
 * first use) and keeps it in ctx: the first call with an expression
 * compiles it (tens of milliseconds), later calls reuse it.
 *   inputs   HOST array of ninputs (1..8) pointers to F64 grids of equal
 *            extents and equal strides.
 *   out      F64 grid of the same extents, distinct from every input;
 *            points outside the bounds are not written.
 * Errors: STENCIL_ERR_ARG (syntax, an offset beyond three cells, an input
 * index beyond ninputs, mismatched grids, aliasing), STENCIL_ERR_DTYPE,
 * STENCIL_ERR_CUDA (NVRTC unavailable or the compilation failed: the
 * message carries the compiler log).  Asynchronous after the first call
 * with an expression (the compilation runs on the host).
 */
STENCIL_API int stencil_apply_expr(stencil_ctx* ctx, const stencil_grid* const* inputs,
                                   int32_t ninputs, const stencil_grid* out,
                                   const char* expr, void* stream);

/*
 * stencil_expr_source -- the CUDA C source stencil_apply_expr generates for
 * expr over ninputs inputs (no device needed): written NUL-terminated into
 * buf (truncated to len - 1 characters; buf may be NULL to validate only),
 * the bounds' radius r into *radius (may be NULL).  Errors: STENCIL_ERR_ARG
 * as stencil_apply_expr.
 */
STENCIL_API int stencil_expr_source(const char* expr, int32_t ninputs, char* buf,
                                    size_t len, int32_t* radius);

/*
 * stencil_average2d -- the paper's running example (Section 2.2, Listing 1):
 * nsweeps sweeps of the four-neighbour average
 *   u'(x, y) = (u(x-1, y) + u(x+1, y) + u(x, y-1) + u(x, y+1)) * 0.25
 * over the interior of every z plane of u (a 2D grid is nz = 1; the z halo
 * planes are not read), out of place, the boundary kept.  Binary64 in the
 * order written (no fused multiply-add): bitwise the definition.
 *   u, u_tmp  F64 grids of equal extents and strides (u_tmp is scratch; its
 *             halo is overwritten with u's); the result ends in u.
 * Asynchronous on `stream`; argument errors as for stencil_jacobi_sweep.
 */
STENCIL_API int stencil_average2d(stencil_ctx* ctx, const stencil_grid* u, const stencil_grid* u_tmp,
                                  int64_t nsweeps, void* stream);

/*
 * stencil_redblack_sweep -- nsweeps red-black Gauss-Seidel sweeps of the
 * same Poisson relaxation (Section 4.1 names the benchmark Gauss-Seidel;
 * the red-black ordering keeps every half sweep data parallel).  One sweep
 * updates every interior point with i+j+k even ("red", halo indices) by
 * u = (sum of its six neighbours + h^2 f) / 6, then every point with i+j+k
 * odd ("black") by the same formula from the updated red values; the
 * result equals the in-place sweeps exactly up to rounding.  It runs
 * through the Jacobi kernel with a colour mask per stage: a pass of
 * 2 x sweeps_per_pass stages applies sweeps_per_pass red-black sweeps while
 * reading and writing each grid once (sweeps_per_pass 0 = 1; at most 2 for
 * FP32/BF16 storage, 1 for F64).  Arguments, dtypes, the work grid, flags,
 * halo handling, errors and asynchrony are those of stencil_jacobi_sweep.
 */
STENCIL_API int stencil_redblack_sweep(stencil_ctx* ctx, const stencil_grid* u,
                                       const stencil_grid* u_tmp, const stencil_grid* f,
                                       const stencil_grid* work, double h, int64_t nsweeps,
                                       int32_t sweeps_per_pass, int32_t flags, void* stream);

/*
 * stencil_autotune_sweep -- the project's autotuner for stencil_jacobi_sweep.
 * For the storage / arithmetic that (u dtype, flags, work) selects, time
 * every compiled configuration of the sweep kernel (sweeps fused per pass,
 * rows per warp, warps per CTA, shared-memory stages, CTAs per SM) on these
 * grids, keep the fastest per pass length in ctx, and make the pass length
 * with the fastest time per sweep the ctx's default (sweeps_per_pass = 0).
 * Arguments as for stencil_jacobi_sweep; trial passes read u and write
 * u_tmp's interior only (u is not changed).  report (nullable): a text line
 * per configuration timed.  Synchronous; not to be called during a stream
 * capture.  No counterpart in the paper (its tile sizes were fixed by hand).
 */
STENCIL_API int stencil_autotune_sweep(stencil_ctx* ctx, const stencil_grid* u,
                                       const stencil_grid* u_tmp,
                                       const stencil_grid* f,
                                       const stencil_grid* work, double h,
                                       int32_t flags, char* report,
                                       size_t report_len, void* stream);

/*
 * Inspect or pin the sweep configuration (for reproducible runs and tests).
 * (dtype, flags, with_work) select the storage / arithmetic exactly as in
 * stencil_jacobi_sweep (with_work != 0: a work grid is passed; F64 fixed
 * point with a work grid and 4 or more sweeps keeps the iterate resident).
 * stencil_sweep_config_count writes the number of compiled configurations
 * for pass length T (0 if none); stencil_sweep_config_select makes
 * configuration `index` the one ctx uses for that pass length.
 */
STENCIL_API int stencil_sweep_config_count(int32_t dtype, int32_t flags,
                                           int32_t with_work, int32_t T,
                                           int32_t* count);
STENCIL_API int stencil_sweep_config_select(stencil_ctx* ctx, int32_t dtype,
                                            int32_t flags, int32_t with_work,
                                            int32_t T, int32_t index);

/*
 * The same for stencil_redblack_sweep: the compiled red-black tile
 * configurations for `sweeps_per_pass` sweeps per pass (1 or 2), and the
 * one ctx uses (index 0, the fastest measured at 512^3, unless selected).
 * Errors: STENCIL_ERR_ARG (null count or ctx, index out of range),
 * STENCIL_ERR_DTYPE.
 */
STENCIL_API int stencil_redblack_config_count(int32_t dtype, int32_t flags,
                                              int32_t with_work,
                                              int32_t sweeps_per_pass,
                                              int32_t* count);
STENCIL_API int stencil_redblack_config_select(stencil_ctx* ctx, int32_t dtype,
                                               int32_t flags, int32_t with_work,
                                               int32_t sweeps_per_pass,
                                               int32_t index);

/*
 * The same for stencil_residual's fixed-point evaluation: the number of
 * compiled tile configurations, and the one ctx uses (index 0 unless
 * selected).  Errors: STENCIL_ERR_ARG (null count or ctx, index out of
 * range).
 */
STENCIL_API int stencil_residual_config_count(int32_t* count);
STENCIL_API int stencil_residual_config_select(stencil_ctx* ctx, int32_t index);

/*
 * The same for stencil_advect_uvw's fixed-point kernel (its thread-block
 * shape, CTAs per SM and z chunk length): the number of compiled
 * configurations, and the
 * one ctx uses (index 0 unless selected).  Errors: STENCIL_ERR_ARG (null
 * count or ctx, index out of range).
 */
STENCIL_API int stencil_advect_config_count(int32_t* count);
STENCIL_API int stencil_advect_config_select(stencil_ctx* ctx, int32_t index);

/*
 * stencil_residual -- the residual of A u = f for the 7-point operator
 *     (A u)[i,j,k] = (6 u[i,j,k] - sum of the six neighbours) / h^2,
 *     r = f - A u on the interior,
 * to binary64 accuracy or better (it decides convergence of the iterative
 * solve).  Grids whose data and row strides are 16-byte aligned (what a TMA
 * descriptor needs) are evaluated in 64-bit fixed point: u and h^2 f at one
 * scale 2^-S per call with 12 max|u| + h^2 max|f| < 2^(62-S) (the maxima of
 * the values read, rounded up to their high words), so 6u minus
 * the six neighbours is exact and each r is within 6.5 2^-S / h^2 of the
 * exact f - A u (finer than a binary64 evaluation of the same expression,
 * whose rounding is up to about 16 eps (12 max|u| / h^2 + max|f|)); r is
 * rounded to binary64 once it is formed.  ||r||^2 is summed exactly (192-bit
 * integers), so the norm does not depend on the summation order.  Other
 * grids take a binary64 evaluation in the written order (bitwise the plain
 * definition).  Non-finite input: norms and r are NaN and the ctx status
 * reports STENCIL_ERR_NONFINITE.  The first call on a ctx reads u and f
 * twice (a range pass fixes S); later calls take the previous call's
 * magnitudes as the scale, check on the device that the values read give
 * the same scale, and repeat the pass at the right scale when they do not,
 * so the result depends on the input alone and a call whose magnitudes keep
 * the scale reads u and f once.
 *   u, f      F64 grids of equal extents (u's halo is the boundary).
 *   r         NULL, or an F64 grid of the same extents, distinct from u and
 *             f (STENCIL_ERR_ARG if it is either): its interior receives r
 *             (halo untouched).
 *   norms_dev DEVICE pointer to 2 doubles: ||r||_2 and ||f||_2 over the
 *             interior (unweighted).  The sum order is fixed (per-block
 *             partial sums combined in block order), so the result is
 *             bitwise reproducible run to run.
 * Uses ctx scratch memory.
 */
STENCIL_API int stencil_residual(stencil_ctx* ctx, const stencil_grid* u,
                     const stencil_grid* f, double h, const stencil_grid* r,
                     double* norms_dev, void* stream);

/* One Poisson instance of a batch. */
typedef struct {
  stencil_grid u;   /* F64 iterate: start on entry, solution on return (halo = Dirichlet values) */
  stencil_grid f;   /* F64 source, same extents */
  double h;         /* grid spacing */
} stencil_problem;

/* Options of stencil_batch_solve (zero-initialise, then set rtol etc.). */
typedef struct {
  double rtol;               /* target ||f - A u||_2 / ||f||_2, e.g. 1e-8 */
  int64_t max_sweeps;        /* inner sweeps per instance before giving up (0 = 10^7) */
  int32_t inner_dtype;       /* STENCIL_F32 or STENCIL_BF16 storage of the correction */
  int32_t sweeps_per_cycle;  /* inner sweeps per refinement cycle (0 = 100) */
  int32_t sweeps_per_pass;   /* sweeps fused per pass of the inner solve (0 = autotuned) */
  int32_t smoother;          /* inner sweeps: 0 = Jacobi, 1 = red-black Gauss-Seidel
                                (stencil_redblack_sweep's, one sweep per pass) */
  double stall_ratio;        /* a cycle with rel > stall_ratio * previous rel escalates
                                BF16 -> F32 storage (0 = 0.9999); F32 stalls end the
                                instance with STENCIL_ERR_NOT_CONVERGED */
} stencil_batch_opts;

/* Per-instance outcome of stencil_batch_solve. */
typedef struct {
  int64_t sweeps;            /* inner sweeps done */
  int32_t cycles;            /* refinement cycles (corrections applied) */
  int32_t status;            /* STENCIL_OK, STENCIL_ERR_NOT_CONVERGED, STENCIL_ERR_NONFINITE */
  double rel_residual;       /* final ||f - A u||_2 / ||f||_2, binary64 */
  int32_t final_dtype;       /* inner storage used by the last cycle */
  int32_t reserved;
} stencil_result;

/*
 * stencil_batch_workspace_size -- device workspace bytes stencil_batch_solve
 * needs for these n problems (written to *bytes).  Host-only, no GPU work.
 */
STENCIL_API int stencil_batch_workspace_size(const stencil_problem* probs, int32_t n,
                                             size_t* bytes);

/*
 * stencil_batch_solve -- solve n independent Poisson problems A u = f (the
 * 7-point operator of stencil_residual, Dirichlet halos) to a relative
 * residual rtol by mixed-precision iterative refinement: each cycle computes
 * r = f - A u and its norm in binary64 (bitwise the stencil_residual values),
 * stops an instance when ||r||/||f|| <= rtol, otherwise rounds r to the inner
 * storage type (round-to-nearest-even), runs sweeps_per_cycle Jacobi (or,
 * with opts.smoother = 1, red-black Gauss-Seidel) sweeps of A e = r from
 * e = 0 with binary32 arithmetic, and adds e to u in binary64.
 * All active instances advance together: every pass of the inner solve is
 * one persistent launch over the tiles of all of them, and one cycle is one
 * CUDA graph (residual, check, cast, passes, update) that is replayed until
 * every instance has finished; the host reads one counter per cycle.
 *
 *   probs      host array of n problem descriptors (device grids; u's must
 *              satisfy the alignment rules of stencil_grid).
 *   opts       see stencil_batch_opts.
 *   workspace  device memory of at least stencil_batch_workspace_size bytes,
 *              256-byte aligned; owned by the caller, clobbered.
 *   results    host array of n results.
 * Synchronous: starts after the work already queued on `stream` and returns
 * when every instance has finished (converged, hit max_sweeps, stalled in
 * F32, or met a non-finite residual); the work itself runs on the context's
 * own stream.  Instances' outcomes are in results[i].status; the return
 * value reports only argument and CUDA errors.  Not to be called during a
 * stream capture.
 */
STENCIL_API int stencil_batch_solve(stencil_ctx* ctx, const stencil_problem* probs, int32_t n,
                                    const stencil_batch_opts* opts, void* workspace,
                                    size_t workspace_bytes, stencil_result* results,
                                    void* stream);

/*
 * Learned warm start (wsnet_*).  A small 3D U-Net maps the source f of a
 * Poisson problem on an n^3 grid to a starting iterate u0 for the Jacobi
 * solve; the solve (plain Jacobi or stencil_batch_solve) then removes the
 * remaining error, and its residual decides the result.  The paper has no
 * learned component: this is the warm-start pattern layered on the solver.
 * Architecture (levels L <= 4 with per-level channels in {16, 32, 64}): two
 * 3x3x3 convolutions with ReLU per level, 2x2x2 average pooling between
 * encoder levels, nearest 2x upsampling between decoder levels whose first
 * convolution adds the encoder feature of the same level before its ReLU,
 * a 1x1x1 output layer and a fixed separable [1,2,1]/4 smoothing filter
 * (it all but removes the checkerboard mode, which Jacobi damps as slowly as
 * the smoothest mode).  Input f / rms(f) over the interior; output
 * u0 = y * rms(f) / (3 pi^2) on the interior (the halo of u is untouched).
 * Activations and gradients are bfloat16, products accumulate in binary32 on
 * the tensor cores; parameters are binary32 (Adam).  Parameter vector layout
 * (wsnet_get_params): per 3x3x3 layer, in forward order (encoder levels
 * 0..L-1 with layers a, b; decoder levels L-2..0 with layers a, b), weights
 * W[co][tap*cin + ci] (tap = 9 dz + 3 dy + dx over offsets -1..1) then
 * biases b[co]; then the output layer's C0 weights and its bias.
 * A net owns its device memory (parameters and the activations of one n^3
 * sample); one net per host thread.
 */
typedef struct wsnet wsnet;

/* Create a net for n^3 grids (n a multiple of 2^(levels-1)); He-normal
 * weights from `seed` (deterministic), zero biases.  Allocates. */
STENCIL_API int wsnet_create(int device, int32_t levels, const int32_t* channels,
                             int32_t n, uint64_t seed, wsnet** out);
/* Free the net and its device memory (synchronises the device). */
STENCIL_API int wsnet_destroy(wsnet* net);
/* Number of binary32 parameters. */
STENCIL_API int wsnet_num_params(const wsnet* net, int64_t* count);
/* Copy the parameters to / from a host array of wsnet_num_params floats. */
STENCIL_API int wsnet_get_params(wsnet* net, float* host, int64_t count);
STENCIL_API int wsnet_set_params(wsnet* net, const float* host, int64_t count);
/* u0 on the interior of u (F64 n^3 grid) from the source f (F64 n^3 grid),
 * enqueued on `stream`. */
STENCIL_API int wsnet_infer(wsnet* net, const stencil_grid* f,
                            const stencil_grid* u, void* stream);
/* One Adam step (lr; betas 0.9, 0.999; eps 1e-8) on the mean squared error
 * between the normalised output and the normalised targets u[s] over
 * `count` samples (host arrays of F64 n^3 grids f[s], u[s]); *loss receives
 * the mean loss.  Synchronises `stream`. */
STENCIL_API int wsnet_train_step(wsnet* net, const stencil_grid* f,
                                 const stencil_grid* u, int32_t count,
                                 float lr, double* loss, void* stream);
/* Save a training checkpoint: the net's configuration, FP32 parameters and
 * Adam state (8-byte magic "WSNET02", int32 levels, int32
 * channels[levels], int32 n, int64 parameter count, the parameters in
 * wsnet_get_params order, int64 Adam step count, the first and second
 * moments in the same order; little endian).  Load one into a net created
 * with the same levels, channels and n: training then continues exactly as
 * if it had not stopped.  Files with the magic "WSNET01" (parameters only,
 * no optimiser state) load too, with the optimiser restarted.
 * STENCIL_ERR_ARG on a mismatch or an unreadable file (the net is then
 * unchanged).  Synchronous. */
STENCIL_API int wsnet_save(wsnet* net, const char* path);
STENCIL_API int wsnet_load(wsnet* net, const char* path);
/* 1 (the default): the 3x3x3 convolutions with at least 16 input and output
 * channels on grids whose rows of 16 to 128 voxels divide 128 run on the
 * tcgen05 tensor cores (accumulators in tensor memory); 0: every
 * convolution uses the warp-level mma.sync kernel.  Both paths sum the
 * bf16 products in binary32 in the same order (taps, then 16-channel
 * chunks). */
STENCIL_API int wsnet_use_tcgen05(wsnet* net, int32_t enable);
/* Read and clear the net's device status: STENCIL_ERR_TIMEOUT if a bounded
 * wait inside a kernel expired (synchronises `stream`). */
STENCIL_API int wsnet_status(wsnet* net, void* stream);
/* One forward and backward pass on a given normalised input x and target t
 * (DEVICE binary32 arrays of n^3 values, z slowest, x fastest); y (device,
 * nullable) receives the output, grads (host, nullable) the gradients, in
 * the parameter layout.  For checking the kernels against a reference. */
STENCIL_API int wsnet_loss_grad(wsnet* net, const float* x, const float* t,
                                float* y, float* grads, double* loss,
                                void* stream);

/*
 * stencil_residual_noalloc -- the same residual and norms as
 * stencil_residual, for callers that cannot allocate device memory: code
 * running where allocation is forbidden or unavailable (a host application
 * that owns all device memory through its own allocator, a no-allocation
 * real-time loop), and that therefore cannot create a stencil_ctx either.  This call allocates nothing and takes
 * no context: its partial sums live in a fixed array built into the
 * library (128 KiB per device that loads the library, held until the
 * process exits).  The paper has no counterpart; it is a deployment
 * convenience.
 *   u, f, h, r, norms_dev   as for stencil_residual; the grids must be on
 *            the current CUDA device, and the call runs on `stream`.
 *   Limit:   ny * nz <= 524288 (one partial sum per 64 rows, 8192 sums);
 *            larger grids are rejected with STENCIL_ERR_ARG before any
 *            launch (use stencil_residual with a context for them).
 *   r is evaluated in binary64 in the written order (bitwise the plain
 *   definition), so it agrees with stencil_residual's to both evaluations'
 *   rounding; the norms use a fixed partition of the sum and are
 *   reproducible run to run.
 *   The first call in each CUDA context on a device looks up the array's
 *   device address (with that device current; again after the context is
 *   replaced, e.g. by cudaDeviceReset); make that first call before any
 *   stream capture on the device.  Every call on a device shares
 *   the one array: calls that overlap on the GPU (different streams, or
 *   threads without ordering) race and give wrong norms.  Each call
 *   overwrites every partial sum it reads, so nothing has to be cleared
 *   between calls.
 */
STENCIL_API int stencil_residual_noalloc(const stencil_grid* u,
                                         const stencil_grid* f, double h,
                                         const stencil_grid* r,
                                         double* norms_dev, void* stream);

/*
 * stencil_advect_uvw -- Piacsek-Williams flux-form momentum advection
 * (Section 4.1: three stencils over u, v, w fused into one region, 63
 * floating-point operations per cell).  Centred second order on a C grid
 * (u on x faces, v on y faces, w on z faces); for interior (i,j,k) and
 * c1 = tzc1[k-1], c2 = tzc2[k-1]:
 *   su = tcx*(u[i-1]*(u+u[i-1]) - u[i+1]*(u+u[i+1]))
 *      + tcy*(u[j-1]*(v[j-1]+v[i+1,j-1]) - u[j+1]*(v+v[i+1]))
 *      + c1*u[k-1]*(w[k-1]+w[i+1,k-1]) - c2*u[k+1]*(w+w[i+1])
 *   sv = tcx*(v[i-1]*(u[i-1]+u[i-1,j+1]) - v[i+1]*(u+u[j+1]))
 *      + tcy*(v[j-1]*(v+v[j-1]) - v[j+1]*(v+v[j+1]))
 *      + c1*v[k-1]*(w[k-1]+w[j+1,k-1]) - c2*v[k+1]*(w+w[j+1])
 *   sw = tcx*(w[i-1]*(u[i-1]+u[i-1,k+1]) - w[i+1]*(u+u[k+1]))
 *      + tcy*(w[j-1]*(v[j-1]+v[j-1,k+1]) - w[j+1]*(v+v[k+1]))
 *      + c1*w[k-1]*(w+w[k-1]) - c2*w[k+1]*(w+w[k+1])
 * (unnamed offsets are 0).  All six grids F64 with equal extents; inputs'
 * halos are filled by the caller; outputs are written on the interior only.
 * tzc1, tzc2: DEVICE arrays of nz doubles.
 * Arithmetic: 64-bit integer fixed point with one scale for u, v, w (from
 * their largest magnitude, halos included) and one for the factors; every
 * sum of two or three values is exact, every product is within 9/4 units
 * of 2^-64 of its exact value (three 32 x 32-bit partial products), and
 * each tendency is rounded to binary64 once: the error is at most about
 * 2^-50 max|u,v,w|^2 max|factor|, the order of a binary64 evaluation's
 * rounding error, and equal fluxes cancel exactly.  If the three fields' (or
 * the factors') largest magnitudes differ by more than 2^8, or an input is
 * not finite, the launch evaluates the formula in binary64 instead (NaN and
 * Inf propagate as in binary64).  The scales follow from the magnitudes the
 * pass reads: the first call on a ctx measures them with a range pass;
 * later calls take the previous call's magnitudes and check on the device
 * that the values read lead to the same scales, repeating the pass when
 * they do not, so the result depends on the input alone.  Uses the
 * context's scratch; asynchronous.
 */
STENCIL_API int stencil_advect_uvw(stencil_ctx* ctx, const stencil_grid* u,
                       const stencil_grid* v, const stencil_grid* w,
                       const stencil_grid* su, const stencil_grid* sv,
                       const stencil_grid* sw, const double* tzc1,
                       const double* tzc2, double tcx, double tcy,
                       void* stream);

#ifdef __cplusplus
}
#endif

#endif /* STENCIL_H_ */
