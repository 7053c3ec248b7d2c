/*
 * oracle.c -- plain CPU oracle for the stencil hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file's library.  The product
 * (the CUDA library under paper_2310_01882_b300/csrc) shares no code,
 * header, helper or constant with it, and never calls it.
 *
 * Every routine is the plain definition, written as loops in the order the
 * formula is stated, in FP64 unless the routine's name says otherwise.  It is
 * compiled with -O2 -ffp-contract=off so that no multiply-add is fused: the
 * left-to-right evaluation order is kept, as the paper's extraction keeps the
 * source order of operations (Section 3: no_reassoc operations are carried
 * into the stencil region unchanged).
 *
 * Layout (Section 2.2, first index fastest as in Fortran): a field with
 * interior extents nx, ny, nz and a one-cell halo is a dense array of
 * (nx+2)*(ny+2)*(nz+2) values, x fastest, then y, then z.  Interior indices
 * run 1..n in each axis; index 0 and n+1 are the halo.
 *
 * Pins: each routine is checked in tests/test_oracle_*.py against closed
 * forms, invariants and brute force (see the docstrings there).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define AT(a, i, j, k) (a)[((size_t)(k) * (size_t)(ny + 2) + (size_t)(j)) * (size_t)(nx + 2) + (size_t)(i)]

static size_t field_len(int64_t nx, int64_t ny, int64_t nz) {
  return (size_t)(nx + 2) * (size_t)(ny + 2) * (size_t)(nz + 2);
}

int oracle_num_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) return nthreads;
  return omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

/*
 * One relaxation sweep of the 3D 7-point stencil (Section 4.1: each cell
 * becomes the average of its six orthogonal neighbours), in the Poisson form
 * with a source term:
 *     out[i,j,k] = (u[i-1]+u[i+1]+u[j-1]+u[j+1]+u[k-1]+u[k+1] + h*h*f) / 6
 * on the interior.  The update is out of place (Section 2.2: a stencil apply
 * reads its input field and yields a new one), i.e. a Jacobi sweep.  With
 * f = 0 it is exactly the paper's Laplace average.  The halo of `out` is
 * copied from `u` (the Dirichlet values).
 */
void oracle_jacobi_sweep_f64(const double* u, double* out, const double* f,
                             int64_t nx, int64_t ny, int64_t nz, double h,
                             int nthreads) {
  const double hh = h * h;
  memcpy(out, u, field_len(nx, ny, nz) * sizeof(double));
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(oracle_num_threads(nthreads))
#endif
  for (int64_t k = 1; k <= nz; ++k)
    for (int64_t j = 1; j <= ny; ++j)
      for (int64_t i = 1; i <= nx; ++i) {
        double s = AT(u, i - 1, j, k) + AT(u, i + 1, j, k);
        s += AT(u, i, j - 1, k);
        s += AT(u, i, j + 1, k);
        s += AT(u, i, j, k - 1);
        s += AT(u, i, j, k + 1);
        s += hh * AT(f, i, j, k);
        AT(out, i, j, k) = s / 6.0;
      }
#ifndef _OPENMP
  (void)nthreads;
#endif
}

/* nsweeps Jacobi sweeps; result in u, tmp is scratch of the same size. */
void oracle_jacobi_f64(double* u, double* tmp, const double* f, int64_t nx,
                       int64_t ny, int64_t nz, double h, int64_t nsweeps,
                       int nthreads) {
  double* a = u;
  double* b = tmp;
  for (int64_t s = 0; s < nsweeps; ++s) {
    oracle_jacobi_sweep_f64(a, b, f, nx, ny, nz, h, nthreads);
    double* t = a; a = b; b = t;
  }
  if (a != u) memcpy(u, a, field_len(nx, ny, nz) * sizeof(double));
}

/*
 * The same sweep with FP32 storage and FP32 arithmetic, in the same order.
 * hh is the FP32 coefficient h*h (the caller rounds it once).  Used by the
 * mixed-precision refinement oracle for its inner sweeps.
 */
void oracle_jacobi_sweep_f32(const float* u, float* out, const float* f,
                             int64_t nx, int64_t ny, int64_t nz, float hh) {
  memcpy(out, u, field_len(nx, ny, nz) * sizeof(float));
  for (int64_t k = 1; k <= nz; ++k)
    for (int64_t j = 1; j <= ny; ++j)
      for (int64_t i = 1; i <= nx; ++i) {
        float s = AT(u, i - 1, j, k) + AT(u, i + 1, j, k);
        s += AT(u, i, j - 1, k);
        s += AT(u, i, j + 1, k);
        s += AT(u, i, j, k - 1);
        s += AT(u, i, j, k + 1);
        s += hh * AT(f, i, j, k);
        AT(out, i, j, k) = s / 6.0f;
      }
}

/*
 * BF16 storage: a bfloat16 is the upper 16 bits of an IEEE binary32.
 * Rounding float -> bf16 is round-to-nearest-even on the discarded 16 bits;
 * NaN stays NaN.
 */
static float bf16_to_float(uint16_t b) {
  uint32_t x = (uint32_t)b << 16;
  float r;
  memcpy(&r, &x, 4);
  return r;
}

static uint16_t float_to_bf16(float v) {
  uint32_t x;
  memcpy(&x, &v, 4);
  if ((x & 0x7f800000u) == 0x7f800000u && (x & 0x007fffffu) != 0)
    return (uint16_t)((x >> 16) | 0x0040u);
  uint32_t lsb = (x >> 16) & 1u;
  x += 0x7fffu + lsb;
  return (uint16_t)(x >> 16);
}

void oracle_f32_to_bf16(const float* in, uint16_t* out, int64_t n) {
  for (int64_t i = 0; i < n; ++i) out[i] = float_to_bf16(in[i]);
}

void oracle_bf16_to_f32(const uint16_t* in, float* out, int64_t n) {
  for (int64_t i = 0; i < n; ++i) out[i] = bf16_to_float(in[i]);
}

/* Sweep with BF16 storage of u, out and f; FP32 arithmetic as above. */
void oracle_jacobi_sweep_bf16(const uint16_t* u, uint16_t* out,
                              const uint16_t* f, int64_t nx, int64_t ny,
                              int64_t nz, float hh) {
  memcpy(out, u, field_len(nx, ny, nz) * sizeof(uint16_t));
  for (int64_t k = 1; k <= nz; ++k)
    for (int64_t j = 1; j <= ny; ++j)
      for (int64_t i = 1; i <= nx; ++i) {
        float s = bf16_to_float(AT(u, i - 1, j, k)) + bf16_to_float(AT(u, i + 1, j, k));
        s += bf16_to_float(AT(u, i, j - 1, k));
        s += bf16_to_float(AT(u, i, j + 1, k));
        s += bf16_to_float(AT(u, i, j, k - 1));
        s += bf16_to_float(AT(u, i, j, k + 1));
        s += hh * bf16_to_float(AT(f, i, j, k));
        AT(out, i, j, k) = float_to_bf16(s / 6.0f);
      }
}

/*
 * The paper's running example (Section 2.2, Listing 1): each interior point
 * of a 2D grid becomes the average of its four neighbours,
 *   out(x, y) = (u(x-1, y) + u(x+1, y) + u(x, y-1) + u(x, y+1)) * 0.25,
 * out of place (a stencil apply), the boundary kept.  A 3D field is taken as
 * a stack of independent 2D planes (k = 1..nz; its z halo planes are not
 * read).  nsweeps sweeps; the result is left in u, tmp is scratch.
 */
void oracle_average2d(double* u, double* tmp, int64_t nx, int64_t ny, int64_t nz, int64_t nsweeps) {
  double* a = u;
  double* b = tmp;
  memcpy(b, a, field_len(nx, ny, nz) * sizeof(double));
  for (int64_t sw = 0; sw < nsweeps; ++sw) {
    for (int64_t k = 1; k <= nz; ++k)
      for (int64_t j = 1; j <= ny; ++j)
        for (int64_t i = 1; i <= nx; ++i) {
          double s = AT(a, i - 1, j, k) + AT(a, i + 1, j, k);
          s += AT(a, i, j - 1, k);
          s += AT(a, i, j + 1, k);
          AT(b, i, j, k) = s * 0.25;
        }
    double* t = a; a = b; b = t;
  }
  if (a != u) memcpy(u, a, field_len(nx, ny, nz) * sizeof(double));
}

/*
 * A general linear stencil apply (Section 2.2: a stencil.apply reads an
 * input field at constant offsets and writes one output value per point of
 * its bounds; here the body is a linear combination):
 *   out(x, y, z) = sum_p c_p * in(x + dx_p, y + dy_p, z + dz_p)
 * terms added in the listed order (each product rounded, then added).  The
 * output bounds are the interior points whose every read lies in the field
 * (halo included): with r = max |d| over the offsets, indices r .. n + 1 - r
 * per axis -- the whole interior for offsets within the one-cell halo.
 * Nothing else of out is written.  offsets: 3 * npoints ints (dx, dy, dz).
 */
void oracle_apply_linear(const double* in, double* out, int64_t nx, int64_t ny, int64_t nz,
                         const int* offsets, const double* coeffs, int npoints) {
  int64_t r = 1;
  for (int p = 0; p < 3 * npoints; ++p) {
    const int64_t a = offsets[p] < 0 ? -offsets[p] : offsets[p];
    if (a > r) r = a;
  }
  for (int64_t k = r; k <= nz + 1 - r; ++k)
    for (int64_t j = r; j <= ny + 1 - r; ++j)
      for (int64_t i = r; i <= nx + 1 - r; ++i) {
        double acc = 0.0;
        for (int p = 0; p < npoints; ++p) {
          const double term = coeffs[p] * AT(in, i + offsets[3 * p], j + offsets[3 * p + 1], k + offsets[3 * p + 2]);
          acc = acc + term;
        }
        AT(out, i, j, k) = acc;
      }
}

/*
 * Red-black Gauss-Seidel.  Section 4.1 names the relaxation benchmark
 * Gauss-Seidel; with the red-black ordering every half sweep stays data
 * parallel.  One sweep updates, in place, first every interior point with
 * i + j + k even ("red") from its six neighbours, then every interior point
 * with i + j + k odd ("black") from its neighbours, which are all red and
 * already updated.  Each update is the Jacobi formula above (same operation
 * order).  A point's neighbours have the other colour, so the order of the
 * updates within one colour does not matter.
 */
void oracle_rbgs_f64(double* u, const double* f, int64_t nx, int64_t ny,
                     int64_t nz, double h, int64_t nsweeps, int nthreads) {
  const double hh = h * h;
  for (int64_t sw = 0; sw < nsweeps; ++sw)
    for (int color = 0; color < 2; ++color) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(oracle_num_threads(nthreads))
#endif
      for (int64_t k = 1; k <= nz; ++k)
        for (int64_t j = 1; j <= ny; ++j)
          for (int64_t i = 1; i <= nx; ++i) {
            if (((i + j + k) & 1) != color) continue;
            double s = AT(u, i - 1, j, k) + AT(u, i + 1, j, k);
            s += AT(u, i, j - 1, k);
            s += AT(u, i, j + 1, k);
            s += AT(u, i, j, k - 1);
            s += AT(u, i, j, k + 1);
            s += hh * AT(f, i, j, k);
            AT(u, i, j, k) = s / 6.0;
          }
    }
#ifndef _OPENMP
  (void)nthreads;
#endif
}

/* The same with FP32 storage and arithmetic (hh the FP32 coefficient). */
void oracle_rbgs_f32(float* u, const float* f, int64_t nx, int64_t ny,
                     int64_t nz, float hh, int64_t nsweeps) {
  for (int64_t sw = 0; sw < nsweeps; ++sw)
    for (int color = 0; color < 2; ++color)
      for (int64_t k = 1; k <= nz; ++k)
        for (int64_t j = 1; j <= ny; ++j)
          for (int64_t i = 1; i <= nx; ++i) {
            if (((i + j + k) & 1) != color) continue;
            float s = AT(u, i - 1, j, k) + AT(u, i + 1, j, k);
            s += AT(u, i, j - 1, k);
            s += AT(u, i, j + 1, k);
            s += AT(u, i, j, k - 1);
            s += AT(u, i, j, k + 1);
            s += hh * AT(f, i, j, k);
            AT(u, i, j, k) = s / 6.0f;
          }
}

/* The same with bf16 storage of u and f, FP32 arithmetic. */
void oracle_rbgs_bf16(uint16_t* u, const uint16_t* f, int64_t nx, int64_t ny,
                      int64_t nz, float hh, int64_t nsweeps) {
  for (int64_t sw = 0; sw < nsweeps; ++sw)
    for (int color = 0; color < 2; ++color)
      for (int64_t k = 1; k <= nz; ++k)
        for (int64_t j = 1; j <= ny; ++j)
          for (int64_t i = 1; i <= nx; ++i) {
            if (((i + j + k) & 1) != color) continue;
            float s = bf16_to_float(AT(u, i - 1, j, k)) + bf16_to_float(AT(u, i + 1, j, k));
            s += bf16_to_float(AT(u, i, j - 1, k));
            s += bf16_to_float(AT(u, i, j + 1, k));
            s += bf16_to_float(AT(u, i, j, k - 1));
            s += bf16_to_float(AT(u, i, j, k + 1));
            s += hh * bf16_to_float(AT(f, i, j, k));
            AT(u, i, j, k) = float_to_bf16(s / 6.0f);
          }
}

/*
 * Residual of the Poisson problem A u = f with the 7-point operator
 *     (A u)[i,j,k] = (6 u[i,j,k] - sum of the six neighbours) / h^2
 *     r = f - A u
 * on the interior, in FP64.  norms[0] = ||r||_2, norms[1] = ||f||_2, both
 * unweighted sums over interior points.  If r is not NULL its interior is
 * written (halo untouched).
 */
void oracle_residual_f64(const double* u, const double* f, int64_t nx,
                         int64_t ny, int64_t nz, double h, double* r,
                         double* norms, int nthreads) {
  const double hh = h * h;
  double rr = 0.0, ff = 0.0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(+ : rr, ff) num_threads(oracle_num_threads(nthreads))
#endif
  for (int64_t k = 1; k <= nz; ++k)
    for (int64_t j = 1; j <= ny; ++j)
      for (int64_t i = 1; i <= nx; ++i) {
        double s = AT(u, i - 1, j, k) + AT(u, i + 1, j, k);
        s += AT(u, i, j - 1, k);
        s += AT(u, i, j + 1, k);
        s += AT(u, i, j, k - 1);
        s += AT(u, i, j, k + 1);
        double au = (6.0 * AT(u, i, j, k) - s) / hh;
        double res = AT(f, i, j, k) - au;
        if (r) AT(r, i, j, k) = res;
        rr += res * res;
        ff += AT(f, i, j, k) * AT(f, i, j, k);
      }
  norms[0] = sqrt(rr);
  norms[1] = sqrt(ff);
#ifndef _OPENMP
  (void)nthreads;
#endif
}

/*
 * Piacsek-Williams flux-form momentum advection (Section 4.1: three stencils
 * over the fields u, v, w fused into one region, 63 floating-point operations
 * per cell).  Centred second order on an Arakawa C grid: u lives on x faces,
 * v on y faces, w on z faces.  For each velocity component the tendency is
 * the divergence of "advected component times the advecting velocity
 * interpolated to the flux point", with the 1/2 factors and 1/dx folded into
 * tcx, tcy and the vertical factors tzc1[k], tzc2[k] (k = 1..nz maps to
 * tzc[k-1]).  Each component costs 21 operations: 6 (x) + 6 (y) + 7 (z) + 2
 * to combine, 63 in total.  Products are evaluated left to right as written.
 * Outputs are written on the interior only; inputs' halos are the caller's.
 */
void oracle_advect_uvw(const double* u, const double* v, const double* w,
                       double* su, double* sv, double* sw, const double* tzc1,
                       const double* tzc2, double tcx, double tcy, int64_t nx,
                       int64_t ny, int64_t nz, int nthreads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(oracle_num_threads(nthreads))
#endif
  for (int64_t k = 1; k <= nz; ++k) {
    const double c1 = tzc1[k - 1], c2 = tzc2[k - 1];
    for (int64_t j = 1; j <= ny; ++j)
      for (int64_t i = 1; i <= nx; ++i) {
        double tx, ty, tz;
        /* u component, at (i+1/2, j, k) */
        tx = tcx * (AT(u, i - 1, j, k) * (AT(u, i, j, k) + AT(u, i - 1, j, k)) -
                    AT(u, i + 1, j, k) * (AT(u, i, j, k) + AT(u, i + 1, j, k)));
        ty = tcy * (AT(u, i, j - 1, k) * (AT(v, i, j - 1, k) + AT(v, i + 1, j - 1, k)) -
                    AT(u, i, j + 1, k) * (AT(v, i, j, k) + AT(v, i + 1, j, k)));
        tz = c1 * AT(u, i, j, k - 1) * (AT(w, i, j, k - 1) + AT(w, i + 1, j, k - 1)) -
             c2 * AT(u, i, j, k + 1) * (AT(w, i, j, k) + AT(w, i + 1, j, k));
        AT(su, i, j, k) = tx + ty + tz;
        /* v component, at (i, j+1/2, k) */
        tx = tcx * (AT(v, i - 1, j, k) * (AT(u, i - 1, j, k) + AT(u, i - 1, j + 1, k)) -
                    AT(v, i + 1, j, k) * (AT(u, i, j, k) + AT(u, i, j + 1, k)));
        ty = tcy * (AT(v, i, j - 1, k) * (AT(v, i, j, k) + AT(v, i, j - 1, k)) -
                    AT(v, i, j + 1, k) * (AT(v, i, j, k) + AT(v, i, j + 1, k)));
        tz = c1 * AT(v, i, j, k - 1) * (AT(w, i, j, k - 1) + AT(w, i, j + 1, k - 1)) -
             c2 * AT(v, i, j, k + 1) * (AT(w, i, j, k) + AT(w, i, j + 1, k));
        AT(sv, i, j, k) = tx + ty + tz;
        /* w component, at (i, j, k+1/2) */
        tx = tcx * (AT(w, i - 1, j, k) * (AT(u, i - 1, j, k) + AT(u, i - 1, j, k + 1)) -
                    AT(w, i + 1, j, k) * (AT(u, i, j, k) + AT(u, i, j, k + 1)));
        ty = tcy * (AT(w, i, j - 1, k) * (AT(v, i, j - 1, k) + AT(v, i, j - 1, k + 1)) -
                    AT(w, i, j + 1, k) * (AT(v, i, j, k) + AT(v, i, j, k + 1)));
        tz = c1 * AT(w, i, j, k - 1) * (AT(w, i, j, k) + AT(w, i, j, k - 1)) -
             c2 * AT(w, i, j, k + 1) * (AT(w, i, j, k) + AT(w, i, j, k + 1));
        AT(sw, i, j, k) = tx + ty + tz;
      }
  }
#ifndef _OPENMP
  (void)nthreads;
#endif
}

/*
 * Mixed-precision iterative refinement of A u = f (the FP32/BF16 storage
 * pattern; the paper itself iterates in FP64 only).  Cycle c = 0, 1, ...:
 *   1. r = f - A u and rel_c = ||r||_2 / ||f||_2, in FP64;
 *   2. stop with status 0 if rel_c <= rtol, with status -7 if sweeps >=
 *      max_sweeps, with status -6 if rel_c is not finite;
 *   3. if c > 0 and rel_c > stall_ratio * rel_{c-1}: BF16 inner storage
 *      escalates to FP32; FP32 inner storage stops with status -7 (stalled);
 *      FP64 inner storage is never checked;
 *   4. r_lo = r rounded to the inner storage type (FP64 -> FP32 round to
 *      nearest even, then FP32 -> BF16 round to nearest even for BF16);
 *   5. e = 0, then m sweeps of A e = r_lo with inner storage and FP32
 *      arithmetic (FP64 for inner = F64): Jacobi sweeps (smoother 0, the
 *      sweep above with f := r_lo) or red-black Gauss-Seidel sweeps
 *      (smoother 1, oracle_rbgs_* in place);
 *   6. u += e in FP64 (interior only); sweeps += m.
 * inner: 0 = F64, 1 = F32, 2 = BF16 (the library's dtype codes).  The zero
 * start is the caller's (u's interior set to 0).  u's halo is the Dirichlet
 * value; e's halo is zero.  Writes *cycles (corrections applied),
 * hist[0..cycles] (rel of every residual evaluated, the last one final),
 * *final_inner and *status; returns the number of sweeps done.
 */
static void add_correction_f64(double* u, const double* e, int64_t nx,
                               int64_t ny, int64_t nz) {
  for (int64_t k = 1; k <= nz; ++k)
    for (int64_t j = 1; j <= ny; ++j)
      for (int64_t i = 1; i <= nx; ++i) AT(u, i, j, k) = AT(u, i, j, k) + AT(e, i, j, k);
}

int64_t oracle_refine(double* u, const double* f, int64_t nx, int64_t ny,
                      int64_t nz, double h, double rtol, int inner, int smoother,
                      int64_t m, int64_t max_sweeps, double stall_ratio,
                      int64_t* cycles, double* hist, int64_t hist_len,
                      int* final_inner, int* status, double* work) {
  /* work: 6 fields' worth of FP64 storage */
  const size_t len = field_len(nx, ny, nz);
  double* r = work;
  double* e64 = work + len;
  double* t64 = work + 2 * len;
  float* r32 = (float*)(work + 3 * len);
  float* e32 = r32 + len;
  float* t32 = e32 + len;
  uint16_t* r16 = (uint16_t*)(work + 5 * len);
  uint16_t* e16 = r16 + len;
  uint16_t* t16 = e16 + len;
  const float hh32 = (float)(h * h);
  int64_t sweeps = 0;
  int cur = inner;
  double prev = INFINITY;
  int64_t c = 0;
  *status = 0;
  memset(r, 0, len * sizeof(double));
  for (;; ++c) {
    double norms[2];
    oracle_residual_f64(u, f, nx, ny, nz, h, r, norms, 1);
    double rel = norms[1] > 0.0 ? norms[0] / norms[1] : norms[0];
    if (c < hist_len) hist[c] = rel;
    if (!isfinite(rel)) { *status = -6; break; }
    if (rel <= rtol) break;
    if (sweeps >= max_sweeps) { *status = -7; break; }
    if (c > 0 && cur != 0 && rel > stall_ratio * prev) {
      if (cur == 2) {
        cur = 1;
      } else {
        *status = -7;
        break;
      }
    }
    prev = rel;
    if (cur == 0) {
      memset(e64, 0, len * sizeof(double));
      if (smoother == 1) {
        oracle_rbgs_f64(e64, r, nx, ny, nz, h, m, 1);
      } else {
        for (int64_t s = 0; s < m; ++s) {
          oracle_jacobi_sweep_f64(e64, t64, r, nx, ny, nz, h, 1);
          double* t = e64; e64 = t64; t64 = t;
        }
      }
      add_correction_f64(u, e64, nx, ny, nz);
    } else if (cur == 1) {
      for (size_t q = 0; q < len; ++q) { r32[q] = (float)r[q]; e32[q] = 0.0f; }
      if (smoother == 1) {
        oracle_rbgs_f32(e32, r32, nx, ny, nz, hh32, m);
      } else {
        for (int64_t s = 0; s < m; ++s) {
          oracle_jacobi_sweep_f32(e32, t32, r32, nx, ny, nz, hh32);
          float* t = e32; e32 = t32; t32 = t;
        }
      }
      for (size_t q = 0; q < len; ++q) t64[q] = (double)e32[q];
      add_correction_f64(u, t64, nx, ny, nz);
    } else {
      for (size_t q = 0; q < len; ++q) { r16[q] = float_to_bf16((float)r[q]); e16[q] = 0; }
      if (smoother == 1) {
        oracle_rbgs_bf16(e16, r16, nx, ny, nz, hh32, m);
      } else {
        for (int64_t s = 0; s < m; ++s) {
          oracle_jacobi_sweep_bf16(e16, t16, r16, nx, ny, nz, hh32);
          uint16_t* t = e16; e16 = t16; t16 = t;
        }
      }
      for (size_t q = 0; q < len; ++q) t64[q] = (double)bf16_to_float(e16[q]);
      add_correction_f64(u, t64, nx, ny, nz);
    }
    sweeps += m;
  }
  *cycles = c;
  *final_inner = cur;
  return sweeps;
}
