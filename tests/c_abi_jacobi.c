/*
 * c_abi_jacobi.c -- a plain C caller of libstencil.so (test helper).
 *
 *   c_abi_jacobi nx ny nz nsweeps u.bin f.bin out.bin
 *
 * Reads u and f (float64, (nz+2)(ny+2)(nx+2) cells with the halo, x
 * fastest), places them in device memory with 16-byte aligned rows, runs
 * nsweeps Jacobi sweeps through stencil_jacobi_sweep (with an FP64 work grid,
 * so the fixed-point iterate stays resident), checks the context status and
 * writes u back to out.bin.  Exit status 0 on success; any library or CUDA
 * error is printed and gives a nonzero status.
 */
#include <cuda_runtime_api.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "stencil.h"

static int cuda_ok(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    fprintf(stderr, "%s: %s\n", what, cudaGetErrorString(e));
    return 0;
  }
  return 1;
}

static int read_all(const char* path, double* buf, size_t n) {
  FILE* fp = fopen(path, "rb");
  if (!fp) return 0;
  const size_t got = fread(buf, sizeof(double), n, fp);
  fclose(fp);
  return got == n;
}

int main(int argc, char** argv) {
  if (argc != 8) {
    fprintf(stderr, "usage: %s nx ny nz nsweeps u.bin f.bin out.bin\n", argv[0]);
    return 2;
  }
  const int64_t nx = atoll(argv[1]), ny = atoll(argv[2]), nz = atoll(argv[3]);
  const int64_t nsweeps = atoll(argv[4]);
  const int64_t X = nx + 2, Y = ny + 2, Z = nz + 2;
  const int64_t sy = (X + 1) / 2 * 2; /* 16-byte rows of float64 */
  const int64_t sz = sy * Y;
  const size_t cells = (size_t)(X * Y * Z);
  double* host = (double*)malloc(2 * cells * sizeof(double));
  if (!host || !read_all(argv[5], host, cells) || !read_all(argv[6], host + cells, cells)) {
    fprintf(stderr, "cannot read the inputs\n");
    return 2;
  }
  void* dev[4] = {NULL, NULL, NULL, NULL}; /* u, u_tmp, f, work */
  const size_t bytes = (size_t)(sz * Z) * sizeof(double);
  for (int b = 0; b < 4; ++b)
    if (!cuda_ok(cudaMalloc(&dev[b], bytes), "cudaMalloc") || !cuda_ok(cudaMemset(dev[b], 0, bytes), "cudaMemset"))
      return 3;
  const size_t pitch = (size_t)sy * sizeof(double), row = (size_t)X * sizeof(double);
  if (!cuda_ok(cudaMemcpy2D(dev[0], pitch, host, row, row, (size_t)(Y * Z), cudaMemcpyHostToDevice), "copy u") ||
      !cuda_ok(cudaMemcpy2D(dev[2], pitch, host + cells, row, row, (size_t)(Y * Z), cudaMemcpyHostToDevice),
               "copy f"))
    return 3;
  stencil_grid g[4];
  for (int b = 0; b < 4; ++b) {
    g[b].data = dev[b];
    g[b].nx = nx;
    g[b].ny = ny;
    g[b].nz = nz;
    g[b].sy = sy;
    g[b].sz = sz;
    g[b].dtype = STENCIL_F64;
    g[b].reserved = 0;
  }
  stencil_ctx* ctx = NULL;
  int rc = stencil_ctx_create(0, &ctx);
  if (!rc) rc = stencil_jacobi_sweep(ctx, &g[0], &g[1], &g[2], &g[3], 1.0 / (double)(nx + 1), nsweeps, 0, 0, NULL);
  if (!rc) rc = stencil_ctx_status(ctx, NULL);
  if (rc) {
    fprintf(stderr, "stencil error %d: %s\n", rc, stencil_last_error());
    return 4;
  }
  if (!cuda_ok(cudaMemcpy2D(host, row, dev[0], pitch, row, (size_t)(Y * Z), cudaMemcpyDeviceToHost), "copy back"))
    return 3;
  stencil_ctx_destroy(ctx);
  for (int b = 0; b < 4; ++b) cudaFree(dev[b]);
  FILE* fp = fopen(argv[7], "wb");
  if (!fp || fwrite(host, sizeof(double), cells, fp) != cells) {
    fprintf(stderr, "cannot write the output\n");
    return 2;
  }
  fclose(fp);
  free(host);
  return 0;
}
