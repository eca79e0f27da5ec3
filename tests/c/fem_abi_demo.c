/*
 * A plain C11 caller of the library: only include/fem.h and the CUDA runtime
 * (cudaMalloc / cudaMemcpy for the caller-owned device vectors), no Python.
 * It checks, on an N^3 unit-cube hexahedral mesh of order p:
 *   - diffusion applied to the constant function vanishes (constants are in
 *     the kernel of the Laplacian);
 *   - the mass matrix applied to the constant function sums to the volume 1;
 *   - Jacobi-PCG for -lap u = 1, u = 0 on the boundary converges to 1e-10;
 *   - elasticity applied to a rigid translation vanishes;
 *   - a bad argument returns a status and a message instead of aborting.
 * Prints "c abi ok" and returns 0, else prints the failing check and
 * returns 1. Build: gcc -std=c11 fem_abi_demo.c -I include -I <cuda>/include
 *   -L <pkg> -lfem -L <cuda>/lib64 -lcudart -lm
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "fem.h"

#define CHECK(cond, what)                                                   \
  do {                                                                      \
    if (!(cond)) {                                                          \
      fprintf(stderr, "check failed: %s (%s)\n", what, fem_last_error());   \
      return 1;                                                             \
    }                                                                       \
  } while (0)

static double max_abs(const double* v, int64_t n) {
  double m = 0.0;
  for (int64_t i = 0; i < n; ++i) m = fabs(v[i]) > m ? fabs(v[i]) : m;
  return m;
}

int main(void) {
  const int N = 3, p = 3, q = p + 2;
  const int64_t nv = (int64_t)(N + 1) * (N + 1) * (N + 1), ne = (int64_t)N * N * N;
  double* coords = malloc(sizeof(double) * 3 * nv);
  int32_t* hex = malloc(sizeof(int32_t) * 8 * ne);
  for (int k = 0; k <= N; ++k)
    for (int j = 0; j <= N; ++j)
      for (int i = 0; i <= N; ++i) {
        const int64_t v = i + (N + 1) * (j + (N + 1) * (int64_t)k);
        coords[3 * v] = (double)i / N;
        coords[3 * v + 1] = (double)j / N;
        coords[3 * v + 2] = (double)k / N;
      }
  for (int k = 0; k < N; ++k)
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i) {
        const int64_t e = i + N * (j + N * (int64_t)k);
#define VID(a, b, c) (int32_t)((i + (a)) + (N + 1) * ((j + (b)) + (N + 1) * (k + (c))))
        const int32_t t[8] = {VID(0, 0, 0), VID(1, 0, 0), VID(1, 1, 0), VID(0, 1, 0),
                              VID(0, 0, 1), VID(1, 0, 1), VID(1, 1, 1), VID(0, 1, 1)};
#undef VID
        memcpy(hex + 8 * e, t, sizeof t);
      }
  fem_mesh* mesh = NULL;
  fem_space* space = NULL;
  CHECK(fem_mesh_create(coords, nv, hex, ne, &mesh) == FEM_OK, "mesh");
  CHECK(fem_space_create(mesh, p, &space) == FEM_OK, "space");
  int64_t ndof = 0, nbdr = 0;
  CHECK(fem_space_info(space, &ndof, &nbdr, NULL, NULL) == FEM_OK, "space info");
  CHECK(ndof == (int64_t)(p * N + 1) * (p * N + 1) * (p * N + 1), "ndof of a structured cube");

  double *x = NULL, *y = NULL, *b = NULL, *g = NULL, *bc = NULL, *fq = NULL;
  const int64_t nq = ne * q * q * q;
  CHECK(cudaMalloc((void**)&x, sizeof(double) * 3 * ndof) == cudaSuccess, "cudaMalloc");
  CHECK(cudaMalloc((void**)&y, sizeof(double) * 3 * ndof) == cudaSuccess, "cudaMalloc");
  CHECK(cudaMalloc((void**)&b, sizeof(double) * ndof) == cudaSuccess, "cudaMalloc");
  CHECK(cudaMalloc((void**)&g, sizeof(double) * ndof) == cudaSuccess, "cudaMalloc");
  CHECK(cudaMalloc((void**)&bc, sizeof(double) * ndof) == cudaSuccess, "cudaMalloc");
  CHECK(cudaMalloc((void**)&fq, sizeof(double) * nq) == cudaSuccess, "cudaMalloc");
  double* h = malloc(sizeof(double) * 3 * ndof);
  for (int64_t i = 0; i < 3 * ndof; ++i) h[i] = 1.0;
  CHECK(cudaMemcpy(x, h, sizeof(double) * 3 * ndof, cudaMemcpyHostToDevice) == cudaSuccess, "copy");

  /* diffusion: A 1 = 0 */
  fem_form* dif = NULL;
  CHECK(fem_form_create(space, FEM_DIFFUSION, q, NULL, NULL, &dif) == FEM_OK, "diffusion form");
  CHECK(fem_apply(dif, FEM_F64, x, y, 0, NULL) == FEM_OK, "diffusion apply");
  CHECK(cudaMemcpy(h, y, sizeof(double) * ndof, cudaMemcpyDeviceToHost) == cudaSuccess, "copy");
  CHECK(max_abs(h, ndof) <= 1e-12, "diffusion of a constant vanishes");

  /* mass: 1^T M 1 = volume */
  fem_form* mass = NULL;
  CHECK(fem_form_create(space, FEM_MASS, q, NULL, NULL, &mass) == FEM_OK, "mass form");
  CHECK(fem_apply(mass, FEM_F64, x, y, 0, NULL) == FEM_OK, "mass apply");
  CHECK(cudaMemcpy(h, y, sizeof(double) * ndof, cudaMemcpyDeviceToHost) == cudaSuccess, "copy");
  double vol = 0.0;
  for (int64_t i = 0; i < ndof; ++i) vol += h[i];
  CHECK(fabs(vol - 1.0) <= 1e-12, "mass of the unit cube");

  /* Poisson: -lap u = 1, u = 0 on the boundary, Jacobi-PCG to 1e-10 */
  int32_t* bdr = malloc(sizeof(int32_t) * nbdr);
  int32_t* d_bdr = NULL;
  CHECK(fem_space_boundary_dofs(space, bdr) == FEM_OK, "boundary dofs");
  CHECK(cudaMalloc((void**)&d_bdr, sizeof(int32_t) * nbdr) == cudaSuccess, "cudaMalloc");
  CHECK(cudaMemcpy(d_bdr, bdr, sizeof(int32_t) * nbdr, cudaMemcpyHostToDevice) == cudaSuccess, "copy");
  CHECK(fem_form_set_essential(dif, d_bdr, nbdr, NULL) == FEM_OK, "essential dofs");
  double* hq = malloc(sizeof(double) * nq);
  for (int64_t i = 0; i < nq; ++i) hq[i] = 1.0;
  CHECK(cudaMemcpy(fq, hq, sizeof(double) * nq, cudaMemcpyHostToDevice) == cudaSuccess, "copy");
  CHECK(fem_rhs(dif, fq, b, NULL) == FEM_OK, "load vector");
  CHECK(cudaMemset(g, 0, sizeof(double) * ndof) == cudaSuccess, "memset");
  CHECK(fem_lift_rhs(dif, b, g, bc, NULL) == FEM_OK, "lift");
  CHECK(cudaMemset(y, 0, sizeof(double) * ndof) == cudaSuccess, "memset");
  fem_solve_opts opts;
  fem_solve_opts_default(&opts);
  fem_solve_info info;
  CHECK(fem_solve(dif, bc, y, &opts, &info, NULL) == FEM_OK, "solve");
  CHECK(info.converged && info.relres <= 1e-10, "solve converged");
  CHECK(cudaMemcpy(h, y, sizeof(double) * ndof, cudaMemcpyDeviceToHost) == cudaSuccess, "copy");
  /* the torsion-like solution of -lap u = 1 on the unit cube peaks at ~0.0562 */
  CHECK(max_abs(h, ndof) > 0.05 && max_abs(h, ndof) < 0.06, "solution magnitude");

  /* elasticity: a rigid translation has no strain */
  double *lam = NULL, *mu = NULL;
  CHECK(cudaMalloc((void**)&lam, sizeof(double) * ne) == cudaSuccess, "cudaMalloc");
  CHECK(cudaMalloc((void**)&mu, sizeof(double) * ne) == cudaSuccess, "cudaMalloc");
  for (int64_t i = 0; i < ne; ++i) hq[i] = 1.0 + 0.1 * (double)(i % 5);
  CHECK(cudaMemcpy(lam, hq, sizeof(double) * ne, cudaMemcpyHostToDevice) == cudaSuccess, "copy");
  CHECK(cudaMemcpy(mu, hq, sizeof(double) * ne, cudaMemcpyHostToDevice) == cudaSuccess, "copy");
  fem_form* el = NULL;
  CHECK(fem_form_create_elasticity(space, q, lam, mu, NULL, &el) == FEM_OK, "elasticity form");
  CHECK(fem_apply(el, FEM_F64, x, y, 0, NULL) == FEM_OK, "elasticity apply");
  CHECK(cudaMemcpy(h, y, sizeof(double) * 3 * ndof, cudaMemcpyDeviceToHost) == cudaSuccess, "copy");
  CHECK(max_abs(h, 3 * ndof) <= 1e-12, "elasticity of a translation vanishes");

  /* errors come back as a status and a message */
  fem_space* bad = NULL;
  CHECK(fem_space_create(mesh, 0, &bad) == FEM_EINVAL && bad == NULL, "p = 0 rejected");
  CHECK(strlen(fem_last_error()) > 0, "error message");

  fem_form_destroy(el);
  fem_form_destroy(mass);
  fem_form_destroy(dif);
  fem_space_destroy(space);
  fem_mesh_destroy(mesh);
  cudaFree(x);
  cudaFree(y);
  cudaFree(b);
  cudaFree(g);
  cudaFree(bc);
  cudaFree(fq);
  cudaFree(d_bdr);
  cudaFree(lam);
  cudaFree(mu);
  free(coords);
  free(hex);
  free(h);
  free(hq);
  free(bdr);
  printf("c abi ok: ndof %lld, PCG %d iterations, relres %.2e\n", (long long)ndof, info.iterations, info.relres);
  return 0;
}
