/*
 * The library from plain C: a Q3 Helmholtz operator on a perturbed hexahedral
 * mesh of the unit cube, applied to host vectors through the C ABI alone.
 *
 * With k^2 = 1 the Laplacian part of A annihilates the constant function, so
 * y = A 1 is the mass matrix applied to 1 and its entries sum to the volume of
 * the domain, 1 (the perturbation keeps the boundary vertices in place).  The
 * program checks that sum, and that a second apply gives the same vector to
 * rounding (the atomic scatter may add in another order).  Exit status 0 on
 * success.
 *
 *   cc -std=c11 -I include helmholtz_host.c -L paper_1903_08243_gb300 -lmfa -o helmholtz_host
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "mfa.h"

#define CHECK(call)                                                          \
  do {                                                                       \
    int rc_ = (call);                                                        \
    if (rc_ != MFA_OK) {                                                     \
      fprintf(stderr, "%s failed (%d): %s\n", #call, rc_, mfa_last_error()); \
      return 1;                                                              \
    }                                                                        \
  } while (0)

/* nx^3 hexahedra of the unit cube; interior vertices moved by a fixed pattern
 * of up to 0.1 h (deterministic, no random generator needed). */
static void box_mesh(int nx, double *coords, int32_t *cell_vert) {
  const int m = nx + 1;
  const double h = 1.0 / nx;
  for (int k = 0; k < m; ++k)
    for (int j = 0; j < m; ++j)
      for (int i = 0; i < m; ++i) {
        const int v = i + m * (j + m * k);
        const int interior = i > 0 && i < nx && j > 0 && j < nx && k > 0 && k < nx;
        const double s = interior ? 0.1 * h : 0.0;
        coords[3 * v + 0] = i * h + s * sin(1.0 + 3.0 * v);
        coords[3 * v + 1] = j * h + s * sin(2.0 + 5.0 * v);
        coords[3 * v + 2] = k * h + s * sin(3.0 + 7.0 * v);
      }
  for (int k = 0; k < nx; ++k)
    for (int j = 0; j < nx; ++j)
      for (int i = 0; i < nx; ++i) {
        const int c = i + nx * (j + nx * k);
        for (int v = 0; v < 8; ++v) {  /* local vertex a + 2b + 4c at corner (a, b, c) */
          const int a = v & 1, b = (v >> 1) & 1, cc = (v >> 2) & 1;
          cell_vert[8 * c + v] = (i + a) + m * ((j + b) + m * (k + cc));
        }
      }
}

int main(void) {
  const int nx = 4, degree = 3;
  const int64_t ncell = (int64_t)nx * nx * nx, nvert = (int64_t)(nx + 1) * (nx + 1) * (nx + 1);
  double *coords = malloc(sizeof(double) * 3 * nvert);
  int32_t *cell_vert = malloc(sizeof(int32_t) * 8 * ncell);
  if (!coords || !cell_vert) return 1;
  box_mesh(nx, coords, cell_vert);

  mfa_ctx *ctx = NULL;
  mfa_mesh *mesh = NULL;
  mfa_space *space = NULL;
  mfa_form *form = NULL;
  CHECK(mfa_create(&ctx, 0, NULL));
  CHECK(mfa_mesh_upload(ctx, MFA_CELL_HEX8, ncell, nvert, coords, cell_vert, &mesh));
  CHECK(mfa_space_create(ctx, mesh, degree, 1, NULL, 0, &space));  /* the library builds the map */
  int64_t ndof = 0;
  CHECK(mfa_space_ndof(space, &ndof));
  mfa_form_params p = {0};
  p.kind = MFA_FORM_HELMHOLTZ;
  p.k2 = 1.0;
  CHECK(mfa_form_create(ctx, space, &p, &form));

  double *x = malloc(sizeof(double) * ndof), *y = malloc(sizeof(double) * ndof);
  if (!x || !y) return 1;
  for (int64_t i = 0; i < ndof; ++i) x[i] = 1.0;
  CHECK(mfa_apply_host(ctx, form, x, y));
  double sum = 0.0;
  for (int64_t i = 0; i < ndof; ++i) sum += y[i];
  printf("Q%d Helmholtz on %d^3 hexes, %lld dofs: sum(A 1) = %.15f\n", degree, nx, (long long)ndof, sum);
  int status = fabs(sum - 1.0) < 1e-12 ? 0 : 2;

  double *y2 = malloc(sizeof(double) * ndof);
  if (!y2) return 1;
  CHECK(mfa_apply_host(ctx, form, x, y2));
  for (int64_t i = 0; i < ndof; ++i)
    if (fabs(y2[i] - y[i]) > 1e-13 * fabs(y[i])) status = 3;

  CHECK(mfa_form_destroy(form));
  CHECK(mfa_space_destroy(space));
  CHECK(mfa_mesh_destroy(mesh));
  CHECK(mfa_destroy(ctx));
  free(coords);
  free(cell_vert);
  free(x);
  free(y);
  free(y2);
  if (status == 0)
    printf("ok\n");
  else
    printf("FAILED (%d)\n", status);
  return status;
}
