/*
 * FP64 CPU oracle for matrix-free finite element operator action.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this code.  It shares no code,
 * header, table or generator with the CUDA library: it computes its own
 * quadrature rules, its own basis functions and its own geometry, directly
 * from their definitions, and evaluates every integral by plain loops over
 * cells, quadrature points and basis functions (no sum factorization, no
 * batching, no reordering).
 *
 * What it computes (Section 2 of arXiv 1903.08243): the assembled linear form
 *   y_i = sum_K sum_q w_q |det J_K(xi_q)| * integrand(phi_i, u_h)(xi_q),
 * i.e. the action of the bilinear forms of the Supplementary material
 * (mass, Helmholtz, Laplacian, elasticity, hyperelasticity) on a vector.
 */
#ifndef FE_ORACLE_H
#define FE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Cell types (ids, not vertex counts): tetrahedron (4 vertices), hexahedron (8),
 * triangle (3) and quadrilateral (4) in the plane z = 0.  A 2D problem is the
 * 3D one with no z dependence: J gets a unit (z, z) entry, reference gradients
 * have no z component, vector fields have 2 components (plane strain). */
enum { ORC_TRI = 3, ORC_TET = 4, ORC_HEX = 8, ORC_QUAD = 40 };
enum {
  ORC_MASS = 0,
  ORC_LAPLACE = 1,
  ORC_HELMHOLTZ = 2,
  ORC_ELASTICITY = 3,
  ORC_HYPER_RES = 4,
  ORC_HYPER_JAC = 5
};
enum { ORC_SVK = 0, ORC_NEOHOOKE = 1 };

typedef struct {
  int32_t cell_type;   /* ORC_TET or ORC_HEX */
  int32_t degree;      /* P_p (tet, p = 1, 2) or Q_p (hex, p >= 1) */
  int32_t ncomp;       /* 1 (scalar) or 3 (vector, dof = 3*node + c) */
  int32_t kind;        /* ORC_MASS ... ORC_HYPER_JAC */
  int32_t law;         /* ORC_SVK or ORC_NEOHOOKE (hyperelastic forms) */
  int32_t qdeg;        /* tet: rule degree; hex: Gauss points per direction */
  int32_t equispaced;  /* hex only: 1 = equispaced nodes, 0 = Gauss-Lobatto */
  int32_t nq_rule;     /* tet/tri: > 0 = integrate with the explicit rule qpts/qw
                          of nq_rule points instead of the collapsed rule of qdeg */
  int64_t ncell, nvert, nnode;
  const double *coords;      /* [nvert][3] */
  const int32_t *cell_vert;  /* [ncell][4 or 8] */
  const int32_t *cell_node;  /* [ncell][nloc] */
  double k2, lambda, mu;
  double b[3];               /* body force of the hyperelastic residual */
  const double *ucoef;       /* [nnode*3] linearisation point of HYPER_JAC */
  const double *qpts;        /* nq_rule > 0: reference points [nq_rule][dim] */
  const double *qw;          /* nq_rule > 0: weights [nq_rule] (they sum to the reference volume) */
} orc_problem;

/* 1D rules on [0,1].  Return the number of points or a negative error. */
int orc_gauss_legendre(int n, double *x, double *w);
/* Gauss-Jacobi for the weight (1-x)^alpha on [0,1] (beta = 0). */
int orc_gauss_jacobi(int n, int alpha, double *x, double *w);
/* Gauss-Lobatto-Legendre nodes (n >= 2) on [0,1], ascending. */
int orc_gll_nodes(int n, double *x);
/* Collapsed (conical product) rule on the reference tet exact to `degree`.
 * pts is [nq][3]; returns nq = m^3 with m = ceil((degree+1)/2). */
int orc_tet_rule(int degree, double *pts, double *w);
/* Lagrange P_p on the reference tet (p = 1..6) by inverting the Vandermonde
 * matrix of monomials at the nodes.  phi [ndof], dphi [ndof][3].  Nodes:
 * P1/P2 vertices, then edge midpoints (0,1), (0,2), (0,3), (1,2), (1,3),
 * (2,3); P3..P6 the lattice points (i, j, l)/p, i + j + l <= p, i fastest,
 * then j, then l. */
int orc_tet_basis(int p, const double xi[3], double *phi, double *dphi);
/* Lagrange Q_p on [0,1]^3; phi [n^3], dphi [n^3][3]. */
int orc_hex_basis(int p, int equispaced, const double xi[3], double *phi, double *dphi);
/* Collapsed rule on the reference triangle exact to `degree`: pts [nq][2],
 * nq = m^2 with m = ceil((degree+1)/2). */
int orc_tri_rule(int degree, double *pts, double *w);
/* Lagrange P_p (p = 1..6) on the reference triangle by inverting the
 * Vandermonde matrix of monomials at the lattice nodes (i, j)/p, i + j <= p, i
 * fastest.  phi [ndof], dphi [ndof][2]. */
int orc_tri_basis(int p, const double xi[2], double *phi, double *dphi);
/* Lagrange Q_p on [0,1]^2 at GLL nodes, node i + n j; phi [n^2], dphi [n^2][2]. */
int orc_quad_basis(int p, const double xi[2], double *phi, double *dphi);

/* y = A(x) restricted to the listed cells (cells == NULL: all cells).
 * y is overwritten.  Returns 0, or a negative error (bad argument,
 * non-positive Jacobian determinant, non-positive deformation J). */
int orc_apply(const orc_problem *pb, const double *x, double *y,
              const int64_t *cells, int64_t ncells);
/* Discrete hyperelastic energy  sum_K sum_q w |det J| Psi(F) - sum_q w|det J| b.u. */
int orc_energy(const orc_problem *pb, const double *u, double *energy);
/* Cell-local element matrix A_K[i][j] = d y_loc[i] / d x_loc[j] (linear forms). */
int orc_element_matrix(const orc_problem *pb, int64_t cell, double *A);

#ifdef __cplusplus
}
#endif
#endif
