/*
 * FP64 CPU oracle for matrix-free finite element operator action.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
 * benchmark's CPU-baseline leg, never by the library.  Everything here is
 * written from definitions, in the order the paper states them:
 *
 *  - global assembly (Section 2.2, Listing 3): for each cell gather the
 *    coordinates and the dofs through the cell maps, run the local kernel,
 *    increment the global vector through the cell->dof map;
 *  - local assembly (Section 2.1, Listing 2 and its description): pull back
 *    to the reference cell, loop over quadrature points, change basis from
 *    dofs to point values and gradients, evaluate the integrand, and
 *    accumulate w_q |det J| times the integrand against every test function.
 *    The Jacobian is evaluated at every quadrature point (the general case
 *    in Section 2.1; constant on affine tetrahedra);
 *  - the integrands of the Supplementary material: mass, Helmholtz,
 *    (vector) Laplacian, elasticity, hyperelasticity residual and its
 *    Gateaux derivative.
 *
 * Nothing is batched, fused or sum-factorised: point values are direct sums
 * over all local basis functions.  Quadrature points and basis functions are
 * computed here from their mathematical definitions in long double.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EARG (-1)
#define ORC_EDET (-2)
#define ORC_EJAC (-3)
#define ORC_EMEM (-4)

#define PI_L 3.141592653589793238462643383279502884L

/* ------------------------------------------------------------------ */
/* One-dimensional rules                                               */
/* ------------------------------------------------------------------ */

/* Jacobi polynomial P_n^{(a,b)}(t) and P_{n-1}^{(a,b)}(t) by the three-term
 * recurrence (Szego, Orthogonal Polynomials, Eq. 4.5.1). */
static void jacobi_eval(int n, long double a, long double b, long double t,
                        long double *pn, long double *pnm1) {
  long double p0 = 1.0L, p1 = 0.5L * ((a + b + 2.0L) * t + (a - b));
  if (n == 0) { *pn = p0; *pnm1 = 0.0L; return; }
  for (int k = 1; k < n; ++k) {
    long double c = 2.0L * k + a + b;
    long double a1 = 2.0L * (k + 1) * (k + a + b + 1.0L) * c;
    long double a2 = (c + 1.0L) * (a * a - b * b);
    long double a3 = c * (c + 1.0L) * (c + 2.0L);
    long double a4 = 2.0L * (k + a) * (k + b) * (c + 2.0L);
    long double p2 = ((a2 + a3 * t) * p1 - a4 * p0) / a1;
    p0 = p1;
    p1 = p2;
  }
  *pn = p1;
  *pnm1 = p0;
}

/* d/dt P_n^{(a,b)} from (2n+a+b)(1-t^2) P_n' = n[(a-b) - (2n+a+b) t] P_n + 2(n+a)(n+b) P_{n-1}
 * (Szego Eq. 4.5.7). */
static long double jacobi_deriv(int n, long double a, long double b, long double t,
                                long double pn, long double pnm1) {
  long double c = 2.0L * n + a + b;
  return (n * ((a - b) - c * t) * pn + 2.0L * (n + a) * (n + b) * pnm1) / (c * (1.0L - t * t));
}

/* Roots of P_n^{(a,b)} on (-1,1), ascending: Newton's method with deflation
 * by the roots already found, started from Chebyshev points. */
static void jacobi_roots(int n, long double a, long double b, long double *t) {
  for (int i = 0; i < n; ++i) {
    long double x = -cosl(PI_L * (2.0L * i + 1.0L) / (2.0L * n));
    if (i > 0 && x <= t[i - 1]) x = 0.5L * (t[i - 1] + 1.0L);
    for (int it = 0; it < 200; ++it) {
      long double pn, pm;
      jacobi_eval(n, a, b, x, &pn, &pm);
      long double dp = jacobi_deriv(n, a, b, x, pn, pm);
      long double s = 0.0L;
      for (int j = 0; j < i; ++j) s += 1.0L / (x - t[j]);
      long double dx = pn / (dp - pn * s);
      x -= dx;
      if (fabsl(dx) < 1e-19L) break;
    }
    t[i] = x;
  }
}

int orc_gauss_jacobi(int n, int alpha, double *x, double *w) {
  if (n < 1 || n > 64 || alpha < 0 || !x || !w) return ORC_EARG;
  long double t[64];
  jacobi_roots(n, (long double)alpha, 0.0L, t);
  for (int i = 0; i < n; ++i) {
    long double pn, pm;
    jacobi_eval(n, (long double)alpha, 0.0L, t[i], &pn, &pm);
    long double dp = jacobi_deriv(n, (long double)alpha, 0.0L, t[i], pn, pm);
    /* Christoffel weight for beta = 0 on [-1,1]: 2^(a+1) / ((1-t^2) P_n'(t)^2);
     * the affine map to [0,1] with weight (1-x)^a divides it by 2^(a+1). */
    long double wt = 1.0L / ((1.0L - t[i] * t[i]) * dp * dp);
    x[i] = (double)(0.5L * (1.0L + t[i]));
    w[i] = (double)wt;
  }
  return n;
}

int orc_gauss_legendre(int n, double *x, double *w) { return orc_gauss_jacobi(n, 0, x, w); }

int orc_gll_nodes(int n, double *x) {
  if (n < 2 || n > 64 || !x) return ORC_EARG;
  int N = n - 1; /* interior nodes are the roots of P_N'(t) */
  long double r[64];
  for (int i = 0; i < N - 1; ++i) {
    long double y = -cosl(PI_L * (i + 1.0L) / N);
    if (i > 0 && y <= r[i - 1]) y = 0.5L * (r[i - 1] + 1.0L);
    for (int it = 0; it < 200; ++it) {
      long double pn, pm;
      jacobi_eval(N, 0.0L, 0.0L, y, &pn, &pm);
      long double d1 = jacobi_deriv(N, 0.0L, 0.0L, y, pn, pm);
      /* Legendre's equation: (1-t^2) P'' = 2 t P' - N(N+1) P */
      long double d2 = (2.0L * y * d1 - (long double)N * (N + 1) * pn) / (1.0L - y * y);
      long double s = 0.0L;
      for (int j = 0; j < i; ++j) s += 1.0L / (y - r[j]);
      long double dy = d1 / (d2 - d1 * s);
      y -= dy;
      if (fabsl(dy) < 1e-19L) break;
    }
    r[i] = y;
  }
  x[0] = 0.0;
  for (int i = 0; i < N - 1; ++i) x[i + 1] = (double)(0.5L * (1.0L + r[i]));
  x[n - 1] = 1.0;
  return n;
}

/* ------------------------------------------------------------------ */
/* Reference-tetrahedron rule: conical product (Stroud) of Gauss rules  */
/* ------------------------------------------------------------------ */

int orc_tet_rule(int degree, double *pts, double *w) {
  if (degree < 0 || degree > 30 || !pts || !w) return ORC_EARG;
  int m = (degree + 2) / 2; /* ceil((degree+1)/2): 2m-1 >= degree */
  double xa[32], wa[32], xb[32], wb[32], xc[32], wc[32];
  orc_gauss_jacobi(m, 0, xa, wa);
  orc_gauss_jacobi(m, 1, xb, wb);
  orc_gauss_jacobi(m, 2, xc, wc);
  int q = 0;
  /* (a,b,c) in [0,1]^3 -> x = a(1-b)(1-c), y = b(1-c), z = c, with the
   * Jacobian (1-b)(1-c)^2 absorbed by the Jacobi weights. */
  for (int k = 0; k < m; ++k)
    for (int j = 0; j < m; ++j)
      for (int i = 0; i < m; ++i) {
        double a = xa[i], b = xb[j], c = xc[k];
        pts[3 * q + 0] = a * (1.0 - b) * (1.0 - c);
        pts[3 * q + 1] = b * (1.0 - c);
        pts[3 * q + 2] = c;
        w[q] = wa[i] * wb[j] * wc[k];
        ++q;
      }
  return q;
}

int orc_tri_rule(int degree, double *pts, double *w) {
  if (degree < 0 || degree > 30 || !pts || !w) return ORC_EARG;
  int m = (degree + 2) / 2;
  double xa[32], wa[32], xb[32], wb[32];
  orc_gauss_jacobi(m, 0, xa, wa);
  orc_gauss_jacobi(m, 1, xb, wb);
  int q = 0;
  /* (a,b) in [0,1]^2 -> x = a(1-b), y = b, the Jacobian (1-b) absorbed by the Jacobi weight */
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < m; ++i) {
      pts[2 * q + 0] = xa[i] * (1.0 - xb[j]);
      pts[2 * q + 1] = xb[j];
      w[q] = wa[i] * wb[j];
      ++q;
    }
  return q;
}

/* ------------------------------------------------------------------ */
/* Basis functions                                                      */
/* ------------------------------------------------------------------ */

/* Monomial exponents of total degree <= p, p <= 2. */
#define ORC_TET_MAXP 6
#define ORC_TET_MAXN 84 /* (p+1)(p+2)(p+3)/6 at p = 6 */

static int tet_monomials(int p, int e[ORC_TET_MAXN][3]) {
  int n = 0;
  for (int d = 0; d <= p; ++d)
    for (int i = d; i >= 0; --i)
      for (int j = d - i; j >= 0; --j) {
        int k = d - i - j;
        e[n][0] = i; e[n][1] = j; e[n][2] = k;
        ++n;
      }
  return n;
}

static long double ipow(long double x, int k) {
  long double r = 1.0L;
  for (int i = 0; i < k; ++i) r *= x;
  return r;
}

/* Reference nodes.  P1/P2: vertices, then midpoints of edges (0,1), (0,2),
 * (0,3), (1,2), (1,3), (2,3).  P3..P6: the equispaced lattice points
 * (i, j, l)/p, i + j + l <= p, with i running fastest, then j, then l. */
static void tet_nodes(int p, long double nodes[ORC_TET_MAXN][3]) {
  static const long double v[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  static const int ed[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
  if (p >= 3) {
    int n = 0;
    for (int l = 0; l <= p; ++l)
      for (int j = 0; j <= p - l; ++j)
        for (int i = 0; i <= p - l - j; ++i) {
          nodes[n][0] = (long double)i / p;
          nodes[n][1] = (long double)j / p;
          nodes[n][2] = (long double)l / p;
          ++n;
        }
    return;
  }
  for (int i = 0; i < 4; ++i)
    for (int d = 0; d < 3; ++d) nodes[i][d] = v[i][d];
  if (p == 2)
    for (int e = 0; e < 6; ++e)
      for (int d = 0; d < 3; ++d) nodes[4 + e][d] = 0.5L * (v[ed[e][0]][d] + v[ed[e][1]][d]);
}

int orc_tet_basis(int p, const double xi[3], double *phi, double *dphi) {
  if (p < 1 || p > ORC_TET_MAXP || !xi || !phi || !dphi) return ORC_EARG;
  int e[ORC_TET_MAXN][3];
  int n = tet_monomials(p, e);
  long double nodes[ORC_TET_MAXN][3];
  tet_nodes(p, nodes);
  /* Vandermonde V[i][j] = m_j(node_i); C = V^{-1} gives phi_a = sum_j C[j][a] m_j. */
  static _Thread_local long double M[ORC_TET_MAXN][2 * ORC_TET_MAXN];
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j)
      M[i][j] = ipow(nodes[i][0], e[j][0]) * ipow(nodes[i][1], e[j][1]) * ipow(nodes[i][2], e[j][2]);
    for (int j = 0; j < n; ++j) M[i][n + j] = (i == j) ? 1.0L : 0.0L;
  }
  for (int c = 0; c < n; ++c) { /* Gauss-Jordan with partial pivoting */
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(M[r][c]) > fabsl(M[piv][c])) piv = r;
    if (fabsl(M[piv][c]) < 1e-30L) return ORC_EARG;
    if (piv != c)
      for (int j = 0; j < 2 * n; ++j) { long double t = M[c][j]; M[c][j] = M[piv][j]; M[piv][j] = t; }
    long double d = M[c][c];
    for (int j = 0; j < 2 * n; ++j) M[c][j] /= d;
    for (int r = 0; r < n; ++r)
      if (r != c) {
        long double f = M[r][c];
        for (int j = 0; j < 2 * n; ++j) M[r][j] -= f * M[c][j];
      }
  }
  long double x = xi[0], y = xi[1], z = xi[2];
  for (int a = 0; a < n; ++a) {
    long double v = 0, gx = 0, gy = 0, gz = 0;
    for (int j = 0; j < n; ++j) {
      long double c = M[j][n + a];
      int i0 = e[j][0], i1 = e[j][1], i2 = e[j][2];
      v += c * ipow(x, i0) * ipow(y, i1) * ipow(z, i2);
      if (i0) gx += c * i0 * ipow(x, i0 - 1) * ipow(y, i1) * ipow(z, i2);
      if (i1) gy += c * i1 * ipow(x, i0) * ipow(y, i1 - 1) * ipow(z, i2);
      if (i2) gz += c * i2 * ipow(x, i0) * ipow(y, i1) * ipow(z, i2 - 1);
    }
    phi[a] = (double)v;
    dphi[3 * a + 0] = (double)gx;
    dphi[3 * a + 1] = (double)gy;
    dphi[3 * a + 2] = (double)gz;
  }
  return n;
}

/* 1D Lagrange polynomial l_i on nodes s and its derivative (product rule). */
static void lagrange1d(int n, const double *s, int i, long double t, long double *v, long double *d) {
  long double val = 1.0L;
  for (int j = 0; j < n; ++j)
    if (j != i) val *= (t - s[j]) / ((long double)s[i] - s[j]);
  long double der = 0.0L;
  for (int k = 0; k < n; ++k) {
    if (k == i) continue;
    long double term = 1.0L / ((long double)s[i] - s[k]);
    for (int j = 0; j < n; ++j)
      if (j != i && j != k) term *= (t - s[j]) / ((long double)s[i] - s[j]);
    der += term;
  }
  *v = val;
  *d = der;
}

static void hex_nodes1d(int p, int equispaced, double *s) {
  if (equispaced)
    for (int i = 0; i <= p; ++i) s[i] = (double)i / p;
  else
    orc_gll_nodes(p + 1, s);
}

int orc_hex_basis(int p, int equispaced, const double xi[3], double *phi, double *dphi) {
  if (p < 1 || p > 16 || !xi || !phi || !dphi) return ORC_EARG;
  int n = p + 1;
  double s[17];
  hex_nodes1d(p, equispaced, s);
  long double v[3][17], d[3][17];
  for (int dim = 0; dim < 3; ++dim)
    for (int i = 0; i < n; ++i) lagrange1d(n, s, i, xi[dim], &v[dim][i], &d[dim][i]);
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        int a = i + n * (j + n * k);
        phi[a] = (double)(v[0][i] * v[1][j] * v[2][k]);
        dphi[3 * a + 0] = (double)(d[0][i] * v[1][j] * v[2][k]);
        dphi[3 * a + 1] = (double)(v[0][i] * d[1][j] * v[2][k]);
        dphi[3 * a + 2] = (double)(v[0][i] * v[1][j] * d[2][k]);
      }
  return n * n * n;
}

int orc_tri_basis(int p, const double xi[2], double *phi, double *dphi) {
  if (p < 1 || p > ORC_TET_MAXP || !xi || !phi || !dphi) return ORC_EARG;
  enum { MAXN = (ORC_TET_MAXP + 1) * (ORC_TET_MAXP + 2) / 2 };
  int e[MAXN][2], n = 0;
  for (int d = 0; d <= p; ++d)
    for (int i = d; i >= 0; --i) {
      e[n][0] = i;
      e[n][1] = d - i;
      ++n;
    }
  long double nodes[MAXN][2];
  int k = 0;
  for (int j = 0; j <= p; ++j)
    for (int i = 0; i <= p - j; ++i) {
      nodes[k][0] = (long double)i / p;
      nodes[k][1] = (long double)j / p;
      ++k;
    }
  long double M[MAXN][2 * MAXN];
  for (int r = 0; r < n; ++r) {
    for (int c = 0; c < n; ++c) M[r][c] = ipow(nodes[r][0], e[c][0]) * ipow(nodes[r][1], e[c][1]);
    for (int c = 0; c < n; ++c) M[r][n + c] = (r == c) ? 1.0L : 0.0L;
  }
  for (int c = 0; c < n; ++c) { /* Gauss-Jordan with partial pivoting */
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(M[r][c]) > fabsl(M[piv][c])) piv = r;
    if (fabsl(M[piv][c]) < 1e-30L) return ORC_EARG;
    if (piv != c)
      for (int j = 0; j < 2 * n; ++j) { long double tt = M[c][j]; M[c][j] = M[piv][j]; M[piv][j] = tt; }
    long double d = M[c][c];
    for (int j = 0; j < 2 * n; ++j) M[c][j] /= d;
    for (int r = 0; r < n; ++r)
      if (r != c) {
        long double f = M[r][c];
        for (int j = 0; j < 2 * n; ++j) M[r][j] -= f * M[c][j];
      }
  }
  long double x = xi[0], y = xi[1];
  for (int a = 0; a < n; ++a) {
    long double v = 0, gx = 0, gy = 0;
    for (int j = 0; j < n; ++j) {
      long double c = M[j][n + a];
      int i0 = e[j][0], i1 = e[j][1];
      v += c * ipow(x, i0) * ipow(y, i1);
      if (i0) gx += c * i0 * ipow(x, i0 - 1) * ipow(y, i1);
      if (i1) gy += c * i1 * ipow(x, i0) * ipow(y, i1 - 1);
    }
    phi[a] = (double)v;
    dphi[2 * a + 0] = (double)gx;
    dphi[2 * a + 1] = (double)gy;
  }
  return n;
}

int orc_quad_basis(int p, const double xi[2], double *phi, double *dphi) {
  if (p < 1 || p > 16 || !xi || !phi || !dphi) return ORC_EARG;
  int n = p + 1;
  double s[17];
  hex_nodes1d(p, 0, s);
  long double v[2][17], d[2][17];
  for (int dim = 0; dim < 2; ++dim)
    for (int i = 0; i < n; ++i) lagrange1d(n, s, i, xi[dim], &v[dim][i], &d[dim][i]);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      int a = i + n * j;
      phi[a] = (double)(v[0][i] * v[1][j]);
      dphi[2 * a + 0] = (double)(d[0][i] * v[1][j]);
      dphi[2 * a + 1] = (double)(v[0][i] * d[1][j]);
    }
  return n * n;
}

/* ------------------------------------------------------------------ */
/* Tabulation of one problem                                            */
/* ------------------------------------------------------------------ */

static int nv_of(int ct) { return ct == ORC_TRI ? 3 : (ct == ORC_TET || ct == ORC_QUAD) ? 4 : 8; }
static int dim_of(int ct) { return (ct == ORC_TRI || ct == ORC_QUAD) ? 2 : 3; }

typedef struct {
  int nq, nloc, nv, nc, dim;
  double *w;      /* [nq] */
  double *phi;    /* [nq][nloc] */
  double *dphi;   /* [nq][nloc][3] reference gradients */
  double *dN;     /* [nq][nv][3] reference gradients of the coordinate basis */
} tables;

static void free_tables(tables *t) {
  free(t->w); free(t->phi); free(t->dphi); free(t->dN);
  memset(t, 0, sizeof(*t));
}

static int nloc_of(const orc_problem *pb) {
  if (pb->cell_type == ORC_TRI) {
    const int p = pb->degree;
    return p >= 1 && p <= ORC_TET_MAXP ? (p + 1) * (p + 2) / 2 : -1;
  }
  if (pb->cell_type == ORC_QUAD) return (pb->degree + 1) * (pb->degree + 1);
  if (pb->cell_type == ORC_TET) {
    const int p = pb->degree;
    return p >= 1 && p <= ORC_TET_MAXP ? (p + 1) * (p + 2) * (p + 3) / 6 : -1;
  }
  int n = pb->degree + 1;
  return n * n * n;
}

static int check_problem(const orc_problem *pb) {
  if (!pb || !pb->coords || !pb->cell_vert || !pb->cell_node) return ORC_EARG;
  const int ct = pb->cell_type;
  if (ct != ORC_TET && ct != ORC_HEX && ct != ORC_TRI && ct != ORC_QUAD) return ORC_EARG;
  if ((ct == ORC_TET || ct == ORC_TRI) && (pb->degree < 1 || pb->degree > ORC_TET_MAXP)) return ORC_EARG;
  if ((ct == ORC_HEX || ct == ORC_QUAD) && (pb->degree < 1 || pb->degree > 16)) return ORC_EARG;
  const int dim = dim_of(ct);
  if (pb->ncomp != 1 && pb->ncomp != dim) return ORC_EARG;
  if (pb->kind < ORC_MASS || pb->kind > ORC_HYPER_JAC) return ORC_EARG;
  if (pb->kind >= ORC_ELASTICITY && pb->ncomp != dim) return ORC_EARG;
  if (pb->kind == ORC_HYPER_JAC && !pb->ucoef) return ORC_EARG;
  if (pb->qdeg < 1) return ORC_EARG;
  if (pb->nq_rule < 0 || (pb->nq_rule > 0 && (!pb->qpts || !pb->qw || (ct != ORC_TET && ct != ORC_TRI))))
    return ORC_EARG;
  if (pb->ncell < 0 || pb->nvert < 0 || pb->nnode < 0) return ORC_EARG;
  int nl = nloc_of(pb);
  for (int64_t c = 0; c < pb->ncell; ++c) {
    for (int v = 0; v < nv_of(ct); ++v) {
      int32_t id = pb->cell_vert[c * nv_of(ct) + v];
      if (id < 0 || id >= pb->nvert) return ORC_EARG;
    }
    for (int a = 0; a < nl; ++a) {
      int32_t id = pb->cell_node[c * nl + a];
      if (id < 0 || id >= pb->nnode) return ORC_EARG;
    }
  }
  return 0;
}

static int build_tables(const orc_problem *pb, tables *t) {
  memset(t, 0, sizeof(*t));
  t->nloc = nloc_of(pb);
  t->nv = nv_of(pb->cell_type);
  t->nc = pb->ncomp;
  t->dim = dim_of(pb->cell_type);
  double *pts;
  if (pb->nq_rule > 0) {
    /* an explicit simplex rule (the symmetric rules of Table 2), points stored with zero padding */
    t->nq = pb->nq_rule;
    pts = calloc(3 * (size_t)t->nq, sizeof(double));
    t->w = malloc(sizeof(double) * t->nq);
    if (!pts || !t->w) { free(pts); free_tables(t); return ORC_EMEM; }
    for (int q = 0; q < t->nq; ++q) {
      for (int e = 0; e < t->dim; ++e) pts[3 * q + e] = pb->qpts[(size_t)q * t->dim + e];
      t->w[q] = pb->qw[q];
    }
  } else if (pb->cell_type == ORC_TRI || pb->cell_type == ORC_QUAD) {
    /* points stored with a zero z coordinate */
    int m = pb->cell_type == ORC_TRI ? (pb->qdeg + 2) / 2 : pb->qdeg;
    if (m > 64) return ORC_EARG;
    t->nq = m * m;
    pts = calloc(3 * (size_t)t->nq, sizeof(double));
    t->w = malloc(sizeof(double) * t->nq);
    double *p2 = malloc(sizeof(double) * 2 * t->nq);
    if (!pts || !t->w || !p2) { free(pts); free(p2); free_tables(t); return ORC_EMEM; }
    if (pb->cell_type == ORC_TRI) {
      orc_tri_rule(pb->qdeg, p2, t->w);
    } else {
      double x1[64], w1[64];
      orc_gauss_legendre(m, x1, w1);
      for (int j = 0; j < m; ++j)
        for (int i = 0; i < m; ++i) {
          p2[2 * (i + m * j)] = x1[i];
          p2[2 * (i + m * j) + 1] = x1[j];
          t->w[i + m * j] = w1[i] * w1[j];
        }
    }
    for (int q = 0; q < t->nq; ++q) {
      pts[3 * q] = p2[2 * q];
      pts[3 * q + 1] = p2[2 * q + 1];
    }
    free(p2);
  } else if (pb->cell_type == ORC_TET) {
    int m = (pb->qdeg + 2) / 2;
    t->nq = m * m * m;
    pts = malloc(sizeof(double) * 3 * t->nq);
    t->w = malloc(sizeof(double) * t->nq);
    if (!pts || !t->w) { free(pts); free_tables(t); return ORC_EMEM; }
    orc_tet_rule(pb->qdeg, pts, t->w);
  } else {
    int m = pb->qdeg;
    t->nq = m * m * m;
    double x1[64], w1[64];
    if (m > 64) return ORC_EARG;
    orc_gauss_legendre(m, x1, w1);
    pts = malloc(sizeof(double) * 3 * t->nq);
    t->w = malloc(sizeof(double) * t->nq);
    if (!pts || !t->w) { free(pts); free_tables(t); return ORC_EMEM; }
    for (int k = 0; k < m; ++k)
      for (int j = 0; j < m; ++j)
        for (int i = 0; i < m; ++i) {
          int q = i + m * (j + m * k);
          pts[3 * q + 0] = x1[i];
          pts[3 * q + 1] = x1[j];
          pts[3 * q + 2] = x1[k];
          t->w[q] = w1[i] * w1[j] * w1[k];
        }
  }
  t->phi = malloc(sizeof(double) * t->nq * t->nloc);
  t->dphi = malloc(sizeof(double) * t->nq * t->nloc * 3);
  t->dN = malloc(sizeof(double) * t->nq * t->nv * 3);
  if (!t->phi || !t->dphi || !t->dN) { free(pts); free_tables(t); return ORC_EMEM; }
  for (int q = 0; q < t->nq; ++q) {
    const double *xq = pts + 3 * q;
    double Nv[8], dNv[24];
    if (t->dim == 2) {
      /* 2D: basis and coordinate-map gradients with a zero z component */
      double phi2[64 * 64], dphi2[2 * 64 * 64], N2[4], dN2[8];
      if (pb->cell_type == ORC_TRI) {
        orc_tri_basis(pb->degree, xq, phi2, dphi2);
        orc_tri_basis(1, xq, N2, dN2);
      } else {
        orc_quad_basis(pb->degree, xq, phi2, dphi2);
        orc_quad_basis(1, xq, N2, dN2);
      }
      for (int a = 0; a < t->nloc; ++a) {
        t->phi[q * t->nloc + a] = phi2[a];
        t->dphi[(q * t->nloc + a) * 3 + 0] = dphi2[2 * a];
        t->dphi[(q * t->nloc + a) * 3 + 1] = dphi2[2 * a + 1];
        t->dphi[(q * t->nloc + a) * 3 + 2] = 0.0;
      }
      for (int v = 0; v < t->nv; ++v) {
        dNv[3 * v] = dN2[2 * v];
        dNv[3 * v + 1] = dN2[2 * v + 1];
        dNv[3 * v + 2] = 0.0;
      }
      memcpy(t->dN + q * t->nv * 3, dNv, sizeof(double) * t->nv * 3);
      continue;
    }
    if (pb->cell_type == ORC_TET) {
      orc_tet_basis(pb->degree, xq, t->phi + q * t->nloc, t->dphi + q * t->nloc * 3);
      orc_tet_basis(1, xq, Nv, dNv);
    } else {
      orc_hex_basis(pb->degree, pb->equispaced, xq, t->phi + q * t->nloc, t->dphi + q * t->nloc * 3);
      orc_hex_basis(1, 1, xq, Nv, dNv); /* trilinear map: Q1 on the cell corners */
    }
    memcpy(t->dN + q * t->nv * 3, dNv, sizeof(double) * t->nv * 3);
  }
  free(pts);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Constitutive laws (Supplementary material; neo-Hookean: textbook)    */
/* ------------------------------------------------------------------ */

static double det3(const double A[3][3]) {
  return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
         A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
         A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

/* Inverse by the adjugate: inv[i][j] = cof[j][i] / det. */
static void inv3(const double A[3][3], double det, double inv[3][3]) {
  inv[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / det;
  inv[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
  inv[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
  inv[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / det;
  inv[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
  inv[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
  inv[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / det;
  inv[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
  inv[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
}

static void matmul(const double A[3][3], const double B[3][3], double C[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[i][k] * B[k][j];
      C[i][j] = s;
    }
}

static void transpose(const double A[3][3], double T[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) T[i][j] = A[j][i];
}

/* St Venant-Kirchhoff: E = (F^T F - I)/2, S = dPsi/dE = lambda tr(E) I + 2 mu E, P = F S. */
static void svk_stress(const double F[3][3], double lam, double mu, double P[3][3], double S[3][3]) {
  double Ft[3][3], C[3][3], E[3][3];
  transpose(F, Ft);
  matmul(Ft, F, C);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) E[i][j] = 0.5 * (C[i][j] - (i == j ? 1.0 : 0.0));
  double tr = E[0][0] + E[1][1] + E[2][2];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) S[i][j] = 2.0 * mu * E[i][j] + (i == j ? lam * tr : 0.0);
  matmul(F, S, P);
}

static double svk_energy(const double F[3][3], double lam, double mu) {
  double Ft[3][3], C[3][3], E[3][3];
  transpose(F, Ft);
  matmul(Ft, F, C);
  double tr = 0.0, ee = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) E[i][j] = 0.5 * (C[i][j] - (i == j ? 1.0 : 0.0));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) ee += E[i][j] * E[j][i];
  for (int i = 0; i < 3; ++i) tr += E[i][i];
  return 0.5 * lam * tr * tr + mu * ee;
}

/* dP = dF S + F dS with dE = sym(F^T dF), dS = lambda tr(dE) I + 2 mu dE. */
static void svk_dstress(const double F[3][3], const double dF[3][3], double lam, double mu, double dP[3][3]) {
  double P[3][3], S[3][3], Ft[3][3], FtdF[3][3], dE[3][3], dS[3][3], t1[3][3], t2[3][3];
  svk_stress(F, lam, mu, P, S);
  transpose(F, Ft);
  matmul(Ft, dF, FtdF);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) dE[i][j] = 0.5 * (FtdF[i][j] + FtdF[j][i]);
  double tr = dE[0][0] + dE[1][1] + dE[2][2];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) dS[i][j] = 2.0 * mu * dE[i][j] + (i == j ? lam * tr : 0.0);
  matmul(dF, S, t1);
  matmul(F, dS, t2);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) dP[i][j] = t1[i][j] + t2[i][j];
}

/* Compressible neo-Hookean: Psi = mu/2 (tr C - 3) - mu ln J + lambda/2 (ln J)^2,
 * P = mu (F - F^{-T}) + lambda ln J F^{-T}. */
static int nh_stress(const double F[3][3], double lam, double mu, double P[3][3]) {
  double J = det3(F);
  if (!(J > 0.0)) return ORC_EJAC;
  double Fi[3][3];
  inv3(F, J, Fi);
  double lnJ = log(J);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) P[i][j] = mu * (F[i][j] - Fi[j][i]) + lam * lnJ * Fi[j][i];
  return 0;
}

static int nh_energy(const double F[3][3], double lam, double mu, double *psi) {
  double J = det3(F);
  if (!(J > 0.0)) return ORC_EJAC;
  double trC = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) trC += F[i][j] * F[i][j];
  double lnJ = log(J);
  *psi = 0.5 * mu * (trC - 3.0) - mu * lnJ + 0.5 * lam * lnJ * lnJ;
  return 0;
}

/* dP = mu dF + (mu - lambda ln J) F^{-T} dF^T F^{-T} + lambda tr(F^{-1} dF) F^{-T}. */
static int nh_dstress(const double F[3][3], const double dF[3][3], double lam, double mu, double dP[3][3]) {
  double J = det3(F);
  if (!(J > 0.0)) return ORC_EJAC;
  double Fi[3][3], FiT[3][3], dFt[3][3], t1[3][3], t2[3][3], FidF[3][3];
  inv3(F, J, Fi);
  transpose(Fi, FiT);
  transpose(dF, dFt);
  matmul(FiT, dFt, t1);
  matmul(t1, FiT, t2);
  matmul(Fi, dF, FidF);
  double tr = FidF[0][0] + FidF[1][1] + FidF[2][2];
  double lnJ = log(J);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) dP[i][j] = mu * dF[i][j] + (mu - lam * lnJ) * t2[i][j] + lam * tr * FiT[i][j];
  return 0;
}

/* ------------------------------------------------------------------ */
/* Local kernel                                                         */
/* ------------------------------------------------------------------ */

/* Geometry at quadrature point q: J[i][j] = dx_i/dxi_j = sum_v X_v[i] dN_v/dxi_j. */
static int geometry(const tables *t, int q, const double *X, double *wdet, double Jinv[3][3]) {
  double J[3][3] = {{0}};
  const double *dN = t->dN + q * t->nv * 3;
  for (int v = 0; v < t->nv; ++v)
    for (int i = 0; i < t->dim; ++i)
      for (int j = 0; j < 3; ++j) J[i][j] += X[3 * v + i] * dN[3 * v + j];
  if (t->dim == 2) J[2][2] = 1.0; /* the plane: no z dependence */
  double det = det3(J);
  if (!(det != 0.0) || !isfinite(det)) return ORC_EDET;
  inv3(J, det, Jinv);
  *wdet = t->w[q] * fabs(det);
  return 0;
}

/* y_loc = local action on cell c.  xl, ul, yl are [nloc][nc]. */
static int cell_kernel(const orc_problem *pb, const tables *t, const double *X, const double *xl,
                       const double *ul, double *yl, double *grad /* [nloc][3] scratch */) {
  const int nl = t->nloc, nc = t->nc;
  for (int i = 0; i < nl * nc; ++i) yl[i] = 0.0;
  for (int q = 0; q < t->nq; ++q) {
    double wdet, Jinv[3][3];
    int rc = geometry(t, q, X, &wdet, Jinv);
    if (rc) return rc;
    const double *phi = t->phi + q * nl;
    const double *dphi = t->dphi + q * nl * 3;
    /* physical gradients: grad phi_a = J^{-T} grad_ref phi_a */
    for (int a = 0; a < nl; ++a)
      for (int j = 0; j < 3; ++j)
        grad[3 * a + j] = dphi[3 * a + 0] * Jinv[0][j] + dphi[3 * a + 1] * Jinv[1][j] + dphi[3 * a + 2] * Jinv[2][j];
    /* change of basis: dofs -> value and gradient at the point */
    double u[3] = {0}, gu[3][3] = {{0}}, gc[3][3] = {{0}};
    for (int a = 0; a < nl; ++a)
      for (int c = 0; c < nc; ++c) {
        u[c] += phi[a] * xl[a * nc + c];
        for (int j = 0; j < 3; ++j) gu[c][j] += xl[a * nc + c] * grad[3 * a + j];
      }
    if (pb->kind == ORC_HYPER_JAC)
      for (int a = 0; a < nl; ++a)
        for (int c = 0; c < nc; ++c)
          for (int j = 0; j < 3; ++j) gc[c][j] += ul[a * nc + c] * grad[3 * a + j];
    /* integrand: f0 multiplies the test value, f1 the test gradient */
    double f0[3] = {0}, f1[3][3] = {{0}};
    switch (pb->kind) {
      case ORC_MASS:
        for (int c = 0; c < nc; ++c) f0[c] = u[c];
        break;
      case ORC_LAPLACE:
        for (int c = 0; c < nc; ++c)
          for (int j = 0; j < 3; ++j) f1[c][j] = gu[c][j];
        break;
      case ORC_HELMHOLTZ:
        for (int c = 0; c < nc; ++c) {
          f0[c] = pb->k2 * u[c];
          for (int j = 0; j < 3; ++j) f1[c][j] = gu[c][j];
        }
        break;
      case ORC_ELASTICITY: {
        double tr = gu[0][0] + gu[1][1] + gu[2][2];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j)
            f1[i][j] = pb->mu * (gu[i][j] + gu[j][i]) + (i == j ? pb->lambda * tr : 0.0);
        break;
      }
      case ORC_HYPER_RES: {
        double F[3][3], P[3][3], S[3][3];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) F[i][j] = (i == j ? 1.0 : 0.0) + gu[i][j];
        if (pb->law == ORC_SVK) svk_stress(F, pb->lambda, pb->mu, P, S);
        else if ((rc = nh_stress(F, pb->lambda, pb->mu, P))) return rc;
        for (int i = 0; i < 3; ++i) {
          f0[i] = -pb->b[i];
          for (int j = 0; j < 3; ++j) f1[i][j] = P[i][j];
        }
        break;
      }
      case ORC_HYPER_JAC: {
        double F[3][3], dP[3][3];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) F[i][j] = (i == j ? 1.0 : 0.0) + gc[i][j];
        if (pb->law == ORC_SVK) svk_dstress(F, gu, pb->lambda, pb->mu, dP);
        else if ((rc = nh_dstress(F, gu, pb->lambda, pb->mu, dP))) return rc;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) f1[i][j] = dP[i][j];
        break;
      }
      default:
        return ORC_EARG;
    }
    for (int a = 0; a < nl; ++a)
      for (int c = 0; c < nc; ++c) {
        double s = f0[c] * phi[a];
        for (int j = 0; j < 3; ++j) s += f1[c][j] * grad[3 * a + j];
        yl[a * nc + c] += wdet * s;
      }
  }
  return 0;
}

static void gather(const orc_problem *pb, const tables *t, int64_t c, const double *x, double *X,
                   double *xl, double *ul) {
  for (int v = 0; v < t->nv; ++v) {
    int64_t id = pb->cell_vert[c * t->nv + v];
    for (int d = 0; d < 3; ++d) X[3 * v + d] = pb->coords[3 * id + d];
  }
  for (int a = 0; a < t->nloc; ++a) {
    int64_t node = pb->cell_node[c * t->nloc + a];
    for (int k = 0; k < t->nc; ++k) {
      xl[a * t->nc + k] = x[node * t->nc + k];
      if (ul) ul[a * t->nc + k] = pb->ucoef[node * t->nc + k];
    }
  }
}

int orc_apply(const orc_problem *pb, const double *x, double *y, const int64_t *cells, int64_t ncells) {
  int rc = check_problem(pb);
  if (rc) return rc;
  if (!x || !y) return ORC_EARG;
  if (cells)
    for (int64_t i = 0; i < ncells; ++i)
      if (cells[i] < 0 || cells[i] >= pb->ncell) return ORC_EARG;
  tables t;
  if ((rc = build_tables(pb, &t))) return rc;
  const int nl = t.nloc, nc = t.nc;
  double *xl = malloc(sizeof(double) * nl * nc), *ul = malloc(sizeof(double) * nl * nc);
  double *yl = malloc(sizeof(double) * nl * nc), *grad = malloc(sizeof(double) * nl * 3);
  if (!xl || !ul || !yl || !grad) { rc = ORC_EMEM; goto done; }
  memset(y, 0, sizeof(double) * pb->nnode * nc);
  int64_t n = cells ? ncells : pb->ncell;
  for (int64_t i = 0; i < n; ++i) {
    int64_t c = cells ? cells[i] : i;
    double X[24];
    gather(pb, &t, c, x, X, xl, pb->kind == ORC_HYPER_JAC ? ul : NULL);
    if ((rc = cell_kernel(pb, &t, X, xl, ul, yl, grad))) goto done;
    for (int a = 0; a < nl; ++a) {
      int64_t node = pb->cell_node[c * nl + a];
      for (int k = 0; k < nc; ++k) y[node * nc + k] += yl[a * nc + k];
    }
  }
done:
  free(xl); free(ul); free(yl); free(grad);
  free_tables(&t);
  return rc;
}

int orc_element_matrix(const orc_problem *pb, int64_t cell, double *A) {
  int rc = check_problem(pb);
  if (rc) return rc;
  if (!A || cell < 0 || cell >= pb->ncell || pb->kind == ORC_HYPER_RES) return ORC_EARG;
  tables t;
  if ((rc = build_tables(pb, &t))) return rc;
  const int nl = t.nloc, nc = t.nc, m = nl * nc;
  double *xl = calloc(m, sizeof(double)), *ul = calloc(m, sizeof(double));
  double *yl = malloc(sizeof(double) * m), *grad = malloc(sizeof(double) * nl * 3);
  double *zero = calloc((size_t)pb->nnode * nc + 1, sizeof(double));
  double X[24];
  if (!xl || !ul || !yl || !grad || !zero) { rc = ORC_EMEM; goto done; }
  gather(pb, &t, cell, zero, X, xl, pb->kind == ORC_HYPER_JAC ? ul : NULL);
  for (int j = 0; j < m; ++j) {
    for (int i = 0; i < m; ++i) xl[i] = (i == j) ? 1.0 : 0.0;
    if ((rc = cell_kernel(pb, &t, X, xl, ul, yl, grad))) goto done;
    for (int i = 0; i < m; ++i) A[i * m + j] = yl[i];
  }
done:
  free(xl); free(ul); free(yl); free(grad); free(zero);
  free_tables(&t);
  return rc;
}

int orc_energy(const orc_problem *pb, const double *u, double *energy) {
  int rc = check_problem(pb);
  if (rc) return rc;
  if (!u || !energy || pb->ncomp != dim_of(pb->cell_type)) return ORC_EARG;
  tables t;
  if ((rc = build_tables(pb, &t))) return rc;
  const int nl = t.nloc, nc = t.nc;
  double *xl = malloc(sizeof(double) * nl * 3), *grad = malloc(sizeof(double) * nl * 3);
  double total = 0.0;
  if (!xl || !grad) { rc = ORC_EMEM; goto done; }
  for (int64_t c = 0; c < pb->ncell; ++c) {
    double X[24];
    gather(pb, &t, c, u, X, xl, NULL);
    for (int q = 0; q < t.nq; ++q) {
      double wdet, Jinv[3][3];
      if ((rc = geometry(&t, q, X, &wdet, Jinv))) goto done;
      const double *phi = t.phi + q * nl;
      const double *dphi = t.dphi + q * nl * 3;
      double uq[3] = {0}, F[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
      for (int a = 0; a < nl; ++a) {
        double g[3];
        for (int j = 0; j < 3; ++j)
          g[j] = dphi[3 * a + 0] * Jinv[0][j] + dphi[3 * a + 1] * Jinv[1][j] + dphi[3 * a + 2] * Jinv[2][j];
        for (int cc = 0; cc < nc; ++cc) {
          uq[cc] += phi[a] * xl[nc * a + cc];
          for (int j = 0; j < 3; ++j) F[cc][j] += xl[nc * a + cc] * g[j];
        }
      }
      double psi;
      if (pb->law == ORC_SVK) psi = svk_energy(F, pb->lambda, pb->mu);
      else if ((rc = nh_energy(F, pb->lambda, pb->mu, &psi))) goto done;
      total += wdet * (psi - (pb->b[0] * uq[0] + pb->b[1] * uq[1] + pb->b[2] * uq[2]));
    }
  }
  *energy = total;
done:
  free(xl); free(grad);
  free_tables(&t);
  return rc;
}
