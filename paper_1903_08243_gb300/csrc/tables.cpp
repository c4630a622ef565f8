// Quadrature rules and basis tabulations of the library, built on the host in
// FP64.
//
// Gauss rules follow Golub and Welsch (1969): the points are the eigenvalues
// of the symmetric tridiagonal Jacobi matrix of the weight, here found by
// Sturm-sequence bisection, and each weight is mu0 times the squared first
// component of the normalised eigenvector, here obtained from the
// eigenvector's three-term recurrence.  Lagrange bases use the barycentric
// formulas (Berrut and Trefethen, 2004).  The reference-tetrahedron basis
// uses the closed forms of P1/P2 in barycentric coordinates.
#include <cmath>
#include <cstring>

#include "mfa_internal.h"

namespace mfa {

namespace {

// Recurrence coefficients of the orthonormal Jacobi polynomials for the
// weight (1-t)^alpha (1+t)^beta on [-1,1]: diagonal a_k, squared off-diagonal b_k.
void jacobi_coefficients(int n, double alpha, double beta, double* a, double* b, double* mu0) {
  const double ab = alpha + beta;
  for (int k = 0; k < n; ++k) {
    if (k == 0) {
      a[k] = (beta - alpha) / (ab + 2.0);
    } else {
      const double c = 2.0 * k + ab;
      a[k] = (beta * beta - alpha * alpha) / (c * (c + 2.0));
    }
  }
  b[0] = 0.0;
  for (int k = 1; k < n; ++k) {
    const double c = 2.0 * k + ab;
    b[k] = 4.0 * k * (k + alpha) * (k + beta) * (k + ab) / (c * c * (c + 1.0) * (c - 1.0));
  }
  *mu0 = std::pow(2.0, ab + 1.0) * std::tgamma(alpha + 1.0) * std::tgamma(beta + 1.0) / std::tgamma(ab + 2.0);
}

// Number of eigenvalues of the Jacobi matrix that are < x (Sturm sequence).
int sturm_count(int n, const double* a, const double* b, double x) {
  int count = 0;
  double q = a[0] - x;
  if (q < 0.0) ++count;
  for (int k = 1; k < n; ++k) {
    if (q == 0.0) q = 1e-300;
    q = a[k] - x - b[k] / q;
    if (q < 0.0) ++count;
  }
  return count;
}

// Golub-Welsch rule on [-1,1] for the Jacobi weight.
void gauss_jacobi_pm1(int n, double alpha, double beta, double* t, double* w) {
  double a[kMaxN + 2], b[kMaxN + 2], mu0;
  jacobi_coefficients(n, alpha, beta, a, b, &mu0);
  for (int k = 0; k < n; ++k) {
    // k-th smallest eigenvalue: the smallest x with count(x) > k, by bisection
    double lo = -1.0, hi = 1.0;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (sturm_count(n, a, b, mid) > k) hi = mid;
      else lo = mid;
    }
    const double lam = 0.5 * (lo + hi);
    // eigenvector components v_j = p_j(lam), p_0 = 1,
    // sqrt(b_{j+1}) p_{j+1} = (lam - a_j) p_j - sqrt(b_j) p_{j-1}
    double pm = 0.0, pc = 1.0, norm = 1.0;
    for (int j = 0; j + 1 < n; ++j) {
      const double pn = ((lam - a[j]) * pc - (j > 0 ? std::sqrt(b[j]) * pm : 0.0)) / std::sqrt(b[j + 1]);
      pm = pc;
      pc = pn;
      norm += pn * pn;
    }
    t[k] = lam;
    w[k] = mu0 / norm;
  }
}

}  // namespace

void gauss_jacobi01(int n, int alpha, double* x, double* w) {
  double t[kMaxN + 2], wt[kMaxN + 2];
  gauss_jacobi_pm1(n, (double)alpha, 0.0, t, wt);
  const double scale = std::pow(2.0, -(alpha + 1.0));  // (1-x)^alpha = 2^-alpha (1-t)^alpha, dx = dt/2
  for (int i = 0; i < n; ++i) {
    x[i] = 0.5 * (1.0 + t[i]);
    w[i] = wt[i] * scale;
  }
}

void gauss_legendre01(int n, double* x, double* w) { gauss_jacobi01(n, 0, x, w); }

void gll01(int n, double* x) {
  // interior GLL points: roots of P'_{n-1}, i.e. of the Jacobi polynomial P^{(1,1)}_{n-2}
  x[0] = 0.0;
  x[n - 1] = 1.0;
  if (n > 2) {
    double t[kMaxN + 2], w[kMaxN + 2];
    gauss_jacobi_pm1(n - 2, 1.0, 1.0, t, w);
    for (int i = 0; i < n - 2; ++i) x[i + 1] = 0.5 * (1.0 + t[i]);
  }
}

void lagrange_matrix(int n, const double* nodes, int m, const double* pts, double* L) {
  double lam[kMaxN + 2];
  for (int j = 0; j < n; ++j) {
    double p = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) p *= (nodes[j] - nodes[k]);
    lam[j] = 1.0 / p;
  }
  for (int q = 0; q < m; ++q) {
    int hit = -1;
    for (int j = 0; j < n; ++j)
      if (pts[q] == nodes[j]) hit = j;
    if (hit >= 0) {
      for (int j = 0; j < n; ++j) L[q * n + j] = (j == hit) ? 1.0 : 0.0;
      continue;
    }
    double den = 0.0;
    for (int j = 0; j < n; ++j) den += lam[j] / (pts[q] - nodes[j]);
    for (int j = 0; j < n; ++j) L[q * n + j] = lam[j] / (pts[q] - nodes[j]) / den;
  }
}

void collocation_derivative(int m, const double* pts, double* D) {
  double lam[kMaxN + 2];
  for (int j = 0; j < m; ++j) {
    double p = 1.0;
    for (int k = 0; k < m; ++k)
      if (k != j) p *= (pts[j] - pts[k]);
    lam[j] = 1.0 / p;
  }
  for (int q = 0; q < m; ++q) {
    double diag = 0.0;
    for (int r = 0; r < m; ++r) {
      if (r == q) continue;
      const double v = (lam[r] / lam[q]) / (pts[q] - pts[r]);
      D[q * m + r] = v;
      diag -= v;  // rows of a derivative matrix sum to zero
    }
    D[q * m + q] = diag;
  }
}

int tet_rule_collapsed(int degree, double* pts, double* w) {
  const int m = (degree + 2) / 2;
  double xa[kMaxN], wa[kMaxN], xb[kMaxN], wb[kMaxN], xc[kMaxN], wc[kMaxN];
  gauss_jacobi01(m, 0, xa, wa);
  gauss_jacobi01(m, 1, xb, wb);
  gauss_jacobi01(m, 2, xc, wc);
  int q = 0;
  for (int k = 0; k < m; ++k)
    for (int j = 0; j < m; ++j)
      for (int i = 0; i < m; ++i) {
        const double a = xa[i], b = xb[j], c = xc[k];
        pts[3 * q + 0] = a * (1.0 - b) * (1.0 - c);
        pts[3 * q + 1] = b * (1.0 - c);
        pts[3 * q + 2] = c;
        w[q] = wa[i] * wb[j] * wc[k];
        ++q;
      }
  return q;
}

void tet_basis(int p, const double* xi, double* phi, double* dphi) {
  const double l[4] = {1.0 - xi[0] - xi[1] - xi[2], xi[0], xi[1], xi[2]};
  static const double gl[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  if (p == 1) {
    for (int i = 0; i < 4; ++i) {
      phi[i] = l[i];
      for (int d = 0; d < 3; ++d) dphi[3 * i + d] = gl[i][d];
    }
    return;
  }
  static const int ed[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
  for (int i = 0; i < 4; ++i) {
    phi[i] = l[i] * (2.0 * l[i] - 1.0);
    for (int d = 0; d < 3; ++d) dphi[3 * i + d] = (4.0 * l[i] - 1.0) * gl[i][d];
  }
  for (int e = 0; e < 6; ++e) {
    const int a = ed[e][0], b = ed[e][1];
    phi[4 + e] = 4.0 * l[a] * l[b];
    for (int d = 0; d < 3; ++d) dphi[3 * (4 + e) + d] = 4.0 * (l[b] * gl[a][d] + l[a] * gl[b][d]);
  }
}

int tet_lattice_size(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

// P_p (p >= 3) by Silvester's product formula for the equispaced simplex lattice: node b = (b0, b1, b2, b3),
// b0 + b1 + b2 + b3 = p, has phi_b = prod_s S_{b_s}(l_s) with S_m(l) = prod_{t<m} (p l - t) / (t + 1), l the
// barycentric coordinates (l0 = 1 - x - y - z, l1 = x, l2 = y, l3 = z).  Nodes in lattice order: (i, j, k)/p with
// i = b1 fastest, then j = b2, then k = b3.
void tet_basis_pk(int p, const double* xi, double* phi, double* dphi) {
  const double l[4] = {1.0 - xi[0] - xi[1] - xi[2], xi[0], xi[1], xi[2]};
  static const double gl[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  // S_m(l_s) and its derivative in l_s, m = 0..p
  double S[4][kTetMaxP + 1], dS[4][kTetMaxP + 1];
  for (int s = 0; s < 4; ++s) {
    S[s][0] = 1.0;
    dS[s][0] = 0.0;
    for (int m = 1; m <= p; ++m) {
      const double f = (p * l[s] - (m - 1)) / m;
      S[s][m] = S[s][m - 1] * f;
      dS[s][m] = dS[s][m - 1] * f + S[s][m - 1] * (double)p / m;
    }
  }
  int n = 0;
  for (int k = 0; k <= p; ++k)
    for (int j = 0; j <= p - k; ++j)
      for (int i = 0; i <= p - k - j; ++i) {
        const int b[4] = {p - i - j - k, i, j, k};
        double v = 1.0;
        for (int s = 0; s < 4; ++s) v *= S[s][b[s]];
        phi[n] = v;
        double g[3] = {0.0, 0.0, 0.0};
        for (int s = 0; s < 4; ++s) {
          double prod = dS[s][b[s]];
          for (int r = 0; r < 4; ++r)
            if (r != s) prod *= S[r][b[r]];
          for (int d = 0; d < 3; ++d) g[d] += prod * gl[s][d];
        }
        for (int d = 0; d < 3; ++d) dphi[3 * n + d] = g[d];
        ++n;
      }
}

// Collapsed rule on the reference triangle exact to `degree`: (a, b) -> (a (1 - b), b), the Jacobian (1 - b) in the
// Jacobi weight of the b direction.  pts [nq][2].
int tri_rule_collapsed(int degree, double* pts, double* w) {
  const int m = (degree + 2) / 2;
  double xa[kMaxN], wa[kMaxN], xb[kMaxN], wb[kMaxN];
  gauss_jacobi01(m, 0, xa, wa);
  gauss_jacobi01(m, 1, xb, wb);
  int q = 0;
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < m; ++i) {
      pts[2 * q + 0] = xa[i] * (1.0 - xb[j]);
      pts[2 * q + 1] = xb[j];
      w[q] = wa[i] * wb[j];
      ++q;
    }
  return q;
}

int tri_lattice_size(int p) { return (p + 1) * (p + 2) / 2; }

// P_p on the equispaced triangle lattice by Silvester's product formula, nodes (i, j)/p with i fastest; barycentric
// l0 = 1 - x - y, l1 = x, l2 = y; dphi [n][2].
void tri_basis_pk(int p, const double* xi, double* phi, double* dphi) {
  const double l[3] = {1.0 - xi[0] - xi[1], xi[0], xi[1]};
  static const double gl[3][2] = {{-1, -1}, {1, 0}, {0, 1}};
  double S[3][kTetMaxP + 1], dS[3][kTetMaxP + 1];
  for (int s = 0; s < 3; ++s) {
    S[s][0] = 1.0;
    dS[s][0] = 0.0;
    for (int m = 1; m <= p; ++m) {
      const double f = (p * l[s] - (m - 1)) / m;
      S[s][m] = S[s][m - 1] * f;
      dS[s][m] = dS[s][m - 1] * f + S[s][m - 1] * (double)p / m;
    }
  }
  int n = 0;
  for (int j = 0; j <= p; ++j)
    for (int i = 0; i <= p - j; ++i) {
      const int b[3] = {p - i - j, i, j};
      phi[n] = S[0][b[0]] * S[1][b[1]] * S[2][b[2]];
      double g[2] = {0.0, 0.0};
      for (int s = 0; s < 3; ++s) {
        double prod = dS[s][b[s]];
        for (int r = 0; r < 3; ++r)
          if (r != s) prod *= S[r][b[r]];
        g[0] += prod * gl[s][0];
        g[1] += prod * gl[s][1];
      }
      dphi[2 * n] = g[0];
      dphi[2 * n + 1] = g[1];
      ++n;
    }
}

}  // namespace mfa
