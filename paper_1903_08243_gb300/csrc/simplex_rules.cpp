// Fully symmetric quadrature rules on the reference triangle and tetrahedron,
// with the point counts of Table 2: 1, 3, 6, 12 (triangle) and 1, 4, 14, 24
// (tetrahedron) for exactness degree 1, 2, 4, 6 (3 and 5 take the next rule).
// The paper prints no points, so the rules are derived here from their
// definition, once per process.
//
// A fully symmetric rule is a union of orbits of the permutations of the
// barycentric coordinates, one weight per orbit:
//   tet  S31 (a,a,a,1-3a): 4 points, S22 (a,a,1/2-a,1/2-a): 6, S211 (a,a,b,1-2a-b): 12
//   tri  S21 (a,a,1-2a): 3 points, S111 (a,b,1-a-b): 6
// with structures  tet: S31 (4), 2 S31 + S22 (14), 3 S31 + S211 (24);
//                  tri: S21 (3), 2 S21 (6), 2 S21 + S111 (12).
// The rule is exact to degree d when it integrates every monomial
// x^i y^j z^k, i + j + k <= d, exactly; the mean of such a monomial over the
// reference simplex is i! j! k! dim! / (i + j + k + dim)!.  The weights and
// orbit parameters solve these equations in the least-squares sense by
// variable projection: the equations are linear in the weights, which are the
// least-squares fit of the current points, and a damped Gauss-Newton
// (Levenberg-Marquardt) iteration on the analytic Jacobian moves the orbit
// parameters from pseudo-random starts inside the simplex, in double; the rule
// taken is then polished by Gauss-Newton on weights and positions together in
// long double.
// Admissible solutions have positive weights and every point
// strictly inside; of those the rule whose smallest barycentric coordinate is
// largest (points farthest from the boundary) is taken.  That choice only
// matters for the 12-point triangle rule, whose moment equations have two
// admissible solutions, and the 3-point one, whose other solution is the edge
// midpoints.  Each tetrahedral structure has a single admissible solution
// (thousands of starts find no other), so its search ends at the first.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <map>
#include <mutex>
#include <vector>

#include "mfa_internal.h"

namespace mfa {

namespace {

using real = long double;

enum OrbitKind { kCentroid, kS31, kS22, kS211, kS21, kS111 };

int nparam_of(OrbitKind k) { return k == kS211 || k == kS111 ? 2 : (k == kCentroid ? 0 : 1); }

// Class of each barycentric slot in the first arrangement of the orbit (the
// other points are the distinct rearrangements).
std::vector<int> pattern_of(OrbitKind k, int dim) {
  switch (k) {
    case kS31: return {0, 0, 0, 1};
    case kS22: return {0, 0, 1, 1};
    case kS211: return {0, 0, 1, 2};
    case kS21: return {0, 0, 1};
    case kS111: return {0, 1, 2};
    default: return std::vector<int>(dim + 1, 0);
  }
}

// The class values as affine functions of the orbit parameters:
// value[c] = base[c] + slope[c][0] x0 + slope[c][1] x1.
void class_affine(OrbitKind k, int dim, real base[3], real slope[3][2]) {
  for (int c = 0; c < 3; ++c) base[c] = slope[c][0] = slope[c][1] = 0;
  switch (k) {
    case kCentroid: base[0] = 1.0L / (dim + 1); break;
    case kS31: slope[0][0] = 1; base[1] = 1; slope[1][0] = -3; break;
    case kS22: slope[0][0] = 1; base[1] = 0.5L; slope[1][0] = -1; break;
    case kS211: slope[0][0] = 1; slope[1][1] = 1; base[2] = 1; slope[2][0] = -2; slope[2][1] = -1; break;
    case kS21: slope[0][0] = 1; base[1] = 1; slope[1][0] = -2; break;
    case kS111: slope[0][0] = 1; slope[1][1] = 1; base[2] = 1; slope[2][0] = -1; slope[2][1] = -1; break;
  }
}

// The degree each structure is solved for: the 14-point tet rule is exact to
// degree 5 and the 6-point triangle rule to degree 4, and requests of a lower
// degree take them (the moment equations of a lower degree would leave a
// family of solutions).
int design_degree(int dim, int degree) {
  if (degree <= 1) return 1;
  if (degree == 2) return 2;
  if (dim == 3) return degree <= 5 ? 5 : 6;
  return degree <= 4 ? 4 : 6;
}

std::vector<OrbitKind> structure_of(int dim, int degree) {
  if (degree <= 1) return {kCentroid};
  if (dim == 3) {
    if (degree == 2) return {kS31};
    if (degree <= 5) return {kS31, kS31, kS22};
    if (degree == 6) return {kS31, kS31, kS31, kS211};
  } else {
    if (degree == 2) return {kS21};
    if (degree <= 4) return {kS21, kS21};
    if (degree <= 6) return {kS21, kS21, kS111};
  }
  return {};
}

struct System {
  int dim = 0, norb = 0, npar = 0, degree = 0;
  std::vector<OrbitKind> orbits;
  std::vector<int> par_off;                 // first parameter of each orbit
  std::vector<int> owner;                   // orbit of each point
  std::vector<std::array<int, 4>> slot_cls; // class of each barycentric slot of each point
  std::vector<std::array<int, 3>> expo;     // monomial exponents
  std::vector<real> mean;                   // monomial means over the simplex

  int nunk() const { return norb + npar; }
  int neq() const { return (int)expo.size(); }
  int npts() const { return (int)owner.size(); }

  // barycentric coordinates of every point and their parameter derivatives
  template <class T>
  void points(const T* par, std::vector<std::array<T, 4>>& lam, std::vector<std::array<std::array<T, 2>, 4>>& dlam) const {
    lam.resize(npts());
    dlam.resize(npts());
    for (int p = 0; p < npts(); ++p) {
      const int o = owner[p];
      real base[3], slope[3][2];
      class_affine(orbits[o], dim, base, slope);
      const T* x = par + par_off[o];
      const int np = nparam_of(orbits[o]);
      for (int s = 0; s <= dim; ++s) {
        const int c = slot_cls[p][s];
        T v = (T)base[c];
        for (int j = 0; j < np; ++j) v += (T)slope[c][j] * x[j];
        lam[p][s] = v;
        dlam[p][s][0] = np > 0 ? (T)slope[c][0] : T(0);
        dlam[p][s][1] = np > 1 ? (T)slope[c][1] : T(0);
      }
    }
  }

  // residual r[q] and (if J) the Jacobian J[q][u], u = (orbit weights, parameters)
  template <class T>
  void eval(const T* u, std::vector<T>& r, std::vector<T>* J) const {
    std::vector<std::array<T, 4>> lam;
    std::vector<std::array<std::array<T, 2>, 4>> dlam;
    points(u + norb, lam, dlam);
    // powers of the reference coordinates (the barycentric coordinates of vertices 1..dim)
    std::vector<T> pw((size_t)npts() * 3 * (degree + 1));
    auto P = [&](int p, int i, int e) -> T& { return pw[((size_t)p * 3 + i) * (degree + 1) + e]; };
    for (int p = 0; p < npts(); ++p)
      for (int i = 0; i < dim; ++i) {
        P(p, i, 0) = T(1);
        for (int e = 1; e <= degree; ++e) P(p, i, e) = P(p, i, e - 1) * lam[p][i + 1];
      }
    r.assign(neq(), T(0));
    if (J) J->assign((size_t)neq() * nunk(), T(0));
    for (int q = 0; q < neq(); ++q) {
      const auto& ex = expo[q];
      T acc = -(T)mean[q];
      T* row = J ? J->data() + (size_t)q * nunk() : nullptr;
      for (int p = 0; p < npts(); ++p) {
        T m = T(1);
        for (int i = 0; i < dim; ++i) m *= P(p, i, ex[i]);
        const int o = owner[p];
        acc += u[o] * m;
        if (!row) continue;
        row[o] += m;
        T dm[3];
        for (int i = 0; i < dim; ++i) {
          T d = ex[i] > 0 ? T(ex[i]) * P(p, i, ex[i] - 1) : T(0);
          for (int k = 0; k < dim; ++k)
            if (k != i) d *= P(p, k, ex[k]);
          dm[i] = d;
        }
        for (int j = 0; j < nparam_of(orbits[o]); ++j) {
          T g = T(0);
          for (int i = 0; i < dim; ++i) g += dm[i] * dlam[p][i + 1][j];
          row[norb + par_off[o] + j] += u[o] * g;
        }
      }
      r[q] = acc;
    }
  }
};

System make_system(int dim, int degree) {
  System s;
  s.dim = dim;
  s.degree = std::max(degree, 1);
  s.orbits = structure_of(dim, degree);
  s.norb = (int)s.orbits.size();
  for (int o = 0; o < s.norb; ++o) {
    s.par_off.push_back(s.npar);
    s.npar += nparam_of(s.orbits[o]);
    std::vector<int> pat = pattern_of(s.orbits[o], dim);
    std::sort(pat.begin(), pat.end());
    do {  // every distinct arrangement of the class pattern is one point
      std::array<int, 4> cls{0, 0, 0, 0};
      for (int i = 0; i <= dim; ++i) cls[i] = pat[i];
      s.owner.push_back(o);
      s.slot_cls.push_back(cls);
    } while (std::next_permutation(pat.begin(), pat.end()));
  }
  auto fact = [](int n) {
    real f = 1;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
  };
  for (int k = 0; k <= (dim == 3 ? degree : 0); ++k)
    for (int j = 0; j + k <= degree; ++j)
      for (int i = 0; i + j + k <= degree; ++i) {
        s.expo.push_back({i, j, k});
        s.mean.push_back(fact(i) * fact(j) * fact(k) * fact(dim) / fact(i + j + k + dim));
      }
  return s;
}

// Solve the n x n system A x = b (Gaussian elimination, partial pivoting).
template <class T>
bool solve_dense(int n, std::vector<T> A, std::vector<T> b, std::vector<T>& x) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)piv * n + c])) piv = r;
    if (!(std::fabs(A[(size_t)piv * n + c]) > T(0))) return false;
    if (piv != c) {
      for (int k = 0; k < n; ++k) std::swap(A[(size_t)c * n + k], A[(size_t)piv * n + k]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < n; ++r) {
      const T f = A[(size_t)r * n + c] / A[(size_t)c * n + c];
      for (int k = c; k < n; ++k) A[(size_t)r * n + k] -= f * A[(size_t)c * n + k];
      b[r] -= f * b[c];
    }
  }
  x.assign(n, T(0));
  for (int r = n - 1; r >= 0; --r) {
    T v = b[r];
    for (int k = r + 1; k < n; ++k) v -= A[(size_t)r * n + k] * x[k];
    x[r] = v / A[(size_t)r * n + r];
  }
  return true;
}

template <class T>
T max_abs(const std::vector<T>& v) {
  T m = T(0);
  for (T x : v) m = std::max(m, (T)std::fabs(x));
  return m;
}

// The weights that best fit the points of u's parameters (normal equations of
// the weight columns V of the Jacobian, which do not depend on the weights):
// written into u.  Also returns the residual and the Jacobian at the result.
template <class T>
bool fit_weights(const System& s, std::vector<T>& u, std::vector<T>& r, std::vector<T>& J) {
  s.eval(u.data(), r, &J);
  const int n = s.nunk(), k = s.norb;
  std::vector<T> A((size_t)k * k), b(k), w;
  for (int a = 0; a < k; ++a) {
    T v = T(0);
    for (int q = 0; q < s.neq(); ++q) v += J[(size_t)q * n + a] * (T)s.mean[q];
    b[a] = v;
    for (int c = 0; c < k; ++c) {
      T m = T(0);
      for (int q = 0; q < s.neq(); ++q) m += J[(size_t)q * n + a] * J[(size_t)q * n + c];
      A[(size_t)a * k + c] = m;
    }
  }
  if (!solve_dense(k, A, b, w)) return false;
  for (int a = 0; a < k; ++a) u[a] = w[a];
  s.eval(u.data(), r, &J);
  return true;
}

// Variable projection (Golub and Pereyra, 1973) with Kaufman's Jacobian: the
// weights are always the least-squares fit of the current points, and a
// damped Gauss-Newton (Levenberg-Marquardt) step moves the orbit parameters
// along the parameter columns of the Jacobian projected off the weight
// columns.  Returns the final max |residual|; a start that is not near a root
// after `give_up` iterations is abandoned.
template <class T>
T levenberg_marquardt(const System& s, std::vector<T>& u, int max_iter, int give_up, T done) {
  const int n = s.nunk(), k = s.norb, np = s.npar, m = s.neq();
  std::vector<T> r, J, rt, Jt;
  if (!fit_weights(s, u, r, J)) return T(1);
  T cost = T(0);
  for (T v : r) cost += v * v;
  T lambda = T(1e-3);
  std::vector<T> K((size_t)m * np), VtV((size_t)k * k), A((size_t)np * np), g(np), dx, col(k), coef;
  for (int it = 0; it < max_iter; ++it) {
    if (max_abs(r) < done) break;
    if (it == give_up && max_abs(r) > T(1e-6)) break;
    // K = D - V (V^T V)^{-1} V^T D, with V the weight columns and D the parameter columns
    for (int a = 0; a < k; ++a)
      for (int c = 0; c < k; ++c) {
        T v = T(0);
        for (int q = 0; q < m; ++q) v += J[(size_t)q * n + a] * J[(size_t)q * n + c];
        VtV[(size_t)a * k + c] = v;
      }
    bool proj_ok = true;
    for (int j = 0; j < np && proj_ok; ++j) {
      for (int a = 0; a < k; ++a) {
        T v = T(0);
        for (int q = 0; q < m; ++q) v += J[(size_t)q * n + a] * J[(size_t)q * n + k + j];
        col[a] = v;
      }
      proj_ok = solve_dense(k, VtV, col, coef);
      for (int q = 0; q < m && proj_ok; ++q) {
        T v = J[(size_t)q * n + k + j];
        for (int a = 0; a < k; ++a) v -= J[(size_t)q * n + a] * coef[a];
        K[(size_t)q * np + j] = v;
      }
    }
    if (!proj_ok) break;
    for (int a = 0; a < np; ++a) {
      T ga = T(0);
      for (int q = 0; q < m; ++q) ga += K[(size_t)q * np + a] * r[q];
      g[a] = -ga;
      for (int b = 0; b < np; ++b) {
        T v = T(0);
        for (int q = 0; q < m; ++q) v += K[(size_t)q * np + a] * K[(size_t)q * np + b];
        A[(size_t)a * np + b] = v;
      }
    }
    bool stepped = false;
    for (int tries = 0; tries < 8 && !stepped; ++tries) {
      std::vector<T> Ad = A;
      for (int a = 0; a < np; ++a) Ad[(size_t)a * np + a] += lambda * (A[(size_t)a * np + a] + T(1e-30));
      if (!solve_dense(np, Ad, g, dx)) {
        lambda *= T(10);
        continue;
      }
      std::vector<T> ut = u;
      for (int a = 0; a < np; ++a) ut[k + a] += dx[a];
      if (!fit_weights(s, ut, rt, Jt)) {
        lambda *= T(4);
        continue;
      }
      T ct = T(0);
      for (T v : rt) ct += v * v;
      if (ct < cost) {
        u.swap(ut);
        r.swap(rt);
        J.swap(Jt);
        cost = ct;
        lambda = std::max(lambda / T(3), T(1e-12));
        stepped = true;
      } else {
        lambda *= T(4);
      }
    }
    if (!stepped) break;
  }
  return max_abs(r);
}

// Undamped Gauss-Newton on weights and positions together: the residual is
// evaluated from u directly, so every step only has to be roughly right and the
// iteration converges to the precision of T (variable projection would refit
// the weights from the normal equations each time, which caps their accuracy
// at cond^2 eps).  Returns the final max |residual|.
template <class T>
T gauss_newton_polish(const System& s, std::vector<T>& u, int iters) {
  const int n = s.nunk(), m = s.neq();
  std::vector<T> r, J, A((size_t)n * n), g(n), du;
  for (int it = 0; it < iters; ++it) {
    s.eval(u.data(), r, &J);
    for (int a = 0; a < n; ++a) {
      T ga = T(0);
      for (int q = 0; q < m; ++q) ga += J[(size_t)q * n + a] * r[q];
      g[a] = -ga;
      for (int b = 0; b < n; ++b) {
        T v = T(0);
        for (int q = 0; q < m; ++q) v += J[(size_t)q * n + a] * J[(size_t)q * n + b];
        A[(size_t)a * n + b] = v;
      }
    }
    if (!solve_dense(n, A, g, du)) break;
    for (int a = 0; a < n; ++a) u[a] += du[a];
  }
  s.eval(u.data(), r, (std::vector<T>*)nullptr);
  return max_abs(r);
}

// SplitMix64 (Steele, Lea and Flood, 2014) as the source of starting points.
struct SplitMix {
  uint64_t s;
  real uniform() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (real)(z >> 11) * (1.0L / 9007199254740992.0L);
  }
};

struct Rule {
  std::vector<double> pts, w;
};

bool derive(int dim, int degree, Rule& out) {
  const System s = make_system(dim, degree);
  if (s.orbits.empty()) return false;
  real fdim = 1;
  for (int i = 2; i <= dim; ++i) fdim *= i;
  if (s.orbits[0] == kCentroid) {
    out.pts.assign(dim, 1.0 / (dim + 1));
    out.w.assign(1, (double)(1 / fdim));
    return true;
  }
  SplitMix rng{0x1903082430000000ULL + 16 * dim + degree};
  const int starts = s.npts() == 24 ? 1200 : 300;
  double best_min = -1;
  std::vector<double> best;
  std::vector<std::array<double, 4>> lam;
  std::vector<std::array<std::array<double, 2>, 4>> dlam;
  for (int t = 0; t < starts; ++t) {
    std::vector<double> u(s.nunk(), 0.0);
    for (int o = 0; o < s.norb; ++o) {  // parameters that keep the orbit inside the simplex
      double* x = u.data() + s.norb + s.par_off[o];
      switch (s.orbits[o]) {
        case kS31: x[0] = (double)rng.uniform() / 3; break;
        case kS22: x[0] = (double)rng.uniform() / 4; break;
        case kS21: x[0] = (double)rng.uniform() / 2; break;
        case kS211: x[0] = (double)rng.uniform() / 2; x[1] = (double)rng.uniform() * (1 - 2 * x[0]); break;
        case kS111: x[0] = (double)rng.uniform(); x[1] = (double)rng.uniform() * (1 - x[0]); break;
        default: break;
      }
    }
    if (levenberg_marquardt(s, u, 100, 30, 1e-15) > 1e-13) continue;
    bool ok = true;
    for (int o = 0; o < s.norb; ++o) ok = ok && u[o] > 0;
    s.points(u.data() + s.norb, lam, dlam);
    double mn = 1;
    for (const auto& l : lam)
      for (int i = 0; i <= dim; ++i) mn = std::min(mn, l[i]);
    if (!ok || mn <= 1e-9) continue;
    if (mn > best_min + 1e-9) {
      best_min = mn;
      best = u;
    }
    if (dim == 3) break;  // the tetrahedral structures have one admissible solution: the first is the rule
  }
  if (best.empty()) return false;
  std::vector<real> ul(best.begin(), best.end());  // polish in extended precision
  // the moment equations of the 24-point rule are ill-conditioned (condition ~4e6): converge in
  // extended precision so that the points are right to well below double rounding
  if (gauss_newton_polish(s, ul, 8) > (real)1e-15L) return false;
  std::vector<std::array<real, 4>> laml;
  std::vector<std::array<std::array<real, 2>, 4>> dlaml;
  s.points(ul.data() + s.norb, laml, dlaml);
  out.pts.clear();
  out.w.clear();
  for (int p = 0; p < s.npts(); ++p) {
    for (int i = 0; i < dim; ++i) out.pts.push_back((double)laml[p][i + 1]);
    out.w.push_back((double)(ul[s.owner[p]] / fdim));
  }
  return true;
}

}  // namespace

int simplex_rule_symmetric(int dim, int degree, std::vector<double>& pts, std::vector<double>& w) {
  if ((dim != 2 && dim != 3) || degree < 0 || degree > 6) return 0;
  static std::mutex mu;
  static std::map<int, Rule> cache;
  std::lock_guard<std::mutex> lock(mu);
  const int design = design_degree(dim, degree);
  const int key = dim * 16 + design;
  auto it = cache.find(key);
  if (it == cache.end()) {
    Rule r;
    if (!derive(dim, design, r)) return -1;
    it = cache.emplace(key, r).first;
  }
  pts = it->second.pts;
  w = it->second.w;
  return (int)w.size();
}

}  // namespace mfa

extern "C" int mfa_simplex_rule(int cell_type, int degree, int max_points, double* pts, double* w, int* nq) {
  if ((cell_type != MFA_CELL_TRI3 && cell_type != MFA_CELL_TET4) || degree < 0 || degree > 6 || !nq ||
      max_points < 0 || (max_points > 0 && (!pts || !w)))
    return mfa::set_error(MFA_ERR_ARG, "mfa_simplex_rule: bad argument");
  const int dim = cell_type == MFA_CELL_TET4 ? 3 : 2;
  std::vector<double> p, wt;
  const int n = mfa::simplex_rule_symmetric(dim, degree, p, wt);
  if (n <= 0) return mfa::set_error(MFA_ERR_UNSUPPORTED, "mfa_simplex_rule: the rule's derivation failed");
  *nq = n;
  if (n > max_points) {
    char msg[96];
    snprintf(msg, sizeof msg, "mfa_simplex_rule: %d points needed", n);
    return mfa::set_error(MFA_ERR_ARG, msg);
  }
  for (int i = 0; i < n * dim; ++i) pts[i] = p[i];
  for (int i = 0; i < n; ++i) w[i] = wt[i];
  return MFA_OK;
}
