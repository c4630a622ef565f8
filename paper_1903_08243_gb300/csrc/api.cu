// C-ABI entry points of the mfa library (declared in include/mfa.h).
//
// The handles mirror the parloop of Section 2.2 of arXiv 1903.08243: a mesh
// holds `coords` and `cell2vert`, a space holds `cell2dof`, a form holds the
// element kernel's tables and stored geometry, and mfa_apply runs the global
// assembly loop on the GPU.
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <algorithm>
#include <vector>

#include "mfa_internal.h"

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

#define MFA_CUDA(call)                                                                          \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) return fail(MFA_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));  \
  } while (0)

int cuda_alloc(void** p, size_t bytes, const char* what) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(MFA_ERR_OOM, "cudaMalloc(%zu) for %s: out of device memory", bytes, what);
  }
  if (e != cudaSuccess) return fail(MFA_ERR_CUDA, "cudaMalloc for %s: %s", what, cudaGetErrorString(e));
  return MFA_OK;
}

int nloc_of(int cell_type, int degree) {
  if (cell_type == MFA_CELL_TET4) {
    if (degree == 1) return 4;
    if (degree == 2) return 10;
    return degree >= 3 && degree <= mfa::kTetMaxP ? mfa::tet_lattice_size(degree) : -1;
  }
  if (cell_type == MFA_CELL_HEX8 && degree >= 1 && degree <= 8) return (degree + 1) * (degree + 1) * (degree + 1);
  if (cell_type == MFA_CELL_TRI3 && degree >= 1 && degree <= mfa::kTetMaxP) return mfa::tri_lattice_size(degree);
  if (cell_type == MFA_CELL_QUAD4 && degree >= 1 && degree <= 8) return (degree + 1) * (degree + 1);
  return -1;
}

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Algorithmic FP operations of one apply (an FMA counts 2), following the
// kernels' arithmetic, which is the operation count of the definitions after
// sum factorisation (hex) or per-point evaluation (tet).
void count_work(mfa_form* f) {
  const mfa_space* sp = f->space;
  const int64_t ncell = sp->mesh->ncell;
  const int64_t ndof = sp->nnode * sp->ncomp;
  const int kind = f->p.kind;
  double per_cell = 0.0, bytes = 0.0;
  double exec_cell = -1.0;  // operations the kernel executes, where fewer than the algorithmic count
  if (mfa::is_planar(sp->mesh->cell_type)) {
    // Planar cells.  Quads: per component B and B^T 2 x 2 (q n^2 + q^2 n), D and D^T 8 q^3 (the Jacobian action
    // also interpolates the linearisation point: 2 (q n^2 + q^2 n) + 4 q^3); per point the pointwise work; scatter
    // adds.  Triangles (dense): per point interpolation 2 (value) + 4 (gradient) per dof and component, test side
    // the same, the pointwise work.  Pointwise: scalar G g 6 + value terms; vector: physical gradient(s) 12 each,
    // the physics (3D laws in plane strain), flux map 13.
    const double nl = sp->nloc, nc = sp->ncomp;
    const bool val = kind == MFA_FORM_MASS || kind == MFA_FORM_HELMHOLTZ, grad = kind != MFA_FORM_MASS;
    const bool jac = kind == MFA_FORM_HYPER_JAC, svk = f->p.law == MFA_LAW_SVK;
    double per_pt;
    if (kind <= MFA_FORM_HELMHOLTZ) per_pt = nc * ((grad ? 6.0 : 0.0) + (val ? 2.0 : 0.0));
    else if (kind == MFA_FORM_ELASTICITY) per_pt = 12.0 + 24.0 + 13.0;
    else if (kind == MFA_FORM_HYPER_RES) per_pt = 12.0 + (svk ? 102.0 : 66.0) + 13.0 + 2.0;
    else per_pt = 24.0 + (svk ? 243.0 : 202.0) + 13.0;
    if (sp->mesh->cell_type == MFA_CELL_QUAD4) {
      const double n = sp->degree + 1, q = f->nq1, bsw = 2.0 * (q * n * n + q * q * n);
      per_cell = nc * (2.0 * bsw + (grad || kind == MFA_FORM_HYPER_RES ? 8.0 * q * q * q : 0.0)) +
                 (jac ? nc * (bsw + 4.0 * q * q * q) : 0.0) + per_pt * q * q + nc * n * n;
      bytes = ncell * (4.0 * n * n + 8.0 * mfa::quad_geom_entries(kind) * q * q);
    } else {
      const double nq = f->nq;
      const bool val_out = val || kind == MFA_FORM_HYPER_RES;
      const double per_q = nl * nc * ((val ? 2.0 : 0.0) + (grad ? 4.0 : 0.0) + (jac ? 4.0 : 0.0)) +
                           nl * nc * ((val_out ? 2.0 : 0.0) + (grad ? 4.0 : 0.0)) + per_pt + 1.0;
      per_cell = nq * per_q + 20.0 + nl * nc;
      bytes = ncell * (4.0 * nl + 12.0) + 24.0 * sp->mesh->nvert;
    }
    if (jac) bytes += 8.0 * ndof;
    bytes += 16.0 * ndof;
    if (f->scatter == MFA_SCATTER_COLOUR) bytes += 4.0 * ncell;
    f->flops = f->flops_executed = per_cell * ncell;
    f->bytes = bytes;
    return;
  }
  if (sp->mesh->cell_type == MFA_CELL_HEX8 && f->launch.variant == MFA_VARIANT_EVEN_ODD) {
    // even-odd line products: per line, forming e/o (2h adds), then per mirror pair of outputs
    // (odd: one multiply) + 2h FMA + 2 adds, and for odd n a middle output
    const int n = sp->degree + 1, h = n / 2, odd = n & 1;
    auto line = [&](int sigma, int acc) {
      double f_ = 2.0 * h + h * (4.0 * h + 2.0 + odd);
      if (odd) f_ += 2.0 * h + (sigma > 0 ? 1.0 : 0.0);
      return f_ + (acc ? n : 0);
    };
    const double L = (double)n * n, P = (double)n * n * n;
    exec_cell = L * 6.0 * line(1, 0) + P;  // B, B^T and the scatter adds
    // D, D^T, G g; the D product along z, fused with B, takes the halves of B's split and forms no e/o of
    // its own (2h flops fewer per line); the fused D^T / B^T pair along z starts its product chains from the
    // accumulator's sum and difference with doubled tables (one addition per half, where three additions
    // were: 4h flops fewer per line, 3h + 1 for odd n, whose middle multiply becomes an FMA and whose middle
    // addition goes into the chain).  Recombining a mirror pair as one FMA instead of two additions changes
    // no flop count.
    if (kind != MFA_FORM_MASS)
      exec_cell += L * (3.0 * line(-1, 0) + 3.0 * line(-1, 1) - 2.0 * h - (odd ? 3.0 * h + 1.0 : 4.0 * h)) + 15.0 * P;
    if (kind != MFA_FORM_LAPLACE) exec_cell += P;  // c0 w|J| u
  }
  if (sp->mesh->cell_type == MFA_CELL_HEX8 && sp->ncomp == 3) {
    // per component: B and B^T sweeps 4 (q n^3 + q^2 n^2 + q^3 n), D and D^T 12 q^4 (the Jacobian action also
    // interpolates the linearisation point's gradient: 2 (q n^3 + q^2 n^2 + q^3 n) + 6 q^4); per point the
    // physical gradient(s) (45 each), the physics and the flux map (54: 9 entries x 5 + w|J|); scatter adds
    // 3 n^3.  Vector Laplacian: three G g products (3 x 15) per point.  q = n for p+1 points.
    const double n = sp->degree + 1, q = f->nq1, PN = n * n * n, PQ = q * q * q;
    const double bsw = 2.0 * (q * n * n * n + q * q * n * n + q * q * q * n);
    const bool jac = kind == MFA_FORM_HYPER_JAC, svk = f->p.law == MFA_LAW_SVK;
    double per_pt = 0.0;
    if (kind == MFA_FORM_LAPLACE) per_pt = 45.0;
    else if (kind == MFA_FORM_ELASTICITY) per_pt = 45.0 + 24.0 + 54.0;
    else if (kind == MFA_FORM_HYPER_RES) per_pt = 45.0 + (svk ? 102.0 : 66.0) + 54.0 + 3.0;
    else per_pt = 90.0 + (svk ? 243.0 : 202.0) + 54.0;
    per_cell = 3.0 * (2.0 * bsw + 12.0 * PQ * q) + (jac ? 3.0 * (bsw + 6.0 * PQ * q) : 0.0) + per_pt * PQ + 3.0 * PN;
    bytes = ncell * (4.0 * PN + 8.0 * mfa::hex_geom_entries(kind) * PQ);
    if (jac) bytes += 8.0 * ndof;
  } else if (sp->mesh->cell_type == MFA_CELL_HEX8) {
    // algorithmic count of collocation sum factorisation, whatever the kernel variant:
    // 24 n^4 for n = nq (B, B^T, D, D^T sweeps) + pointwise physics + scatter adds
    const double n = sp->degree + 1, q = f->nq1;
    const double sweeps = 2.0 * (q * n * n * n + q * q * n * n + q * q * q * n);  // one direction set
    per_cell = 2.0 * sweeps + n * n * n;                                            // B, B^T and the scatter add
    if (kind != MFA_FORM_MASS) per_cell += 12.0 * q * q * q * q + 15.0 * q * q * q;  // D, D^T, G g
    if (kind != MFA_FORM_LAPLACE) per_cell += q * q * q;                            // c0 w|J| u
    const double esz = f->p.precision == MFA_PREC_FP64 ? 8.0 : (f->p.precision == MFA_PREC_FP32 ? 4.0 : 2.0);
    bytes = ncell * (4.0 * n * n * n + esz * mfa::hex_geom_entries(kind) * q * q * q);
    if (f->launch.otf) {
      // trilinear Jacobian from 8 vertices (~200), adjugate, determinant and G (~70) at every point; the vertex
      // coordinates and map replace the stored factors
      per_cell += 270.0 * q * q * q;
      bytes = ncell * (4.0 * n * n * n + 32.0) + 24.0 * sp->mesh->nvert;
    }
  } else if (sp->degree == 2 && sp->ncomp == 3 && (kind == MFA_FORM_HYPER_RES || kind == MFA_FORM_HYPER_JAC)) {
    // moment kernel: per field 10x3x12 FMA moments + 36 mapped entries (900), per point the
    // gradient(s) (54 each), wd and wd*xi (4), the physics, the moment sums (72); per cell the
    // map back (180), the outputs (720), the body force (60, residual) and the scatter adds (30).
    // ln J and one division count as one flop each.
    const bool res = kind == MFA_FORM_HYPER_RES, svk = f->p.law == MFA_LAW_SVK;
    const double phys = res ? (svk ? 102.0 : 66.0) : (svk ? 243.0 : 202.0);
    const double fields = res ? 1.0 : 2.0;
    per_cell = 60.0 + 900.0 * fields + f->nq * (54.0 * fields + 76.0 + phys) + 180.0 + 720.0 + (res ? 60.0 : 0.0) + 30.0;
    // neo-Hookean residual: the mu F part of the stress leaves the point loop (its moments have a closed form in
    // the rule's weight moments): per point 29 flops fewer (the identity, mu F and its addition; one multiply
    // more), per cell ~330 more (the closed form)
    if (res && !svk) per_cell += -29.0 * f->nq + 330.0;
    bytes = ncell * (4.0 * sp->nloc + 16.0) + 24.0 * sp->mesh->nvert;
    if (kind == MFA_FORM_HYPER_JAC) bytes += 8.0 * ndof;
  } else if (sp->degree >= 3) {
    // dense tabulation, per point: interpolation (value 2, gradient 6 per dof and component; the Jacobian
    // action also the linearisation point's gradient), the physics, and the test-side sums (value 2,
    // gradient 6 per dof and component); per cell the affine geometry (~70) and the scatter adds
    const double nl = sp->nloc, nc = sp->ncomp, nq = f->nq;
    const bool val_in = kind == MFA_FORM_MASS || kind == MFA_FORM_HELMHOLTZ;
    const bool val_out = val_in || kind == MFA_FORM_HYPER_RES;
    const bool grad = kind != MFA_FORM_MASS, jac = kind == MFA_FORM_HYPER_JAC, svk = f->p.law == MFA_LAW_SVK;
    double per_q = nl * nc * ((val_in ? 2.0 : 0.0) + (grad ? 6.0 : 0.0) + (jac ? 6.0 : 0.0));
    per_q += nl * nc * ((val_out ? 2.0 : 0.0) + (grad ? 6.0 : 0.0));
    if (kind <= MFA_FORM_HELMHOLTZ) per_q += nc * ((grad ? 3.0 * 5.0 + 3.0 : 0.0) + (val_in ? 2.0 : 0.0)) + 1.0;
    else if (kind == MFA_FORM_ELASTICITY) per_q += 45.0 + 24.0 + 54.0 + 1.0;
    else if (kind == MFA_FORM_HYPER_RES) per_q += 45.0 + (svk ? 102.0 : 66.0) + 54.0 + 4.0;
    else per_q += 90.0 + (svk ? 243.0 : 202.0) + 54.0 + 1.0;
    per_cell = nq * per_q + 70.0 + nl * nc;
    bytes = ncell * (4.0 * nl + 16.0) + 24.0 * sp->mesh->nvert;
    if (jac) bytes += 8.0 * ndof;
  } else {
    const double nl = sp->nloc, nc = sp->ncomp, nq = f->nq;
    double per_q = 0.0;
    const bool value = kind == MFA_FORM_MASS || kind == MFA_FORM_HELMHOLTZ;
    const bool grad = kind != MFA_FORM_MASS;
    if (value) per_q += 2.0 * nl * nc + 2.0 * nl * nc + 2.0 * nc;  // interpolate, integrate, scale
    if (grad) per_q += 6.0 * nl * nc + 6.0 * nl * nc;              // reference gradient in and out
    if (kind <= MFA_FORM_HELMHOLTZ && grad) per_q += nc * (15.0 + 18.0);
    if (kind == MFA_FORM_ELASTICITY) per_q += 45.0 + 23.0 + 54.0;
    if (kind == MFA_FORM_HYPER_RES) per_q += 45.0 + 54.0 + (f->p.law == MFA_LAW_SVK ? 100.0 : 60.0) + 6.0;
    if (kind == MFA_FORM_HYPER_JAC) per_q += 45.0 + 45.0 + 6.0 * nl * 3 + 54.0 + (f->p.law == MFA_LAW_SVK ? 190.0 : 170.0);
    per_cell = nq * per_q + 60.0 + nl * nc;  // affine geometry + scatter adds
    bytes = ncell * (4.0 * nl + 16.0) + 24.0 * sp->mesh->nvert;
    if (kind == MFA_FORM_HYPER_JAC) bytes += 8.0 * ndof;
  }
  bytes += 16.0 * ndof;  // x read once, y written once
  if (f->scatter == MFA_SCATTER_COLOUR) bytes += 4.0 * ncell;
  f->flops = per_cell * ncell;
  f->flops_executed = (exec_cell >= 0.0 ? exec_cell : per_cell) * ncell;
  f->bytes = bytes;
}

int build_colouring(mfa_space* sp) {
  if (sp->d_colour_cells) return MFA_OK;
  const int64_t ncell = sp->mesh->ncell;
  std::vector<int32_t> map((size_t)ncell * sp->nloc);
  MFA_CUDA(cudaMemcpy(map.data(), sp->d_cell_node, map.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
  std::vector<int32_t> order;
  std::vector<int64_t> offsets;
  const int ncol = mfa::greedy_colour(ncell, sp->nloc, map.data(), sp->nnode, order, offsets);
  if (ncol <= 0) return fail(MFA_ERR_UNSUPPORTED, "greedy colouring needs more than 64 colours");
  int rc = cuda_alloc((void**)&sp->d_colour_cells, order.size() * sizeof(int32_t), "colour lists");
  if (rc) return rc;
  MFA_CUDA(cudaMemcpy(sp->d_colour_cells, order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  sp->ncolours = ncol;
  sp->colour_offsets = offsets;
  return MFA_OK;
}

int hex_tables(mfa_form* f) {
  const int n = f->space->degree + 1, q = f->nq1;
  double gll[mfa::kMaxN], xg[mfa::kMaxN], wg[mfa::kMaxN];
  mfa::gll01(n, gll);
  mfa::gauss_legendre01(q, xg, wg);
  mfa::lagrange_matrix(n, gll, q, xg, f->hex.B);
  mfa::collocation_derivative(q, xg, f->hex.D);
  for (int i = 0; i < q; ++i) {
    f->hex.x1[i] = xg[i];
    f->hex.w1[i] = wg[i];
  }
  return MFA_OK;
}

bool tet_pk_cell_ok(const mfa_form* f);

// Simplex rules come from simplex_rule_choice (below): the symmetric rule where
// the integral is exact (or the form asks for MFA_RULE_SYMMETRIC), else the
// collapsed rule of degree qdeg, which then defines the result.
// P3..P6: dense tables in device memory for the warp-per-cell kernel (layouts in TetDenseArgs).
static int tet_dense_tables(mfa_form* f, const std::vector<double>& pts, const std::vector<double>& w) {
  const int p = f->space->degree, nl = f->space->nloc;
  const int nq = (int)w.size();
  std::vector<double> phi((size_t)nq * nl), dphi((size_t)nq * nl * 3);
  for (int q = 0; q < nq; ++q) mfa::tet_basis_pk(p, &pts[3 * q], &phi[(size_t)q * nl], &dphi[(size_t)q * nl * 3]);
  const size_t nb = (size_t)nl * nq;
  std::vector<double> buf(8 * nb + nq);
  double* phi_aq = buf.data();
  double* dphi_aeq = phi_aq + nb;
  double* phi_qa = dphi_aeq + 3 * nb;
  double* dphi_qae = phi_qa + nb;
  double* wq = dphi_qae + 3 * nb;
  for (int q = 0; q < nq; ++q)
    for (int a = 0; a < nl; ++a) {
      const double v = phi[(size_t)q * nl + a];
      phi_aq[(size_t)a * nq + q] = v;
      phi_qa[(size_t)q * nl + a] = v;
      for (int e = 0; e < 3; ++e) {
        const double d = dphi[((size_t)q * nl + a) * 3 + e];
        dphi_aeq[((size_t)a * 3 + e) * nq + q] = d;
        dphi_qae[((size_t)q * nl + a) * 3 + e] = d;
      }
    }
  for (int q = 0; q < nq; ++q) wq[q] = w[q];
  if (tet_pk_cell_ok(f)) {  // the same tables as a kernel parameter of the thread-per-cell kernel
    f->tpk.nq = nq;
    for (int q = 0; q < nq; ++q) {
      f->tpk.w[q] = w[q];
      for (int a = 0; a < nl; ++a) {
        f->tpk.phi[q * nl + a] = phi[(size_t)q * nl + a];
        for (int e = 0; e < 3; ++e) f->tpk.dphi[(q * nl + a) * 3 + e] = dphi[((size_t)q * nl + a) * 3 + e];
      }
    }
  }
  int rc = cuda_alloc((void**)&f->d_tdense, sizeof(double) * buf.size(), "tet tables");
  if (!rc && cudaMemcpy(f->d_tdense, buf.data(), sizeof(double) * buf.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    rc = fail(MFA_ERR_CUDA, "tet tables: upload");
  if (rc) return rc;
  f->tdense_nq = nq;
  f->nq = nq;
  return MFA_OK;
}

// Triangles P1..P6: dense tables for the warp-per-cell kernel, gradients with 2 components.
// The simplex rule of a form.  The integrand has degree d on affine cells
// (-1: not a polynomial); the rule's degree is d when d <= qdeg (exact), else
// qdeg.  MFA_RULE_AUTO takes the symmetric rule where the integral is exact
// and the degree <= 6, MFA_RULE_SYMMETRIC wherever the degree <= 6; the
// collapsed product rule otherwise.
struct SimplexRuleChoice {
  int degree;
  bool symmetric;
};

SimplexRuleChoice simplex_rule_choice(const mfa_form* f) {
  const int p = f->space->degree, kind = f->p.kind;
  int qdeg = f->p.qdeg;
  if (qdeg <= 0) qdeg = (kind == MFA_FORM_HYPER_RES || kind == MFA_FORM_HYPER_JAC) ? (p > 2 ? 2 * p : 4) : 2 * p;
  int poly = -1;
  if (kind == MFA_FORM_MASS || kind == MFA_FORM_HELMHOLTZ) poly = 2 * p;
  if (kind == MFA_FORM_LAPLACE || kind == MFA_FORM_ELASTICITY) poly = 2 * (p - 1);
  if ((kind == MFA_FORM_HYPER_RES || kind == MFA_FORM_HYPER_JAC) && f->p.law == MFA_LAW_SVK) poly = 4 * (p - 1);
  const bool exact = poly >= 0 && poly <= qdeg;
  const int deg = exact ? poly : qdeg;
  return {deg, deg <= 6 && (exact || f->p.rule == MFA_RULE_SYMMETRIC)};
}

// Points of the rule simplex_rule_choice picks (without deriving it).
int simplex_rule_points(const mfa_form* f, int dim) {
  const SimplexRuleChoice c = simplex_rule_choice(f);
  if (c.symmetric) {
    static const int tri[7] = {1, 1, 3, 6, 6, 12, 12}, tet[7] = {1, 1, 4, 14, 14, 14, 24};
    return dim == 3 ? tet[c.degree] : tri[c.degree];
  }
  const int m = c.degree / 2 + 1;
  return dim == 3 ? m * m * m : m * m;
}

int simplex_form_rule(const mfa_form* f, int dim, std::vector<double>& pts, std::vector<double>& w) {
  const SimplexRuleChoice c = simplex_rule_choice(f);
  if (c.symmetric) {
    if (mfa::simplex_rule_symmetric(dim, c.degree, pts, w) <= 0)
      return fail(MFA_ERR_UNSUPPORTED, "symmetric simplex rule of degree %d", c.degree);
    return MFA_OK;
  }
  const int m = c.degree / 2 + 1;
  if (m > mfa::kMaxN) return fail(MFA_ERR_UNSUPPORTED, "simplex rule of degree %d", c.degree);
  const int nq = dim == 3 ? m * m * m : m * m;
  pts.resize((size_t)dim * nq);
  w.resize(nq);
  const int got = dim == 3 ? mfa::tet_rule_collapsed(c.degree, pts.data(), w.data())
                           : mfa::tri_rule_collapsed(c.degree, pts.data(), w.data());
  if (got != nq) return fail(MFA_ERR_UNSUPPORTED, "simplex rule of degree %d", c.degree);
  return MFA_OK;
}

// The thread-per-cell triangle kernel covers P1..P4 with at most 25 points (P4 Jacobian action: no).
bool tri_cell_ok(const mfa_form* f) {
  if (f->space->mesh->cell_type != MFA_CELL_TRI3 || f->space->degree > 4) return false;
  if (f->space->degree == 4 && f->p.kind == MFA_FORM_HYPER_JAC) return false;  // register-bound: one warp per cell
  return simplex_rule_points(f, 2) <= mfa::kTriMaxQ;
}

// The thread-per-cell P3/P4 tet kernel covers the scalar forms on rules of at most 24 points (Table 2's
// symmetric rules of degree <= 6: P3 mass, Laplace and Helmholtz, P4 Laplace).
bool tet_pk_cell_ok(const mfa_form* f) {
  const mfa_space* sp = f->space;
  if (sp->mesh->cell_type != MFA_CELL_TET4 || sp->ncomp != 1 || sp->degree < 3 || sp->degree > 4) return false;
  if (f->p.kind > MFA_FORM_HELMHOLTZ) return false;
  return simplex_rule_points(f, 3) <= mfa::kTetPkMaxQ;
}

int tri_tables(mfa_form* f) {
  const int p = f->space->degree, nl = f->space->nloc;
  std::vector<double> pts, w;
  const int rrc = simplex_form_rule(f, 2, pts, w);
  if (rrc) return rrc;
  const int nq = (int)w.size();
  if (tri_cell_ok(f) && nq > mfa::kTriMaxQ) return fail(MFA_ERR_UNSUPPORTED, "triangle rule of %d points", nq);
  std::vector<double> phi((size_t)nq * nl), dphi((size_t)nq * nl * 2);
  for (int q = 0; q < nq; ++q) mfa::tri_basis_pk(p, &pts[2 * q], &phi[(size_t)q * nl], &dphi[(size_t)q * nl * 2]);
  const size_t nb = (size_t)nl * nq;
  std::vector<double> buf(6 * nb + nq);
  double* phi_aq = buf.data();
  double* dphi_aeq = phi_aq + nb;
  double* phi_qa = dphi_aeq + 2 * nb;
  double* dphi_qae = phi_qa + nb;
  double* wq = dphi_qae + 2 * nb;
  for (int q = 0; q < nq; ++q)
    for (int a = 0; a < nl; ++a) {
      const double v = phi[(size_t)q * nl + a];
      phi_aq[(size_t)a * nq + q] = v;
      phi_qa[(size_t)q * nl + a] = v;
      for (int e = 0; e < 2; ++e) {
        const double d = dphi[((size_t)q * nl + a) * 2 + e];
        dphi_aeq[((size_t)a * 2 + e) * nq + q] = d;
        dphi_qae[((size_t)q * nl + a) * 2 + e] = d;
      }
    }
  for (int q = 0; q < nq; ++q) wq[q] = w[q];
  if (tri_cell_ok(f)) {  // the same tables as a kernel parameter of the thread-per-cell kernel
    f->tri.nq = nq;
    for (int q = 0; q < nq; ++q) {
      f->tri.w[q] = w[q];
      for (int a = 0; a < nl; ++a) {
        f->tri.phi[q * mfa::kTriMaxNl + a] = phi[(size_t)q * nl + a];
        for (int e = 0; e < 2; ++e)
          f->tri.dphi[(q * mfa::kTriMaxNl + a) * 2 + e] = dphi[((size_t)q * nl + a) * 2 + e];
      }
    }
  }
  int rc = cuda_alloc((void**)&f->d_tdense, sizeof(double) * buf.size(), "triangle tables");
  if (!rc && cudaMemcpy(f->d_tdense, buf.data(), sizeof(double) * buf.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    rc = fail(MFA_ERR_CUDA, "triangle tables: upload");
  if (rc) return rc;
  f->tdense_nq = nq;
  f->nq = nq;
  return MFA_OK;
}

int tet_tables(mfa_form* f) {
  const int p = f->space->degree, kind = f->p.kind;
  std::vector<double> rpts, rw;
  const int rrc = simplex_form_rule(f, 3, rpts, rw);
  if (rrc) return rrc;
  if (p >= 3) return tet_dense_tables(f, rpts, rw);
  const int nq = (int)rw.size();
  if (!mfa::tet_rule_compiled(p, f->space->ncomp, kind, nq))
    return fail(MFA_ERR_UNSUPPORTED, "P%d form %d: no kernel for a rule of %d points", p, kind, nq);
  const double* pts = rpts.data();
  for (int q = 0; q < nq; ++q) f->tet.w[q] = rw[q];
  f->tet.nq = nq;
  const int nl = f->space->nloc;
  for (int i = 0; i < nq; ++i) mfa::tet_basis(p, pts + 3 * i, f->tet.phi + i * nl, f->tet.dphi + i * nl * 3);
  for (int i = 0; i < 3 * nq; ++i) f->tet.pts[i] = pts[i];
  if (p == 2) {  // the P2 reference gradients are linear: alpha = grad(0), beta[.][f] = grad(e_f) - grad(0)
    double phi0[10], g0[30], phif[10], gf[30];
    const double origin[3] = {0.0, 0.0, 0.0};
    mfa::tet_basis(2, origin, phi0, g0);
    for (int a = 0; a < 10; ++a)
      for (int e = 0; e < 3; ++e) f->tet.alpha[a * 3 + e] = g0[a * 3 + e];
    for (int fd = 0; fd < 3; ++fd) {
      double ef[3] = {0.0, 0.0, 0.0};
      ef[fd] = 1.0;
      mfa::tet_basis(2, ef, phif, gf);
      for (int a = 0; a < 10; ++a)
        for (int e = 0; e < 3; ++e) f->tet.beta[a * 9 + e * 3 + fd] = gf[a * 3 + e] - g0[a * 3 + e];
    }
    for (int a = 0; a < 10; ++a) {
      double m = 0.0;
      for (int q = 0; q < nq; ++q) m += f->tet.w[q] * f->tet.phi[q * nl + a];
      f->tet.mvec[a] = m;
    }
    for (int k = 0; k < 13; ++k) f->tet.wmom[k] = 0.0;
    for (int q = 0; q < nq; ++q) {
      const double w = f->tet.w[q], *xq = f->tet.pts + 3 * q;
      f->tet.wmom[0] += w;
      for (int fd = 0; fd < 3; ++fd) {
        f->tet.wmom[1 + fd] += w * xq[fd];
        for (int g = 0; g < 3; ++g) f->tet.wmom[4 + 3 * fd + g] += w * xq[fd] * xq[g];
      }
    }
  }
  f->nq = nq;
  return MFA_OK;
}

mfa::TetApplyArgs tet_args(mfa_form* f, const double* x, double* y) {
  mfa::TetApplyArgs a{};
  a.x = x;
  a.y = y;
  a.coords = f->space->mesh->d_coords;
  a.cell_vert = f->space->mesh->d_cell_vert;
  a.cell_node = f->space->d_cell_node;
  a.ucoef = f->d_coef;
  a.cell_list = nullptr;
  a.count = f->space->mesh->ncell;
  a.k2 = f->p.k2;
  a.lambda = f->p.lambda;
  a.mu = f->p.mu;
  a.b0 = f->p.b[0];
  a.b1 = f->p.b[1];
  a.b2 = f->p.b[2];
  a.err = f->ctx->d_err;
  return a;
}

}  // namespace

namespace mfa {
int set_error(int code, const char* msg) { return fail(code, "%s", msg); }

static int apply_form_raw(mfa_form* f, const double* x, double* y, cudaStream_t stream);

// y += A x, or with Dirichlet constraints y += R A R x + (I - R) x (R zeroes the constrained dofs).
int apply_form(mfa_form* f, const double* x, double* y, cudaStream_t stream) {
  clear_stale_error();
  if (!f->d_dir_mask) return apply_form_raw(f, x, y, stream);
  const int64_t n = f->space->nnode * f->space->ncomp;
  cudaError_t e = dirichlet_mask_launch(x, f->d_dir_mask, f->d_dir_x, n, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->d_dir_y, 0, sizeof(double) * n, stream);
  if (e != cudaSuccess) return fail(MFA_ERR_CUDA, "constrained apply: %s", cudaGetErrorString(e));
  const int rc = apply_form_raw(f, f->d_dir_x, f->d_dir_y, stream);
  if (rc) return rc;
  e = dirichlet_combine_launch(f->d_dir_y, x, f->d_dir_mask, y, n, stream);
  return e == cudaSuccess ? MFA_OK : fail(MFA_ERR_CUDA, "constrained apply: %s", cudaGetErrorString(e));
}

static int apply_form_raw(mfa_form* f, const double* x, double* y, cudaStream_t stream) {
  mfa_space* sp = f->space;
  mfa_ctx* ctx = f->ctx;
  const mfa::GridBudget budget{ctx->sm_count, f->launch.max_blocks};
  const bool colour = f->scatter == MFA_SCATTER_COLOUR;
  const int ncol = colour ? sp->ncolours : 1;
  for (int k = 0; k < ncol; ++k) {
    const int32_t* list = colour ? sp->d_colour_cells + sp->colour_offsets[k] : nullptr;
    const int64_t count = colour ? sp->colour_offsets[k + 1] - sp->colour_offsets[k] : sp->mesh->ncell;
    cudaError_t e;
    if (sp->mesh->cell_type == MFA_CELL_QUAD4) {
      mfa::QuadArgs a{x, y, sp->d_cell_node, static_cast<const double*>(f->d_geom), f->d_coef, list, count,
                      f->p.lambda, f->p.mu, f->p.b[0], f->p.b[1], ctx->d_err};
      e = mfa::quad_apply_launch(sp->degree + 1, f->nq1, sp->ncomp, f->p.kind, f->p.law, colour, f->hex, a,
                                 budget, stream);
    } else if (sp->mesh->cell_type == MFA_CELL_TRI3) {
      const int64_t nb = (int64_t)sp->nloc * f->tdense_nq;
      mfa::TetDenseArgs a{};
      a.x = x;
      a.y = y;
      a.coords = sp->mesh->d_coords;
      a.cell_vert = sp->mesh->d_cell_vert;
      a.cell_node = sp->d_cell_node;
      a.ucoef = f->d_coef;
      a.cell_list = list;
      a.count = count;
      a.phi_aq = f->d_tdense;
      a.dphi_aeq = a.phi_aq + nb;
      a.phi_qa = a.dphi_aeq + 2 * nb;
      a.dphi_qae = a.phi_qa + nb;
      a.w = a.dphi_qae + 2 * nb;
      a.nq = f->tdense_nq;
      a.k2 = f->p.k2;
      a.lambda = f->p.lambda;
      a.mu = f->p.mu;
      a.b0 = f->p.b[0];
      a.b1 = f->p.b[1];
      a.b2 = 0.0;
      a.err = ctx->d_err;
      if (f->launch.variant == MFA_VARIANT_CELL)
        e = mfa::tri_cell_launch(sp->degree, sp->ncomp, f->p.kind, f->p.law, colour, f->launch.cb ? f->launch.cb : 128,
                                 f->tri, a, budget, stream);
      else
        e = mfa::tri_dense_launch(sp->degree, sp->ncomp, f->p.kind, f->p.law, colour, a, budget, stream);
    } else if (sp->mesh->cell_type == MFA_CELL_HEX8 && sp->ncomp == 3) {
      mfa::HexVecArgs a{x, y, sp->d_cell_node, static_cast<const double*>(f->d_geom), f->d_coef, list, count,
                        f->gstride, f->p.lambda, f->p.mu, f->p.b[0], f->p.b[1], f->p.b[2], ctx->d_err};
      const int n = sp->degree + 1;
      e = n <= 5 ? mfa::hex_vector_launch_a(n, f->nq1, f->p.kind, f->p.law, colour, f->hex, a, budget, stream)
                 : mfa::hex_vector_launch_b(n, f->nq1, f->p.kind, f->p.law, colour, f->hex, a, budget, stream);
    } else if (sp->mesh->cell_type == MFA_CELL_HEX8) {
      mfa::HexApplyArgs a{x, y, sp->d_cell_node, f->d_geom, list, count, ctx->d_err, f->gstride};
      a.coords = sp->mesh->d_coords;
      a.cell_vert = sp->mesh->d_cell_vert;
      a.c0 = f->p.kind == MFA_FORM_HELMHOLTZ ? f->p.k2 : 1.0;
      mfa::LaunchConfig lc = f->launch;
      lc.agg = f->scatter == MFA_SCATTER_WARP;
      e = mfa::hex_apply_launch(sp->degree + 1, f->nq1, f->p.kind, f->p.precision, colour, lc, f->hex, a,
                                budget, stream);
    } else if (sp->degree >= 3) {
      const int64_t nb = (int64_t)sp->nloc * f->tdense_nq;
      mfa::TetDenseArgs a{};
      a.x = x;
      a.y = y;
      a.coords = sp->mesh->d_coords;
      a.cell_vert = sp->mesh->d_cell_vert;
      a.cell_node = sp->d_cell_node;
      a.ucoef = f->d_coef;
      a.cell_list = list;
      a.count = count;
      a.phi_aq = f->d_tdense;
      a.dphi_aeq = a.phi_aq + nb;
      a.phi_qa = a.dphi_aeq + 3 * nb;
      a.dphi_qae = a.phi_qa + nb;
      a.w = a.dphi_qae + 3 * nb;
      a.nq = f->tdense_nq;
      a.k2 = f->p.k2;
      a.lambda = f->p.lambda;
      a.mu = f->p.mu;
      a.b0 = f->p.b[0];
      a.b1 = f->p.b[1];
      a.b2 = f->p.b[2];
      a.err = ctx->d_err;
      if (f->launch.variant == MFA_VARIANT_CELL)
        e = mfa::tet_pk_cell_launch(sp->degree, f->p.kind, colour, f->launch.cb ? f->launch.cb : 128, f->tpk, a,
                                    budget, stream);
      else
        e = mfa::tet_dense_launch(sp->degree, sp->ncomp, f->p.kind, f->p.law, colour, a, budget, stream);
    } else {
      mfa::TetApplyArgs a = tet_args(f, x, y);
      a.cell_list = list;
      a.count = count;
      e = mfa::tet_apply_launch(sp->degree, sp->ncomp, f->p.kind, f->p.law, colour, f->scatter == MFA_SCATTER_WARP,
                                f->launch.cb ? f->launch.cb : 128, f->tet, a, budget, stream);
    }
    if (e != cudaSuccess) return fail(MFA_ERR_CUDA, "apply kernel launch: %s", cudaGetErrorString(e));
  }
  return MFA_OK;
}

}  // namespace mfa

extern "C" {

const char* mfa_last_error(void) { return g_err; }
int mfa_version(void) { return MFA_VERSION; }

int mfa_create(mfa_ctx** out, int device, void* stream) {
  if (!out) return fail(MFA_ERR_ARG, "mfa_create: out is NULL");
  *out = nullptr;
  int ndev = 0;
  MFA_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(MFA_ERR_ARG, "mfa_create: device %d of %d", device, ndev);
  MFA_CUDA(cudaSetDevice(device));
  mfa_ctx* c = new (std::nothrow) mfa_ctx();
  if (!c) return fail(MFA_ERR_OOM, "mfa_create: host allocation");
  c->device = device;
  c->stream = (cudaStream_t)stream;
  cudaError_t e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  int rc = e == cudaSuccess ? MFA_OK : fail(MFA_ERR_CUDA, "SM count: %s", cudaGetErrorString(e));
  if (!rc) rc = cuda_alloc((void**)&c->d_err, sizeof(int), "error flag");
  if (!rc) rc = cuda_alloc((void**)&c->d_scratch, sizeof(double) * (mfa::dot_partials() + 8), "dot scratch");
  if (!rc && cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess) rc = fail(MFA_ERR_CUDA, "memset error flag");
  if (rc) {
    mfa_destroy(c);
    return rc;
  }
  *out = c;
  return MFA_OK;
}

int mfa_set_stream(mfa_ctx* ctx, void* stream) {
  if (!ctx) return fail(MFA_ERR_ARG, "mfa_set_stream: ctx is NULL");
  ctx->stream = (cudaStream_t)stream;
  return MFA_OK;
}

int mfa_destroy(mfa_ctx* ctx) {
  if (!ctx) return MFA_OK;
  cudaSetDevice(ctx->device);
  if (ctx->copy_in) cudaStreamDestroy(ctx->copy_in);
  if (ctx->copy_out) cudaStreamDestroy(ctx->copy_out);
  for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
  cudaFree(ctx->d_err);
  cudaFree(ctx->d_scratch);
  delete ctx;
  return MFA_OK;
}

int mfa_mesh_upload(mfa_ctx* ctx, int cell_type, int64_t ncell, int64_t nvert, const double* coords,
                    const int32_t* cell_vert, mfa_mesh** out) {
  if (!ctx || !out || !coords || !cell_vert) return fail(MFA_ERR_ARG, "mfa_mesh_upload: NULL argument");
  *out = nullptr;
  if (cell_type != MFA_CELL_TET4 && cell_type != MFA_CELL_HEX8 && cell_type != MFA_CELL_TRI3 &&
      cell_type != MFA_CELL_QUAD4)
    return fail(MFA_ERR_ARG, "mfa_mesh_upload: cell_type %d", cell_type);
  const int nv = mfa::verts_of(cell_type);
  if (ncell < 0 || nvert <= 0 || nvert > INT32_MAX || ncell > INT32_MAX)
    return fail(MFA_ERR_ARG, "mfa_mesh_upload: ncell %lld nvert %lld", (long long)ncell, (long long)nvert);
  for (int64_t i = 0; i < ncell * nv; ++i)
    if (cell_vert[i] < 0 || cell_vert[i] >= nvert)
      return fail(MFA_ERR_RANGE, "mfa_mesh_upload: cell_vert[%lld] = %d outside [0, %lld)", (long long)i,
                  cell_vert[i], (long long)nvert);
  MFA_CUDA(cudaSetDevice(ctx->device));
  mfa_mesh* m = new (std::nothrow) mfa_mesh();
  if (!m) return fail(MFA_ERR_OOM, "mfa_mesh_upload: host allocation");
  m->ctx = ctx;
  m->device = ctx->device;
  m->cell_type = cell_type;
  m->ncell = ncell;
  m->nvert = nvert;
  int rc = cuda_alloc((void**)&m->d_coords, sizeof(double) * 3 * nvert, "coords");
  if (!rc) rc = cuda_alloc((void**)&m->d_cell_vert, sizeof(int32_t) * nv * ncell, "cell_vert");
  if (!rc && cudaMemcpy(m->d_coords, coords, sizeof(double) * 3 * nvert, cudaMemcpyHostToDevice) != cudaSuccess)
    rc = fail(MFA_ERR_CUDA, "mfa_mesh_upload: copy coords");
  if (!rc && ncell > 0 &&
      cudaMemcpy(m->d_cell_vert, cell_vert, sizeof(int32_t) * nv * ncell, cudaMemcpyHostToDevice) != cudaSuccess)
    rc = fail(MFA_ERR_CUDA, "mfa_mesh_upload: copy cell_vert");
  if (rc) {
    mfa_mesh_destroy(m);
    return rc;
  }
  *out = m;
  return MFA_OK;
}

int mfa_mesh_destroy(mfa_mesh* m) {
  if (!m) return MFA_OK;
  cudaSetDevice(m->device);
  cudaFree(m->d_coords);
  cudaFree(m->d_cell_vert);
  delete m;
  return MFA_OK;
}

int mfa_space_create(mfa_ctx* ctx, mfa_mesh* mesh, int degree, int ncomp, const int32_t* cell_node, int64_t nnode,
                     mfa_space** out) {
  if (!ctx || !mesh || !out) return fail(MFA_ERR_ARG, "mfa_space_create: NULL argument");
  *out = nullptr;
  const int nl = nloc_of(mesh->cell_type, degree);
  if (nl < 0) return fail(MFA_ERR_UNSUPPORTED, "mfa_space_create: degree %d on cell type %d", degree, mesh->cell_type);
  std::vector<int32_t> built;
  if (!cell_node) {  // build the map from the mesh's vertex connectivity
    std::vector<int32_t> cv((size_t)mesh->ncell * mfa::verts_of(mesh->cell_type));
    if (!cv.empty())
      MFA_CUDA(cudaMemcpy(cv.data(), mesh->d_cell_vert, cv.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    built.resize((size_t)mesh->ncell * nl);
    int rc = mfa_build_cell_node(mesh->cell_type, degree, mesh->ncell, cv.data(), mesh->nvert, built.data(), &nnode);
    if (rc) return rc;
    cell_node = built.data();
  }
  const bool planar = mfa::is_planar(mesh->cell_type);
  if (ncomp != 1 && ncomp != (planar ? 2 : 3))
    return fail(MFA_ERR_ARG, "mfa_space_create: ncomp %d (1 or %d on this mesh)", ncomp, planar ? 2 : 3);
  if (nnode <= 0 || nnode * ncomp > INT32_MAX) return fail(MFA_ERR_ARG, "mfa_space_create: nnode %lld", (long long)nnode);
  {
    std::vector<int64_t> stamp(nnode, -1);
    for (int64_t c = 0; c < mesh->ncell; ++c)
      for (int a = 0; a < nl; ++a) {
        const int32_t v = cell_node[c * nl + a];
        if (v < 0 || v >= nnode)
          return fail(MFA_ERR_RANGE, "mfa_space_create: cell_node[%lld][%d] = %d outside [0, %lld)", (long long)c, a, v,
                      (long long)nnode);
        if (stamp[v] == c)
          return fail(MFA_ERR_ARG, "mfa_space_create: node %d repeated in cell %lld", v, (long long)c);
        stamp[v] = c;
      }
  }
  MFA_CUDA(cudaSetDevice(ctx->device));
  mfa_space* s = new (std::nothrow) mfa_space();
  if (!s) return fail(MFA_ERR_OOM, "mfa_space_create: host allocation");
  s->ctx = ctx;
  s->device = ctx->device;
  s->mesh = mesh;
  s->degree = degree;
  s->ncomp = ncomp;
  s->nloc = nl;
  s->nnode = nnode;
  const size_t bytes = sizeof(int32_t) * nl * mesh->ncell;
  int rc = cuda_alloc((void**)&s->d_cell_node, bytes, "cell_node");
  if (!rc && bytes && cudaMemcpy(s->d_cell_node, cell_node, bytes, cudaMemcpyHostToDevice) != cudaSuccess)
    rc = fail(MFA_ERR_CUDA, "mfa_space_create: copy cell_node");
  if (rc) {
    mfa_space_destroy(s);
    return rc;
  }
  *out = s;
  return MFA_OK;
}

int mfa_space_ndof(const mfa_space* s, int64_t* ndof) {
  if (!s || !ndof) return fail(MFA_ERR_ARG, "mfa_space_ndof: NULL argument");
  *ndof = s->nnode * s->ncomp;
  return MFA_OK;
}

int mfa_space_get_cell_node(const mfa_space* s, int32_t* out) {
  if (!s || !out) return fail(MFA_ERR_ARG, "mfa_space_get_cell_node: NULL argument");
  const size_t bytes = sizeof(int32_t) * (size_t)s->nloc * s->mesh->ncell;
  MFA_CUDA(cudaSetDevice(s->device));
  if (bytes) MFA_CUDA(cudaMemcpy(out, s->d_cell_node, bytes, cudaMemcpyDeviceToHost));
  return MFA_OK;
}

int mfa_space_destroy(mfa_space* s) {
  if (!s) return MFA_OK;
  cudaSetDevice(s->device);
  cudaFree(s->d_cell_node);
  cudaFree(s->d_colour_cells);
  delete s;
  return MFA_OK;
}

static int default_variant(const mfa_space* sp, int nq, int precision) {
  if (sp->mesh->cell_type == MFA_CELL_QUAD4) return MFA_VARIANT_POINT;
  if (sp->mesh->cell_type == MFA_CELL_TRI3) return MFA_VARIANT_CELL_WARP;
  if (sp->mesh->cell_type != MFA_CELL_HEX8) return sp->degree >= 3 ? MFA_VARIANT_CELL_WARP : MFA_VARIANT_CELL;
  if (sp->ncomp == 3) return MFA_VARIANT_POINT;  // the vector forms have the point kernel only
  return mfa::hex_default_variant(sp->degree + 1, nq, precision);
}

// Compiled cells-per-block choices of `variant` for this form (default first).
static int cb_options(const mfa_form* f, int variant, int* out) {
  const mfa_space* sp = f->space;
  const int n = sp->degree + 1, nq = f->p.qdeg > 0 ? f->p.qdeg : n;
  if (sp->mesh->cell_type == MFA_CELL_QUAD4) {
    if (variant != MFA_VARIANT_POINT) return 0;
    out[0] = mfa::quad_cells_per_block(n, nq);
    return 1;
  }
  if (sp->mesh->cell_type == MFA_CELL_TRI3) {
    if (variant == MFA_VARIANT_CELL) return tri_cell_ok(f) ? mfa::tet_cb_options(out) : 0;  // threads per block
    if (variant != MFA_VARIANT_CELL_WARP) return 0;
    out[0] = 8;  // one warp per cell, 8 warps per block
    return 1;
  }
  if (sp->mesh->cell_type != MFA_CELL_HEX8) {
    if (sp->degree >= 3) {
      if (variant == MFA_VARIANT_CELL) return tet_pk_cell_ok(f) ? mfa::tet_cb_options(out) : 0;  // threads per block
      if (variant != MFA_VARIANT_CELL_WARP) return 0;
      out[0] = 8;  // one warp per cell, 8 warps per block
      return 1;
    }
    return variant == MFA_VARIANT_CELL ? mfa::tet_cb_options(out) : 0;
  }
  if (sp->ncomp == 3) {
    if (variant != MFA_VARIANT_POINT) return 0;
    out[0] = mfa::hex_cells_per_block(n, n);
    return 1;
  }
  if (f->p.precision == MFA_PREC_FP64) {
    if (variant == MFA_VARIANT_POINT) return mfa::hex_point_cb_options(n, nq, out);
    if (variant == MFA_VARIANT_EVEN_ODD) return nq == n ? mfa::hex_eo_cb_options(n, out) : 0;
    return 0;
  }
  if (variant == MFA_VARIANT_LINE || variant == MFA_VARIANT_LINE_STAGED) return mfa::hex_line_cb_options(n, out);
  return 0;
}

// Every compiled configuration of the form: the creation-time one first, then
// variant by variant, cells per block in option order, atomic before colour.
static std::vector<mfa_launch_config> form_configs(const mfa_form* f) {
  std::vector<mfa_launch_config> all;
  const bool hex = f->space->mesh->cell_type == MFA_CELL_HEX8;
  std::vector<int> variants;
  const int ctype = f->space->mesh->cell_type;
  if (ctype == MFA_CELL_QUAD4) variants = {MFA_VARIANT_POINT};
  else if (ctype == MFA_CELL_TRI3 && tri_cell_ok(f)) variants = {MFA_VARIANT_CELL, MFA_VARIANT_CELL_WARP};
  else if (ctype == MFA_CELL_TRI3) variants = {MFA_VARIANT_CELL_WARP};
  else if (!hex && tet_pk_cell_ok(f)) variants = {MFA_VARIANT_CELL, MFA_VARIANT_CELL_WARP};
  else if (!hex) variants = {f->space->degree >= 3 ? MFA_VARIANT_CELL_WARP : MFA_VARIANT_CELL};
  else if (f->p.precision == MFA_PREC_FP64) variants = {MFA_VARIANT_POINT, MFA_VARIANT_EVEN_ODD};
  else variants = {MFA_VARIANT_LINE, MFA_VARIANT_LINE_STAGED};
  const bool colour_ok = f->p.precision == MFA_PREC_FP64;
  const int n = f->space->degree + 1;
  const bool stored = !hex || f->d_geom != nullptr;  // the on-the-fly forms have no stored factors
  // on-the-fly geometry: the FP64 scalar point kernel with p+1 points, default cells per block
  const bool otf_ok = hex && f->p.precision == MFA_PREC_FP64 && f->space->ncomp == 1 && f->nq1 == n &&
                      f->p.kind <= MFA_FORM_HELMHOLTZ;
  for (int v : variants) {
    int opts[4];
    const int nopt = cb_options(f, v, opts);
    for (int i = 0; i < nopt; ++i) {
      for (int geo = 0; geo < 2; ++geo) {
        if (geo == 0 && !stored) continue;
        if (geo == 1 && !(otf_ok && v == MFA_VARIANT_POINT && i == 0)) continue;
        // warp-aggregated scatter: tets, and the scalar point kernel with p+1 points at its default cells per block
        const bool warp_ok = colour_ok && geo == 0 &&
                             ((v == MFA_VARIANT_CELL && ctype == MFA_CELL_TET4) ||
                              (v == MFA_VARIANT_POINT && hex && f->space->ncomp == 1 && f->nq1 == n && i == 0));
        const int scatters[3] = {MFA_SCATTER_ATOMIC, MFA_SCATTER_COLOUR, MFA_SCATTER_WARP};
        for (int sc = 0; sc < (colour_ok ? (warp_ok ? 3 : 2) : 1); ++sc) {
          mfa_launch_config c{};
          c.variant = v;
          c.cells_per_block = opts[i];
          c.scatter = scatters[sc];
          c.geometry = geo ? MFA_GEOM_ONTHEFLY : MFA_GEOM_STORED;
          all.push_back(c);
        }
      }
    }
  }
  // move the creation-time configuration to the front
  int dopts[4];
  const int dn = cb_options(f, f->launch.variant, dopts);
  const int dcb = f->launch.cb ? f->launch.cb : (dn > 0 ? dopts[0] : 0);
  const int dgeo = f->launch.otf ? MFA_GEOM_ONTHEFLY : MFA_GEOM_STORED;
  for (size_t i = 0; i < all.size(); ++i)
    if (all[i].variant == f->launch.variant && all[i].cells_per_block == dcb && all[i].scatter == f->scatter &&
        all[i].geometry == dgeo) {
      std::rotate(all.begin(), all.begin() + i, all.begin() + i + 1);
      break;
    }
  return all;
}

int mfa_form_create(mfa_ctx* ctx, mfa_space* sp, const mfa_form_params* prm, mfa_form** out) {
  if (!ctx || !sp || !prm || !out) return fail(MFA_ERR_ARG, "mfa_form_create: NULL argument");
  *out = nullptr;
  const double t0 = now_ms();
  const int kind = prm->kind, ct = sp->mesh->cell_type;
  if (kind < MFA_FORM_MASS || kind > MFA_FORM_HYPER_JAC) return fail(MFA_ERR_ARG, "mfa_form_create: kind %d", kind);
  if (prm->scatter < MFA_SCATTER_AUTO || prm->scatter > MFA_SCATTER_WARP)
    return fail(MFA_ERR_ARG, "mfa_form_create: scatter %d", prm->scatter);
  if (prm->law != MFA_LAW_SVK && prm->law != MFA_LAW_NEOHOOKE) return fail(MFA_ERR_ARG, "mfa_form_create: law %d", prm->law);
  if (prm->precision < MFA_PREC_FP64 || prm->precision > MFA_PREC_BF16)
    return fail(MFA_ERR_ARG, "mfa_form_create: precision %d", prm->precision);
  if (prm->geometry != MFA_GEOM_STORED && prm->geometry != MFA_GEOM_ONTHEFLY)
    return fail(MFA_ERR_ARG, "mfa_form_create: geometry %d", prm->geometry);
  if (prm->rule != MFA_RULE_AUTO && prm->rule != MFA_RULE_SYMMETRIC)
    return fail(MFA_ERR_ARG, "mfa_form_create: rule %d", prm->rule);
  if (prm->geometry == MFA_GEOM_ONTHEFLY &&
      (ct != MFA_CELL_HEX8 || sp->ncomp != 1 || kind > MFA_FORM_HELMHOLTZ || prm->precision != MFA_PREC_FP64 ||
       (prm->qdeg > 0 && prm->qdeg != sp->degree + 1) || prm->scatter == MFA_SCATTER_WARP ||
       prm->cells_per_block != 0))
    return fail(MFA_ERR_UNSUPPORTED,
                "mfa_form_create: on-the-fly geometry covers FP64 scalar hex forms with p+1 points (atomic or colour "
                "scatter, default cells per block)");
  if (prm->precision != MFA_PREC_FP64 && (ct != MFA_CELL_HEX8 || (prm->qdeg > 0 && prm->qdeg != sp->degree + 1) ||
                                          prm->scatter == MFA_SCATTER_COLOUR || prm->scatter == MFA_SCATTER_WARP))
    return fail(MFA_ERR_UNSUPPORTED,
                "mfa_form_create: FP32/BF16 cover hex forms with p+1 points per direction and the atomic scatter");
  const bool planar = mfa::is_planar(ct);
  if (kind >= MFA_FORM_ELASTICITY && sp->ncomp != (planar ? 2 : 3))
    return fail(MFA_ERR_ARG, "mfa_form_create: form %d needs a vector space", kind);
  if (planar) {
    const int n = sp->degree + 1, nq = prm->qdeg > 0 ? prm->qdeg : n;
    const bool hyper = kind == MFA_FORM_HYPER_RES || kind == MFA_FORM_HYPER_JAC;
    bool ok = (sp->ncomp == 1 && kind <= MFA_FORM_HELMHOLTZ) ||
              (sp->ncomp == 2 && kind >= MFA_FORM_LAPLACE && kind != MFA_FORM_HELMHOLTZ);
    ok = ok && prm->precision == MFA_PREC_FP64 && prm->scatter != MFA_SCATTER_WARP;
    if (ct == MFA_CELL_QUAD4) ok = ok && (nq == n || (nq == n + 1 && n + 1 <= mfa::kMaxN) ||
                                          (hyper && nq == 2 * n && 2 * n <= mfa::kMaxN));
    if (!ok)
      return fail(MFA_ERR_UNSUPPORTED,
                  "mfa_form_create: planar cells cover FP64 mass/Laplace/Helmholtz and vector Laplace/elasticity/"
                  "hyperelasticity (quads: p+1 or p+2 points, 2p+2 for the hyperelastic forms), atomic or colour "
                  "scatter");
  }
  if (ct == MFA_CELL_HEX8 && sp->ncomp == 1 && kind > MFA_FORM_HELMHOLTZ)
    return fail(MFA_ERR_UNSUPPORTED, "mfa_form_create: scalar hex kernels cover mass/Laplace/Helmholtz");
  if (ct == MFA_CELL_HEX8 && sp->ncomp == 3) {
    const int n = sp->degree + 1, nq = prm->qdeg > 0 ? prm->qdeg : n;
    const bool hyper = kind == MFA_FORM_HYPER_RES || kind == MFA_FORM_HYPER_JAC;
    const bool rule_ok = nq == n || (!hyper && nq == n + 1 && n <= 7) || (hyper && nq == 2 * n && n <= 4);
    if (kind == MFA_FORM_MASS || kind == MFA_FORM_HELMHOLTZ || prm->precision != MFA_PREC_FP64 || !rule_ok)
      return fail(MFA_ERR_UNSUPPORTED,
                  "mfa_form_create: vector hex kernels cover FP64 Laplace/elasticity (p+1 or p+2 points) and "
                  "hyperelasticity (p+1, or 2p+2 for p <= 3)");
  }
  if (ct == MFA_CELL_TET4) {
    const bool ok = (sp->ncomp == 1 && kind <= MFA_FORM_HELMHOLTZ) ||
                    (sp->degree >= 2 && sp->ncomp == 3 && kind >= MFA_FORM_LAPLACE && kind != MFA_FORM_HELMHOLTZ);
    if (!ok) return fail(MFA_ERR_UNSUPPORTED, "mfa_form_create: form %d on P%d x %d", kind, sp->degree, sp->ncomp);
    if (sp->degree >= 3 && prm->scatter == MFA_SCATTER_WARP)
      return fail(MFA_ERR_UNSUPPORTED, "mfa_form_create: warp-aggregated scatter on P%d", sp->degree);
  }
  MFA_CUDA(cudaSetDevice(ctx->device));
  mfa_form* f = new (std::nothrow) mfa_form();
  if (!f) return fail(MFA_ERR_OOM, "mfa_form_create: host allocation");
  f->ctx = ctx;
  f->device = ctx->device;
  f->space = sp;
  f->p = *prm;
  f->scatter = prm->scatter == MFA_SCATTER_AUTO ? MFA_SCATTER_ATOMIC : prm->scatter;
  f->launch.variant = default_variant(sp, prm->qdeg > 0 ? prm->qdeg : sp->degree + 1, prm->precision);
  if (tri_cell_ok(f) || tet_pk_cell_ok(f)) f->launch.variant = MFA_VARIANT_CELL;
  int rc = MFA_OK;
  if (f->scatter == MFA_SCATTER_WARP) {
    // the warp-aggregated scatter is compiled for the point kernel (scalar hex, p+1 points) and the tet kernels
    if (ct == MFA_CELL_HEX8 && (sp->ncomp != 1 || (prm->qdeg > 0 && prm->qdeg != sp->degree + 1)))
      rc = fail(MFA_ERR_UNSUPPORTED, "mfa_form_create: warp-aggregated scatter on this hex form");
    if (ct == MFA_CELL_HEX8) f->launch.variant = MFA_VARIANT_POINT;
  }
  if (prm->cells_per_block != 0) {
    int opts[4];
    const int nopt = cb_options(f, f->launch.variant, opts);
    bool found = false;
    for (int i = 0; i < nopt; ++i) found = found || opts[i] == prm->cells_per_block;
    if (!found)
      rc = fail(MFA_ERR_UNSUPPORTED, "mfa_form_create: %d cells per block is not compiled for this form",
                prm->cells_per_block);
    f->launch.cb = prm->cells_per_block;
  }
  if (!rc && ct == MFA_CELL_QUAD4) {
    const int n = sp->degree + 1;
    f->nq1 = prm->qdeg > 0 ? prm->qdeg : n;
    rc = hex_tables(f);  // 1D tables: the same B, D, points and weights
    f->nq = f->nq1 * f->nq1;
    if (!rc) {
      const int ng = mfa::quad_geom_entries(kind);
      f->gstride = (int64_t)ng * f->nq;
      rc = cuda_alloc((void**)&f->d_geom, sizeof(double) * f->gstride * sp->mesh->ncell, "geometric factors");
      if (!rc) {
        mfa::clear_stale_error();
        cudaError_t e = mfa::quad_geometry_launch(f->nq1, kind, kind == MFA_FORM_HELMHOLTZ ? prm->k2 : 1.0, f->hex,
                                                  sp->mesh->d_coords, sp->mesh->d_cell_vert, sp->mesh->ncell,
                                                  static_cast<double*>(f->d_geom), ctx->d_err, ctx->stream);
        if (e != cudaSuccess) rc = fail(MFA_ERR_CUDA, "geometry kernel: %s", cudaGetErrorString(e));
      }
      if (!rc) rc = mfa_sync(ctx);
    }
  } else if (!rc && ct == MFA_CELL_TRI3) {
    rc = tri_tables(f);
  } else if (!rc && ct == MFA_CELL_HEX8) {
    const int n = sp->degree + 1;
    f->nq1 = prm->qdeg > 0 ? prm->qdeg : n;
    const bool vec_2n = sp->ncomp == 3 && f->nq1 == 2 * n && n <= 4;  // validated above for the hyperelastic forms
    if (!(f->nq1 == n || (f->nq1 == n + 1 && n <= 7) || vec_2n) || n > 9)
      rc = fail(MFA_ERR_UNSUPPORTED, "mfa_form_create: Q%d with %d Gauss points per direction", sp->degree, f->nq1);
    if (!rc) rc = hex_tables(f);
    f->nq = f->nq1 * f->nq1 * f->nq1;
    if (!rc && prm->geometry == MFA_GEOM_ONTHEFLY) {
      // the trilinear map is recomputed at every point from the vertices: nothing to store
      f->launch.otf = true;
      f->launch.variant = MFA_VARIANT_POINT;
    } else if (!rc) {
      const int ng = mfa::hex_geom_entries(kind);
      const size_t esz = prm->precision == MFA_PREC_FP64 ? 8 : (prm->precision == MFA_PREC_FP32 ? 4 : 2);
      // FP32/BF16 blocks (line kernels) are padded to 16 bytes per cell, for the bulk copies, and further to
      // spread the kernels' factor reads over the shared-memory banks; their points run with x slowest
      f->gstride = (int64_t)ng * f->nq;
      if (prm->precision != MFA_PREC_FP64) f->gstride = mfa::line_geom_stride(f->nq1, ng, (int)esz);
      rc = cuda_alloc((void**)&f->d_geom, esz * f->gstride * sp->mesh->ncell, "geometric factors");
      const double c0 = kind == MFA_FORM_HELMHOLTZ ? prm->k2 : 1.0;
      if (!rc) {
        mfa::clear_stale_error();
        cudaError_t e = mfa::hex_geometry_launch(f->nq1, kind, prm->precision, c0, f->hex, sp->mesh->d_coords,
                                                 sp->mesh->d_cell_vert, sp->mesh->ncell, f->d_geom, f->gstride,
                                                 ctx->d_err, ctx->stream);
        if (e != cudaSuccess) rc = fail(MFA_ERR_CUDA, "geometry kernel: %s", cudaGetErrorString(e));
      }
      if (!rc) rc = mfa_sync(ctx);
    }
  } else if (!rc) {
    rc = tet_tables(f);
  }
  if (!rc && f->scatter == MFA_SCATTER_COLOUR) rc = build_colouring(sp);
  if (rc) {
    mfa_form_destroy(f);
    return rc;
  }
  count_work(f);
  f->setup_ms = now_ms() - t0;
  *out = f;
  return MFA_OK;
}

int mfa_form_set_coefficient(mfa_form* f, const double* u) {
  if (!f || !u) return fail(MFA_ERR_ARG, "mfa_form_set_coefficient: NULL argument");
  f->d_coef = u;
  return MFA_OK;
}

int mfa_form_get_info(const mfa_form* f, mfa_form_info* info) {
  if (!f || !info) return fail(MFA_ERR_ARG, "mfa_form_get_info: NULL argument");
  info->ncell = f->space->mesh->ncell;
  info->ndof = f->space->nnode * f->space->ncomp;
  info->nloc = f->space->nloc;
  info->nq = f->nq;
  info->ncolours = f->space->ncolours;
  info->scatter = f->scatter;
  info->flops = f->flops;
  info->flops_executed = f->flops_executed;
  info->bytes = f->bytes;
  info->setup_ms = f->setup_ms;
  return MFA_OK;
}

int mfa_form_set_dirichlet(mfa_form* f, const int32_t* dofs, int64_t n) {
  if (!f || n < 0 || (n > 0 && !dofs)) return fail(MFA_ERR_ARG, "mfa_form_set_dirichlet: bad argument");
  const int64_t ndof = f->space->nnode * f->space->ncomp;
  std::vector<uint8_t> mask(ndof, 0);
  for (int64_t i = 0; i < n; ++i) {
    if (dofs[i] < 0 || dofs[i] >= ndof)
      return fail(MFA_ERR_RANGE, "mfa_form_set_dirichlet: dof %d outside [0, %lld)", dofs[i], (long long)ndof);
    mask[dofs[i]] = 1;
  }
  MFA_CUDA(cudaSetDevice(f->ctx->device));
  MFA_CUDA(cudaStreamSynchronize(f->ctx->stream));  // no apply of this form may still use the old buffers
  cudaFree(f->d_dir_mask);
  cudaFree(f->d_dir_x);
  cudaFree(f->d_dir_y);
  f->d_dir_mask = nullptr;
  f->d_dir_x = f->d_dir_y = nullptr;
  f->ndir = 0;
  if (n == 0) return MFA_OK;
  int rc = cuda_alloc((void**)&f->d_dir_mask, ndof > 0 ? ndof : 1, "dirichlet mask");
  if (!rc) rc = cuda_alloc((void**)&f->d_dir_x, sizeof(double) * (ndof > 0 ? ndof : 1), "dirichlet work");
  if (!rc) rc = cuda_alloc((void**)&f->d_dir_y, sizeof(double) * (ndof > 0 ? ndof : 1), "dirichlet work");
  if (!rc && cudaMemcpy(f->d_dir_mask, mask.data(), ndof, cudaMemcpyHostToDevice) != cudaSuccess)
    rc = fail(MFA_ERR_CUDA, "mfa_form_set_dirichlet: upload");
  if (rc) {
    cudaFree(f->d_dir_mask);
    cudaFree(f->d_dir_x);
    cudaFree(f->d_dir_y);
    f->d_dir_mask = nullptr;
    f->d_dir_x = f->d_dir_y = nullptr;
    return rc;
  }
  int64_t count = 0;
  for (uint8_t m : mask) count += m;
  f->ndir = count;
  return MFA_OK;
}

int mfa_form_list_configs(const mfa_form* f, mfa_launch_config* out, int max, int* count) {
  if (!f || !count || max < 0 || (max > 0 && !out)) return fail(MFA_ERR_ARG, "mfa_form_list_configs: bad argument");
  const std::vector<mfa_launch_config> all = form_configs(f);
  for (int i = 0; i < max && i < (int)all.size(); ++i) out[i] = all[i];
  *count = (int)all.size();
  return MFA_OK;
}

int mfa_form_get_config(const mfa_form* f, mfa_launch_config* cfg) {
  if (!f || !cfg) return fail(MFA_ERR_ARG, "mfa_form_get_config: NULL argument");
  int opts[4];
  const int nopt = cb_options(f, f->launch.variant, opts);
  *cfg = mfa_launch_config{};
  cfg->variant = f->launch.variant;
  cfg->cells_per_block = f->launch.cb ? f->launch.cb : (nopt > 0 ? opts[0] : 0);
  cfg->scatter = f->scatter;
  cfg->geometry = f->launch.otf ? MFA_GEOM_ONTHEFLY : MFA_GEOM_STORED;
  cfg->max_blocks = f->launch.max_blocks;
  cfg->ms = f->tuned_ms;
  return MFA_OK;
}

int mfa_form_set_config(mfa_form* f, const mfa_launch_config* cfg) {
  if (!f || !cfg) return fail(MFA_ERR_ARG, "mfa_form_set_config: NULL argument");
  mfa_launch_config want = *cfg;
  if (want.max_blocks < 0) return fail(MFA_ERR_ARG, "mfa_form_set_config: max_blocks %d < 0", want.max_blocks);
  const mfa_space* sp = f->space;
  if (want.variant == MFA_VARIANT_AUTO) {
    want.variant = default_variant(sp, f->nq1, f->p.precision);
    if (tri_cell_ok(f) || tet_pk_cell_ok(f)) want.variant = MFA_VARIANT_CELL;
    if (sp->mesh->cell_type == MFA_CELL_HEX8 && !f->d_geom) want.variant = MFA_VARIANT_POINT;
  }
  if (want.cells_per_block == 0) {
    int opts[4];
    if (cb_options(f, want.variant, opts) > 0) want.cells_per_block = opts[0];
  }
  bool found = false;
  for (const mfa_launch_config& c : form_configs(f))
    found = found || (c.variant == want.variant && c.cells_per_block == want.cells_per_block &&
                      c.scatter == want.scatter && c.geometry == want.geometry);
  if (!found)
    return fail(MFA_ERR_UNSUPPORTED,
                "mfa_form_set_config: variant %d, %d cells per block, scatter %d, geometry %d not available",
                want.variant, want.cells_per_block, want.scatter, want.geometry);
  if (want.scatter == MFA_SCATTER_COLOUR) {
    int rc = build_colouring(f->space);
    if (rc) return rc;
  }
  f->launch.variant = want.variant;
  f->launch.cb = want.cells_per_block;
  f->launch.otf = want.geometry == MFA_GEOM_ONTHEFLY;
  f->launch.max_blocks = want.max_blocks;
  f->scatter = want.scatter;
  f->tuned_ms = 0.0;
  count_work(f);
  return MFA_OK;
}

int mfa_form_autotune(mfa_ctx* ctx, mfa_form* f, const double* x, double* y, int reps, mfa_launch_config* tried,
                      int max_tried, int* ntried) {
  if (!ctx || !f || !x || !y || !ntried || reps < 1 || max_tried < 0 || (max_tried > 0 && !tried))
    return fail(MFA_ERR_ARG, "mfa_form_autotune: bad argument");
  if (f->ctx != ctx) return fail(MFA_ERR_ARG, "mfa_form_autotune: form belongs to another context");
  if ((const void*)x == (const void*)y) return fail(MFA_ERR_ARG, "mfa_form_autotune: x and y alias");
  if (f->p.kind == MFA_FORM_HYPER_JAC && !f->d_coef)
    return fail(MFA_ERR_ARG, "mfa_form_autotune: HYPER_JAC needs mfa_form_set_coefficient");
  MFA_CUDA(cudaSetDevice(ctx->device));
  std::vector<mfa_launch_config> all = form_configs(f);
  const mfa::LaunchConfig keep_launch = f->launch;
  const int keep_scatter = f->scatter;
  cudaEvent_t ev[2];
  MFA_CUDA(cudaEventCreate(&ev[0]));
  if (cudaEventCreate(&ev[1]) != cudaSuccess) {
    cudaEventDestroy(ev[0]);
    return fail(MFA_ERR_CUDA, "mfa_form_autotune: cudaEventCreate");
  }
  int best = -1, rc = MFA_OK;
  for (size_t i = 0; i < all.size() && rc == MFA_OK; ++i) {
    mfa_launch_config& c = all[i];
    c.ms = -1.0;
    if (mfa_form_set_config(f, &c) != MFA_OK) continue;  // e.g. colouring needs more than 64 colours
    // untimed first apply (first-use setup of the variant).  A refused launch
    // leaves the context intact and skips the configuration; an error seen at
    // the synchronisation (a device fault or a kernel's error flag) ends the
    // tuning with that status.
    int r = mfa_apply(ctx, f, x, y, 0);
    int s = mfa_sync(ctx);
    if (s != MFA_OK) {
      rc = s;
      break;
    }
    if (r != MFA_OK) continue;
    cudaEventRecord(ev[0], ctx->stream);
    for (int k = 0; k < reps && r == MFA_OK; ++k) r = mfa_apply(ctx, f, x, y, 0);
    cudaEventRecord(ev[1], ctx->stream);
    s = mfa_sync(ctx);
    if (s != MFA_OK) {
      rc = s;
      break;
    }
    if (r != MFA_OK) continue;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess) continue;
    c.ms = ms / reps;
    if (best < 0 || c.ms < all[best].ms) best = (int)i;
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  for (int i = 0; i < max_tried && i < (int)all.size(); ++i) tried[i] = all[i];
  *ntried = (int)all.size();
  if (rc == MFA_OK && best < 0) rc = fail(MFA_ERR_CUDA, "mfa_form_autotune: no configuration ran");
  if (rc != MFA_OK) {
    f->launch = keep_launch;
    f->scatter = keep_scatter;
    count_work(f);
    return rc;
  }
  rc = mfa_form_set_config(f, &all[best]);
  if (rc == MFA_OK) f->tuned_ms = all[best].ms;
  return rc;
}

int mfa_form_destroy(mfa_form* f) {
  if (!f) return MFA_OK;
  cudaSetDevice(f->device);
  cudaFree(f->d_geom);
  cudaFree(f->d_tdense);
  cudaFree(f->d_dir_mask);
  cudaFree(f->d_dir_x);
  cudaFree(f->d_dir_y);
  cudaFree(f->d_stage_x);
  cudaFree(f->d_stage_y);
  delete f;
  return MFA_OK;
}

int mfa_apply(mfa_ctx* ctx, mfa_form* f, const double* x, double* y, int accumulate) {
  if (!ctx || !f || !x || !y) return fail(MFA_ERR_ARG, "mfa_apply: NULL argument");
  if (f->ctx != ctx) return fail(MFA_ERR_ARG, "mfa_apply: form belongs to another context");
  if ((const void*)x == (const void*)y) return fail(MFA_ERR_ARG, "mfa_apply: x and y alias");
  if (f->p.kind == MFA_FORM_HYPER_JAC && !f->d_coef)
    return fail(MFA_ERR_ARG, "mfa_apply: HYPER_JAC needs mfa_form_set_coefficient");
  MFA_CUDA(cudaSetDevice(ctx->device));
  const int64_t ndof = f->space->nnode * f->space->ncomp;
  if (!accumulate) MFA_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * ndof, ctx->stream));
  return mfa::apply_form(f, x, y, ctx->stream);
}

int mfa_apply_f32(mfa_ctx* ctx, mfa_form* f, const float* x, float* y, int accumulate) {
  if (!ctx || !f || !x || !y) return fail(MFA_ERR_ARG, "mfa_apply_f32: NULL argument");
  if (f->ctx != ctx) return fail(MFA_ERR_ARG, "mfa_apply_f32: form belongs to another context");
  if ((const void*)x == (const void*)y) return fail(MFA_ERR_ARG, "mfa_apply_f32: x and y alias");
  if (f->p.precision == MFA_PREC_FP64) return fail(MFA_ERR_ARG, "mfa_apply_f32: needs an FP32 or BF16 form");
  if (f->d_dir_mask) return fail(MFA_ERR_UNSUPPORTED, "mfa_apply_f32: forms with Dirichlet constraints");
  MFA_CUDA(cudaSetDevice(ctx->device));
  mfa_space* sp = f->space;
  const int64_t ndof = sp->nnode * sp->ncomp;
  if (!accumulate) MFA_CUDA(cudaMemsetAsync(y, 0, sizeof(float) * ndof, ctx->stream));
  cudaError_t e = mfa::hex_apply_launch_f32(sp->degree + 1, f->p.kind, f->p.precision, x, y, sp->d_cell_node,
                                            f->d_geom, sp->mesh->ncell, f->gstride, ctx->d_err, mfa::GridBudget{ctx->sm_count, f->launch.max_blocks},
                                            ctx->stream);
  if (e != cudaSuccess) return fail(MFA_ERR_CUDA, "mfa_apply_f32: %s", cudaGetErrorString(e));
  return MFA_OK;
}

int mfa_convert_f64_to_f32(mfa_ctx* ctx, const double* x, float* y, int64_t n) {
  if (!ctx || (n > 0 && (!x || !y)) || n < 0) return fail(MFA_ERR_ARG, "mfa_convert_f64_to_f32: bad arguments");
  MFA_CUDA(cudaSetDevice(ctx->device));
  cudaError_t e = mfa::convert_d2f_launch(x, y, n, ctx->stream);
  return e == cudaSuccess ? MFA_OK : fail(MFA_ERR_CUDA, "mfa_convert_f64_to_f32: %s", cudaGetErrorString(e));
}

int mfa_convert_f32_to_f64(mfa_ctx* ctx, const float* x, double* y, int64_t n) {
  if (!ctx || (n > 0 && (!x || !y)) || n < 0) return fail(MFA_ERR_ARG, "mfa_convert_f32_to_f64: bad arguments");
  MFA_CUDA(cudaSetDevice(ctx->device));
  cudaError_t e = mfa::convert_f2d_launch(x, y, n, ctx->stream);
  return e == cudaSuccess ? MFA_OK : fail(MFA_ERR_CUDA, "mfa_convert_f32_to_f64: %s", cudaGetErrorString(e));
}

int mfa_apply_host(mfa_ctx* ctx, mfa_form* f, const double* xh, double* yh) {
  if (!ctx || !f || !xh || !yh) return fail(MFA_ERR_ARG, "mfa_apply_host: NULL argument");
  MFA_CUDA(cudaSetDevice(ctx->device));
  const int64_t ndof = f->space->nnode * f->space->ncomp;
  int rc = MFA_OK;
  if (!f->d_stage_x) rc = cuda_alloc((void**)&f->d_stage_x, sizeof(double) * ndof, "staging x");
  if (!rc && !f->d_stage_y) rc = cuda_alloc((void**)&f->d_stage_y, sizeof(double) * ndof, "staging y");
  if (rc) return rc;
  MFA_CUDA(cudaMemcpyAsync(f->d_stage_x, xh, sizeof(double) * ndof, cudaMemcpyHostToDevice, ctx->stream));
  rc = mfa_apply(ctx, f, f->d_stage_x, f->d_stage_y, 0);
  if (rc) return rc;
  MFA_CUDA(cudaMemcpyAsync(yh, f->d_stage_y, sizeof(double) * ndof, cudaMemcpyDeviceToHost, ctx->stream));
  return mfa_sync(ctx);
}

int mfa_apply_host_many(mfa_ctx* ctx, int n, mfa_form* const* forms, const double* const* xh, double* const* yh) {
  if (!ctx || n < 0 || (n > 0 && (!forms || !xh || !yh))) return fail(MFA_ERR_ARG, "mfa_apply_host_many: bad argument");
  for (int i = 0; i < n; ++i) {
    if (!forms[i] || !xh[i] || !yh[i]) return fail(MFA_ERR_ARG, "mfa_apply_host_many: NULL entry %d", i);
    for (int j = 0; j < i; ++j)
      if (forms[j] == forms[i]) return fail(MFA_ERR_ARG, "mfa_apply_host_many: form %d repeated", i);
  }
  MFA_CUDA(cudaSetDevice(ctx->device));
  if (!ctx->copy_in) MFA_CUDA(cudaStreamCreateWithFlags(&ctx->copy_in, cudaStreamNonBlocking));
  if (!ctx->copy_out) MFA_CUDA(cudaStreamCreateWithFlags(&ctx->copy_out, cudaStreamNonBlocking));
  while ((int)ctx->events.size() < 2 * n + 1) {
    cudaEvent_t e;
    MFA_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ctx->events.push_back(e);
  }
  for (int i = 0; i < n; ++i) {
    mfa_form* f = forms[i];
    const int64_t ndof = f->space->nnode * f->space->ncomp;
    int rc = MFA_OK;
    if (!f->d_stage_x) rc = cuda_alloc((void**)&f->d_stage_x, sizeof(double) * ndof, "staging x");
    if (!rc && !f->d_stage_y) rc = cuda_alloc((void**)&f->d_stage_y, sizeof(double) * ndof, "staging y");
    if (rc) return rc;
  }
  // the copies in start after whatever the context stream already holds (a staging buffer may still be in use)
  cudaEvent_t start = ctx->events[2 * n];
  MFA_CUDA(cudaEventRecord(start, ctx->stream));
  MFA_CUDA(cudaStreamWaitEvent(ctx->copy_in, start, 0));
  for (int i = 0; i < n; ++i) {
    mfa_form* f = forms[i];
    const int64_t ndof = f->space->nnode * f->space->ncomp;
    cudaEvent_t in_done = ctx->events[2 * i], applied = ctx->events[2 * i + 1];
    MFA_CUDA(cudaMemcpyAsync(f->d_stage_x, xh[i], sizeof(double) * ndof, cudaMemcpyHostToDevice, ctx->copy_in));
    MFA_CUDA(cudaEventRecord(in_done, ctx->copy_in));
    MFA_CUDA(cudaStreamWaitEvent(ctx->stream, in_done, 0));
    const int rc = mfa_apply(ctx, f, f->d_stage_x, f->d_stage_y, 0);
    if (rc) {
      cudaStreamSynchronize(ctx->copy_in);
      cudaStreamSynchronize(ctx->copy_out);
      return rc;
    }
    MFA_CUDA(cudaEventRecord(applied, ctx->stream));
    MFA_CUDA(cudaStreamWaitEvent(ctx->copy_out, applied, 0));
    MFA_CUDA(cudaMemcpyAsync(yh[i], f->d_stage_y, sizeof(double) * ndof, cudaMemcpyDeviceToHost, ctx->copy_out));
  }
  MFA_CUDA(cudaStreamSynchronize(ctx->copy_in));
  MFA_CUDA(cudaStreamSynchronize(ctx->copy_out));
  return mfa_sync(ctx);
}

int mfa_sync(mfa_ctx* ctx) {
  if (!ctx) return fail(MFA_ERR_ARG, "mfa_sync: ctx is NULL");
  MFA_CUDA(cudaSetDevice(ctx->device));
  MFA_CUDA(cudaStreamSynchronize(ctx->stream));
  int flag = 0;
  MFA_CUDA(cudaMemcpy(&flag, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    MFA_CUDA(cudaMemset(ctx->d_err, 0, sizeof(int)));
    if (flag & 4) return fail(MFA_ERR_TIMEOUT, "a kernel gave up waiting for a bulk copy");
    if (flag & 8) return fail(MFA_ERR_RANGE, "a halo node id was outside [0, nnode)");
    return fail(MFA_ERR_DOMAIN, "kernel reported %s%s", (flag & 1) ? "det J == 0 or non-finite " : "",
                (flag & 2) ? "deformation with J <= 0" : "");
  }
  return MFA_OK;
}

int mfa_diagonal(mfa_ctx* ctx, mfa_form* f, double* d) {
  if (!ctx || !f || !d) return fail(MFA_ERR_ARG, "mfa_diagonal: NULL argument");
  if (f->p.kind == MFA_FORM_HYPER_RES || f->p.kind == MFA_FORM_HYPER_JAC)
    return fail(MFA_ERR_UNSUPPORTED, "mfa_diagonal: linear forms only");
  MFA_CUDA(cudaSetDevice(ctx->device));
  mfa_space* sp = f->space;
  const int ct = sp->mesh->cell_type;
  const int64_t ndof = sp->nnode * sp->ncomp;
  if ((ct == MFA_CELL_HEX8 || ct == MFA_CELL_QUAD4) && f->p.precision != MFA_PREC_FP64)
    return fail(MFA_ERR_UNSUPPORTED, "mfa_diagonal: FP64 forms only");
  if ((ct == MFA_CELL_HEX8 || ct == MFA_CELL_QUAD4) && !f->d_geom)
    return fail(MFA_ERR_UNSUPPORTED, "mfa_diagonal: needs stored geometric factors");
  MFA_CUDA(cudaMemsetAsync(d, 0, sizeof(double) * ndof, ctx->stream));
  mfa::clear_stale_error();
  cudaError_t e;
  const auto dense_args = [&]() {  // the [q][a] tables of the P3+ tets and the triangles
    const int dim = ct == MFA_CELL_TRI3 ? 2 : 3;
    const int64_t nb = (int64_t)sp->nloc * f->tdense_nq;
    mfa::TetDenseArgs a{};
    a.coords = sp->mesh->d_coords;
    a.cell_vert = sp->mesh->d_cell_vert;
    a.cell_node = sp->d_cell_node;
    a.count = sp->mesh->ncell;
    a.phi_aq = f->d_tdense;
    a.dphi_aeq = a.phi_aq + nb;
    a.phi_qa = a.dphi_aeq + dim * nb;
    a.dphi_qae = a.phi_qa + nb;
    a.w = a.dphi_qae + dim * nb;
    a.nq = f->tdense_nq;
    a.k2 = f->p.k2;
    a.lambda = f->p.lambda;
    a.mu = f->p.mu;
    a.err = ctx->d_err;
    return a;
  };
  if (ct == MFA_CELL_HEX8 && sp->ncomp == 1) {
    e = mfa::hex_diagonal_launch(sp->degree + 1, f->nq1, f->p.kind, f->hex, sp->d_cell_node,
                                 static_cast<const double*>(f->d_geom),
                                 sp->mesh->ncell, d, mfa::GridBudget{ctx->sm_count, 0}, ctx->stream);
  } else if (ct == MFA_CELL_HEX8 || ct == MFA_CELL_QUAD4) {
    e = mfa::tensor_diagonal_launch(ct == MFA_CELL_HEX8 ? 3 : 2, sp->ncomp, sp->degree + 1, f->nq1, f->p.kind, f->hex,
                                    sp->d_cell_node, static_cast<const double*>(f->d_geom), f->gstride,
                                    sp->mesh->ncell, f->p.lambda, f->p.mu, d, ctx->stream);
  } else if (ct == MFA_CELL_TRI3 || sp->degree >= 3) {
    e = mfa::simplex_diagonal_launch(ct == MFA_CELL_TRI3 ? 2 : 3, sp->ncomp, sp->nloc, f->p.kind, dense_args(), d,
                                     ctx->stream);
  } else {
    mfa::TetApplyArgs a = tet_args(f, nullptr, nullptr);
    e = mfa::tet_diagonal_launch(sp->degree, sp->ncomp, f->p.kind, f->tet, a, d, ctx->stream);
  }
  if (e == cudaSuccess && f->d_dir_mask) e = mfa::dirichlet_diag_launch(f->d_dir_mask, d, ndof, ctx->stream);
  if (e != cudaSuccess) return fail(MFA_ERR_CUDA, "diagonal kernel: %s", cudaGetErrorString(e));
  return MFA_OK;
}

int mfa_cg(mfa_ctx* ctx, mfa_form* f, int precond, const double* b, double* x, double rtol, int maxit, int* iters,
           double* relres) {
  if (!ctx || !f || !b || !x) return fail(MFA_ERR_ARG, "mfa_cg: NULL argument");
  if (precond != MFA_PC_NONE && precond != MFA_PC_JACOBI) return fail(MFA_ERR_ARG, "mfa_cg: precond %d", precond);
  if (f->p.kind > MFA_FORM_ELASTICITY && f->p.kind != MFA_FORM_HYPER_JAC)
    return fail(MFA_ERR_ARG, "mfa_cg: the residual form is not linear");
  if (!(rtol > 0.0) || maxit < 0) return fail(MFA_ERR_ARG, "mfa_cg: rtol %g maxit %d", rtol, maxit);
  MFA_CUDA(cudaSetDevice(ctx->device));
  const int64_t n = f->space->nnode * f->space->ncomp;
  cudaStream_t s = ctx->stream;
  double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *dinv = nullptr;
  int rc = cuda_alloc((void**)&r, n * 8, "cg r");
  if (!rc) rc = cuda_alloc((void**)&z, n * 8, "cg z");
  if (!rc) rc = cuda_alloc((void**)&p, n * 8, "cg p");
  if (!rc) rc = cuda_alloc((void**)&q, n * 8, "cg q");
  if (!rc && precond == MFA_PC_JACOBI) rc = cuda_alloc((void**)&dinv, n * 8, "cg diag");
  double* partial = ctx->d_scratch;
  double* dres = ctx->d_scratch + mfa::dot_partials();
  auto dot = [&](const double* u, const double* v, double* out) -> int {
    cudaError_t e = mfa::dot_launch(u, v, n, partial, dres, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dres, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? MFA_OK : fail(MFA_ERR_CUDA, "mfa_cg dot: %s", cudaGetErrorString(e));
  };
  auto precondition = [&](const double* in, double* outv) -> int {
    cudaError_t e = precond == MFA_PC_JACOBI ? mfa::pointwise_mul_launch(dinv, in, outv, n, s)
                                             : cudaMemcpyAsync(outv, in, n * 8, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? MFA_OK : fail(MFA_ERR_CUDA, "mfa_cg precondition: %s", cudaGetErrorString(e));
  };
  int it = 0;
  double bnorm = 0.0, rr = 0.0, rz = 0.0, res = 0.0;
  if (!rc && precond == MFA_PC_JACOBI) {
    rc = mfa_diagonal(ctx, f, dinv);
    if (!rc && mfa::reciprocal_launch(dinv, dinv, n, s) != cudaSuccess) rc = fail(MFA_ERR_CUDA, "mfa_cg: reciprocal");
  }
  if (!rc) rc = dot(b, b, &bnorm);
  if (!rc) {
    bnorm = std::sqrt(bnorm);
    rc = mfa_apply(ctx, f, x, r, 0);  // r = b - A x
  }
  if (!rc && mfa::axpby_launch(1.0, b, -1.0, r, n, s) != cudaSuccess) rc = fail(MFA_ERR_CUDA, "mfa_cg: axpby");
  if (!rc) rc = dot(r, r, &rr);
  if (!rc) rc = precondition(r, z);
  if (!rc) rc = dot(r, z, &rz);
  if (!rc && cudaMemcpyAsync(p, z, n * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess) rc = fail(MFA_ERR_CUDA, "copy");
  res = bnorm > 0.0 ? std::sqrt(rr) / bnorm : std::sqrt(rr);
  if (!rc && (!std::isfinite(bnorm) || !std::isfinite(rr) || !std::isfinite(rz)))
    rc = fail(MFA_ERR_BREAKDOWN, "mfa_cg: non-finite right-hand side or initial residual");
  while (!rc && res > rtol && it < maxit) {
    double pq = 0.0;
    rc = mfa_apply(ctx, f, p, q, 0);
    if (!rc) rc = dot(p, q, &pq);
    if (rc) break;
    if (!(pq > 0.0) || !std::isfinite(pq) || !std::isfinite(rz)) {
      rc = fail(MFA_ERR_BREAKDOWN, "mfa_cg: breakdown at iteration %d (p.Ap = %g)", it, pq);
      break;
    }
    const double alpha = rz / pq;
    if (mfa::axpby_launch(alpha, p, 1.0, x, n, s) != cudaSuccess ||
        mfa::axpby_launch(-alpha, q, 1.0, r, n, s) != cudaSuccess) {
      rc = fail(MFA_ERR_CUDA, "mfa_cg: update");
      break;
    }
    rc = dot(r, r, &rr);
    ++it;
    if (rc) break;
    if (!std::isfinite(rr)) {
      rc = fail(MFA_ERR_BREAKDOWN, "mfa_cg: non-finite residual at iteration %d", it);
      break;
    }
    res = bnorm > 0.0 ? std::sqrt(rr) / bnorm : std::sqrt(rr);
    if (res <= rtol) break;
    double rz_new = 0.0;
    rc = precondition(r, z);
    if (!rc) rc = dot(r, z, &rz_new);
    if (rc) break;
    const double beta = rz_new / rz;
    rz = rz_new;
    if (mfa::axpby_launch(1.0, z, beta, p, n, s) != cudaSuccess) {
      rc = fail(MFA_ERR_CUDA, "mfa_cg: direction update");
      break;
    }
  }
  if (!rc) {
    int r2 = mfa_sync(ctx);
    if (r2) rc = r2;
  }
  if (!rc && res > rtol) rc = fail(MFA_ERR_NOT_CONVERGED, "mfa_cg: relative residual %g after %d iterations", res, it);
  if (iters) *iters = it;
  if (relres) *relres = res;
  cudaFree(r);
  cudaFree(z);
  cudaFree(p);
  cudaFree(q);
  cudaFree(dinv);
  return rc;
}

}  // extern "C"
