// Tetrahedral kernels: P1/P2 Lagrange on affine cells, one CUDA thread per
// cell.
//
// This is the GPU form of the paper's cross-element vectorisation (Section
// 3.1): the loop over cells is split across lanes, each lane runs the whole
// local kernel of one cell (Listing 2) and every lane executes the same
// instruction stream, with the quadrature and basis tables shared by all
// lanes (uniform loads from the constant bank).  The Jacobian is constant on
// an affine cell and computed once per cell (Listing 2, lines 8-20).
//
// Forms (Supplementary material): mass, Laplacian, Helmholtz (P1/P2 scalar,
// P2 vector Laplacian), linear elasticity, and the hyperelastic residual and
// Jacobian action for St Venant-Kirchhoff and compressible neo-Hookean laws.
#include "mfa_internal.h"
#include "physics.cuh"
#include "scatter.cuh"

namespace mfa {
namespace {

// SC: scatter mode, 0 atomic, 1 colour (plain read-modify-write), 2 warp-aggregated atomic.
template <int P, int NC, int KIND, int LAW, int NQ, int SC>
__global__ void __launch_bounds__(128) tet_apply_kernel(const __grid_constant__ TetTables tb, const TetApplyArgs a) {
  constexpr int NL = P == 1 ? 4 : 10;
  constexpr bool kValue = (KIND == MFA_FORM_MASS || KIND == MFA_FORM_HELMHOLTZ);
  constexpr bool kGrad = (KIND != MFA_FORM_MASS);
  constexpr bool kVector = (KIND >= MFA_FORM_ELASTICITY);
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < a.count;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = a.cell_list ? (int64_t)__ldg(a.cell_list + idx) : idx;
    // affine geometry: J[d][e] = X_{e+1}[d] - X_0[d]
    double X0[3], J[3][3];
    {
      const int32_t v0 = __ldg(a.cell_vert + 4 * cell);
#pragma unroll
      for (int d = 0; d < 3; ++d) X0[d] = __ldg(a.coords + 3 * (int64_t)v0 + d);
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        const int32_t ve = __ldg(a.cell_vert + 4 * cell + e + 1);
#pragma unroll
        for (int d = 0; d < 3; ++d) J[d][e] = __ldg(a.coords + 3 * (int64_t)ve + d) - X0[d];
      }
    }
    double cof[3][3];
    const double det = det3(J, cof);
    if (!(det != 0.0) || !isfinite(det)) {
      atomicOr(a.err, 1);
      continue;
    }
    const double idet = 1.0 / det;
    double Ji[3][3];  // J^{-1}[e][j] = cof[j][e] / det
#pragma unroll
    for (int e = 0; e < 3; ++e)
#pragma unroll
      for (int j = 0; j < 3; ++j) Ji[e][j] = cof[j][e] * idet;
    const double adet = fabs(det);

    int32_t node[NL];
    double xl[NL][NC], yl[NL][NC];
#pragma unroll
    for (int i = 0; i < NL; ++i) {
      node[i] = __ldg(a.cell_node + NL * cell + i);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        xl[i][c] = __ldg(a.x + (int64_t)NC * node[i] + c);
        yl[i][c] = 0.0;
      }
    }
    bool ok = true;
#pragma unroll 1
    for (int q = 0; q < NQ; ++q) {
      const double wd = tb.w[q] * adet;
      const double* phi = tb.phi + q * NL;
      const double* dphi = tb.dphi + q * NL * 3;
      double u[NC];
      double gr[NC][3];  // reference gradient d u_c / d xi_e
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        u[c] = 0.0;
        gr[c][0] = gr[c][1] = gr[c][2] = 0.0;
      }
#pragma unroll
      for (int i = 0; i < NL; ++i)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          if constexpr (kValue) u[c] = fma(phi[i], xl[i][c], u[c]);
          if constexpr (kGrad) {
            gr[c][0] = fma(xl[i][c], dphi[3 * i + 0], gr[c][0]);
            gr[c][1] = fma(xl[i][c], dphi[3 * i + 1], gr[c][1]);
            gr[c][2] = fma(xl[i][c], dphi[3 * i + 2], gr[c][2]);
          }
        }
      // h[c][e] = wd * sum_j f1[c][j] Ji[e][j]: the test-gradient flux pulled back to the reference cell
      double h[NC][3];
      double f0[NC];
      if constexpr (!kVector) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          f0[c] = 0.0;
          if constexpr (kValue) f0[c] = wd * (KIND == MFA_FORM_HELMHOLTZ ? a.k2 : 1.0) * u[c];
          if constexpr (kGrad) {
            double gx[3];
#pragma unroll
            for (int j = 0; j < 3; ++j) gx[j] = gr[c][0] * Ji[0][j] + gr[c][1] * Ji[1][j] + gr[c][2] * Ji[2][j];
#pragma unroll
            for (int e = 0; e < 3; ++e) h[c][e] = wd * (gx[0] * Ji[e][0] + gx[1] * Ji[e][1] + gx[2] * Ji[e][2]);
          }
        }
      } else {
        double gu[3][3], gc[3][3], f1[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int j = 0; j < 3; ++j) gu[c][j] = gr[c][0] * Ji[0][j] + gr[c][1] * Ji[1][j] + gr[c][2] * Ji[2][j];
        if constexpr (KIND == MFA_FORM_HYPER_JAC) {
          double gcr[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
          for (int i = 0; i < NL; ++i) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const double uc = __ldg(a.ucoef + 3 * (int64_t)node[i] + c);
              gcr[c][0] = fma(uc, dphi[3 * i + 0], gcr[c][0]);
              gcr[c][1] = fma(uc, dphi[3 * i + 1], gcr[c][1]);
              gcr[c][2] = fma(uc, dphi[3 * i + 2], gcr[c][2]);
            }
          }
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int j = 0; j < 3; ++j) gc[c][j] = gcr[c][0] * Ji[0][j] + gcr[c][1] * Ji[1][j] + gcr[c][2] * Ji[2][j];
        }
        ok = ok && physics<KIND, LAW>(gu, gc, a.lambda, a.mu, f1);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
#pragma unroll
          for (int e = 0; e < 3; ++e) h[c][e] = wd * (f1[c][0] * Ji[e][0] + f1[c][1] * Ji[e][1] + f1[c][2] * Ji[e][2]);
          f0[c] = 0.0;
        }
        if constexpr (KIND == MFA_FORM_HYPER_RES) {
          f0[0] = -wd * a.b0;
          f0[1] = -wd * a.b1;
          f0[2] = -wd * a.b2;
        }
      }
#pragma unroll
      for (int i = 0; i < NL; ++i)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          double s = yl[i][c];
          if constexpr (kValue || KIND == MFA_FORM_HYPER_RES) s = fma(f0[c], phi[i], s);
          if constexpr (kGrad) {
            s = fma(h[c][0], dphi[3 * i + 0], s);
            s = fma(h[c][1], dphi[3 * i + 1], s);
            s = fma(h[c][2], dphi[3 * i + 2], s);
          }
          yl[i][c] = s;
        }
    }
    if (!ok) atomicOr(a.err, 2);
#pragma unroll
    for (int i = 0; i < NL; ++i)
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int64_t at = (int64_t)NC * node[i] + c;
        if constexpr (SC == 1) a.y[at] += yl[i][c];
        else if constexpr (SC == 2) warp_aggregated_add(a.y, at, yl[i][c]);
        else atomicAdd(a.y + at, yl[i][c]);
      }
  }
}

// P2 vector hyperelastic forms by moments.  On an affine cell the reference
// gradient of each P2 basis function is linear, grad phi_a(xi) = alpha_a +
// beta_a xi, so with G0 = sum_a x_a alpha_a^T J^{-1} and G_f = sum_a x_a
// beta_a(.,f)^T J^{-1} the displacement gradient at a point is
// G0 + sum_f xi_f G_f (27 FMA instead of 117), and the test-side integral
// sum_q wd_q f1_q : grad phi_a(xi_q) only needs the moments
// K0 = sum_q wd_q f1_q and K_f = sum_q wd_q xi_qf f1_q (39 FMA per point
// instead of 120), mapped back once per cell.  The body force term is
// -b |det J| sum_q w_q phi_a(xi_q).  Same quadrature and physics as
// tet_apply_kernel; only the order of the sums changes.
//
// Neo-Hookean residual: P = mu F + s cof(F), s = (lambda ln J - mu) / J.
// F = I + G0 + sum_f xi_f G_f is linear in xi, so the moments of mu F are
// mu |det J| (W0 F0 + sum_f W1_f G_f) for K0 and
// mu |det J| (W1_f F0 + sum_g W2_fg G_g) for K_f, with F0 = I + G0 and the
// rule's weight moments W0 = sum_q w_q, W1_f = sum_q w_q xi_f,
// W2_fg = sum_q w_q xi_f xi_g: the point loop keeps only s cof(F).
template <int KIND, int LAW, int SC>
__global__ void __launch_bounds__(128) tet_moment_kernel(const __grid_constant__ TetTables tb, const TetApplyArgs a) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < a.count;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = a.cell_list ? (int64_t)__ldg(a.cell_list + idx) : idx;
    double X0[3], J[3][3];
    {
      const int32_t v0 = __ldg(a.cell_vert + 4 * cell);
#pragma unroll
      for (int d = 0; d < 3; ++d) X0[d] = __ldg(a.coords + 3 * (int64_t)v0 + d);
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        const int32_t ve = __ldg(a.cell_vert + 4 * cell + e + 1);
#pragma unroll
        for (int d = 0; d < 3; ++d) J[d][e] = __ldg(a.coords + 3 * (int64_t)ve + d) - X0[d];
      }
    }
    double cof[3][3];
    const double det = det3(J, cof);
    if (!(det != 0.0) || !isfinite(det)) {
      atomicOr(a.err, 1);
      continue;
    }
    const double idet = 1.0 / det;
    double Ji[3][3];
#pragma unroll
    for (int e = 0; e < 3; ++e)
#pragma unroll
      for (int j = 0; j < 3; ++j) Ji[e][j] = cof[j][e] * idet;
    const double adet = fabs(det);
    int32_t node[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) node[i] = __ldg(a.cell_node + 10 * cell + i);

    // moments of the gradient of a vector field with nodal values v (reference, then physical)
    auto moments = [&](const double* v, double (*G0)[3], double (*Gf)[3][3]) {
      double A[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, Bm[3][3][3];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int e = 0; e < 3; ++e)
#pragma unroll
          for (int f = 0; f < 3; ++f) Bm[c][e][f] = 0.0;
#pragma unroll
      for (int i = 0; i < 10; ++i)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const double xc = __ldg(v + 3 * (int64_t)node[i] + c);
#pragma unroll
          for (int e = 0; e < 3; ++e) {
            A[c][e] = fma(xc, tb.alpha[i * 3 + e], A[c][e]);
#pragma unroll
            for (int f = 0; f < 3; ++f) Bm[c][e][f] = fma(xc, tb.beta[i * 9 + e * 3 + f], Bm[c][e][f]);
          }
        }
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          G0[c][j] = A[c][0] * Ji[0][j] + A[c][1] * Ji[1][j] + A[c][2] * Ji[2][j];
#pragma unroll
          for (int f = 0; f < 3; ++f) Gf[f][c][j] = Bm[c][0][f] * Ji[0][j] + Bm[c][1][f] * Ji[1][j] + Bm[c][2][f] * Ji[2][j];
        }
    };
    double G0[3][3], Gf[3][3][3];
    moments(a.x, G0, Gf);
    double C0[3][3], Cf[3][3][3];
    if constexpr (KIND == MFA_FORM_HYPER_JAC) moments(a.ucoef, C0, Cf);

    double K0[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, K1[3][3][3];
#pragma unroll
    for (int f = 0; f < 3; ++f)
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int j = 0; j < 3; ++j) K1[f][c][j] = 0.0;
    bool ok = true;
    constexpr bool kSplitNH = KIND == MFA_FORM_HYPER_RES && LAW != MFA_LAW_SVK;
    if constexpr (kSplitNH) {
      G0[0][0] += 1.0;  // F0 = I + G0
      G0[1][1] += 1.0;
      G0[2][2] += 1.0;
#pragma unroll 1
      for (int q = 0; q < tb.nq; ++q) {
        const double x0 = tb.pts[3 * q], x1 = tb.pts[3 * q + 1], x2 = tb.pts[3 * q + 2];
        double F[3][3], cf[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int j = 0; j < 3; ++j) F[c][j] = fma(x2, Gf[2][c][j], fma(x1, Gf[1][c][j], fma(x0, Gf[0][c][j], G0[c][j])));
        const double Jq = det3(F, cf);
        if (!(Jq > 0.0)) {
          ok = false;
          continue;
        }
        const double t = tb.w[q] * adet * ((a.lambda * log(Jq) - a.mu) / Jq);
        const double t0 = t * x0, t1 = t * x1, t2 = t * x2;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            K0[c][j] = fma(t, cf[c][j], K0[c][j]);
            K1[0][c][j] = fma(t0, cf[c][j], K1[0][c][j]);
            K1[1][c][j] = fma(t1, cf[c][j], K1[1][c][j]);
            K1[2][c][j] = fma(t2, cf[c][j], K1[2][c][j]);
          }
      }
      const double ma = a.mu * adet;
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          double s0 = tb.wmom[0] * G0[c][j];
#pragma unroll
          for (int g = 0; g < 3; ++g) s0 = fma(tb.wmom[1 + g], Gf[g][c][j], s0);
          K0[c][j] = fma(ma, s0, K0[c][j]);
#pragma unroll
          for (int f = 0; f < 3; ++f) {
            double sf = tb.wmom[1 + f] * G0[c][j];
#pragma unroll
            for (int g = 0; g < 3; ++g) sf = fma(tb.wmom[4 + 3 * f + g], Gf[g][c][j], sf);
            K1[f][c][j] = fma(ma, sf, K1[f][c][j]);
          }
        }
    }
#pragma unroll 1
    for (int q = 0; q < (kSplitNH ? 0 : tb.nq); ++q) {
      const double x0 = tb.pts[3 * q], x1 = tb.pts[3 * q + 1], x2 = tb.pts[3 * q + 2];
      const double wd = tb.w[q] * adet;
      double gu[3][3], gc[3][3], f1[3][3];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          gu[c][j] = fma(x2, Gf[2][c][j], fma(x1, Gf[1][c][j], fma(x0, Gf[0][c][j], G0[c][j])));
          if constexpr (KIND == MFA_FORM_HYPER_JAC)
            gc[c][j] = fma(x2, Cf[2][c][j], fma(x1, Cf[1][c][j], fma(x0, Cf[0][c][j], C0[c][j])));
        }
      ok = ok && physics<KIND, LAW>(gu, gc, a.lambda, a.mu, f1);
      const double w0 = wd * x0, w1 = wd * x1, w2 = wd * x2;
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          K0[c][j] = fma(wd, f1[c][j], K0[c][j]);
          K1[0][c][j] = fma(w0, f1[c][j], K1[0][c][j]);
          K1[1][c][j] = fma(w1, f1[c][j], K1[1][c][j]);
          K1[2][c][j] = fma(w2, f1[c][j], K1[2][c][j]);
        }
    }
    if (!ok) atomicOr(a.err, 2);
    // back to the reference gradients: H0[c][e] = sum_j K0[c][j] Ji[e][j], H1[f][c][e] likewise
    double H0[3][3], H1[3][3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        H0[c][e] = K0[c][0] * Ji[e][0] + K0[c][1] * Ji[e][1] + K0[c][2] * Ji[e][2];
#pragma unroll
        for (int f = 0; f < 3; ++f) H1[f][c][e] = K1[f][c][0] * Ji[e][0] + K1[f][c][1] * Ji[e][1] + K1[f][c][2] * Ji[e][2];
      }
    const double bb[3] = {a.b0, a.b1, a.b2};
#pragma unroll
    for (int i = 0; i < 10; ++i)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double s = 0.0;
        if constexpr (KIND == MFA_FORM_HYPER_RES) s = -bb[c] * adet * tb.mvec[i];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          s = fma(tb.alpha[i * 3 + e], H0[c][e], s);
#pragma unroll
          for (int f = 0; f < 3; ++f) s = fma(tb.beta[i * 9 + e * 3 + f], H1[f][c][e], s);
        }
        const int64_t at = 3 * (int64_t)node[i] + c;
        if constexpr (SC == 1) a.y[at] += s;
        else if constexpr (SC == 2) warp_aggregated_add(a.y, at, s);
        else atomicAdd(a.y + at, s);
      }
  }
}

// Persistent grid of `threads`-thread blocks (one cell per thread), capped at
// the resident blocks of all SMs; `bps` caches the occupancy per block size.
template <typename Kern>
cudaError_t launch_cells(Kern kern, int (&bps)[4], int threads, const TetTables& tb, const TetApplyArgs& a,
                         GridBudget budget, cudaStream_t s) {
  if (a.count == 0) return cudaSuccess;
  if (threads != 32 && threads != 64 && threads != 128) return cudaErrorInvalidValue;
  int& b = bps[threads / 32 - 1];
  if (b < 0) {
    int v = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, threads, 0);
    if (e != cudaSuccess) return e;
    b = v < 1 ? 1 : v;
  }
  int64_t blocks = (a.count + threads - 1) / threads;
  const int64_t cap = budget.cap(b);
  if (blocks > cap) blocks = cap;
  kern<<<(unsigned)blocks, threads, 0, s>>>(tb, a);
  return cudaGetLastError();
}

// sc: scatter mode as for the kernels (0 atomic, 1 colour, 2 warp-aggregated)
template <int KIND, int LAW>
cudaError_t launch_moment(int sc, int threads, const TetTables& tb, const TetApplyArgs& a, GridBudget budget,
                          cudaStream_t s) {
  static int bps[3][4] = {{-1, -1, -1, -1}, {-1, -1, -1, -1}, {-1, -1, -1, -1}};  // per scatter mode and block size
  if (sc == 1) return launch_cells(tet_moment_kernel<KIND, LAW, 1>, bps[1], threads, tb, a, budget, s);
  if (sc == 2) return launch_cells(tet_moment_kernel<KIND, LAW, 2>, bps[2], threads, tb, a, budget, s);
  return launch_cells(tet_moment_kernel<KIND, LAW, 0>, bps[0], threads, tb, a, budget, s);
}

template <int P, int NC, int KIND, int LAW, int NQ, int SC>
cudaError_t launch(int threads, const TetTables& tb, const TetApplyArgs& a, GridBudget budget, cudaStream_t s) {
  static int bps[4] = {-1, -1, -1, -1};
  return launch_cells(tet_apply_kernel<P, NC, KIND, LAW, NQ, SC>, bps, threads, tb, a, budget, s);
}

template <int P, int NC, int KIND, int LAW, int NQ>
cudaError_t launch2(int sc, int threads, const TetTables& tb, const TetApplyArgs& a, GridBudget budget,
                    cudaStream_t s) {
  if (sc == 1) return launch<P, NC, KIND, LAW, NQ, 1>(threads, tb, a, budget, s);
  if (sc == 2) return launch<P, NC, KIND, LAW, NQ, 2>(threads, tb, a, budget, s);
  return launch<P, NC, KIND, LAW, NQ, 0>(threads, tb, a, budget, s);
}

// Diagonal of the linear forms, per local dof and cell:
//   scalar:      sum_q w|J| (c0 phi_a^2 + |grad phi_a|^2)
//   vector Lap.: sum_q w|J| |grad phi_a|^2
//   elasticity:  sum_q w|J| (mu |grad phi_a|^2 + (mu + lambda) (d_c phi_a)^2)
template <int NL, int NC>
__global__ void tet_diag_kernel(const __grid_constant__ TetTables tb, const TetApplyArgs a, int kind, double* d) {
  for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < a.count;
       cell += (int64_t)gridDim.x * blockDim.x) {
    double X0[3], J[3][3];
    const int32_t v0 = a.cell_vert[4 * cell];
    for (int k = 0; k < 3; ++k) X0[k] = a.coords[3 * (int64_t)v0 + k];
    for (int e = 0; e < 3; ++e) {
      const int32_t ve = a.cell_vert[4 * cell + e + 1];
      for (int k = 0; k < 3; ++k) J[k][e] = a.coords[3 * (int64_t)ve + k] - X0[k];
    }
    double cof[3][3];
    const double det = det3(J, cof);
    if (!(det != 0.0) || !isfinite(det)) {
      atomicOr(a.err, 1);
      continue;
    }
    const double adet = fabs(det);
    double c0 = kind == MFA_FORM_MASS ? 1.0 : (kind == MFA_FORM_HELMHOLTZ ? a.k2 : 0.0);
    const bool grad = kind != MFA_FORM_MASS;
    for (int i = 0; i < NL; ++i) {
      double acc[NC];
      for (int c = 0; c < NC; ++c) acc[c] = 0.0;
      for (int q = 0; q < tb.nq; ++q) {
        const double wd = tb.w[q] * adet;
        const double ph = tb.phi[q * NL + i];
        double g[3];
        for (int j = 0; j < 3; ++j)
          g[j] = (tb.dphi[(q * NL + i) * 3 + 0] * cof[j][0] + tb.dphi[(q * NL + i) * 3 + 1] * cof[j][1] +
                  tb.dphi[(q * NL + i) * 3 + 2] * cof[j][2]) / det;
        const double gg = grad ? g[0] * g[0] + g[1] * g[1] + g[2] * g[2] : 0.0;
        for (int c = 0; c < NC; ++c) {
          if (kind == MFA_FORM_ELASTICITY) acc[c] += wd * (a.mu * gg + (a.mu + a.lambda) * g[c] * g[c]);
          else acc[c] += wd * (c0 * ph * ph + gg);
        }
      }
      const int32_t node = a.cell_node[NL * cell + i];
      for (int c = 0; c < NC; ++c) atomicAdd(d + (int64_t)NC * node + c, acc[c]);
    }
  }
}

}  // namespace

cudaError_t tet_diagonal_launch(int p, int ncomp, int kind, const TetTables& tb, const TetApplyArgs& a, double* d,
                                cudaStream_t s) {
  if (a.count == 0) return cudaSuccess;
  int64_t blocks = (a.count + 127) / 128;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (p == 1 && ncomp == 1) tet_diag_kernel<4, 1><<<(unsigned)blocks, 128, 0, s>>>(tb, a, kind, d);
  else if (p == 2 && ncomp == 1) tet_diag_kernel<10, 1><<<(unsigned)blocks, 128, 0, s>>>(tb, a, kind, d);
  else if (p == 2 && ncomp == 3) tet_diag_kernel<10, 3><<<(unsigned)blocks, 128, 0, s>>>(tb, a, kind, d);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

int tet_cb_options(int* out) {
  out[0] = 128;
  out[1] = 64;
  out[2] = 32;
  return 3;
}

// Rules by form: P1 Laplace 1 point (degree 0), P1 mass / Helmholtz 4 (degree
// 2), P2 scalar mass / Helmholtz 14 (degree 4), P2 Laplace and elasticity 4
// (degree 2); the P2 hyperelastic moment kernel takes any rule of up to 27
// points (14 symmetric, 27 collapsed).
bool tet_rule_compiled(int p, int ncomp, int kind, int nq) {
  if (p == 1 && ncomp == 1)
    return (kind == MFA_FORM_LAPLACE && nq == 1) || ((kind == MFA_FORM_MASS || kind == MFA_FORM_HELMHOLTZ) && nq == 4);
  if (p == 2 && ncomp == 1)
    return (kind == MFA_FORM_LAPLACE && nq == 4) || ((kind == MFA_FORM_MASS || kind == MFA_FORM_HELMHOLTZ) && nq == 14);
  if (p == 2 && ncomp == 3) {
    if (kind == MFA_FORM_LAPLACE || kind == MFA_FORM_ELASTICITY) return nq == 4;
    if (kind == MFA_FORM_HYPER_RES || kind == MFA_FORM_HYPER_JAC) return nq >= 1 && nq <= kTetMaxQ;
  }
  return false;
}

cudaError_t tet_apply_launch(int p, int ncomp, int kind, int law, bool colour, bool agg, int threads,
                             const TetTables& tb, const TetApplyArgs& a, GridBudget budget, cudaStream_t s) {
  const int sc = colour ? 1 : (agg ? 2 : 0);
  if (!tet_rule_compiled(p, ncomp, kind, tb.nq)) return cudaErrorInvalidValue;
  if (p == 1) {
    switch (kind) {
      case MFA_FORM_MASS: return launch2<1, 1, MFA_FORM_MASS, 0, 4>(sc, threads, tb, a, budget, s);
      case MFA_FORM_LAPLACE: return launch2<1, 1, MFA_FORM_LAPLACE, 0, 1>(sc, threads, tb, a, budget, s);
      case MFA_FORM_HELMHOLTZ: return launch2<1, 1, MFA_FORM_HELMHOLTZ, 0, 4>(sc, threads, tb, a, budget, s);
    }
  }
  if (p == 2 && ncomp == 1) {
    switch (kind) {
      case MFA_FORM_MASS: return launch2<2, 1, MFA_FORM_MASS, 0, 14>(sc, threads, tb, a, budget, s);
      case MFA_FORM_LAPLACE: return launch2<2, 1, MFA_FORM_LAPLACE, 0, 4>(sc, threads, tb, a, budget, s);
      case MFA_FORM_HELMHOLTZ: return launch2<2, 1, MFA_FORM_HELMHOLTZ, 0, 14>(sc, threads, tb, a, budget, s);
    }
  }
  if (p == 2 && ncomp == 3) {
    switch (kind) {
      case MFA_FORM_LAPLACE: return launch2<2, 3, MFA_FORM_LAPLACE, 0, 4>(sc, threads, tb, a, budget, s);
      case MFA_FORM_ELASTICITY: return launch2<2, 3, MFA_FORM_ELASTICITY, 0, 4>(sc, threads, tb, a, budget, s);
      case MFA_FORM_HYPER_RES:
        return law == MFA_LAW_SVK ? launch_moment<MFA_FORM_HYPER_RES, MFA_LAW_SVK>(sc, threads, tb, a, budget, s)
                                  : launch_moment<MFA_FORM_HYPER_RES, MFA_LAW_NEOHOOKE>(sc, threads, tb, a, budget, s);
      case MFA_FORM_HYPER_JAC:
        return law == MFA_LAW_SVK ? launch_moment<MFA_FORM_HYPER_JAC, MFA_LAW_SVK>(sc, threads, tb, a, budget, s)
                                  : launch_moment<MFA_FORM_HYPER_JAC, MFA_LAW_NEOHOOKE>(sc, threads, tb, a, budget, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace mfa
