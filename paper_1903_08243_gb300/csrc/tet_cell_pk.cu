// Scalar P3/P4 tetrahedra, one thread per cell (the paper's one lane per
// entity, Section 3.1), on rules of at most 24 points.
//
// The warp-per-cell kernel (tet_dense.cu) spreads a cell's quadrature points
// over the lanes; on Table 2's fully symmetric rules (14 or 24 points) a
// quarter to a half of its lanes have no point.  Here each thread runs the
// whole local kernel of its cell: the affine geometry, then per point the
// value and reference gradient of u (a dense sum over the 20 or 35 local
// dofs), the pointwise term w|det J| (c0 u, G grad u), and the test-side sums
// into the cell's local result, all in registers.  The tabulated basis is a
// kernel parameter, read at the same address by every lane.
#include "mfa_internal.h"
#include "physics.cuh"

namespace mfa {
namespace {

template <int NL, int KIND, bool COLOUR>
__global__ void __launch_bounds__(128) tet_pk_cell_kernel(const __grid_constant__ TetPkTables tb,
                                                          const TetDenseArgs a) {
  constexpr bool kVal = KIND == MFA_FORM_MASS || KIND == MFA_FORM_HELMHOLTZ;
  constexpr bool kGrad = KIND != MFA_FORM_MASS;
  const int nq = tb.nq;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < a.count;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = a.cell_list ? (int64_t)__ldg(a.cell_list + idx) : idx;
    double J[3][3];
    {
      const int32_t v0 = __ldg(a.cell_vert + 4 * cell);
      double X0[3];
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
    const double idet = 1.0 / det, adet = fabs(det);
    // G[e][f] = sum_j (J^-1)[e][j] (J^-1)[f][j], (J^-1)[e][j] = cof[j][e] / det
    double G[3][3];
#pragma unroll
    for (int e = 0; e < 3; ++e)
#pragma unroll
      for (int f = e; f < 3; ++f) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < 3; ++j) s = fma(cof[j][e], cof[j][f], s);
        G[e][f] = G[f][e] = s * idet * idet;
      }
    double xl[NL], yl[NL];
#pragma unroll
    for (int al = 0; al < NL; ++al) {
      xl[al] = __ldg(a.x + __ldg(a.cell_node + NL * cell + al));
      yl[al] = 0.0;
    }
    const double c0 = KIND == MFA_FORM_HELMHOLTZ ? a.k2 : 1.0;
#pragma unroll 1
    for (int q = 0; q < nq; ++q) {
      const double* phi = tb.phi + q * NL;
      const double* dphi = tb.dphi + q * NL * 3;
      double u = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
#pragma unroll
      for (int al = 0; al < NL; ++al) {
        if constexpr (kVal) u = fma(phi[al], xl[al], u);
        if constexpr (kGrad) {
          g0 = fma(dphi[3 * al], xl[al], g0);
          g1 = fma(dphi[3 * al + 1], xl[al], g1);
          g2 = fma(dphi[3 * al + 2], xl[al], g2);
        }
      }
      const double wd = tb.w[q] * adet;
      const double sv = c0 * wd * u;
      double h0 = 0.0, h1 = 0.0, h2 = 0.0;
      if constexpr (kGrad) {
        h0 = wd * fma(G[0][0], g0, fma(G[0][1], g1, G[0][2] * g2));
        h1 = wd * fma(G[1][0], g0, fma(G[1][1], g1, G[1][2] * g2));
        h2 = wd * fma(G[2][0], g0, fma(G[2][1], g1, G[2][2] * g2));
      }
#pragma unroll
      for (int al = 0; al < NL; ++al) {
        double s = yl[al];
        if constexpr (kVal) s = fma(phi[al], sv, s);
        if constexpr (kGrad) {
          s = fma(dphi[3 * al], h0, s);
          s = fma(dphi[3 * al + 1], h1, s);
          s = fma(dphi[3 * al + 2], h2, s);
        }
        yl[al] = s;
      }
    }
#pragma unroll
    for (int al = 0; al < NL; ++al) {  // the map is read again here rather than kept in registers
      const int32_t node = __ldg(a.cell_node + NL * cell + al);
      if constexpr (COLOUR) a.y[node] += yl[al];
      else atomicAdd(a.y + node, yl[al]);
    }
  }
}

template <int NL, int KIND, bool COLOUR>
cudaError_t launch(int threads, const TetPkTables& tb, const TetDenseArgs& a, GridBudget budget, cudaStream_t s) {
  if (a.count == 0) return cudaSuccess;
  if (threads != 32 && threads != 64 && threads != 128) return cudaErrorInvalidValue;
  auto kern = tet_pk_cell_kernel<NL, KIND, COLOUR>;
  static int bps[4] = {-1, -1, -1, -1};
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

template <int NL, bool COLOUR>
cudaError_t by_kind(int kind, int threads, const TetPkTables& tb, const TetDenseArgs& a, GridBudget budget,
                    cudaStream_t s) {
  switch (kind) {
    case MFA_FORM_MASS: return launch<NL, MFA_FORM_MASS, COLOUR>(threads, tb, a, budget, s);
    case MFA_FORM_LAPLACE: return launch<NL, MFA_FORM_LAPLACE, COLOUR>(threads, tb, a, budget, s);
    case MFA_FORM_HELMHOLTZ: return launch<NL, MFA_FORM_HELMHOLTZ, COLOUR>(threads, tb, a, budget, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t tet_pk_cell_launch(int p, int kind, bool colour, int threads, const TetPkTables& tb,
                               const TetDenseArgs& a, GridBudget budget, cudaStream_t s) {
  if (tb.nq < 1 || tb.nq > kTetPkMaxQ) return cudaErrorInvalidValue;
  if (p == 3) return colour ? by_kind<20, true>(kind, threads, tb, a, budget, s)
                            : by_kind<20, false>(kind, threads, tb, a, budget, s);
  if (p == 4) return colour ? by_kind<35, true>(kind, threads, tb, a, budget, s)
                            : by_kind<35, false>(kind, threads, tb, a, budget, s);
  return cudaErrorInvalidValue;
}

}  // namespace mfa
