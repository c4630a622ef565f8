// Triangles P1..P4, one thread per cell: the planar counterpart of the P1/P2
// tet kernel (the paper's one lane per entity, Section 3.1).  A low-order
// triangle has 3-15 dofs and 1-25 quadrature points: too little work for a
// warp, so each thread runs the whole local kernel of its cell with the basis
// tables as kernel parameters (uniform loads).  Vector forms: plane strain.
#include "mfa_internal.h"
#include "physics.cuh"

namespace mfa {
namespace {

template <int NL, int NC, int KIND, int LAW, bool COLOUR>
__global__ void __launch_bounds__(128) tri_cell_kernel(const __grid_constant__ TriTables tb, const TetDenseArgs a) {
  constexpr bool kValIn = KIND == MFA_FORM_MASS || KIND == MFA_FORM_HELMHOLTZ;
  constexpr bool kValOut = kValIn || KIND == MFA_FORM_HYPER_RES;
  constexpr bool kGrad = KIND != MFA_FORM_MASS;
  constexpr bool kJac = KIND == MFA_FORM_HYPER_JAC;
  const int nq = tb.nq;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < a.count;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = a.cell_list ? (int64_t)__ldg(a.cell_list + idx) : idx;
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 1.0}};  // J_zz = 1: the plane
    {
      const int32_t v0 = __ldg(a.cell_vert + 3 * cell);
      const double X0[2] = {__ldg(a.coords + 3 * (int64_t)v0), __ldg(a.coords + 3 * (int64_t)v0 + 1)};
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int32_t ve = __ldg(a.cell_vert + 3 * cell + e + 1);
#pragma unroll
        for (int d = 0; d < 2; ++d) J[d][e] = __ldg(a.coords + 3 * (int64_t)ve + d) - X0[d];
      }
    }
    double cof[3][3];
    const double det = det3(J, cof);
    if (!(det != 0.0) || !isfinite(det)) {
      atomicOr(a.err, 1);
      continue;
    }
    const double idet = 1.0 / det, adet = fabs(det);
    double Ji[2][2];
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
      for (int j = 0; j < 2; ++j) Ji[e][j] = cof[j][e] * idet;
    const double G00 = Ji[0][0] * Ji[0][0] + Ji[0][1] * Ji[0][1], G11 = Ji[1][0] * Ji[1][0] + Ji[1][1] * Ji[1][1],
                 G01 = Ji[0][0] * Ji[1][0] + Ji[0][1] * Ji[1][1];
    int32_t node[NL];
    double xl[NL][NC], ul[NL][NC], yl[NL][NC];
#pragma unroll
    for (int al = 0; al < NL; ++al) {
      node[al] = __ldg(a.cell_node + NL * cell + al);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        xl[al][c] = __ldg(a.x + (int64_t)NC * node[al] + c);
        ul[al][c] = kJac ? __ldg(a.ucoef + (int64_t)NC * node[al] + c) : 0.0;
        yl[al][c] = 0.0;
      }
    }
    bool ok = true;
#pragma unroll 1
    for (int q = 0; q < nq; ++q) {
      const double* phi = tb.phi + q * kTriMaxNl;
      const double* dphi = tb.dphi + q * kTriMaxNl * 2;
      double u[NC], g[NC][2], gk[NC][2];
#pragma unroll
      for (int c = 0; c < NC; ++c) u[c] = g[c][0] = g[c][1] = gk[c][0] = gk[c][1] = 0.0;
#pragma unroll
      for (int al = 0; al < NL; ++al)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          if constexpr (kValIn) u[c] = fma(phi[al], xl[al][c], u[c]);
          if constexpr (kGrad) {
            g[c][0] = fma(dphi[2 * al], xl[al][c], g[c][0]);
            g[c][1] = fma(dphi[2 * al + 1], xl[al][c], g[c][1]);
          }
          if constexpr (kJac) {
            gk[c][0] = fma(dphi[2 * al], ul[al][c], gk[c][0]);
            gk[c][1] = fma(dphi[2 * al + 1], ul[al][c], gk[c][1]);
          }
        }
      const double wd = tb.w[q] * adet;
      double sv[NC], sh[NC][2];
      if constexpr (KIND <= MFA_FORM_HELMHOLTZ) {
        const double c0 = KIND == MFA_FORM_HELMHOLTZ ? a.k2 : 1.0;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          sv[c] = c0 * wd * u[c];
          sh[c][0] = wd * (G00 * g[c][0] + G01 * g[c][1]);
          sh[c][1] = wd * (G01 * g[c][0] + G11 * g[c][1]);
        }
      } else {
        double gu[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, gc[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, f1[3][3];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            gu[c][j] = g[c][0] * Ji[0][j] + g[c][1] * Ji[1][j];
            if constexpr (kJac) gc[c][j] = gk[c][0] * Ji[0][j] + gk[c][1] * Ji[1][j];
          }
        ok = physics<KIND, LAW>(gu, gc, a.lambda, a.mu, f1) && ok;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          sv[c] = KIND == MFA_FORM_HYPER_RES ? -(c == 0 ? a.b0 : a.b1) * wd : 0.0;
#pragma unroll
          for (int e = 0; e < 2; ++e) sh[c][e] = wd * (f1[c][0] * Ji[e][0] + f1[c][1] * Ji[e][1]);
        }
      }
#pragma unroll
      for (int al = 0; al < NL; ++al)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          double s = yl[al][c];
          if constexpr (kValOut) s = fma(phi[al], sv[c], s);
          if constexpr (kGrad) {
            s = fma(dphi[2 * al], sh[c][0], s);
            s = fma(dphi[2 * al + 1], sh[c][1], s);
          }
          yl[al][c] = s;
        }
    }
    if (!ok) atomicOr(a.err, 2);
#pragma unroll
    for (int al = 0; al < NL; ++al)
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        double* dst = a.y + (int64_t)NC * node[al] + c;
        if constexpr (COLOUR) *dst += yl[al][c];
        else atomicAdd(dst, yl[al][c]);
      }
  }
}

template <int NL, int NC, int KIND, int LAW, bool COLOUR>
cudaError_t launch(int threads, const TriTables& tb, const TetDenseArgs& a, GridBudget budget, cudaStream_t s) {
  if (a.count == 0) return cudaSuccess;
  if (threads != 32 && threads != 64 && threads != 128) return cudaErrorInvalidValue;
  auto kern = tri_cell_kernel<NL, NC, KIND, LAW, COLOUR>;
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

template <int NL, int NC, int KIND, int LAW>
cudaError_t launch2(bool colour, int threads, const TriTables& tb, const TetDenseArgs& a, GridBudget budget,
                    cudaStream_t s) {
  return colour ? launch<NL, NC, KIND, LAW, true>(threads, tb, a, budget, s)
                : launch<NL, NC, KIND, LAW, false>(threads, tb, a, budget, s);
}

template <int NL>
cudaError_t by_form(int ncomp, int kind, int law, bool colour, int threads, const TriTables& tb,
                    const TetDenseArgs& a, GridBudget budget, cudaStream_t s) {
  const bool nh = law == MFA_LAW_NEOHOOKE;
  if (ncomp == 1) {
    switch (kind) {
      case MFA_FORM_MASS: return launch2<NL, 1, MFA_FORM_MASS, 0>(colour, threads, tb, a, budget, s);
      case MFA_FORM_LAPLACE: return launch2<NL, 1, MFA_FORM_LAPLACE, 0>(colour, threads, tb, a, budget, s);
      case MFA_FORM_HELMHOLTZ: return launch2<NL, 1, MFA_FORM_HELMHOLTZ, 0>(colour, threads, tb, a, budget, s);
    }
    return cudaErrorInvalidValue;
  }
  switch (kind) {
    case MFA_FORM_LAPLACE: return launch2<NL, 2, MFA_FORM_LAPLACE, 0>(colour, threads, tb, a, budget, s);
    case MFA_FORM_ELASTICITY: return launch2<NL, 2, MFA_FORM_ELASTICITY, 0>(colour, threads, tb, a, budget, s);
    case MFA_FORM_HYPER_RES:
      return nh ? launch2<NL, 2, MFA_FORM_HYPER_RES, MFA_LAW_NEOHOOKE>(colour, threads, tb, a, budget, s)
                : launch2<NL, 2, MFA_FORM_HYPER_RES, MFA_LAW_SVK>(colour, threads, tb, a, budget, s);
    case MFA_FORM_HYPER_JAC:
      if constexpr (NL <= 10) {
        return nh ? launch2<NL, 2, MFA_FORM_HYPER_JAC, MFA_LAW_NEOHOOKE>(colour, threads, tb, a, budget, s)
                  : launch2<NL, 2, MFA_FORM_HYPER_JAC, MFA_LAW_SVK>(colour, threads, tb, a, budget, s);
      } else {
        return cudaErrorInvalidValue;  // P4: the linearisation point would spill; one warp per cell instead
      }
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t tri_cell_launch(int p, int ncomp, int kind, int law, bool colour, int threads, const TriTables& tb,
                            const TetDenseArgs& a, GridBudget budget, cudaStream_t s) {
  switch (p) {
    case 1: return by_form<3>(ncomp, kind, law, colour, threads, tb, a, budget, s);
    case 2: return by_form<6>(ncomp, kind, law, colour, threads, tb, a, budget, s);
    case 3: return by_form<10>(ncomp, kind, law, colour, threads, tb, a, budget, s);
    case 4: return by_form<15>(ncomp, kind, law, colour, threads, tb, a, budget, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mfa
