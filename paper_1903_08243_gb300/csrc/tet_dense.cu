// Simplex action by dense tabulation, one warp per cell: tetrahedra P3..P6 and triangles P1..P6.
//
// The paper's tet kernels (Listing 2) loop over quadrature points and local
// dofs with tabulated basis values; from P3 on a cell has 20-84 dofs and
// 27-343 points, too much work and state for one thread.  Here a warp owns a
// cell: in the point phase each lane takes one quadrature point of a chunk of
// 32 and interpolates the field and its reference gradient from the cell's
// dofs (staged in shared memory), evaluates the pointwise physics on the
// affine cell, and stages the fluxes; in the dof phase each lane takes
// (local dof, component) pairs and accumulates the test-side sums over the
// chunk's points (a vector P3 cell has 60 such pairs: two rounds of 32 lanes,
// 94% busy, where one lane per dof with its three components kept 20 of 32
// lanes busy).  Both
// phases read the basis tables (FP64, in global memory, cached in L1/L2) with
// consecutive lanes on consecutive addresses: [a][q] layout for the point
// phase, [q][a] for the dof phase.
#include "mfa_internal.h"
#include "physics.cuh"

namespace mfa {
namespace {

constexpr int kWarps = 8;  // cells (warps) per block

template <int NL, int NC, int KIND>
struct DenseShape {
  // staged per point: value term and reference flux (up to 3 directions) of each component
  static constexpr int S = 4 * NC;
  static constexpr int R = (NL * NC + 31) / 32;  // (dof, component) pairs per lane
  static constexpr int SMEM_WARP = 2 * NL * NC + 32 * S;  // doubles: x (and the coefficient), stage
};

// DIM = 3: tetrahedra (4 vertices); DIM = 2: triangles in the plane (3 vertices, plane strain for NC = 2).
template <int DIM, int NL, int NC, int KIND, int LAW, bool COLOUR>
__global__ void __launch_bounds__(32 * kWarps) simplex_dense_kernel(const TetDenseArgs a) {
  using SH = DenseShape<NL, NC, KIND>;
  constexpr int NV = DIM + 1;
  constexpr bool kValue = KIND == MFA_FORM_MASS || KIND == MFA_FORM_HELMHOLTZ || KIND == MFA_FORM_HYPER_RES;
  constexpr bool kGrad = KIND != MFA_FORM_MASS;
  constexpr bool kJac = KIND == MFA_FORM_HYPER_JAC;
  extern __shared__ __align__(16) double smem_d[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double* xl = smem_d + wid * SH::SMEM_WARP;  // [NL][NC]
  double* ul = xl + NL * NC;                  // [NL][NC] linearisation point
  double* st = ul + NL * NC;                  // [32][S]
  const int nq = a.nq;
  const double bb[3] = {a.b0, a.b1, a.b2};
  for (int64_t idx = blockIdx.x * (int64_t)kWarps + wid; idx < a.count; idx += (int64_t)gridDim.x * kWarps) {
    const int64_t cell = a.cell_list ? (int64_t)__ldg(a.cell_list + idx) : idx;
    // affine geometry (every lane, broadcast loads), embedded in 3x3 with J_zz = 1 in the plane
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    {
      const int32_t v0 = __ldg(a.cell_vert + NV * cell);
      double X0[3];
#pragma unroll
      for (int d = 0; d < DIM; ++d) X0[d] = __ldg(a.coords + 3 * (int64_t)v0 + d);
#pragma unroll
      for (int e = 0; e < DIM; ++e) {
        const int32_t ve = __ldg(a.cell_vert + NV * cell + e + 1);
#pragma unroll
        for (int d = 0; d < DIM; ++d) J[d][e] = __ldg(a.coords + 3 * (int64_t)ve + d) - X0[d];
      }
      if constexpr (DIM == 2) J[2][2] = 1.0;
    }
    double cof[3][3];
    const double det = det3(J, cof);
    if (!(det != 0.0) || !isfinite(det)) {
      if (lane == 0) atomicOr(a.err, 1);
      continue;  // uniform across the warp
    }
    const double idet = 1.0 / det, adet = fabs(det);
    double Ji[3][3];
#pragma unroll
    for (int e = 0; e < 3; ++e)
#pragma unroll
      for (int j = 0; j < 3; ++j) Ji[e][j] = cof[j][e] * idet;
    double G[3][3];  // J^{-1} J^{-T}
#pragma unroll
    for (int e = 0; e < 3; ++e)
#pragma unroll
      for (int f = 0; f < 3; ++f) G[e][f] = Ji[e][0] * Ji[f][0] + Ji[e][1] * Ji[f][1] + Ji[e][2] * Ji[f][2];

    // gather the cell's dofs
    for (int i = lane; i < NL * NC; i += 32) {
      const int al = i / NC, c = i - al * NC;
      const int64_t at = (int64_t)NC * __ldg(a.cell_node + cell * NL + al) + c;
      xl[i] = __ldg(a.x + at);
      if constexpr (kJac) ul[i] = __ldg(a.ucoef + at);
    }
    __syncwarp();

    double acc[SH::R];
#pragma unroll
    for (int r = 0; r < SH::R; ++r) acc[r] = 0.0;
    bool ok = true;

    for (int q0 = 0; q0 < nq; q0 += 32) {
      // ---- point phase: lane = point q
      const int q = q0 + lane;
      double sv[NC], sh[NC][3];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        sv[c] = 0.0;
        sh[c][0] = sh[c][1] = sh[c][2] = 0.0;
      }
      if (q < nq) {
        double u[NC], g[NC][3], gk[NC][3];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          u[c] = 0.0;
          g[c][0] = g[c][1] = g[c][2] = 0.0;
          gk[c][0] = gk[c][1] = gk[c][2] = 0.0;
        }
#pragma unroll 4
        for (int al = 0; al < NL; ++al) {
          const double ph = kValue && KIND != MFA_FORM_HYPER_RES ? __ldg(a.phi_aq + (int64_t)al * nq + q) : 0.0;
          double d[3] = {0.0, 0.0, 0.0};
          if constexpr (kGrad) {
#pragma unroll
            for (int e = 0; e < DIM; ++e) d[e] = __ldg(a.dphi_aeq + ((int64_t)al * DIM + e) * nq + q);
          }
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const double xv = xl[al * NC + c];
            if constexpr (kValue && KIND != MFA_FORM_HYPER_RES) u[c] = fma(ph, xv, u[c]);
            if constexpr (kGrad) {
#pragma unroll
              for (int e = 0; e < DIM; ++e) g[c][e] = fma(d[e], xv, g[c][e]);
            }
            if constexpr (kJac) {
              const double uv = ul[al * NC + c];
#pragma unroll
              for (int e = 0; e < DIM; ++e) gk[c][e] = fma(d[e], uv, gk[c][e]);
            }
          }
        }
        const double wd = __ldg(a.w + q) * adet;
        if constexpr (KIND == MFA_FORM_MASS || KIND == MFA_FORM_HELMHOLTZ || KIND == MFA_FORM_LAPLACE) {
          const double c0 = KIND == MFA_FORM_HELMHOLTZ ? a.k2 : 1.0;
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            if constexpr (KIND != MFA_FORM_LAPLACE) sv[c] = c0 * wd * u[c];
            if constexpr (kGrad) {
#pragma unroll
              for (int e = 0; e < DIM; ++e) sh[c][e] = wd * (G[e][0] * g[c][0] + G[e][1] * g[c][1] + G[e][2] * g[c][2]);
            }
          }
        } else {
          double gu[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, gc[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, f1[3][3];
#pragma unroll
          for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int j = 0; j < DIM; ++j) {
              gu[c][j] = g[c][0] * Ji[0][j] + g[c][1] * Ji[1][j] + g[c][2] * Ji[2][j];
              gc[c][j] = kJac ? gk[c][0] * Ji[0][j] + gk[c][1] * Ji[1][j] + gk[c][2] * Ji[2][j] : 0.0;
            }
          ok = physics<KIND, LAW>(gu, gc, a.lambda, a.mu, f1) && ok;
#pragma unroll
          for (int c = 0; c < NC; ++c) {
#pragma unroll
            for (int e = 0; e < DIM; ++e) sh[c][e] = wd * (f1[c][0] * Ji[e][0] + f1[c][1] * Ji[e][1] + f1[c][2] * Ji[e][2]);
            if constexpr (KIND == MFA_FORM_HYPER_RES) sv[c] = -bb[c] * wd;
          }
        }
      }
      double* mine = st + lane * SH::S;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        mine[4 * c + 0] = sv[c];
        mine[4 * c + 1] = sh[c][0];
        mine[4 * c + 2] = sh[c][1];
        mine[4 * c + 3] = sh[c][2];
      }
      __syncwarp();
      // ---- dof phase: lane = (local dof, component) pairs lane, lane + 32, ... (pair i: dof i / NC, component
      // i % NC)
      const int nqc = nq - q0 < 32 ? nq - q0 : 32;
#pragma unroll
      for (int r = 0; r < SH::R; ++r) {
        const int task = lane + 32 * r;
        if (task < NL * NC) {
          const int al = task / NC, c = task - al * NC;
          double s = acc[r];
          for (int tq = 0; tq < nqc; ++tq) {
            const int64_t qa = (int64_t)(q0 + tq) * NL + al;
            const double* sp = st + tq * SH::S + 4 * c;
            if constexpr (kValue) s = fma(__ldg(a.phi_qa + qa), sp[0], s);
            if constexpr (kGrad) {
#pragma unroll
              for (int e = 0; e < DIM; ++e) s = fma(__ldg(a.dphi_qae + DIM * qa + e), sp[1 + e], s);
            }
          }
          acc[r] = s;
        }
      }
      __syncwarp();
    }
    if (!ok) atomicOr(a.err, 2);
    // scatter
#pragma unroll
    for (int r = 0; r < SH::R; ++r) {
      const int task = lane + 32 * r;
      if (task < NL * NC) {
        const int al = task / NC, c = task - al * NC;
        const int32_t node = __ldg(a.cell_node + cell * NL + al);
        double* dst = a.y + (int64_t)NC * node + c;
        if constexpr (COLOUR) *dst += acc[r];
        else atomicAdd(dst, acc[r]);
      }
    }
    __syncwarp();  // xl/ul/st are rewritten by the next cell
  }
}

template <int DIM, int NL, int NC, int KIND, int LAW, bool COLOUR>
cudaError_t launch(const TetDenseArgs& a, GridBudget budget, cudaStream_t s) {
  if (a.count == 0) return cudaSuccess;
  auto kern = simplex_dense_kernel<DIM, NL, NC, KIND, LAW, COLOUR>;
  constexpr int smem = kWarps * DenseShape<NL, NC, KIND>::SMEM_WARP * (int)sizeof(double);
  static int bps = -1;
  if (bps < 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int v = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, 32 * kWarps, smem);
    if (e != cudaSuccess) return e;
    bps = v < 1 ? 1 : v;
  }
  int64_t blocks = (a.count + kWarps - 1) / kWarps;
  const int64_t cap = budget.cap(bps);
  if (blocks > cap) blocks = cap;
  kern<<<(unsigned)blocks, 32 * kWarps, smem, s>>>(a);
  return cudaGetLastError();
}

template <int DIM, int NL, int NC, int KIND, int LAW>
cudaError_t launch2(bool colour, const TetDenseArgs& a, GridBudget budget, cudaStream_t s) {
  return colour ? launch<DIM, NL, NC, KIND, LAW, true>(a, budget, s)
                : launch<DIM, NL, NC, KIND, LAW, false>(a, budget, s);
}

template <int DIM, int NL>
cudaError_t by_form(int ncomp, int kind, int law, bool colour, const TetDenseArgs& a, GridBudget budget, cudaStream_t s) {
  const bool nh = law == MFA_LAW_NEOHOOKE;
  if (ncomp == 1) {
    switch (kind) {
      case MFA_FORM_MASS: return launch2<DIM, NL, 1, MFA_FORM_MASS, 0>(colour, a, budget, s);
      case MFA_FORM_LAPLACE: return launch2<DIM, NL, 1, MFA_FORM_LAPLACE, 0>(colour, a, budget, s);
      case MFA_FORM_HELMHOLTZ: return launch2<DIM, NL, 1, MFA_FORM_HELMHOLTZ, 0>(colour, a, budget, s);
    }
    return cudaErrorInvalidValue;
  }
  if (ncomp != DIM) return cudaErrorInvalidValue;
  switch (kind) {
    case MFA_FORM_LAPLACE: return launch2<DIM, NL, DIM, MFA_FORM_LAPLACE, 0>(colour, a, budget, s);
    case MFA_FORM_ELASTICITY: return launch2<DIM, NL, DIM, MFA_FORM_ELASTICITY, 0>(colour, a, budget, s);
    case MFA_FORM_HYPER_RES:
      return nh ? launch2<DIM, NL, DIM, MFA_FORM_HYPER_RES, MFA_LAW_NEOHOOKE>(colour, a, budget, s)
                : launch2<DIM, NL, DIM, MFA_FORM_HYPER_RES, MFA_LAW_SVK>(colour, a, budget, s);
    case MFA_FORM_HYPER_JAC:
      return nh ? launch2<DIM, NL, DIM, MFA_FORM_HYPER_JAC, MFA_LAW_NEOHOOKE>(colour, a, budget, s)
                : launch2<DIM, NL, DIM, MFA_FORM_HYPER_JAC, MFA_LAW_SVK>(colour, a, budget, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t tet_dense_launch(int p, int ncomp, int kind, int law, bool colour, const TetDenseArgs& a, GridBudget budget,
                             cudaStream_t s) {
  switch (p) {
    case 3: return by_form<3, 20>(ncomp, kind, law, colour, a, budget, s);
    case 4: return by_form<3, 35>(ncomp, kind, law, colour, a, budget, s);
    case 5: return by_form<3, 56>(ncomp, kind, law, colour, a, budget, s);
    case 6: return by_form<3, 84>(ncomp, kind, law, colour, a, budget, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t tri_dense_launch(int p, int ncomp, int kind, int law, bool colour, const TetDenseArgs& a, GridBudget budget,
                             cudaStream_t s) {
  switch (p) {
    case 1: return by_form<2, 3>(ncomp, kind, law, colour, a, budget, s);
    case 2: return by_form<2, 6>(ncomp, kind, law, colour, a, budget, s);
    case 3: return by_form<2, 10>(ncomp, kind, law, colour, a, budget, s);
    case 4: return by_form<2, 15>(ncomp, kind, law, colour, a, budget, s);
    case 5: return by_form<2, 21>(ncomp, kind, law, colour, a, budget, s);
    case 6: return by_form<2, 28>(ncomp, kind, law, colour, a, budget, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mfa
