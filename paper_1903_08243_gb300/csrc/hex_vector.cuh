// Sum-factorised FP64 action of the vector forms on Q_p hexahedra: the vector
// Laplacian, linear elasticity, and the hyperelastic residual and Jacobian
// action (St Venant-Kirchhoff and neo-Hookean) -- the laplacian, elasticity
// and hyperelasticity operators of Section 4.1 and Table 2 on hex meshes.
//
// One thread per tensor point, as in the scalar point kernel
// (hex_kernels.cuh), whose shared-memory layout and 1D tables it reuses.  The
// three components pass through the same sweeps one after the other: for
// component c, B in x, y and z gives u_c at the Gauss points and the three
// collocation derivatives give its reference gradient, which the thread
// keeps in registers.  With all three (and, for the Jacobian, the three of the
// linearisation point) in registers, the thread forms the physical gradient
// with the stored J^{-1}, evaluates the stress, and maps the flux back with
// w|det J| J^{-T}.  Each component's flux then runs through D^T and B^T and is
// scattered, so the shared-memory footprint is that of the scalar kernel.
// Vector dofs are node-interleaved: dof = 3 node + c.
#pragma once

#include "hex_kernels.cuh"
#include "physics.cuh"

namespace mfa {
namespace hexv {

using hexk::Shape;
using hexk::Smem;

template <int N, int NQ, int KIND, int LAW, bool COLOUR>
__device__ __forceinline__ void cell_batch(const HexVecArgs& a, int64_t batch, const Smem<N, NQ, MFA_PREC_FP64>& sm,
                                           int32_t node_ahead) {  // node_ahead: this point's node (0 for none)
  using S = Shape<N, NQ>;
  constexpr int PN = S::PN, PQ = S::PQ, CB = S::CB;
  constexpr bool JAC = KIND == MFA_FORM_HYPER_JAC;
  const double* sB = sm.sB;  // [NQ][N]
  const double* sD = sm.sD;  // [NQ][NQ]
  double* A = sm.A;
  double* Bf = sm.Bf;
  double* F0 = sm.F0;
  double* F1 = sm.F1;
  double* F2 = sm.F2;
  const int cl = sm.cl, pt = sm.pt;
  const int64_t idx = batch * CB + cl;
  const bool valid = cl < CB && idx < a.count;
  int64_t cell = 0;
  int32_t node = node_ahead;
  if (valid) cell = a.cell_list ? (int64_t)__ldg(a.cell_list + idx) : idx;
  const bool atq = valid && pt < PQ;  // this thread owns Gauss point pt
  const int qi = pt % NQ, qj = (pt / NQ) % NQ, qk = pt / (NQ * NQ);

  // reference gradient of component c of the nodal field v at Gauss point pt
  auto ref_grad = [&](const double* v, int c, double g[3]) {
    if (valid && pt < PN) A[pt] = __ldg(v + 3 * (int64_t)node + c);
    __syncthreads();
    if (valid && pt < NQ * N * N) {  // B in x: (NQ, N, N) <- (N, N, N)
      const int i = pt % NQ, jk = pt / NQ;
      double s = 0.0;
#pragma unroll
      for (int m = 0; m < N; ++m) s = fma(sB[i * N + m], A[m + N * jk], s);
      Bf[pt] = s;
    }
    __syncthreads();
    if (valid && pt < NQ * NQ * N) {  // B in y: (NQ, NQ, N) <- (NQ, N, N)
      const int i = pt % NQ, j = (pt / NQ) % NQ, k = pt / (NQ * NQ);
      double s = 0.0;
#pragma unroll
      for (int m = 0; m < N; ++m) s = fma(sB[j * N + m], Bf[i + NQ * (m + N * k)], s);
      A[pt] = s;
    }
    __syncthreads();
    if (atq) {  // B in z: (NQ, NQ, NQ) <- (NQ, NQ, N), u_c at the Gauss points
      double s = 0.0;
#pragma unroll
      for (int m = 0; m < N; ++m) s = fma(sB[qk * N + m], A[qi + NQ * (qj + NQ * m)], s);
      Bf[pt] = s;
    }
    __syncthreads();
    double d0 = 0.0, d1 = 0.0, d2 = 0.0;
    if (atq) {  // collocation derivatives on the Gauss points
#pragma unroll
      for (int m = 0; m < NQ; ++m) {
        d0 = fma(sD[qi * NQ + m], Bf[m + NQ * (qj + NQ * qk)], d0);
        d1 = fma(sD[qj * NQ + m], Bf[qi + NQ * (m + NQ * qk)], d1);
        d2 = fma(sD[qk * NQ + m], Bf[qi + NQ * (qj + NQ * m)], d2);
      }
    }
    g[0] = d0;
    g[1] = d1;
    g[2] = d2;
    // no barrier: the next writer of Bf (the next x sweep) runs after the next gather's barrier
  };

  // components unrolled so that the gradients stay in registers
  double g[3][3];  // g[c][e] = d u_c / d xi_e
#pragma unroll
  for (int c = 0; c < 3; ++c) ref_grad(a.x, c, g[c]);
  double gk[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  // the linearisation point's (Jacobian action)
  if constexpr (JAC) {
#pragma unroll
    for (int c = 0; c < 3; ++c) ref_grad(a.ucoef, c, gk[c]);
  }

  // pointwise: reference flux h[c][e] and the value term of the residual's body force
  double h[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  double v0[3] = {0.0, 0.0, 0.0};
  bool ok = true;
  if (atq) {
    const double* gp = a.geom + cell * a.geom_stride + pt;
    if constexpr (KIND == MFA_FORM_LAPLACE) {
      // G = w|J| J^{-1} J^{-T}: (00, 11, 22, 01, 02, 12), one scalar Laplacian per component
      double G[6];
#pragma unroll
      for (int e = 0; e < 6; ++e) G[e] = __ldg(gp + e * PQ);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        h[c][0] = fma(G[0], g[c][0], fma(G[3], g[c][1], G[4] * g[c][2]));
        h[c][1] = fma(G[3], g[c][0], fma(G[1], g[c][1], G[5] * g[c][2]));
        h[c][2] = fma(G[4], g[c][0], fma(G[5], g[c][1], G[2] * g[c][2]));
      }
    } else {
      double Ji[3][3];
#pragma unroll
      for (int e = 0; e < 9; ++e) Ji[e / 3][e % 3] = __ldg(gp + e * PQ);
      const double wdet = __ldg(gp + 9 * PQ);
      double gu[3][3], gc[3][3], f1[3][3];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
          gu[c][jj] = fma(g[c][0], Ji[0][jj], fma(g[c][1], Ji[1][jj], g[c][2] * Ji[2][jj]));
          gc[c][jj] = JAC ? fma(gk[c][0], Ji[0][jj], fma(gk[c][1], Ji[1][jj], gk[c][2] * Ji[2][jj])) : 0.0;
        }
      ok = physics<KIND, LAW>(gu, gc, a.lam, a.mu, f1);
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int e = 0; e < 3; ++e)
          h[c][e] = wdet * fma(f1[c][0], Ji[e][0], fma(f1[c][1], Ji[e][1], f1[c][2] * Ji[e][2]));
      if constexpr (KIND == MFA_FORM_HYPER_RES) {
        v0[0] = -a.b0 * wdet;
        v0[1] = -a.b1 * wdet;
        v0[2] = -a.b2 * wdet;
      }
    }
  }
  if (!ok) atomicOr(a.err, 2);

  // integrate back and scatter, one component at a time
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (atq) {
      F0[pt] = h[c][0];
      F1[pt] = h[c][1];
      F2[pt] = h[c][2];
    }
    __syncthreads();
    if (atq) {  // r = v0 + sum_d D_d^T f_d
      double r = v0[c];
#pragma unroll
      for (int m = 0; m < NQ; ++m) {
        r = fma(sD[m * NQ + qi], F0[m + NQ * (qj + NQ * qk)], r);
        r = fma(sD[m * NQ + qj], F1[qi + NQ * (m + NQ * qk)], r);
        r = fma(sD[m * NQ + qk], F2[qi + NQ * (qj + NQ * m)], r);
      }
      A[pt] = r;
    }
    __syncthreads();
    if (valid && pt < NQ * NQ * N) {  // B^T in z: (NQ, NQ, N) <- (NQ, NQ, NQ)
      const int ij = pt % (NQ * NQ), k = pt / (NQ * NQ);
      double s = 0.0;
#pragma unroll
      for (int m = 0; m < NQ; ++m) s = fma(sB[m * N + k], A[ij + NQ * NQ * m], s);
      Bf[pt] = s;
    }
    __syncthreads();
    if (valid && pt < NQ * N * N) {  // B^T in y: (NQ, N, N) <- (NQ, NQ, N)
      const int i = pt % NQ, b = (pt / NQ) % N, k = pt / (NQ * N);
      double s = 0.0;
#pragma unroll
      for (int m = 0; m < NQ; ++m) s = fma(sB[m * N + b], Bf[i + NQ * (m + NQ * k)], s);
      A[pt] = s;
    }
    __syncthreads();
    if (valid && pt < PN) {  // B^T in x and scatter-add: (N, N, N) <- (NQ, N, N)
      const int i = pt % N, bc = pt / N;
      double s = 0.0;
#pragma unroll
      for (int m = 0; m < NQ; ++m) s = fma(sB[m * N + i], A[m + NQ * bc], s);
      double* dst = a.y + 3 * (int64_t)node + c;
      if constexpr (COLOUR) *dst += s;  // no other cell of this colour touches `node`
      else atomicAdd(dst, s);
    }
    // the next component's D^T writes A only after the barrier that follows its flux stores
  }
  __syncthreads();
}

template <int N, int NQ, int KIND, int LAW, bool COLOUR>
__global__ void __launch_bounds__(Shape<N, NQ>::T) apply_kernel(const __grid_constant__ HexTables tb,
                                                                const HexVecArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<N, NQ, MFA_PREC_FP64> sm;
  sm.init(smem_raw, tb);
  constexpr int CB = Shape<N, NQ>::CB, PN = Shape<N, NQ>::PN;
  const int64_t nbatch = (a.count + CB - 1) / CB;
  // this thread's node in a batch (0 for no point), requested a batch ahead so the gathers wait on one load
  auto node_of = [&](int64_t batch) -> int32_t {
    const int64_t idx = batch * CB + sm.cl;
    if (!(sm.cl < CB && idx < a.count && sm.pt < PN)) return 0;
    const int64_t cell = a.cell_list ? (int64_t)__ldg(a.cell_list + idx) : idx;
    return __ldg(a.cell_node + cell * PN + sm.pt);
  };
  int32_t next = (int64_t)blockIdx.x < nbatch ? node_of(blockIdx.x) : 0;
  for (int64_t batch = blockIdx.x; batch < nbatch; batch += gridDim.x) {
    const int32_t node = next;
    if (batch + gridDim.x < nbatch) next = node_of(batch + gridDim.x);
    cell_batch<N, NQ, KIND, LAW, COLOUR>(a, batch, sm, node);
  }
}

template <int N, int NQ, int KIND, int LAW, bool COLOUR>
cudaError_t launch(const HexTables& tb, const HexVecArgs& a, GridBudget budget, cudaStream_t s) {
  using S = Shape<N, NQ>;
  auto kern = apply_kernel<N, NQ, KIND, LAW, COLOUR>;
  static int blocks_per_sm = -1;
  if (blocks_per_sm < 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
    if (e != cudaSuccess) return e;
    int b = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, S::T, S::SMEM);
    if (e != cudaSuccess) return e;
    blocks_per_sm = b < 1 ? 1 : b;
  }
  const int64_t nbatch = (a.count + S::CB - 1) / S::CB;
  if (nbatch == 0) return cudaSuccess;
  const int64_t cap = budget.cap(blocks_per_sm);
  kern<<<(unsigned)(nbatch < cap ? nbatch : cap), S::T, S::SMEM, s>>>(tb, a);
  return cudaGetLastError();
}

// Linear vector forms (vector Laplacian, elasticity) at NQ points per direction.
template <int N, int NQ>
cudaError_t dispatch_linear(int kind, bool colour, const HexTables& tb, const HexVecArgs& a, GridBudget budget,
                            cudaStream_t s) {
  switch (kind) {
    case MFA_FORM_LAPLACE:
      return colour ? launch<N, NQ, MFA_FORM_LAPLACE, 0, true>(tb, a, budget, s)
                    : launch<N, NQ, MFA_FORM_LAPLACE, 0, false>(tb, a, budget, s);
    case MFA_FORM_ELASTICITY:
      return colour ? launch<N, NQ, MFA_FORM_ELASTICITY, 0, true>(tb, a, budget, s)
                    : launch<N, NQ, MFA_FORM_ELASTICITY, 0, false>(tb, a, budget, s);
  }
  return cudaErrorInvalidValue;
}

// Hyperelastic forms at NQ points per direction.
template <int N, int NQ>
cudaError_t dispatch_hyper(int kind, int law, bool colour, const HexTables& tb, const HexVecArgs& a, GridBudget budget,
                           cudaStream_t s) {
  const bool nh = law == MFA_LAW_NEOHOOKE;
#define MFA_HEXV_CASE(KIND, LAW) \
  return colour ? launch<N, NQ, KIND, LAW, true>(tb, a, budget, s) : launch<N, NQ, KIND, LAW, false>(tb, a, budget, s)
  switch (kind) {
    case MFA_FORM_HYPER_RES:
      if (nh) MFA_HEXV_CASE(MFA_FORM_HYPER_RES, MFA_LAW_NEOHOOKE);
      MFA_HEXV_CASE(MFA_FORM_HYPER_RES, MFA_LAW_SVK);
    case MFA_FORM_HYPER_JAC:
      if (nh) MFA_HEXV_CASE(MFA_FORM_HYPER_JAC, MFA_LAW_NEOHOOKE);
      MFA_HEXV_CASE(MFA_FORM_HYPER_JAC, MFA_LAW_SVK);
  }
#undef MFA_HEXV_CASE
  return cudaErrorInvalidValue;
}

// p+1 points (every form), p+2 points (linear forms, Table 2's elasticity rule, n <= 7) and 2p+2 points
// (hyperelastic forms, Table 2's hyperelasticity rule, n <= 4).
template <int N>
cudaError_t dispatch(int nq, int kind, int law, bool colour, const HexTables& tb, const HexVecArgs& a, GridBudget budget,
                     cudaStream_t s) {
  const bool hyper = kind == MFA_FORM_HYPER_RES || kind == MFA_FORM_HYPER_JAC;
  if (nq == N) return hyper ? dispatch_hyper<N, N>(kind, law, colour, tb, a, budget, s)
                            : dispatch_linear<N, N>(kind, colour, tb, a, budget, s);
  if constexpr (N + 1 <= 8) {  // n + 1 points: up to 512 threads per cell
    if (nq == N + 1 && !hyper) return dispatch_linear<N, N + 1>(kind, colour, tb, a, budget, s);
  }
  if constexpr (2 * N <= 8) {
    if (nq == 2 * N && hyper) return dispatch_hyper<N, 2 * N>(kind, law, colour, tb, a, budget, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hexv
}  // namespace mfa
