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

template <int N, int KIND, int LAW, bool COLOUR>
__device__ __forceinline__ void cell_batch(const HexVecArgs& a, int64_t batch, const Smem<N, N, MFA_PREC_FP64>& sm) {
  using S = Shape<N, N>;
  constexpr int P = S::P, CB = S::CB;
  constexpr bool JAC = KIND == MFA_FORM_HYPER_JAC;
  const double* sB = sm.sB;
  const double* sD = sm.sD;
  double* A = sm.A;
  double* Bf = sm.Bf;
  double* F0 = sm.F0;
  double* F1 = sm.F1;
  double* F2 = sm.F2;
  const int cl = sm.cl, pt = sm.pt;
  const int64_t idx = batch * CB + cl;
  const bool active = cl < CB && idx < a.count && pt < P;
  int64_t cell = 0;
  int32_t node = 0;
  if (active) {
    cell = a.cell_list ? (int64_t)__ldg(a.cell_list + idx) : idx;
    node = __ldg(a.cell_node + cell * P + pt);
  }
  const int i = pt % N, j = (pt / N) % N, k = pt / (N * N);

  // reference gradient of component c of the nodal field v at this thread's point
  auto ref_grad = [&](const double* v, int c, double g[3]) {
    if (active) A[pt] = __ldg(v + 3 * (int64_t)node + c);
    __syncthreads();
    if (active) {  // B in x
      double s = 0.0;
#pragma unroll
      for (int m = 0; m < N; ++m) s = fma(sB[i * N + m], A[m + N * (j + N * k)], s);
      Bf[pt] = s;
    }
    __syncthreads();
    if (active) {  // B in y
      double s = 0.0;
#pragma unroll
      for (int m = 0; m < N; ++m) s = fma(sB[j * N + m], Bf[i + N * (m + N * k)], s);
      A[pt] = s;
    }
    __syncthreads();
    if (active) {  // B in z: u_c at the Gauss points
      double s = 0.0;
#pragma unroll
      for (int m = 0; m < N; ++m) s = fma(sB[k * N + m], A[i + N * (j + N * m)], s);
      Bf[pt] = s;
    }
    __syncthreads();
    double d0 = 0.0, d1 = 0.0, d2 = 0.0;
    if (active) {  // collocation derivatives
#pragma unroll
      for (int m = 0; m < N; ++m) {
        d0 = fma(sD[i * N + m], Bf[m + N * (j + N * k)], d0);
        d1 = fma(sD[j * N + m], Bf[i + N * (m + N * k)], d1);
        d2 = fma(sD[k * N + m], Bf[i + N * (j + N * m)], d2);
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
  if (active) {
    const double* gp = a.geom + cell * a.geom_stride + pt;
    if constexpr (KIND == MFA_FORM_LAPLACE) {
      // G = w|J| J^{-1} J^{-T}: (00, 11, 22, 01, 02, 12), one scalar Laplacian per component
      double G[6];
#pragma unroll
      for (int e = 0; e < 6; ++e) G[e] = __ldg(gp + e * P);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        h[c][0] = fma(G[0], g[c][0], fma(G[3], g[c][1], G[4] * g[c][2]));
        h[c][1] = fma(G[3], g[c][0], fma(G[1], g[c][1], G[5] * g[c][2]));
        h[c][2] = fma(G[4], g[c][0], fma(G[5], g[c][1], G[2] * g[c][2]));
      }
    } else {
      double Ji[3][3];
#pragma unroll
      for (int e = 0; e < 9; ++e) Ji[e / 3][e % 3] = __ldg(gp + e * P);
      const double wdet = __ldg(gp + 9 * P);
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
    const double vc = v0[c];
    if (active) {
      F0[pt] = h[c][0];
      F1[pt] = h[c][1];
      F2[pt] = h[c][2];
    }
    __syncthreads();
    if (active) {  // r = v0 + sum_d D_d^T f_d
      double r = vc;
#pragma unroll
      for (int m = 0; m < N; ++m) {
        r = fma(sD[m * N + i], F0[m + N * (j + N * k)], r);
        r = fma(sD[m * N + j], F1[i + N * (m + N * k)], r);
        r = fma(sD[m * N + k], F2[i + N * (j + N * m)], r);
      }
      A[pt] = r;
    }
    __syncthreads();
    if (active) {  // B^T in z
      double s = 0.0;
#pragma unroll
      for (int m = 0; m < N; ++m) s = fma(sB[m * N + k], A[i + N * (j + N * m)], s);
      Bf[pt] = s;
    }
    __syncthreads();
    if (active) {  // B^T in y
      double s = 0.0;
#pragma unroll
      for (int m = 0; m < N; ++m) s = fma(sB[m * N + j], Bf[i + N * (m + N * k)], s);
      A[pt] = s;
    }
    __syncthreads();
    if (active) {  // B^T in x and scatter-add
      double s = 0.0;
#pragma unroll
      for (int m = 0; m < N; ++m) s = fma(sB[m * N + i], A[m + N * (j + N * k)], s);
      double* dst = a.y + 3 * (int64_t)node + c;
      if constexpr (COLOUR) *dst += s;  // no other cell of this colour touches `node`
      else atomicAdd(dst, s);
    }
    // the next component's D^T writes A only after the barrier that follows its flux stores
  }
  __syncthreads();
}

template <int N, int KIND, int LAW, bool COLOUR>
__global__ void __launch_bounds__(Shape<N, N>::T) apply_kernel(const __grid_constant__ HexTables tb,
                                                               const HexVecArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<N, N, MFA_PREC_FP64> sm;
  sm.init(smem_raw, tb);
  constexpr int CB = Shape<N, N>::CB;
  const int64_t nbatch = (a.count + CB - 1) / CB;
  for (int64_t batch = blockIdx.x; batch < nbatch; batch += gridDim.x) cell_batch<N, KIND, LAW, COLOUR>(a, batch, sm);
}

template <int N, int KIND, int LAW, bool COLOUR>
cudaError_t launch(const HexTables& tb, const HexVecArgs& a, int sm_count, cudaStream_t s) {
  using S = Shape<N, N>;
  auto kern = apply_kernel<N, KIND, LAW, COLOUR>;
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
  const int64_t cap = (int64_t)sm_count * blocks_per_sm;
  kern<<<(unsigned)(nbatch < cap ? nbatch : cap), S::T, S::SMEM, s>>>(tb, a);
  return cudaGetLastError();
}

template <int N>
cudaError_t dispatch(int kind, int law, bool colour, const HexTables& tb, const HexVecArgs& a, int sm_count,
                     cudaStream_t s) {
  const bool nh = law == MFA_LAW_NEOHOOKE;
#define MFA_HEXV_CASE(KIND, LAW) \
  return colour ? launch<N, KIND, LAW, true>(tb, a, sm_count, s) : launch<N, KIND, LAW, false>(tb, a, sm_count, s)
  switch (kind) {
    case MFA_FORM_LAPLACE: MFA_HEXV_CASE(MFA_FORM_LAPLACE, 0);
    case MFA_FORM_ELASTICITY: MFA_HEXV_CASE(MFA_FORM_ELASTICITY, 0);
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

}  // namespace hexv
}  // namespace mfa
