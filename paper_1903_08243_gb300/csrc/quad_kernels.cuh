// Quadrilateral Q_p action (FP64), sum-factorised in 2D: the quad column of
// Table 2 (mass, Helmholtz, vector Laplacian, elasticity and hyperelasticity
// in plane strain).
//
// Same algorithm as the hex point kernel with one direction less: one thread
// per tensor point, CB cells per block, B in x and y gives the values at the
// Gauss points and the collocation derivative D their reference gradient;
// the pointwise physics uses stored per-point geometry (bilinear map: the
// Jacobian varies over the cell); D^T and B^T integrate back; atomic or
// colour scatter.  Vector forms take the 2 components one after the other
// through the same shared-memory sweeps and evaluate the laws of the 3D
// forms with a zero out-of-plane gradient (F_zz = 1).
#pragma once

#include "mfa_internal.h"
#include "physics.cuh"

namespace mfa {
namespace {

constexpr int ceil32q(int x) { return (x + 31) / 32 * 32; }

template <int N, int NQ>
struct QShape {
  static constexpr int PN = N * N;
  static constexpr int PQ = NQ * NQ;
  static constexpr int M = N > NQ ? N : NQ;
  static constexpr int P = M * M;
  static constexpr int CB = P <= 128 ? 256 / P : 1;
  static constexpr int T = ceil32q(CB * P);
  static constexpr int SMEM = (NQ * N + NQ * NQ + 2 * CB * P + 2 * CB * PQ) * 8;
};

// Geometric factors per point: mass c0 w|J|; Laplacian G = w|J| J^{-1} J^{-T} (00, 11, 01); Helmholtz G and
// c0 w|J|; elasticity / hyperelasticity J^{-1} (row-major) and w|J|.
__host__ __device__ constexpr int quad_geom_entries_for(int kind) {
  return kind == MFA_FORM_MASS ? 1 : (kind == MFA_FORM_LAPLACE ? 3 : (kind == MFA_FORM_HELMHOLTZ ? 4 : 5));
}

template <int N, int NQ, int NC, int KIND, int LAW, bool COLOUR>
__global__ void __launch_bounds__(QShape<N, NQ>::T) quad_apply_kernel(const __grid_constant__ HexTables tb,
                                                                      const QuadArgs a) {
  using S = QShape<N, NQ>;
  constexpr int P = S::P, PN = S::PN, PQ = S::PQ, CB = S::CB, NG = quad_geom_entries_for(KIND);
  constexpr bool JAC = KIND == MFA_FORM_HYPER_JAC;
  constexpr bool kGrad = KIND != MFA_FORM_MASS;
  extern __shared__ __align__(16) double smq[];
  double* sB = smq;                // [NQ][N]
  double* sD = sB + NQ * N;        // [NQ][NQ]
  double* bufA = sD + NQ * NQ;     // [CB][P]
  double* bufB = bufA + CB * P;    // [CB][P]
  double* bufF = bufB + CB * P;    // [2][CB][PQ]
  const int t = threadIdx.x;
  for (int i = t; i < NQ * N; i += blockDim.x) sB[i] = tb.B[i];
  for (int i = t; i < NQ * NQ; i += blockDim.x) sD[i] = tb.D[i];
  const int cl = t / P, pt = t - cl * P;
  double* A = bufA + cl * P;
  double* Bf = bufB + cl * P;
  double* F0 = bufF + cl * PQ;
  double* F1 = F0 + CB * PQ;
  const int qi = pt % NQ, qj = pt / NQ;
  const int64_t nbatch = (a.count + CB - 1) / CB;
  // this thread's node in a batch (0 for no point), requested a batch ahead so the gather waits on one load
  auto node_of = [&](int64_t batch) -> int32_t {
    const int64_t idx = batch * CB + cl;
    if (!(cl < CB && idx < a.count && pt < PN)) return 0;
    const int64_t cell = a.cell_list ? (int64_t)__ldg(a.cell_list + idx) : idx;
    return __ldg(a.cell_node + cell * PN + pt);
  };
  int32_t next = (int64_t)blockIdx.x < nbatch ? node_of(blockIdx.x) : 0;
  __syncthreads();
  for (int64_t batch = blockIdx.x; batch < nbatch; batch += gridDim.x) {
    const int64_t idx = batch * CB + cl;
    const bool valid = cl < CB && idx < a.count;
    const bool atq = valid && pt < PQ;
    int64_t cell = 0;
    const int32_t node = next;
    if (batch + gridDim.x < nbatch) next = node_of(batch + gridDim.x);
    if (valid) cell = a.cell_list ? (int64_t)__ldg(a.cell_list + idx) : idx;

    // value and reference gradient of component c of the nodal field v at Gauss point pt
    auto interp = [&](const double* v, int c, double& u, double& g0, double& g1) {
      if (valid && pt < PN) A[pt] = __ldg(v + (int64_t)NC * node + c);
      __syncthreads();
      if (valid && pt < NQ * N) {  // B in x: (NQ, N) <- (N, N)
        const int i = pt % NQ, j = pt / NQ;
        double s = 0.0;
#pragma unroll
        for (int m = 0; m < N; ++m) s = fma(sB[i * N + m], A[m + N * j], s);
        Bf[pt] = s;
      }
      __syncthreads();
      if (atq) {  // B in y: (NQ, NQ) <- (NQ, N)
        double s = 0.0;
#pragma unroll
        for (int m = 0; m < N; ++m) s = fma(sB[qj * N + m], Bf[qi + NQ * m], s);
        A[pt] = s;
      }
      __syncthreads();
      u = g0 = g1 = 0.0;
      if (atq) {
        u = A[pt];
        if constexpr (kGrad) {
#pragma unroll
          for (int m = 0; m < NQ; ++m) {
            g0 = fma(sD[qi * NQ + m], A[m + NQ * qj], g0);
            g1 = fma(sD[qj * NQ + m], A[qi + NQ * m], g1);
          }
        }
      }
      __syncthreads();  // A is rewritten by the next gather
    };

    double u[NC], g[NC][2], gk[NC][2];
#pragma unroll
    for (int c = 0; c < NC; ++c) interp(a.x, c, u[c], g[c][0], g[c][1]);
#pragma unroll
    for (int c = 0; c < NC; ++c) gk[c][0] = gk[c][1] = 0.0;
    if constexpr (JAC) {
      double dummy;
#pragma unroll
      for (int c = 0; c < NC; ++c) interp(a.ucoef, c, dummy, gk[c][0], gk[c][1]);
    }

    double v0[NC], h[NC][2];
#pragma unroll
    for (int c = 0; c < NC; ++c) v0[c] = h[c][0] = h[c][1] = 0.0;
    bool ok = true;
    if (atq) {
      const double* gp = a.geom + cell * (int64_t)NG * PQ + pt;
      double ge[NG];
#pragma unroll
      for (int e = 0; e < NG; ++e) ge[e] = __ldg(gp + e * PQ);
      if constexpr (KIND <= MFA_FORM_HELMHOLTZ) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          if constexpr (KIND == MFA_FORM_MASS) v0[c] = ge[0] * u[c];
          if constexpr (KIND == MFA_FORM_HELMHOLTZ) v0[c] = ge[3] * u[c];
          if constexpr (kGrad) {
            h[c][0] = fma(ge[0], g[c][0], ge[2] * g[c][1]);
            h[c][1] = fma(ge[2], g[c][0], ge[1] * g[c][1]);
          }
        }
      } else {
        const double Ji[2][2] = {{ge[0], ge[1]}, {ge[2], ge[3]}};
        const double wdet = ge[4];
        double gu[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, gc[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, f1[3][3];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            gu[c][j] = fma(g[c][0], Ji[0][j], g[c][1] * Ji[1][j]);
            if constexpr (JAC) gc[c][j] = fma(gk[c][0], Ji[0][j], gk[c][1] * Ji[1][j]);
          }
        ok = physics<KIND, LAW>(gu, gc, a.lambda, a.mu, f1);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
#pragma unroll
          for (int e = 0; e < 2; ++e) h[c][e] = wdet * fma(f1[c][0], Ji[e][0], f1[c][1] * Ji[e][1]);
          if constexpr (KIND == MFA_FORM_HYPER_RES) v0[c] = -(c == 0 ? a.b0 : a.b1) * wdet;
        }
      }
    }
    if (!ok) atomicOr(a.err, 2);

#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (atq) {
        F0[pt] = h[c][0];
        F1[pt] = h[c][1];
      }
      __syncthreads();
      if (atq) {  // r = value term + D_x^T f0 + D_y^T f1
        double r = v0[c];
        if constexpr (kGrad || KIND == MFA_FORM_HYPER_RES) {
#pragma unroll
          for (int m = 0; m < NQ; ++m) {
            r = fma(sD[m * NQ + qi], F0[m + NQ * qj], r);
            r = fma(sD[m * NQ + qj], F1[qi + NQ * m], r);
          }
        }
        A[pt] = r;
      }
      __syncthreads();
      if (valid && pt < NQ * N) {  // B^T in y: (NQ, N) <- (NQ, NQ)
        const int i = pt % NQ, b = pt / NQ;
        double s = 0.0;
#pragma unroll
        for (int m = 0; m < NQ; ++m) s = fma(sB[m * N + b], A[i + NQ * m], s);
        Bf[pt] = s;
      }
      __syncthreads();
      if (valid && pt < PN) {  // B^T in x and scatter-add: (N, N) <- (NQ, N)
        const int i = pt % N, b = pt / N;
        double s = 0.0;
#pragma unroll
        for (int m = 0; m < NQ; ++m) s = fma(sB[m * N + i], Bf[m + NQ * b], s);
        double* dst = a.y + (int64_t)NC * node + c;
        if constexpr (COLOUR) *dst += s;  // no other cell of this colour touches `node`
        else atomicAdd(dst, s);
      }
      __syncthreads();
    }
  }
}

template <int N, int NQ, int NC, int KIND, int LAW, bool COLOUR>
cudaError_t launch(const HexTables& tb, const QuadArgs& a, GridBudget budget, cudaStream_t s) {
  using S = QShape<N, NQ>;
  auto kern = quad_apply_kernel<N, NQ, NC, KIND, LAW, COLOUR>;
  static int bps = -1;
  if (bps < 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
    if (e != cudaSuccess) return e;
    int v = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, S::T, S::SMEM);
    if (e != cudaSuccess) return e;
    bps = v < 1 ? 1 : v;
  }
  const int64_t nbatch = (a.count + S::CB - 1) / S::CB;
  if (nbatch == 0) return cudaSuccess;
  const int64_t cap = budget.cap(bps);
  kern<<<(unsigned)(nbatch < cap ? nbatch : cap), S::T, S::SMEM, s>>>(tb, a);
  return cudaGetLastError();
}

template <int N, int NQ, int NC, int KIND, int LAW>
cudaError_t launch2(bool colour, const HexTables& tb, const QuadArgs& a, GridBudget budget, cudaStream_t s) {
  return colour ? launch<N, NQ, NC, KIND, LAW, true>(tb, a, budget, s)
                : launch<N, NQ, NC, KIND, LAW, false>(tb, a, budget, s);
}

template <int N, int NQ>
cudaError_t by_form(int ncomp, int kind, int law, bool colour, const HexTables& tb, const QuadArgs& a, GridBudget budget,
                    cudaStream_t s) {
  const bool nh = law == MFA_LAW_NEOHOOKE;
  if (ncomp == 1) {
    switch (kind) {
      case MFA_FORM_MASS: return launch2<N, NQ, 1, MFA_FORM_MASS, 0>(colour, tb, a, budget, s);
      case MFA_FORM_LAPLACE: return launch2<N, NQ, 1, MFA_FORM_LAPLACE, 0>(colour, tb, a, budget, s);
      case MFA_FORM_HELMHOLTZ: return launch2<N, NQ, 1, MFA_FORM_HELMHOLTZ, 0>(colour, tb, a, budget, s);
    }
    return cudaErrorInvalidValue;
  }
  switch (kind) {
    case MFA_FORM_LAPLACE: return launch2<N, NQ, 2, MFA_FORM_LAPLACE, 0>(colour, tb, a, budget, s);
    case MFA_FORM_ELASTICITY: return launch2<N, NQ, 2, MFA_FORM_ELASTICITY, 0>(colour, tb, a, budget, s);
    case MFA_FORM_HYPER_RES:
      return nh ? launch2<N, NQ, 2, MFA_FORM_HYPER_RES, MFA_LAW_NEOHOOKE>(colour, tb, a, budget, s)
                : launch2<N, NQ, 2, MFA_FORM_HYPER_RES, MFA_LAW_SVK>(colour, tb, a, budget, s);
    case MFA_FORM_HYPER_JAC:
      return nh ? launch2<N, NQ, 2, MFA_FORM_HYPER_JAC, MFA_LAW_NEOHOOKE>(colour, tb, a, budget, s)
                : launch2<N, NQ, 2, MFA_FORM_HYPER_JAC, MFA_LAW_SVK>(colour, tb, a, budget, s);
  }
  return cudaErrorInvalidValue;
}

// p+1 and p+2 points per direction for every form, 2p+2 for the hyperelastic forms (2n <= 10).
template <int N>
cudaError_t by_rule(int nq, int ncomp, int kind, int law, bool colour, const HexTables& tb, const QuadArgs& a,
                    GridBudget budget, cudaStream_t s) {
  if (nq == N) return by_form<N, N>(ncomp, kind, law, colour, tb, a, budget, s);
  if constexpr (N + 1 <= kMaxN) {
    if (nq == N + 1) return by_form<N, N + 1>(ncomp, kind, law, colour, tb, a, budget, s);
  }
  if constexpr (2 * N <= kMaxN && 2 * N != N + 1) {
    if (nq == 2 * N && (kind == MFA_FORM_HYPER_RES || kind == MFA_FORM_HYPER_JAC))
      return by_form<N, 2 * N>(ncomp, kind, law, colour, tb, a, budget, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace mfa
