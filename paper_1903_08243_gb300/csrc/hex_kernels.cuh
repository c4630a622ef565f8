// Sum-factorised FP64 operator action on Q_p hexahedra (mass, Laplacian,
// Helmholtz), one CUDA thread per tensor point of a cell.
//
// Local assembly (Section 2.1 of arXiv 1903.08243) on a tensor-product cell
// factorises into 1D contractions (the sum factorisation TSFC applies to
// tensor-product elements, Sections 3 and 4.2.4):
//   u_q   = (B x B x B) u                  values at Gauss points, 3 sweeps
//   g_d   = D_d u_q                        collocation derivatives, 3 sweeps
//   f     = G(q) g  (+ c0 w|J| u_q)        pointwise physics with stored geometry
//   r     = sum_d D_d^T f_d (+ mass term)  3 transposed sweeps
//   y_loc = (B^T x B^T x B^T) r            3 transposed sweeps
// B is the GLL-node basis at the Gauss points and D the derivative of the
// Lagrange basis on the Gauss points, so that D B equals the derivative of
// the node basis at the Gauss points.
//
// The FP64 pipe of GB300 issues 2 DFMA lanes per clock per SM, about 1/64 of
// the FP32 rate; every other instruction class (loads, shared memory,
// integer) is nearly free by comparison.  So the kernel minimises FP64
// operations: geometry is precomputed once in FP64 and read per point
// (56 B per point against ~70 DFMA), and the 12 n^4 DFMA of the contractions
// are the only FP64 work besides ~10 per point for the physics.
//
// Cross-element batching (Section 3.1) maps to CB cells per thread block,
// each cell a slab of n^3 threads; blocks loop persistently over batches.
#pragma once

#include <cuda_bf16.h>

#include "mfa_internal.h"
#include "scatter.cuh"

namespace mfa {
namespace hexk {

// Arithmetic and storage types of one precision variant.  FP64: everything
// in double.  FP32: float arithmetic, geometric factors stored as float.
// BF16: the streamed operands (x and the geometric factors) and the 1D
// tables are rounded to bfloat16, arithmetic and accumulation are float.
// The geometric factors are always computed in FP64 and only then rounded.
template <int PREC>
struct Prec;
template <>
struct Prec<MFA_PREC_FP64> {
  using T = double;
  using TG = double;
  static __device__ __forceinline__ T in(double v) { return v; }
  static __device__ __forceinline__ T geo(const TG* p) { return __ldg(p); }
};
template <>
struct Prec<MFA_PREC_FP32> {
  using T = float;
  using TG = float;
  static __device__ __forceinline__ T in(double v) { return (float)v; }
  static __device__ __forceinline__ T geo(const TG* p) { return __ldg(p); }
};
template <>
struct Prec<MFA_PREC_BF16> {
  using T = float;
  using TG = __nv_bfloat16;
  static __device__ __forceinline__ T in(double v) { return __bfloat162float(__double2bfloat16(v)); }
  static __device__ __forceinline__ T geo(const TG* p) { return __bfloat162float(*p); }
};

constexpr int ceil32(int x) { return (x + 31) / 32 * 32; }

// CBX > 0 overrides the default number of cells per block (autotuner choices).
template <int N, int NQ, int ELEM = 8, int CBX = 0>
struct Shape {
  static constexpr int PN = N * N * N;
  static constexpr int PQ = NQ * NQ * NQ;
  static constexpr int M = N > NQ ? N : NQ;
  static constexpr int P = M * M * M;
  static constexpr int CB0 = P <= 128 ? 256 / P : 1;  // default cells per block
  static constexpr int CB = CBX > 0 ? CBX : CB0;      // cells per block
  static constexpr int T = ceil32(CB * P);           // threads per block
  static constexpr int SMEM = (NQ * N + NQ * NQ + 2 * CB * P + 3 * CB * PQ) * ELEM;
};

template <int KIND>
__host__ __device__ constexpr int geom_entries() {
  return KIND == MFA_FORM_MASS ? 1 : (KIND == MFA_FORM_LAPLACE ? 6 : 7);
}

// Shared-memory working set of one block (types by precision).
template <int N, int NQ, int PREC, int CBX = 0>
struct Smem {
  using S = Shape<N, NQ, 8, CBX>;
  using T = typename Prec<PREC>::T;
  T* sB;  // [NQ][N]
  T* sD;  // [NQ][NQ]
  T* A;   // this thread's cell slot of buffer A
  T* Bf;  // this thread's cell slot of buffer B
  T* F0;
  T* F1;
  T* F2;
  int cl, pt;
  __device__ __forceinline__ void init(unsigned char* raw, const HexTables& tb) {
    constexpr int P = S::P, PQ = S::PQ, CB = S::CB;
    T* smem = reinterpret_cast<T*>(raw);
    sB = smem;
    sD = sB + NQ * N;
    T* bufA = sD + NQ * NQ;
    T* bufB = bufA + CB * P;
    T* F = bufB + CB * P;
    const int t = threadIdx.x;
    for (int i = t; i < NQ * N; i += blockDim.x) sB[i] = Prec<PREC>::in(tb.B[i]);
    for (int i = t; i < NQ * NQ; i += blockDim.x) sD[i] = Prec<PREC>::in(tb.D[i]);
    cl = t / P;
    pt = t - cl * P;
    A = bufA + cl * P;
    Bf = bufB + cl * P;
    F0 = F + cl * PQ;
    F1 = F0 + CB * PQ;
    F2 = F1 + CB * PQ;
  }
};

// One batch of CB cells of one form: gather, sum-factorised local kernel,
// scatter.  Every thread of the block calls it (it contains barriers).
// Geometric factors of Gauss point (qi, qj, qk) from the cell's vertices X[8][3] (shared memory): the
// trilinear Jacobian J, then G = w |det J| J^{-1} J^{-T} = (w / |det J|) adj(J)^T adj(J) (6 entries) and
// c0 w |det J|, in the stored layout's entry order.  Returns false if det J is zero or not finite.
template <int NG>
__device__ __forceinline__ bool point_geometry(const double* X, const HexTables& tb, int qi, int qj, int qk,
                                               double c0, double g[NG]) {
  const double xi[3] = {tb.x1[qi], tb.x1[qj], tb.x1[qk]};
  const double w = tb.w1[qi] * tb.w1[qj] * tb.w1[qk];
  double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    const double fx = (v & 1) ? xi[0] : 1.0 - xi[0], fy = (v & 2) ? xi[1] : 1.0 - xi[1],
                 fz = (v & 4) ? xi[2] : 1.0 - xi[2];
    const double dN[3] = {((v & 1) ? fy : -fy) * fz, fx * ((v & 2) ? fz : -fz), fx * ((v & 4) ? fy : -fy)};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double Xd = X[3 * v + d];
#pragma unroll
      for (int e = 0; e < 3; ++e) J[d][e] = fma(Xd, dN[e], J[d][e]);
    }
  }
  // cofactors: cof[r][c] of J; adj(J) = cof^T, J^{-1} = cof^T / det
  double cof[3][3];
  cof[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  cof[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  cof[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  cof[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  cof[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  cof[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  cof[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  cof[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  cof[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  const double det = J[0][0] * cof[0][0] + J[0][1] * cof[0][1] + J[0][2] * cof[0][2];
  if (!(det != 0.0) || !isfinite(det)) {
#pragma unroll
    for (int e = 0; e < NG; ++e) g[e] = 0.0;
    return false;
  }
  const double adet = fabs(det);
  if constexpr (NG == 1) {
    g[0] = c0 * w * adet;
  } else {
    const double s = w / adet;
    // G[a][b] = s * sum_k cof[k][a] cof[k][b]: (00, 11, 22, 01, 02, 12)
    const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int e = 0; e < 6; ++e)
      g[e] = s * (cof[0][ia[e]] * cof[0][ib[e]] + cof[1][ia[e]] * cof[1][ib[e]] + cof[2][ia[e]] * cof[2][ib[e]]);
    if constexpr (NG == 7) g[6] = c0 * w * adet;
  }
  return true;
}

// Node of this thread's point in batch `batch` (-1 for no point): requested a
// batch ahead, so the gather waits on one load instead of two.
template <int N, int NQ, int CBX>
__device__ __forceinline__ int32_t point_node(const HexApplyArgs& a, int64_t batch, int cl, int pt) {
  using S = Shape<N, NQ, 8, CBX>;
  const int64_t idx = batch * S::CB + cl;
  if (cl >= S::CB || idx >= a.count || pt >= S::PN) return -1;
  const int64_t cell = a.cell_list ? (int64_t)__ldg(a.cell_list + idx) : idx;
  return __ldg(a.cell_node + cell * S::PN + pt);
}

// `node_ahead`: this point's node, loaded ahead by point_node (-1: load it here).
template <int N, int NQ, int KIND, bool COLOUR, int PREC, int CBX = 0, bool AGG = false, bool OTF = false>
__device__ __forceinline__ void hex_cell_batch(const HexApplyArgs& a, int64_t batch,
                                               const Smem<N, NQ, PREC, CBX>& sm, const HexTables& tb,
                                               double* sX, int32_t node_ahead = -1) {
  using S = Shape<N, NQ, 8, CBX>;
  using T = typename Prec<PREC>::T;
  using TG = typename Prec<PREC>::TG;
  constexpr int PN = S::PN, PQ = S::PQ, CB = S::CB;
  constexpr int NG = geom_entries<KIND>();
  const TG* geom = static_cast<const TG*>(a.geom);
  const T* sB = sm.sB;
  const T* sD = sm.sD;
  T* A = sm.A;
  T* Bf = sm.Bf;
  T* F0 = sm.F0;
  T* F1 = sm.F1;
  T* F2 = sm.F2;
  const int cl = sm.cl, pt = sm.pt;
  {
    const int64_t idx = batch * CB + cl;
    const bool valid = (cl < CB) && (idx < a.count);
    int64_t cell = 0;
    if (valid) cell = a.cell_list ? (int64_t)__ldg(a.cell_list + idx) : idx;

    // gather x through the cell->node map; keep the node for the scatter
    int32_t node = 0;
    if (valid && pt < PN) {
      node = node_ahead >= 0 ? node_ahead : __ldg(a.cell_node + cell * PN + pt);
      A[pt] = Prec<PREC>::in(__ldg(a.x + node));
    }
    // geometric factors of this point (consumed after three sweeps): stored, or from the vertices
    T g[NG];
    if constexpr (OTF) {
      if (valid && pt < PN)  // 24 coordinates per cell (a Q1 cell has only 8 threads)
        for (int i = pt; i < 24; i += PN)
          sX[cl * 24 + i] = __ldg(a.coords + 3 * (int64_t)__ldg(a.cell_vert + 8 * cell + i / 3) + i % 3);
      __syncthreads();
      if (valid && pt < PQ) {
        double gd[NG];
        if (!point_geometry<NG>(sX + cl * 24, tb, pt % NQ, (pt / NQ) % NQ, pt / (NQ * NQ), a.c0, gd)) atomicOr(a.err, 1);
#pragma unroll
        for (int e = 0; e < NG; ++e) g[e] = gd[e];
      }
    } else {
      if (valid && pt < PQ) {
#pragma unroll
        for (int e = 0; e < NG; ++e) g[e] = Prec<PREC>::geo(geom + (cell * NG + e) * PQ + pt);
      }
      __syncthreads();
    }

    // B in x: (NQ, N, N) <- (N, N, N)
    if (valid && pt < NQ * N * N) {
      const int i = pt % NQ, jk = pt / NQ;
      T s = 0;
#pragma unroll
      for (int m = 0; m < N; ++m) s = fma(sB[i * N + m], A[m + N * jk], s);
      Bf[pt] = s;
    }
    __syncthreads();
    // B in y: (NQ, NQ, N) <- (NQ, N, N)
    if (valid && pt < NQ * NQ * N) {
      const int i = pt % NQ, j = (pt / NQ) % NQ, k = pt / (NQ * NQ);
      T s = 0;
#pragma unroll
      for (int m = 0; m < N; ++m) s = fma(sB[j * N + m], Bf[i + NQ * (m + N * k)], s);
      A[pt] = s;
    }
    __syncthreads();
    // B in z: (NQ, NQ, NQ) <- (NQ, NQ, N)
    if (valid && pt < PQ) {
      const int ij = pt % (NQ * NQ), k = pt / (NQ * NQ);
      T s = 0;
#pragma unroll
      for (int m = 0; m < N; ++m) s = fma(sB[k * N + m], A[ij + NQ * NQ * m], s);
      Bf[pt] = s;
    }
    __syncthreads();

    if constexpr (KIND == MFA_FORM_MASS) {
      if (valid && pt < PQ) A[pt] = g[0] * Bf[pt];
    } else {
      T v0 = 0;
      if (valid && pt < PQ) {
        const int i = pt % NQ, j = (pt / NQ) % NQ, k = pt / (NQ * NQ);
        T d0 = 0, d1 = 0, d2 = 0;
#pragma unroll
        for (int m = 0; m < NQ; ++m) {
          d0 = fma(sD[i * NQ + m], Bf[m + NQ * (j + NQ * k)], d0);
          d1 = fma(sD[j * NQ + m], Bf[i + NQ * (m + NQ * k)], d1);
          d2 = fma(sD[k * NQ + m], Bf[i + NQ * (j + NQ * m)], d2);
        }
        // G = w|J| J^{-1} J^{-T}: (00, 11, 22, 01, 02, 12)
        F0[pt] = fma(g[0], d0, fma(g[3], d1, g[4] * d2));
        F1[pt] = fma(g[3], d0, fma(g[1], d1, g[5] * d2));
        F2[pt] = fma(g[4], d0, fma(g[5], d1, g[2] * d2));
        if constexpr (KIND == MFA_FORM_HELMHOLTZ) v0 = g[6] * Bf[pt];
      }
      __syncthreads();
      if (valid && pt < PQ) {
        const int i = pt % NQ, j = (pt / NQ) % NQ, k = pt / (NQ * NQ);
        T r = v0;
#pragma unroll
        for (int m = 0; m < NQ; ++m) {
          r = fma(sD[m * NQ + i], F0[m + NQ * (j + NQ * k)], r);
          r = fma(sD[m * NQ + j], F1[i + NQ * (m + NQ * k)], r);
          r = fma(sD[m * NQ + k], F2[i + NQ * (j + NQ * m)], r);
        }
        A[pt] = r;
      }
    }
    __syncthreads();

    // B^T in z: (NQ, NQ, N) <- (NQ, NQ, NQ)
    if (valid && pt < NQ * NQ * N) {
      const int ij = pt % (NQ * NQ), c = pt / (NQ * NQ);
      T s = 0;
#pragma unroll
      for (int m = 0; m < NQ; ++m) s = fma(sB[m * N + c], A[ij + NQ * NQ * m], s);
      Bf[pt] = s;
    }
    __syncthreads();
    // B^T in y: (NQ, N, N) <- (NQ, NQ, N)
    if (valid && pt < NQ * N * N) {
      const int i = pt % NQ, b = (pt / NQ) % N, c = pt / (NQ * N);
      T s = 0;
#pragma unroll
      for (int m = 0; m < NQ; ++m) s = fma(sB[m * N + b], Bf[i + NQ * (m + NQ * c)], s);
      A[pt] = s;
    }
    __syncthreads();
    // B^T in x and scatter-add: (N, N, N) <- (NQ, N, N)
    if (valid && pt < PN) {
      const int i = pt % N, bc = pt / N;
      T s = 0;
#pragma unroll
      for (int m = 0; m < NQ; ++m) s = fma(sB[m * N + i], A[m + NQ * bc], s);
      if constexpr (COLOUR) {
        a.y[node] += (double)s;  // no other cell of this colour touches `node`
      } else if constexpr (AGG) {
        warp_aggregated_add(a.y, node, (double)s);
      } else {
        atomicAdd(a.y + node, (double)s);
      }
    }
    __syncthreads();
  }
}

template <int N, int NQ, int KIND, bool COLOUR, int PREC, int CBX = 0, bool AGG = false, bool OTF = false>
__global__ void __launch_bounds__(Shape<N, NQ, 8, CBX>::T) hex_apply_kernel(const __grid_constant__ HexTables tb,
                                                                           const HexApplyArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int CB = Shape<N, NQ, 8, CBX>::CB;
  __shared__ double sX[OTF ? CB * 24 : 1];  // the batch's vertex coordinates (on-the-fly geometry)
  Smem<N, NQ, PREC, CBX> sm;
  sm.init(smem_raw, tb);
  const int64_t nbatch = (a.count + CB - 1) / CB;
  int32_t next = (int64_t)blockIdx.x < nbatch ? point_node<N, NQ, CBX>(a, blockIdx.x, sm.cl, sm.pt) : -1;
  for (int64_t batch = blockIdx.x; batch < nbatch; batch += gridDim.x) {
    const int32_t node = next;
    if (batch + gridDim.x < nbatch) next = point_node<N, NQ, CBX>(a, batch + gridDim.x, sm.cl, sm.pt);
    hex_cell_batch<N, NQ, KIND, COLOUR, PREC, CBX, AGG, OTF>(a, batch, sm, tb, sX, node);
  }
}

// Many forms of one (n, nq, kind, precision) class in one persistent launch:
// the global batch index runs over all forms' batches (prefix sums in
// `first`), so blocks move from one operator to the next without a launch.
template <int N, int NQ, int KIND, int PREC>
__global__ void __launch_bounds__(Shape<N, NQ>::T) hex_apply_group_kernel(const __grid_constant__ HexTables tb,
                                                                          const HexApplyArgs* __restrict__ items,
                                                                          const int64_t* __restrict__ first,
                                                                          int nitems) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<N, NQ, PREC> sm;
  sm.init(smem_raw, tb);
  const int64_t total = first[nitems];
  int k = 0;
  for (int64_t gb = blockIdx.x; gb < total; gb += gridDim.x) {
    while (k + 1 < nitems && gb >= first[k + 1]) ++k;  // batches only increase within a block
    const HexApplyArgs a = items[k];
    hex_cell_batch<N, NQ, KIND, false, PREC>(a, gb - first[k], sm, tb, nullptr);
  }
}

template <int N, int NQ, int KIND, bool COLOUR, int PREC, int CBX = 0, bool AGG = false, bool OTF = false>
cudaError_t launch_apply(const HexTables& tb, const HexApplyArgs& a, GridBudget budget, cudaStream_t s) {
  using S = Shape<N, NQ, (int)sizeof(typename Prec<PREC>::T), CBX>;
  auto kern = hex_apply_kernel<N, NQ, KIND, COLOUR, PREC, CBX, AGG, OTF>;
  static int blocks_per_sm = -1;
  if (blocks_per_sm < 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, S::T, S::SMEM);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  const int64_t nbatch = (a.count + S::CB - 1) / S::CB;
  if (nbatch == 0) return cudaSuccess;
  const int64_t grid = nbatch < budget.cap(blocks_per_sm) ? nbatch : budget.cap(blocks_per_sm);
  kern<<<(unsigned)grid, S::T, S::SMEM, s>>>(tb, a);
  return cudaGetLastError();
}

template <int N, int NQ, int KIND, int PREC>
cudaError_t launch_group(const HexTables& tb, const HexApplyArgs* items, const int64_t* first, int nitems,
                         int64_t total_batches, GridBudget budget, cudaStream_t s) {
  using S = Shape<N, NQ, (int)sizeof(typename Prec<PREC>::T)>;
  auto kern = hex_apply_group_kernel<N, NQ, KIND, PREC>;
  static int blocks_per_sm = -1;
  if (blocks_per_sm < 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, S::T, S::SMEM);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  if (total_batches == 0) return cudaSuccess;
  const int64_t cap = budget.cap(blocks_per_sm);
  kern<<<(unsigned)(total_batches < cap ? total_batches : cap), S::T, S::SMEM, s>>>(tb, items, first, nitems);
  return cudaGetLastError();
}

#define MFA_HEX_GROUP_CASES(NN, PREC)                                                                   \
  if (n == NN) {                                                                                       \
    switch (kind) {                                                                                    \
      case MFA_FORM_MASS:                                                                              \
        return launch_group<NN, NN, MFA_FORM_MASS, PREC>(tb, items, first, nitems, total, budget, s); \
      case MFA_FORM_LAPLACE:                                                                           \
        return launch_group<NN, NN, MFA_FORM_LAPLACE, PREC>(tb, items, first, nitems, total, budget, s); \
      case MFA_FORM_HELMHOLTZ:                                                                         \
        return launch_group<NN, NN, MFA_FORM_HELMHOLTZ, PREC>(tb, items, first, nitems, total, budget, s); \
      default:                                                                                         \
        return cudaErrorInvalidValue;                                                                  \
    }                                                                                                  \
  }

// Dispatch over the supported (n, nq) pairs for one precision.
#define MFA_HEX_KIND_CASES(NN, NQQ, PREC)                                                              \
  if (n == NN && nq == NQQ) {                                                                          \
    switch (kind) {                                                                                    \
      case MFA_FORM_MASS:                                                                              \
        return colour ? launch_apply<NN, NQQ, MFA_FORM_MASS, true, PREC>(tb, a, budget, s)           \
                      : launch_apply<NN, NQQ, MFA_FORM_MASS, false, PREC>(tb, a, budget, s);         \
      case MFA_FORM_LAPLACE:                                                                           \
        return colour ? launch_apply<NN, NQQ, MFA_FORM_LAPLACE, true, PREC>(tb, a, budget, s)        \
                      : launch_apply<NN, NQQ, MFA_FORM_LAPLACE, false, PREC>(tb, a, budget, s);      \
      case MFA_FORM_HELMHOLTZ:                                                                         \
        return colour ? launch_apply<NN, NQQ, MFA_FORM_HELMHOLTZ, true, PREC>(tb, a, budget, s)      \
                      : launch_apply<NN, NQQ, MFA_FORM_HELMHOLTZ, false, PREC>(tb, a, budget, s);    \
      default:                                                                                         \
        return cudaErrorInvalidValue;                                                                  \
    }                                                                                                  \
  }

// Same, for an explicit number of cells per block CBB (autotuner choices).
#define MFA_HEX_KIND_CASES_CB(NN, NQQ, CBB, PREC)                                                     \
  if (n == NN && nq == NQQ && cb == CBB) {                                                             \
    switch (kind) {                                                                                    \
      case MFA_FORM_MASS:                                                                              \
        return colour ? launch_apply<NN, NQQ, MFA_FORM_MASS, true, PREC, CBB>(tb, a, budget, s)      \
                      : launch_apply<NN, NQQ, MFA_FORM_MASS, false, PREC, CBB>(tb, a, budget, s);    \
      case MFA_FORM_LAPLACE:                                                                           \
        return colour ? launch_apply<NN, NQQ, MFA_FORM_LAPLACE, true, PREC, CBB>(tb, a, budget, s)   \
                      : launch_apply<NN, NQQ, MFA_FORM_LAPLACE, false, PREC, CBB>(tb, a, budget, s); \
      case MFA_FORM_HELMHOLTZ:                                                                         \
        return colour ? launch_apply<NN, NQQ, MFA_FORM_HELMHOLTZ, true, PREC, CBB>(tb, a, budget, s) \
                      : launch_apply<NN, NQQ, MFA_FORM_HELMHOLTZ, false, PREC, CBB>(tb, a, budget, s); \
      default:                                                                                         \
        return cudaErrorInvalidValue;                                                                  \
    }                                                                                                  \
  }

// Matrix-free diagonal d_i = sum_K A_K[i][i] (for Jacobi preconditioning).
// With phi_i = l_a(x) l_b(y) l_c(z) and stored G, the diagonal is a sum of 7
// tensor terms, sum_q G_t(q) U_t[q_x][a] V_t[q_y][b] W_t[q_z][c], each
// contracted by three 1D sweeps (z, then y, then x) over the Gauss points.
template <int N, int NQ, int KIND>
__global__ void __launch_bounds__(Shape<N, NQ>::T) hex_diag_kernel(const __grid_constant__ HexTables tb,
                                                                   const int32_t* __restrict__ cell_node,
                                                                   const double* __restrict__ geom, int64_t ncell,
                                                                   double* __restrict__ d) {
  using S = Shape<N, NQ>;
  constexpr int P = S::P, PN = S::PN, PQ = S::PQ, CB = S::CB;
  constexpr int NG = geom_entries<KIND>();
  extern __shared__ double smem[];
  double* B2 = smem;             // [NQ][N] B*B
  double* DB2 = B2 + NQ * N;     // [NQ][N] (D B)*(D B)
  double* X = DB2 + NQ * N;      // [NQ][N] (D B)*B
  double* bufA = X + NQ * N;     // [CB][P]
  double* bufB = bufA + CB * P;  // [CB][P]
  const int t = threadIdx.x;
  for (int e = t; e < NQ * N; e += blockDim.x) {
    const int q = e / N, a = e % N;
    double db = 0.0;
    for (int r = 0; r < NQ; ++r) db += tb.D[q * NQ + r] * tb.B[r * N + a];
    const double b = tb.B[q * N + a];
    B2[e] = b * b;
    DB2[e] = db * db;
    X[e] = db * b;
  }
  const int cl = t / P, pt = t - cl * P;
  double* A = bufA + cl * P;
  double* Bf = bufB + cl * P;
  const int64_t nbatch = (ncell + CB - 1) / CB;
  // term t: geometry entry, factor for x, y, z (0: B2, 1: DB2, 2: X), multiplier
  constexpr int nterm = KIND == MFA_FORM_MASS ? 1 : (KIND == MFA_FORM_LAPLACE ? 6 : 7);
  const int tg[7] = {0, 1, 2, 3, 4, 5, 6};
  const int fx[7] = {1, 0, 0, 2, 2, 0, 0}, fy[7] = {0, 1, 0, 2, 0, 2, 0}, fz[7] = {0, 0, 1, 0, 2, 2, 0};
  const double mult[7] = {1, 1, 1, 2, 2, 2, 1};
  __syncthreads();
  for (int64_t batch = blockIdx.x; batch < nbatch; batch += gridDim.x) {
    const int64_t cell = batch * CB + cl;
    const bool valid = (cl < CB) && (cell < ncell);
    double acc = 0.0;
    for (int term = 0; term < nterm; ++term) {
      const int ge = KIND == MFA_FORM_MASS ? 0 : tg[term];
      const int ix = KIND == MFA_FORM_MASS ? 0 : fx[term], iy = KIND == MFA_FORM_MASS ? 0 : fy[term],
                iz = KIND == MFA_FORM_MASS ? 0 : fz[term];
      const double* U = ix == 0 ? B2 : (ix == 1 ? DB2 : X);
      const double* V = iy == 0 ? B2 : (iy == 1 ? DB2 : X);
      const double* W = iz == 0 ? B2 : (iz == 1 ? DB2 : X);
      if (valid && pt < PQ) A[pt] = mult[term] * geom[(cell * NG + ge) * PQ + pt];
      __syncthreads();
      if (valid && pt < NQ * NQ * N) {  // z: (NQ, NQ, N) <- (NQ, NQ, NQ)
        const int ij = pt % (NQ * NQ), c = pt / (NQ * NQ);
        double s = 0.0;
        for (int m = 0; m < NQ; ++m) s = fma(W[m * N + c], A[ij + NQ * NQ * m], s);
        Bf[pt] = s;
      }
      __syncthreads();
      if (valid && pt < NQ * N * N) {  // y: (NQ, N, N) <- (NQ, NQ, N)
        const int i = pt % NQ, b = (pt / NQ) % N, c = pt / (NQ * N);
        double s = 0.0;
        for (int m = 0; m < NQ; ++m) s = fma(V[m * N + b], Bf[i + NQ * (m + NQ * c)], s);
        A[pt] = s;
      }
      __syncthreads();
      if (valid && pt < PN) {  // x: (N, N, N) <- (NQ, N, N)
        const int i = pt % N, bc = pt / N;
        double s = 0.0;
        for (int m = 0; m < NQ; ++m) s = fma(U[m * N + i], A[m + NQ * bc], s);
        acc += s;
      }
      __syncthreads();
    }
    if (valid && pt < PN) atomicAdd(d + cell_node[cell * PN + pt], acc);
  }
}

template <int N, int NQ, int KIND>
cudaError_t launch_diag(const HexTables& tb, const int32_t* cell_node, const double* geom, int64_t ncell, double* d,
                        GridBudget budget, cudaStream_t s) {
  using S = Shape<N, NQ>;
  auto kern = hex_diag_kernel<N, NQ, KIND>;
  const int smem = (3 * NQ * N + 2 * S::CB * S::P) * 8;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int64_t nbatch = (ncell + S::CB - 1) / S::CB;
  if (nbatch == 0) return cudaSuccess;
  const int64_t grid = nbatch < budget.cap(4) ? nbatch : budget.cap(4);
  kern<<<(unsigned)grid, S::T, smem, s>>>(tb, cell_node, geom, ncell, d);
  return cudaGetLastError();
}

}  // namespace hexk
}  // namespace mfa
