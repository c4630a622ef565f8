// Diagonals of the linear forms without a sum-factorised diagonal kernel:
// simplices from their tabulated basis (tetrahedra P3..P6, triangles) and
// tensor cells from their 1D tables and stored factors (quadrilaterals, hex
// vector forms).  One thread per (cell, local dof) sums over the quadrature
// points of the cell
//   scalar:      w|J| (c0 phi_a^2 + grad phi_a . grad phi_a)   (c0 = 1 mass, k^2 Helmholtz, 0 Laplace)
//   vector Lap.: w|J| |grad phi_a|^2 for every component
//   elasticity:  w|J| (mu |grad phi_a|^2 + (mu + lambda) (d_c phi_a)^2) for component c,
// the diagonal entries a(phi_a e_c, phi_a e_c) of the forms of Section 2 (for
// elasticity sigma(u) : eps(u) with u = phi_a e_c), and adds them at the
// dof's node.  On tensor cells the reference gradient of a basis function is
// the 1D derivative of the GLL basis at the Gauss points, D B (D the
// collocation derivative), in one direction times B in the others.
#include "mfa_internal.h"
#include "physics.cuh"

namespace mfa {
namespace {

// Adds the diagonal terms of one quadrature point: wd = w |J| (scalar/elasticity forms with physical
// gradient g), or G-weighted forms through gg = grad phi^T G grad phi and the value term c0w phi^2.
template <int NC>
__device__ __forceinline__ void add_terms(int kind, double lambda, double mu, double wd, const double g[3],
                                          double gg, double value, double* acc) {
  if (kind == MFA_FORM_ELASTICITY) {
    const double gsq = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] += wd * (mu * gsq + (mu + lambda) * g[c] * g[c]);
  } else {
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] += gg + value;
  }
}

template <int DIM, int NC>
__global__ void simplex_diag_kernel(const TetDenseArgs a, int nl, int kind, double* d) {
  constexpr int NV = DIM + 1;
  const double c0 = kind == MFA_FORM_MASS ? 1.0 : (kind == MFA_FORM_HELMHOLTZ ? a.k2 : 0.0);
  const bool grad = kind != MFA_FORM_MASS;
  const int64_t total = a.count * nl;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = idx / nl;
    const int al = (int)(idx - cell * nl);
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    {
      const int32_t v0 = __ldg(a.cell_vert + NV * cell);
      double X0[3];
#pragma unroll
      for (int k = 0; k < DIM; ++k) X0[k] = __ldg(a.coords + 3 * (int64_t)v0 + k);
#pragma unroll
      for (int e = 0; e < DIM; ++e) {
        const int32_t ve = __ldg(a.cell_vert + NV * cell + e + 1);
#pragma unroll
        for (int k = 0; k < DIM; ++k) J[k][e] = __ldg(a.coords + 3 * (int64_t)ve + k) - X0[k];
      }
      if constexpr (DIM == 2) J[2][2] = 1.0;  // the plane embedded in 3D
    }
    double cof[3][3];
    const double det = det3(J, cof);
    if (!(det != 0.0) || !isfinite(det)) {
      if (al == 0) atomicOr(a.err, 1);
      continue;
    }
    const double idet = 1.0 / det, adet = fabs(det);
    double acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0.0;
    for (int q = 0; q < a.nq; ++q) {
      const int64_t qa = (int64_t)q * nl + al;
      const double ph = __ldg(a.phi_qa + qa);
      double dr[3] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int e = 0; e < DIM; ++e) dr[e] = __ldg(a.dphi_qae + DIM * qa + e);
      double g[3];  // physical gradient: g_j = sum_e dr_e (J^{-1})_{ej}, (J^{-1})_{ej} = cof_{je} / det
#pragma unroll
      for (int j = 0; j < 3; ++j) g[j] = (dr[0] * cof[j][0] + dr[1] * cof[j][1] + dr[2] * cof[j][2]) * idet;
      const double wd = __ldg(a.w + q) * adet;
      const double gg = grad ? wd * (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]) : 0.0;
      add_terms<NC>(kind, a.lambda, a.mu, wd, g, gg, wd * c0 * ph * ph, acc);
    }
    const int32_t node = __ldg(a.cell_node + cell * nl + al);
#pragma unroll
    for (int c = 0; c < NC; ++c) atomicAdd(d + (int64_t)NC * node + c, acc[c]);
  }
}

// Stored factors per point ([cell][entry][point]):
//   quads (DIM 2): mass c0w|J|; Laplace G00, G11, G01; Helmholtz G00, G11, G01, c0w|J|;
//                  elasticity J^{-1} row-major (4) and w|J|
//   hex vector (DIM 3): Laplace G00, G11, G22, G01, G02, G12; elasticity J^{-1} row-major (9) and w|J|
template <int DIM, int NC>
__global__ void tensor_diag_kernel(const __grid_constant__ HexTables tb, const int32_t* __restrict__ cell_node,
                                   const double* __restrict__ geom, int64_t gstride, int64_t ncell, int n, int nq,
                                   int kind, double lambda, double mu, double* d) {
  __shared__ double sDB[kMaxN * kMaxN];  // [q][a]: derivative of the GLL basis a at Gauss point q
  for (int i = threadIdx.x; i < nq * n; i += blockDim.x) {
    const int q = i / n, al = i - q * n;
    double s = 0.0;
    for (int r = 0; r < nq; ++r) s += tb.D[q * nq + r] * tb.B[r * n + al];
    sDB[i] = s;
  }
  __syncthreads();
  const int nl = DIM == 3 ? n * n * n : n * n, pq = DIM == 3 ? nq * nq * nq : nq * nq;
  const int64_t total = ncell * nl;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = idx / nl;
    const int al = (int)(idx - cell * nl);
    const int ax = al % n, ay = (al / n) % n, az = DIM == 3 ? al / (n * n) : 0;
    double acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0.0;
    const double* gc = geom + cell * gstride;
    for (int q = 0; q < pq; ++q) {
      const int qx = q % nq, qy = (q / nq) % nq, qz = DIM == 3 ? q / (nq * nq) : 0;
      const double bx = tb.B[qx * n + ax], by = tb.B[qy * n + ay], bz = DIM == 3 ? tb.B[qz * n + az] : 1.0;
      const double dx = sDB[qx * n + ax], dy = sDB[qy * n + ay], dz = DIM == 3 ? sDB[qz * n + az] : 0.0;
      const double ph = bx * by * bz;
      const double dr[3] = {dx * by * bz, bx * dy * bz, DIM == 3 ? bx * by * dz : 0.0};
      const double* gp = gc + q;
      double g[3] = {0.0, 0.0, 0.0}, gg = 0.0, value = 0.0, wd = 0.0;
      if (kind == MFA_FORM_ELASTICITY) {
        constexpr int NJ = DIM * DIM;
#pragma unroll
        for (int j = 0; j < DIM; ++j)
#pragma unroll
          for (int e = 0; e < DIM; ++e) g[j] += dr[e] * __ldg(gp + (int64_t)(e * DIM + j) * pq);
        wd = __ldg(gp + (int64_t)NJ * pq);
      } else if (kind == MFA_FORM_MASS) {
        value = __ldg(gp) * ph * ph;
      } else if (DIM == 2) {
        const double G00 = __ldg(gp), G11 = __ldg(gp + pq), G01 = __ldg(gp + 2 * (int64_t)pq);
        gg = G00 * dr[0] * dr[0] + G11 * dr[1] * dr[1] + 2.0 * G01 * dr[0] * dr[1];
        if (kind == MFA_FORM_HELMHOLTZ) value = __ldg(gp + 3 * (int64_t)pq) * ph * ph;
      } else {  // hex vector Laplacian
        const double G00 = __ldg(gp), G11 = __ldg(gp + pq), G22 = __ldg(gp + 2 * (int64_t)pq);
        const double G01 = __ldg(gp + 3 * (int64_t)pq), G02 = __ldg(gp + 4 * (int64_t)pq),
                     G12 = __ldg(gp + 5 * (int64_t)pq);
        gg = G00 * dr[0] * dr[0] + G11 * dr[1] * dr[1] + G22 * dr[2] * dr[2] +
             2.0 * (G01 * dr[0] * dr[1] + G02 * dr[0] * dr[2] + G12 * dr[1] * dr[2]);
      }
      add_terms<NC>(kind, lambda, mu, wd, g, gg, value, acc);
    }
    const int32_t node = __ldg(cell_node + cell * nl + al);
#pragma unroll
    for (int c = 0; c < NC; ++c) atomicAdd(d + (int64_t)NC * node + c, acc[c]);
  }
}

int64_t diag_blocks(int64_t total) {
  int64_t b = (total + 255) / 256;
  return b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b);
}

}  // namespace

cudaError_t simplex_diagonal_launch(int dim, int ncomp, int nl, int kind, const TetDenseArgs& a, double* d,
                                    cudaStream_t s) {
  if (a.count == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)diag_blocks(a.count * nl);
  if (dim == 3 && ncomp == 1) simplex_diag_kernel<3, 1><<<blocks, 256, 0, s>>>(a, nl, kind, d);
  else if (dim == 3 && ncomp == 3) simplex_diag_kernel<3, 3><<<blocks, 256, 0, s>>>(a, nl, kind, d);
  else if (dim == 2 && ncomp == 1) simplex_diag_kernel<2, 1><<<blocks, 256, 0, s>>>(a, nl, kind, d);
  else if (dim == 2 && ncomp == 2) simplex_diag_kernel<2, 2><<<blocks, 256, 0, s>>>(a, nl, kind, d);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t tensor_diagonal_launch(int dim, int ncomp, int n, int nq, int kind, const HexTables& tb,
                                   const int32_t* cell_node, const double* geom, int64_t gstride, int64_t ncell,
                                   double lambda, double mu, double* d, cudaStream_t s) {
  if (ncell == 0) return cudaSuccess;
  if (n > kMaxN || nq > kMaxN) return cudaErrorInvalidValue;
  const int64_t nl = dim == 3 ? (int64_t)n * n * n : (int64_t)n * n;
  const unsigned blocks = (unsigned)diag_blocks(ncell * nl);
  if (dim == 2 && ncomp == 1)
    tensor_diag_kernel<2, 1><<<blocks, 256, 0, s>>>(tb, cell_node, geom, gstride, ncell, n, nq, kind, lambda, mu, d);
  else if (dim == 2 && ncomp == 2)
    tensor_diag_kernel<2, 2><<<blocks, 256, 0, s>>>(tb, cell_node, geom, gstride, ncell, n, nq, kind, lambda, mu, d);
  else if (dim == 3 && ncomp == 3)
    tensor_diag_kernel<3, 3><<<blocks, 256, 0, s>>>(tb, cell_node, geom, gstride, ncell, n, nq, kind, lambda, mu, d);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace mfa
