// Hexahedral kernels: geometry precompute and dispatch of the sum-factorised
// action (see hex_kernels.cuh for the algorithm).
#include <type_traits>

#include "hex_kernels.cuh"

namespace mfa {

int hex_cells_per_block(int n, int nq) {
  const int m = n > nq ? n : nq;
  const int p = m * m * m;
  return p <= 128 ? 256 / p : 1;  // hexk::Shape<N, NQ>::CB
}

int hex_line_cells_per_block(int n) { return line_cb_for(n, 256); }  // hexl::LShape<N>::CB

int hex_geom_entries(int kind) {
  if (kind >= MFA_FORM_ELASTICITY) return 10;  // J^{-1} (row-major) and w|det J|
  return kind == MFA_FORM_MASS ? 1 : (kind == MFA_FORM_LAPLACE ? 6 : 7);
}

namespace {

// Per Gauss point of a trilinear cell: J = sum_v X_v (grad_ref N_v)^T, then
// G = w|det J| J^{-1} J^{-T} (6 entries) and c0 w|det J| (Sections 2.1 and
// 4.1: the Jacobian of a bilinear/trilinear map is evaluated at every
// quadrature point).  Computed once in FP64 and stored [cell][entry][q], the
// points x fastest for FP64 and x slowest for FP32/BF16 (the line kernels).
template <typename TG>
__device__ __forceinline__ void store_geo(TG* p, double v);
template <>
__device__ __forceinline__ void store_geo<double>(double* p, double v) { *p = v; }
template <>
__device__ __forceinline__ void store_geo<float>(float* p, double v) { *p = (float)v; }
template <>
__device__ __forceinline__ void store_geo<__nv_bfloat16>(__nv_bfloat16* p, double v) { *p = __double2bfloat16(v); }

template <typename TG>
__global__ void hex_geometry_kernel(const __grid_constant__ HexTables tb, int nq1, int ng, double c0,
                                    const double* __restrict__ coords, const int32_t* __restrict__ cell_vert,
                                    int64_t ncell, TG* __restrict__ geom, int64_t stride, int* err) {
  const int pq = nq1 * nq1 * nq1;
  const int64_t total = ncell * pq;
  for (int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gid < total;
       gid += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = gid / pq;
    // point qw of the stored block (consecutive threads write consecutive elements): FP64 blocks order the
    // points x fastest, FP32/BF16 blocks (the line kernels', whose pointwise step runs on x-lines) x slowest
    const int qw = (int)(gid - cell * pq);
    int qi, qj, qk;
    if (std::is_same<TG, double>::value) {
      qi = qw % nq1, qj = (qw / nq1) % nq1, qk = qw / (nq1 * nq1);
    } else {
      qj = qw % nq1, qk = (qw / nq1) % nq1, qi = qw / (nq1 * nq1);
    }
    const double xi[3] = {tb.x1[qi], tb.x1[qj], tb.x1[qk]};
    const double w = tb.w1[qi] * tb.w1[qj] * tb.w1[qk];
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int v = 0; v < 8; ++v) {
      const int32_t vid = cell_vert[cell * 8 + v];
      const int bits[3] = {v & 1, (v >> 1) & 1, (v >> 2) & 1};
      double f[3], df[3];
      for (int d = 0; d < 3; ++d) {
        f[d] = bits[d] ? xi[d] : 1.0 - xi[d];
        df[d] = bits[d] ? 1.0 : -1.0;
      }
      const double dN[3] = {df[0] * f[1] * f[2], f[0] * df[1] * f[2], f[0] * f[1] * df[2]};
      for (int d = 0; d < 3; ++d) {
        const double X = coords[3 * (int64_t)vid + d];
        for (int e = 0; e < 3; ++e) J[d][e] += X * dN[e];
      }
    }
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    if (!(det != 0.0) || !isfinite(det)) {
      atomicOr(err, 1);
      for (int e = 0; e < ng; ++e) store_geo(geom + cell * stride + e * pq + qw, 0.0);
      continue;
    }
    // inverse by the adjugate: Ji[i][j] = cof[j][i] / det
    double Ji[3][3];
    Ji[0][0] = c00 / det;
    Ji[1][0] = c01 / det;
    Ji[2][0] = c02 / det;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    const double wdet = w * fabs(det);
    TG* out = geom + cell * stride + qw;
    if (ng == 1) {
      store_geo(out, c0 * wdet);
      continue;
    }
    if (ng == 10) {  // vector forms: J^{-1} row-major, then w|det J|
      for (int e = 0; e < 9; ++e) store_geo(out + e * pq, Ji[e / 3][e % 3]);
      store_geo(out + 9 * pq, wdet);
      continue;
    }
    const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
    for (int e = 0; e < 6; ++e) {
      const int r = ia[e], c = ib[e];
      store_geo(out + e * pq, wdet * (Ji[r][0] * Ji[c][0] + Ji[r][1] * Ji[c][1] + Ji[r][2] * Ji[c][2]));
    }
    if (ng == 7) store_geo(out + 6 * pq, c0 * wdet);
  }
}

}  // namespace

cudaError_t hex_geometry_launch(int nq, int kind, int prec, double c0, const HexTables& tb, const double* coords,
                                const int32_t* cell_vert, int64_t ncell, void* geom, int64_t stride, int* err,
                                cudaStream_t s) {
  const int64_t total = ncell * nq * nq * nq;
  if (total == 0) return cudaSuccess;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 65535 * 8) blocks = 65535 * 8;
  const int ng = hex_geom_entries(kind);
  if (prec == MFA_PREC_FP64)
    hex_geometry_kernel<double><<<(unsigned)blocks, 256, 0, s>>>(tb, nq, ng, c0, coords, cell_vert, ncell,
                                                                 static_cast<double*>(geom), stride, err);
  else if (prec == MFA_PREC_FP32)
    hex_geometry_kernel<float><<<(unsigned)blocks, 256, 0, s>>>(tb, nq, ng, c0, coords, cell_vert, ncell,
                                                                static_cast<float*>(geom), stride, err);
  else
    hex_geometry_kernel<__nv_bfloat16><<<(unsigned)blocks, 256, 0, s>>>(tb, nq, ng, c0, coords, cell_vert, ncell,
                                                                        static_cast<__nv_bfloat16*>(geom), stride, err);
  return cudaGetLastError();
}

int hex_default_variant(int n, int nq, int prec) {
  if (prec == MFA_PREC_BF16) return MFA_VARIANT_LINE_STAGED;
  if (prec == MFA_PREC_FP32) return MFA_VARIANT_LINE_STAGED;
  return hex_use_eo(n, nq, prec) ? MFA_VARIANT_EVEN_ODD : MFA_VARIANT_POINT;
}

// Default, then half and double the default where the block stays within 512
// threads (hex_kernels_tune.cu instantiates the extra ones, p+1 points only).
int hex_point_cb_options(int n, int nq, int* out) {
  const int m = n > nq ? n : nq, p = m * m * m;
  const int cb0 = hex_cells_per_block(n, nq);
  int k = 0;
  out[k++] = cb0;
  if (nq != n || n > 6) return k;
  if (cb0 / 2 >= 1 && cb0 / 2 != cb0) out[k++] = cb0 / 2;
  if (2 * cb0 * p <= 512) out[k++] = 2 * cb0;
  return k;
}

cudaError_t hex_apply_launch(int n, int nq, int kind, int prec, bool colour, const LaunchConfig& lc,
                             const HexTables& tb, const HexApplyArgs& a, GridBudget budget, cudaStream_t s) {
  if (prec != MFA_PREC_FP64) return hex_apply_launch_mixed(n, nq, kind, prec, colour, lc, tb, a, budget, s);
  const int variant = lc.variant == MFA_VARIANT_AUTO ? hex_default_variant(n, nq, prec) : lc.variant;
  if (variant == MFA_VARIANT_EVEN_ODD) {
    if (nq != n || n < 5 || n > 9 || lc.agg || lc.otf) return cudaErrorInvalidValue;
    if (lc.cb == 0 || lc.cb == hex_eo_cells_per_block(n)) return hex_eo_apply_launch(n, kind, colour, a, budget, s);
    return hex_eo_apply_launch_cb(n, kind, colour, lc.cb, a, budget, s);
  }
  if (variant != MFA_VARIANT_POINT) return cudaErrorInvalidValue;
  if (lc.otf) {
    if (lc.agg || (lc.cb != 0 && lc.cb != hex_cells_per_block(n, nq))) return cudaErrorInvalidValue;
    return hex_point_launch_otf(n, nq, kind, colour, tb, a, budget, s);
  }
  if (lc.agg) {
    if (colour || (lc.cb != 0 && lc.cb != hex_cells_per_block(n, nq))) return cudaErrorInvalidValue;
    return hex_point_launch_agg(n, nq, kind, tb, a, budget, s);
  }
  if (lc.cb != 0 && lc.cb != hex_cells_per_block(n, nq))
    return hex_point_launch_cb(n, nq, kind, colour, lc.cb, tb, a, budget, s);
  using namespace hexk;
  MFA_HEX_KIND_CASES(2, 2, MFA_PREC_FP64)
  MFA_HEX_KIND_CASES(3, 3, MFA_PREC_FP64)
  MFA_HEX_KIND_CASES(4, 4, MFA_PREC_FP64)
  MFA_HEX_KIND_CASES(5, 5, MFA_PREC_FP64)
  MFA_HEX_KIND_CASES(6, 6, MFA_PREC_FP64)
  MFA_HEX_KIND_CASES(7, 7, MFA_PREC_FP64)
  MFA_HEX_KIND_CASES(8, 8, MFA_PREC_FP64)
  MFA_HEX_KIND_CASES(9, 9, MFA_PREC_FP64)
  MFA_HEX_KIND_CASES(2, 3, MFA_PREC_FP64)
  MFA_HEX_KIND_CASES(3, 4, MFA_PREC_FP64)
  MFA_HEX_KIND_CASES(4, 5, MFA_PREC_FP64)
  MFA_HEX_KIND_CASES(5, 6, MFA_PREC_FP64)
  MFA_HEX_KIND_CASES(6, 7, MFA_PREC_FP64)
  MFA_HEX_KIND_CASES(7, 8, MFA_PREC_FP64)
  return cudaErrorInvalidValue;
}

cudaError_t hex_group_launch(int n, int kind, int prec, const HexTables& tb, const HexApplyArgs* items,
                             const int64_t* first, int nitems, int64_t total, GridBudget budget, cudaStream_t s) {
  if (prec != MFA_PREC_FP64) return hex_group_launch_mixed(n, kind, prec, tb, items, first, nitems, total, budget, s);
  if (hex_use_eo(n, n, prec)) return hex_eo_group_launch(n, kind, items, first, nitems, total, budget, s);
  using namespace hexk;
  MFA_HEX_GROUP_CASES(2, MFA_PREC_FP64)
  MFA_HEX_GROUP_CASES(3, MFA_PREC_FP64)
  MFA_HEX_GROUP_CASES(4, MFA_PREC_FP64)
  MFA_HEX_GROUP_CASES(5, MFA_PREC_FP64)
  MFA_HEX_GROUP_CASES(6, MFA_PREC_FP64)
  MFA_HEX_GROUP_CASES(7, MFA_PREC_FP64)
  MFA_HEX_GROUP_CASES(8, MFA_PREC_FP64)
  MFA_HEX_GROUP_CASES(9, MFA_PREC_FP64)
  return cudaErrorInvalidValue;
}

#define MFA_HEX_DIAG_CASE(NN, NQQ)                                                                    \
  if (n == NN && nq == NQQ) {                                                                         \
    switch (kind) {                                                                                   \
      case MFA_FORM_MASS:                                                                             \
        return hexk::launch_diag<NN, NQQ, MFA_FORM_MASS>(tb, cell_node, geom, ncell, d, budget, s); \
      case MFA_FORM_LAPLACE:                                                                          \
        return hexk::launch_diag<NN, NQQ, MFA_FORM_LAPLACE>(tb, cell_node, geom, ncell, d, budget, s); \
      case MFA_FORM_HELMHOLTZ:                                                                        \
        return hexk::launch_diag<NN, NQQ, MFA_FORM_HELMHOLTZ>(tb, cell_node, geom, ncell, d, budget, s); \
      default:                                                                                        \
        return cudaErrorInvalidValue;                                                                 \
    }                                                                                                 \
  }

cudaError_t hex_diagonal_launch(int n, int nq, int kind, const HexTables& tb, const int32_t* cell_node,
                                const double* geom, int64_t ncell, double* d, GridBudget budget, cudaStream_t s) {
  MFA_HEX_DIAG_CASE(2, 2)
  MFA_HEX_DIAG_CASE(3, 3)
  MFA_HEX_DIAG_CASE(4, 4)
  MFA_HEX_DIAG_CASE(5, 5)
  MFA_HEX_DIAG_CASE(6, 6)
  MFA_HEX_DIAG_CASE(7, 7)
  MFA_HEX_DIAG_CASE(8, 8)
  MFA_HEX_DIAG_CASE(9, 9)
  MFA_HEX_DIAG_CASE(2, 3)
  MFA_HEX_DIAG_CASE(3, 4)
  MFA_HEX_DIAG_CASE(4, 5)
  MFA_HEX_DIAG_CASE(5, 6)
  MFA_HEX_DIAG_CASE(6, 7)
  MFA_HEX_DIAG_CASE(7, 8)
  return cudaErrorInvalidValue;
}

}  // namespace mfa
