// Quadrilateral kernels: geometry and dispatch (templates in quad_kernels.cuh; the instantiations live in
// quad_kernels_a.cu (n = 2..5) and quad_kernels_b.cu (n = 6..9), compiled in parallel).
#include "quad_kernels.cuh"

namespace mfa {
namespace {

__global__ void quad_geometry_kernel(const __grid_constant__ HexTables tb, int nq1, int kind, double c0,
                                     const double* __restrict__ coords, const int32_t* __restrict__ cell_vert,
                                     int64_t ncell, double* __restrict__ geom, int* err) {
  const int pq = nq1 * nq1, ng = quad_geom_entries_for(kind);
  const int64_t total = ncell * pq;
  for (int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gid < total;
       gid += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = gid / pq;
    const int q = (int)(gid - cell * pq);
    const int qi = q % nq1, qj = q / nq1;
    const double xi[2] = {tb.x1[qi], tb.x1[qj]};
    const double w = tb.w1[qi] * tb.w1[qj];
    double J[2][2] = {{0, 0}, {0, 0}};
    for (int v = 0; v < 4; ++v) {
      const int32_t vid = cell_vert[cell * 4 + v];
      const double fx = (v & 1) ? xi[0] : 1.0 - xi[0], fy = (v & 2) ? xi[1] : 1.0 - xi[1];
      const double dN[2] = {((v & 1) ? 1.0 : -1.0) * fy, fx * ((v & 2) ? 1.0 : -1.0)};
      for (int d = 0; d < 2; ++d) {
        const double X = coords[3 * (int64_t)vid + d];
        J[d][0] += X * dN[0];
        J[d][1] += X * dN[1];
      }
    }
    const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    double* out = geom + cell * (int64_t)ng * pq + q;
    if (!(det != 0.0) || !isfinite(det)) {
      atomicOr(err, 1);
      for (int e = 0; e < ng; ++e) out[e * pq] = 0.0;
      continue;
    }
    const double Ji[2][2] = {{J[1][1] / det, -J[0][1] / det}, {-J[1][0] / det, J[0][0] / det}};
    const double wdet = w * fabs(det);
    if (ng == 1) {
      out[0] = c0 * wdet;
    } else if (ng == 5) {
      out[0] = Ji[0][0];
      out[pq] = Ji[0][1];
      out[2 * pq] = Ji[1][0];
      out[3 * pq] = Ji[1][1];
      out[4 * pq] = wdet;
    } else {
      out[0] = wdet * (Ji[0][0] * Ji[0][0] + Ji[0][1] * Ji[0][1]);
      out[pq] = wdet * (Ji[1][0] * Ji[1][0] + Ji[1][1] * Ji[1][1]);
      out[2 * pq] = wdet * (Ji[0][0] * Ji[1][0] + Ji[0][1] * Ji[1][1]);
      if (ng == 4) out[3 * pq] = c0 * wdet;
    }
  }
}

}  // namespace

cudaError_t quad_apply_launch_a(int n, int nq, int ncomp, int kind, int law, bool colour, const HexTables& tb,
                                const QuadArgs& a, GridBudget budget, cudaStream_t s);
cudaError_t quad_apply_launch_b(int n, int nq, int ncomp, int kind, int law, bool colour, const HexTables& tb,
                                const QuadArgs& a, GridBudget budget, cudaStream_t s);

int quad_geom_entries(int kind) { return quad_geom_entries_for(kind); }

cudaError_t quad_geometry_launch(int nq, int kind, double c0, const HexTables& tb, const double* coords,
                                 const int32_t* cell_vert, int64_t ncell, double* geom, int* err, cudaStream_t s) {
  const int64_t total = ncell * nq * nq;
  if (total == 0) return cudaSuccess;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 65535 * 8) blocks = 65535 * 8;
  quad_geometry_kernel<<<(unsigned)blocks, 256, 0, s>>>(tb, nq, kind, c0, coords, cell_vert, ncell, geom, err);
  return cudaGetLastError();
}

int quad_cells_per_block(int n, int nq) {
  const int m = n > nq ? n : nq;
  return m * m <= 128 ? 256 / (m * m) : 1;
}

cudaError_t quad_apply_launch(int n, int nq, int ncomp, int kind, int law, bool colour, const HexTables& tb,
                              const QuadArgs& a, GridBudget budget, cudaStream_t s) {
  return n <= 5 ? quad_apply_launch_a(n, nq, ncomp, kind, law, colour, tb, a, budget, s)
                : quad_apply_launch_b(n, nq, ncomp, kind, law, colour, tb, a, budget, s);
}

}  // namespace mfa
