// Internal declarations of the mfa library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mfa.h"

namespace mfa {

constexpr int kMaxN = 10;  // nodes or quadrature points per direction (Q_p, p <= 8; p+2 points)

// Grid of a persistent launch: each block walks work units (batches of cells)
// with a stride of gridDim.x.  By default one wave of `bps` resident blocks on
// every SM; with max_blocks > 0 at most that many blocks, so that each block
// walks more units (mfa_launch_config.max_blocks).
struct GridBudget {
  int sms = 0;
  int max_blocks = 0;
  int64_t cap(int bps) const {
    const int64_t c = (int64_t)sms * (bps > 0 ? bps : 1);
    return max_blocks > 0 && max_blocks < c ? max_blocks : c;
  }
};

// ---------------------------------------------------------------- tables.cpp
// Quadrature rules and 1D/3D basis tabulations built on the host in FP64.
void gauss_jacobi01(int n, int alpha, double* x, double* w);  // weight (1-x)^alpha on [0,1]
void gauss_legendre01(int n, double* x, double* w);
void gll01(int n, double* x);
// Lagrange basis on `nodes` (n) evaluated at `pts` (m): L[q*n + a] = l_a(pts[q]).
void lagrange_matrix(int n, const double* nodes, int m, const double* pts, double* L);
// Collocation derivative on `pts` (m points): D[q*m + r] = l_r'(pts[q]).
void collocation_derivative(int m, const double* pts, double* D);
// Reference-tet rules.  Returns the number of points.
int tet_rule_collapsed(int degree, double* pts, double* w);  // conical product, m = ceil((deg+1)/2)
// Table 2's fully symmetric rule of degree <= 6 on the reference triangle (dim 2)
// or tetrahedron (dim 3): pts [nq][dim], w [nq]; returns nq, 0 above degree 6,
// -1 if the derivation fails (simplex_rules.cpp).
int simplex_rule_symmetric(int dim, int degree, std::vector<double>& pts, std::vector<double>& w);
// P1 / P2 basis on the reference tet (closed forms in barycentric coordinates).
void tet_basis(int p, const double* xi, double* phi, double* dphi);
// P3..P6 on the equispaced lattice (Silvester's product formula); nodes (i, j, k)/p, i fastest, then j, then k.
constexpr int kTetMaxP = 6;
int tet_lattice_size(int p);
void tet_basis_pk(int p, const double* xi, double* phi, double* dphi);
// Triangles: collapsed rule (pts [nq][2]) and the P_p lattice basis (nodes (i, j)/p, i fastest; dphi [n][2]).
int tri_rule_collapsed(int degree, double* pts, double* w);
int tri_lattice_size(int p);
void tri_basis_pk(int p, const double* xi, double* phi, double* dphi);
// Vertices per cell of each cell type, and whether it is planar.
inline int verts_of(int ct) { return ct == MFA_CELL_TRI3 ? 3 : ((ct == MFA_CELL_TET4 || ct == MFA_CELL_QUAD4) ? 4 : 8); }
inline bool is_planar(int ct) { return ct == MFA_CELL_TRI3 || ct == MFA_CELL_QUAD4; }

// ---------------------------------------------------------------- colour.cpp
// Greedy first-fit colouring: cells sharing a node get different colours.
// Returns the number of colours (0 on failure); `order` lists cells grouped by
// colour and `offsets` has ncolours + 1 entries.
int greedy_colour(int64_t ncell, int nloc, const int32_t* cell_node, int64_t nnode,
                  std::vector<int32_t>& order, std::vector<int64_t>& offsets);

// ---------------------------------------------------------------- hex kernels
struct HexTables {
  double B[kMaxN * kMaxN];   // [nq][n]: basis at Gauss points
  double D[kMaxN * kMaxN];   // [nq][nq]: collocation derivative at Gauss points
  double w1[kMaxN];          // 1D Gauss weights on [0,1]
  double x1[kMaxN];          // 1D Gauss points on [0,1]
};

struct HexApplyArgs {
  const double* x;
  double* y;
  const int32_t* cell_node;  // [ncell][n^3]
  const void* geom;          // [ncell][ng][nq^3], double / float / bfloat16 by precision
  const int32_t* cell_list;  // cells to process (nullptr: 0..count-1)
  int64_t count;             // number of cells to process
  int* err;
  int64_t geom_stride;       // elements per cell of geom (ng * nq^3, padded to 16 bytes for FP32/BF16)
  // on-the-fly geometry (FP64 point kernel): the trilinear map from the vertices, c0 = k2 (Helmholtz) or 1
  const double* coords = nullptr;
  const int32_t* cell_vert = nullptr;
  double c0 = 1.0;
};

// Vector forms on hexes (ncomp = 3, dof = 3 node + c), FP64, p+1 points per direction.
struct HexVecArgs {
  const double* x;
  double* y;
  const int32_t* cell_node;
  const double* geom;        // [ncell][ng][n^3]: G (6, vector Laplacian) or J^{-1} row-major + w|det J| (10)
  const double* ucoef;       // HYPER_JAC linearisation point
  const int32_t* cell_list;  // cells to process (nullptr: 0..count-1)
  int64_t count;
  int64_t geom_stride;       // doubles per cell of geom
  double lam, mu, b0, b1, b2;
  int* err;
};
// nq: n (every form), n + 1 (vector Laplacian, elasticity), 2n (hyperelastic forms, n <= 4)
cudaError_t hex_vector_launch_a(int n, int nq, int kind, int law, bool colour, const HexTables& tb,
                                const HexVecArgs& a, GridBudget budget, cudaStream_t s);  // n = 2..5
cudaError_t hex_vector_launch_b(int n, int nq, int kind, int law, bool colour, const HexTables& tb,
                                const HexVecArgs& a, GridBudget budget, cudaStream_t s);  // n = 6..9

// Launch the sum-factorised FP64 action for cells [list].  Returns a cudaError_t.
struct LaunchConfig;
cudaError_t hex_apply_launch(int n, int nq, int kind, int prec, bool colour, const LaunchConfig& lc,
                             const HexTables& tb, const HexApplyArgs& a, GridBudget budget, cudaStream_t s);
cudaError_t hex_apply_launch_mixed(int n, int nq, int kind, int prec, bool colour, const LaunchConfig& lc,
                                   const HexTables& tb, const HexApplyArgs& a, GridBudget budget, cudaStream_t s);
// One persistent launch over many forms of the same (n, n, kind, precision).
cudaError_t hex_group_launch(int n, int kind, int prec, const HexTables& tb, const HexApplyArgs* items,
                             const int64_t* first, int nitems, int64_t total, GridBudget budget, cudaStream_t s);
cudaError_t hex_group_launch_mixed(int n, int kind, int prec, const HexTables& tb, const HexApplyArgs* items,
                                   const int64_t* first, int nitems, int64_t total, GridBudget budget, cudaStream_t s);
int hex_cells_per_block(int n, int nq);
int hex_line_cells_per_block(int n);
// FP64 even-odd action for n = 5..9, p+1 points (hex_eo.cuh).
cudaError_t hex_eo_apply_launch(int n, int kind, bool colour, const HexApplyArgs& a, GridBudget budget, cudaStream_t s);
cudaError_t hex_eo_group_launch(int n, int kind, const HexApplyArgs* items, const int64_t* first, int nitems,
                                int64_t total, GridBudget budget, cudaStream_t s);
int hex_eo_cells_per_block(int n);
// FP64 kernel choice.  The even-odd line kernel issues 16-30% fewer FP64
// instructions (n = 5..9) but, with n^2 threads per cell, keeps the FP64 pipe
// busy ~80% of the time against ~93% for the point kernel; measured on GB300
// it wins from n = 7 (Q6: 14.15 vs 14.86 ms) and loses at n = 5, 6.
// FP64 hex with p+1 points: the even-odd kernel from Q4 up (the autotuner picks it there on 64^3: 11% ahead of
// the point kernel at Q4).
inline bool hex_use_eo(int n, int nq, int prec) { return prec == MFA_PREC_FP64 && nq == n && n >= 5 && n <= 9; }

// ---------------------------------------------------------------- launch configurations
// Kernel variant (MFA_VARIANT_*) and cells per block of one apply; cb = 0 is
// the variant's default.  Only the compiled choices listed by the *_cb_options
// functions are accepted by the launchers.
struct LaunchConfig {
  int variant = MFA_VARIANT_AUTO;
  int cb = 0;
  bool agg = false;  // warp-aggregated atomic scatter (MFA_SCATTER_WARP)
  bool otf = false;  // geometry recomputed at every point from the vertices (MFA_GEOM_ONTHEFLY)
  int max_blocks = 0;  // grid cap (GridBudget::max_blocks); 0: one wave of resident blocks
};
// Cells per block of a kernel with `per_cell` threads per cell for a target block size.
constexpr int cells_for_target(int per_cell, int target) { return target / per_cell > 0 ? target / per_cell : 1; }
// Line kernels (FP32/BF16 hex): lanes of a warp that carry lines in the sweeps.  For n = 7 a warp takes four
// whole rows of 7 lines (28 lanes): with the padded plane layout that makes the sweeps in all three directions
// free of bank conflicts.  Other n use all 32 lanes on consecutive lines.
__host__ __device__ constexpr int line_lanes(int n) { return n == 7 ? 28 : 32; }
// Cells per block of the line kernels for a target block size (a multiple of 32 threads).
__host__ __device__ constexpr int line_cb_for(int n, int target) {
  return (target / 32) * line_lanes(n) / (n * n) > 0 ? (target / 32) * line_lanes(n) / (n * n) : 1;
}
// Elements per cell of an FP32/BF16 factor block (ng entries of n^3 points, x the slowest point index): the
// smallest multiple of 16 bytes (line_geom_stride_base), plus up to kLineGeomPadMax further 16-byte units,
// chosen to spread the line kernels' factor reads over the most shared-memory banks.
constexpr int kLineGeomPadMax = 8;
__host__ __device__ constexpr int64_t line_geom_stride_base(int n, int ng, int esz) {
  return ((int64_t)ng * n * n * n * esz + 15) / 16 * 16 / esz;
}
__host__ __device__ constexpr int64_t line_geom_stride_max(int n, int ng, int esz) {
  return line_geom_stride_base(n, ng, esz) + kLineGeomPadMax * 16 / esz;
}
int64_t line_geom_stride(int n, int ng, int esz);
int hex_default_variant(int n, int nq, int prec);
// Compiled cells-per-block choices, the default first; return the count (<= 4).
int hex_point_cb_options(int n, int nq, int* out);
int hex_eo_cb_options(int n, int* out);
int hex_line_cb_options(int n, int* out);
int tet_cb_options(int* out);
cudaError_t hex_point_launch_cb(int n, int nq, int kind, bool colour, int cb, const HexTables& tb,
                                const HexApplyArgs& a, GridBudget budget, cudaStream_t s);
cudaError_t hex_eo_apply_launch_cb(int n, int kind, bool colour, int cb, const HexApplyArgs& a, GridBudget budget,
                                   cudaStream_t s);
cudaError_t hex_point_launch_agg(int n, int nq, int kind, const HexTables& tb, const HexApplyArgs& a, GridBudget budget,
                                 cudaStream_t s);
cudaError_t hex_point_launch_otf(int n, int nq, int kind, bool colour, const HexTables& tb, const HexApplyArgs& a,
                                 GridBudget budget, cudaStream_t s);
// FP32/BF16 action with float vectors.
cudaError_t hex_apply_launch_f32(int n, int kind, int prec, const float* x, float* y, const int32_t* cell_node,
                                 const void* geom, int64_t count, int64_t gstride, int* err, GridBudget budget,
                                 cudaStream_t s);
cudaError_t hex_geometry_launch(int nq, int kind, int prec, double c0, const HexTables& tb, const double* coords,
                                const int32_t* cell_vert, int64_t ncell, void* geom, int64_t stride, int* err,
                                cudaStream_t s);
cudaError_t hex_diagonal_launch(int n, int nq, int kind, const HexTables& tb, const int32_t* cell_node,
                                const double* geom, int64_t ncell, double* d, GridBudget budget, cudaStream_t s);
int hex_geom_entries(int kind);  // stored FP64 values per quadrature point

// ---------------------------------------------------------------- tet kernels
constexpr int kTetMaxQ = 27;
struct TetTables {
  int nq;
  double w[kTetMaxQ];
  double phi[kTetMaxQ * 10];      // [q][a]
  double dphi[kTetMaxQ * 10 * 3]; // [q][a][d] reference gradients
  // P2 only: reference gradient of basis a is alpha[a] + beta[a] xi (linear in xi)
  double pts[kTetMaxQ * 3];       // [q][3] quadrature points
  double alpha[10 * 3];           // [a][e]
  double beta[10 * 9];            // [a][e][f]
  double mvec[10];                // sum_q w_q phi_a(xi_q)
  double wmom[13];                // sum_q w_q (1, xi_f, xi_f xi_g): [0], [1 + f], [4 + 3 f + g]
};

struct TetApplyArgs {
  const double* x;
  double* y;
  const double* coords;
  const int32_t* cell_vert;
  const int32_t* cell_node;
  const double* ucoef;       // HYPER_JAC linearisation point
  const int32_t* cell_list;
  int64_t count;
  double k2, lambda, mu, b0, b1, b2;
  int* err;
};

// threads: threads (cells) per block, one of tet_cb_options.
// Whether tet_apply_launch has a kernel for P_p (p = 1, 2) with ncomp
// components, form `kind` and an nq-point rule.
bool tet_rule_compiled(int p, int ncomp, int kind, int nq);
cudaError_t tet_apply_launch(int p, int ncomp, int kind, int law, bool colour, bool agg, int threads,
                             const TetTables& tb, const TetApplyArgs& a, GridBudget budget, cudaStream_t s);
// ---------------------------------------------------------------- quad kernels (quad_kernels.cu)
struct QuadArgs {
  const double* x;
  double* y;
  const int32_t* cell_node;  // [ncell][n^2]
  const double* geom;        // [ncell][ng][nq^2] (quad_geom_entries)
  const double* ucoef;       // HYPER_JAC linearisation point
  const int32_t* cell_list;
  int64_t count;
  double lambda, mu, b0, b1;
  int* err;
};
int quad_geom_entries(int kind);
int quad_cells_per_block(int n, int nq);
cudaError_t quad_geometry_launch(int nq, int kind, double c0, const HexTables& tb, const double* coords,
                                 const int32_t* cell_vert, int64_t ncell, double* geom, int* err, cudaStream_t s);
cudaError_t quad_apply_launch(int n, int nq, int ncomp, int kind, int law, bool colour, const HexTables& tb,
                              const QuadArgs& a, GridBudget budget, cudaStream_t s);

// P3..P6 (dense tabulation, one warp per cell).  Tables in device memory, nl local dofs, nq points.
struct TetDenseArgs {
  const double* x;
  double* y;
  const double* coords;
  const int32_t* cell_vert;
  const int32_t* cell_node;
  const double* ucoef;
  const int32_t* cell_list;
  int64_t count;
  const double* phi_aq;    // [nl][nq]
  const double* dphi_aeq;  // [nl][3][nq]
  const double* phi_qa;    // [nq][nl]
  const double* dphi_qae;  // [nq][nl][3]
  const double* w;         // [nq]
  int nq;
  double k2, lambda, mu, b0, b1, b2;
  int* err;
};
cudaError_t tet_dense_launch(int p, int ncomp, int kind, int law, bool colour, const TetDenseArgs& a, GridBudget budget,
                             cudaStream_t s);
// Diagonals without a sum-factorised kernel (diag.cu): simplices from the
// dense [q][a] tables (tets P3..P6, triangles), tensor cells from the 1D
// tables and stored factors (quads, hex vector forms).
cudaError_t simplex_diagonal_launch(int dim, int ncomp, int nl, int kind, const TetDenseArgs& a, double* d,
                                    cudaStream_t s);
cudaError_t tensor_diagonal_launch(int dim, int ncomp, int n, int nq, int kind, const HexTables& tb,
                                   const int32_t* cell_node, const double* geom, int64_t gstride, int64_t ncell,
                                   double lambda, double mu, double* d, cudaStream_t s);
// Triangles P1..P4, one thread per cell (tri_kernels.cu): tables as a kernel parameter (9.2 KB), at most 25 points.
constexpr int kTriMaxNl = 15, kTriMaxQ = 25;
struct TriTables {
  int nq;
  double w[kTriMaxQ];
  double phi[kTriMaxQ * kTriMaxNl];       // [q][a]
  double dphi[kTriMaxQ * kTriMaxNl * 2];  // [q][a][e]
};
cudaError_t tri_cell_launch(int p, int ncomp, int kind, int law, bool colour, int threads, const TriTables& tb,
                            const TetDenseArgs& a, GridBudget budget, cudaStream_t s);
// Triangles P1..P6 with the same kernel in the plane (gradient tables with 2 components: [nl][2][nq], [nq][nl][2]).
cudaError_t tri_dense_launch(int p, int ncomp, int kind, int law, bool colour, const TetDenseArgs& a, GridBudget budget,
                             cudaStream_t s);
cudaError_t tet_diagonal_launch(int p, int ncomp, int kind, const TetTables& tb, const TetApplyArgs& a,
                                double* d, cudaStream_t s);
// Scalar P3/P4 tets, one thread per cell (tet_cell_pk.cu), on rules of at most 24 points: the tables as a kernel
// parameter (27 KB at most), phi [q][a] and the reference gradients [q][a][e] with a local-dof stride of NL.
constexpr int kTetPkMaxNl = 35, kTetPkMaxQ = 24;
struct TetPkTables {
  int nq;
  double w[kTetPkMaxQ];
  double phi[kTetPkMaxQ * kTetPkMaxNl];
  double dphi[kTetPkMaxQ * kTetPkMaxNl * 3];
};
cudaError_t tet_pk_cell_launch(int p, int kind, bool colour, int threads, const TetPkTables& tb,
                               const TetDenseArgs& a, GridBudget budget, cudaStream_t s);

// ---------------------------------------------------------------- blas
cudaError_t dot_launch(const double* a, const double* b, int64_t n, double* partial, double* out, cudaStream_t s);
cudaError_t axpby_launch(double alpha, const double* x, double beta, double* y, int64_t n, cudaStream_t s);
cudaError_t pointwise_mul_launch(const double* a, const double* b, double* out, int64_t n, cudaStream_t s);
// Dirichlet constraints (mask[i] != 0: constrained): out = R x; y += R ax + (I - R) x; d[i] = 1 where constrained.
cudaError_t dirichlet_mask_launch(const double* x, const uint8_t* mask, double* out, int64_t n, cudaStream_t s);
cudaError_t dirichlet_combine_launch(const double* ax, const double* x, const uint8_t* mask, double* y, int64_t n,
                                     cudaStream_t s);
cudaError_t dirichlet_diag_launch(const uint8_t* mask, double* d, int64_t n, cudaStream_t s);
cudaError_t reciprocal_launch(const double* a, double* out, int64_t n, cudaStream_t s);
cudaError_t convert_d2f_launch(const double* x, float* y, int64_t n, cudaStream_t s);
cudaError_t dot32_launch(const float* a, const float* b, int64_t n, double* partial, double* out, cudaStream_t s);
cudaError_t jacobi_init32_launch(const float* d, const float* r, float* z, float* p, int64_t n, double* partial,
                                 double* out, cudaStream_t s);
cudaError_t cg_update32_launch(const float* p, const float* q, float* r, float* x, const float* d, float* z,
                               int64_t n, const double* rz, const double* pq, double* partial, double* rz_new,
                               cudaStream_t s);
cudaError_t xpby32_launch(const float* z, float* p, int64_t n, const double* num, const double* den, cudaStream_t s);
cudaError_t convert_f2d_launch(const float* x, double* y, int64_t n, cudaStream_t s);
cudaError_t axpy_ratio_launch(const double* x, double* y, int64_t n, const double* num, const double* den, double sign,
                              cudaStream_t s);
cudaError_t xpby_ratio_launch(const double* z, double* p, int64_t n, const double* num, const double* den,
                              cudaStream_t s);
int dot_partials();

// Record `msg` as the calling thread's mfa_last_error() and return `code`.
int set_error(int code, const char* msg);
// Drop a non-sticky error that an earlier, unrelated runtime call left behind (that call already returned it),
// so that the cudaGetLastError after the next launch reports that launch.  A sticky device error stays.
inline void clear_stale_error() { (void)cudaGetLastError(); }
// z = M(r) of a learned preconditioner, float vectors, on stream s.
int precond_apply_f32(mfa_precond* pc, const float* r, float* z, cudaStream_t s);
bool precond_is_linear(const mfa_precond* pc);
cudaError_t axpy32_ratio_launch(const float* x, float* y, int64_t n, const double* num, const double* den, float sign,
                                cudaStream_t s);
cudaError_t xpay32_ratio_launch(const float* z, float* p, int64_t n, const double* num, const double* den, float sign,
                                cudaStream_t s);
// Enqueue one form's action on `s` (y must already hold zeros or the sum to add to).
int apply_form(mfa_form* f, const double* x, double* y, cudaStream_t s);

}  // namespace mfa

// ---------------------------------------------------------------- handle types
struct mfa_ctx {
  int device = 0;
  int sm_count = 0;
  cudaStream_t stream = nullptr;
  int* d_err = nullptr;          // kernel error flags (bit 0: det J <= 0, bit 1: J <= 0)
  double* d_scratch = nullptr;   // reduction scratch (partials + result)
  cudaStream_t copy_in = nullptr, copy_out = nullptr;  // mfa_apply_host_many's copy streams (created on first use)
  std::vector<cudaEvent_t> events;                    // and its events, two per form, kept for reuse
};

struct mfa_mesh {
  mfa_ctx* ctx = nullptr;
  int device = 0;                // CUDA device of the handle's memory (destroy does not read ctx)
  int cell_type = 0;
  int64_t ncell = 0, nvert = 0;
  double* d_coords = nullptr;
  int32_t* d_cell_vert = nullptr;
};

struct mfa_space {
  mfa_ctx* ctx = nullptr;
  int device = 0;                // CUDA device of the handle's memory (destroy does not read ctx)
  mfa_mesh* mesh = nullptr;
  int degree = 0, ncomp = 1, nloc = 0;
  int64_t nnode = 0;
  int32_t* d_cell_node = nullptr;
  std::vector<int32_t> h_cell_node;  // kept for colouring
  // colouring (built on first coloured form)
  int ncolours = 0;
  std::vector<int64_t> colour_offsets;
  int32_t* d_colour_cells = nullptr;
};

struct mfa_form {
  mfa_ctx* ctx = nullptr;
  int device = 0;                // CUDA device of the handle's memory (destroy does not read ctx)
  mfa_space* space = nullptr;
  mfa_form_params p{};
  int nq1 = 0;                   // hex: points per direction
  int nq = 0;                    // points per cell
  int scatter = MFA_SCATTER_ATOMIC;
  mfa::LaunchConfig launch{};    // variant and cells per block used by apply_form
  double tuned_ms = 0.0;         // time of `launch` measured by mfa_form_autotune
  mfa::HexTables hex{};
  mfa::TetTables tet{};
  double* d_tdense = nullptr;    // P3..P6 tables (TetDenseArgs layouts), tdense_nq points
  mfa::TriTables tri{};          // triangles P1..P4: tables of the thread-per-cell kernel (tri.nq = 0: none)
  mfa::TetPkTables tpk{};        // scalar P3/P4 tets: tables of the thread-per-cell kernel (tpk.nq = 0: none)
  int tdense_nq = 0;
  void* d_geom = nullptr;
  int64_t gstride = 0;           // elements per cell of d_geom
  const double* d_coef = nullptr;
  uint8_t* d_dir_mask = nullptr; // Dirichlet constraints: 1 at constrained dofs (nullptr: none)
  double* d_dir_x = nullptr;     // R x and A R x work vectors of the constrained apply
  double* d_dir_y = nullptr;
  int64_t ndir = 0;
  double* d_stage_x = nullptr;   // mfa_apply_host staging
  double* d_stage_y = nullptr;
  double flops = 0.0, bytes = 0.0, setup_ms = 0.0;
  double flops_executed = 0.0;
};
