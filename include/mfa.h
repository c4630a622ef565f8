/*
 * mfa.h -- matrix-free finite element operator action on GB300 (sm_103a).
 *
 * The library evaluates y = A(x): the global assembly of a linear (residual)
 * form L(x; v) over every cell of a tetrahedral or hexahedral mesh, as in
 * Section 2 of arXiv 1903.08243 ("A study of vectorization for matrix-free
 * finite element methods").  One apply is the parloop of Section 2.2,
 *
 *     parloop(kernel, cells, y(cell2dof, INC), coords(cell2vert, R), x(cell2dof, R)),
 *
 * i.e. for every cell: gather the vertex coordinates through the
 * cell->vertex map and the dofs through the cell->node map, evaluate the
 * local element kernel at the quadrature points (Section 2.1, Listing 2), and
 * add the local result into y through the cell->node map (Listing 3).  The
 * element kernels are the operators of the paper's Supplementary material:
 * mass, Helmholtz, (vector) Laplacian, linear elasticity and hyperelasticity
 * (residual and its Gateaux derivative).
 *
 * Conventions
 *  - Every function returns an mfa_status; 0 is success.  Nothing aborts.
 *    mfa_last_error() returns a message for the calling thread's last failure.
 *  - Handles are created and owned by the library; destroy them with the
 *    matching *_destroy call (a NULL handle is accepted and ignored).
 *  - Host arrays passed to *_upload / *_create are copied; the caller keeps
 *    ownership and may free them on return.
 *  - Vectors passed to mfa_apply are device pointers owned by the caller
 *    (e.g. PyTorch tensors), FP64, contiguous, 8-byte aligned.  Work is
 *    enqueued on the context's stream and is asynchronous with respect to the
 *    host; mfa_sync() waits for it and reports errors found by kernels.
 *  - Reference tetrahedron: vertices (0,0,0), (1,0,0), (0,1,0), (0,0,1).
 *    Reference hexahedron: [0,1]^3, local vertex a + 2b + 4c at corner (a,b,c).
 *  - P2 local nodes: 0..3 vertices, 4..9 midpoints of edges (0,1), (0,2),
 *    (0,3), (1,2), (1,3), (2,3).  Q_p local node i + n*j + n*n*k (n = p + 1)
 *    sits at the tensor product of the Gauss-Lobatto-Legendre points.
 *  - A vector field with ncomp = 3 stores dof 3*node + c.
 */
#ifndef MFA_H
#define MFA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MFA_VERSION 1

#if defined(__GNUC__)
#define MFA_API __attribute__((visibility("default")))
#else
#define MFA_API
#endif

typedef enum {
  MFA_OK = 0,
  MFA_ERR_ARG = 1,           /* null pointer, bad size, bad enum value            */
  MFA_ERR_RANGE = 2,         /* a map entry outside [0, n)                          */
  MFA_ERR_UNSUPPORTED = 3,   /* degree / cell / form / precision combination        */
  MFA_ERR_CUDA = 4,          /* a CUDA runtime call failed                          */
  MFA_ERR_OOM = 5,           /* device or host allocation failed                    */
  MFA_ERR_TIMEOUT = 6,       /* a bounded device wait ran out                       */
  MFA_ERR_NOT_CONVERGED = 7, /* an iterative solver reached maxit                   */
  MFA_ERR_BREAKDOWN = 8,     /* CG breakdown: p.Ap <= 0 or a non-finite scalar      */
  MFA_ERR_DOMAIN = 9         /* a kernel met det J <= 0 or a deformation with J <= 0 */
} mfa_status;

/* Cell types (ids, not vertex counts): tetrahedra (4 vertices), hexahedra (8),
 * and in the plane z = 0 triangles (3) and quadrilaterals (4, local vertex v at
 * corner (v & 1, v >> 1 & 1)).  On planar meshes coords keep 3 entries per
 * vertex (z ignored), vector fields have 2 components and the vector forms are
 * plane strain. */
enum { MFA_CELL_TRI3 = 3, MFA_CELL_TET4 = 4, MFA_CELL_HEX8 = 8, MFA_CELL_QUAD4 = 40 };

/* Forms of the Supplementary material (bilinear forms taken by their action). */
enum {
  MFA_FORM_MASS = 0,       /* y_i = int phi_i u                                       */
  MFA_FORM_LAPLACE = 1,    /* y_i = int grad phi_i : grad u   (vector Laplacian if ncomp=3) */
  MFA_FORM_HELMHOLTZ = 2,  /* y_i = int grad phi_i . grad u + k2 phi_i u              */
  MFA_FORM_ELASTICITY = 3, /* y_i = int sigma(u) : eps(phi_i), sigma = 2 mu eps + lambda tr(eps) I */
  MFA_FORM_HYPER_RES = 4,  /* y_i = int P(F) : grad phi_i - b . phi_i, F = I + grad x  */
  MFA_FORM_HYPER_JAC = 5   /* y_i = int dP(F; grad x) : grad phi_i, F = I + grad u (coefficient) */
};

enum { MFA_LAW_SVK = 0, MFA_LAW_NEOHOOKE = 1 };
/* Arithmetic of the element kernel.  FP64: everything in double.  FP32: float
 * arithmetic with geometric factors computed in FP64 and stored as float.
 * BF16: x, the geometric factors and the 1D tables rounded to bfloat16, float
 * arithmetic and accumulation.  x and y stay FP64 in memory for all three.
 * FP32/BF16 cover hexahedral forms with p+1 points per direction. */
enum { MFA_PREC_FP64 = 0, MFA_PREC_FP32 = 1, MFA_PREC_BF16 = 2 };
/* Geometry of hexahedral forms.  STORED: w |det J| J^{-1} J^{-T} (and c0 w |det J|)
 * computed once per Gauss point at form creation and streamed by every apply.
 * ONTHEFLY: recomputed at every Gauss point of every apply from the cell's 8
 * vertices, as Section 4.1 describes for bilinear/trilinear cells (~270 more
 * FP64 operations per point, no stored factors; FP64 scalar hex forms with
 * p+1 points, atomic or colour scatter). */
enum { MFA_GEOM_STORED = 0, MFA_GEOM_ONTHEFLY = 1 };
/* Scatter-add of the local results into y (Section 2.2's INC access):
 * COLOUR  cells of one colour share no node: plain read-modify-write, one launch
 *         per colour, bitwise reproducible;
 * ATOMIC  one FP64 atomic add per local dof (the default);
 * WARP    atomic adds aggregated within a warp: lanes that add into the same
 *         entry are summed first (FP64 point kernel with p+1 points and tets). */
enum { MFA_SCATTER_AUTO = 0, MFA_SCATTER_COLOUR = 1, MFA_SCATTER_ATOMIC = 2, MFA_SCATTER_WARP = 3 };
/* Quadrature on simplices (tetrahedra, triangles).  The integrand of mass and
 * Helmholtz has degree 2p on an affine cell, Laplace and elasticity 2(p-1),
 * St Venant-Kirchhoff 4(p-1); call it d.  The rule's degree is d when d <= qdeg
 * (the integral is then exact), else qdeg.  Rules: Table 2's fully symmetric
 * ones up to degree 6 (1, 4, 14, 24 points on tets for degree 1, 2, 3-5, 6;
 * 1, 3, 6, 12 on triangles for degree 1, 2, 3-4, 5-6; see mfa_simplex_rule),
 * collapsed Gauss-Jacobi products above (m^3 or m^2 points, m = floor(deg/2)+1).
 * AUTO       the symmetric rule where the integral is exact and its degree is
 *            <= 6; the collapsed rule otherwise (the neo-Hookean integrand,
 *            or qdeg < d), so a rule only ever changes rounding;
 * SYMMETRIC  the symmetric rule whenever the rule's degree is <= 6, whatever
 *            the integrand (Table 2's choice, also for neo-Hookean).
 * Hexahedra and quadrilaterals ignore it (Gauss-Legendre products). */
enum { MFA_RULE_AUTO = 0, MFA_RULE_SYMMETRIC = 1 };

typedef struct {
  int32_t kind;            /* MFA_FORM_*                                               */
  int32_t law;             /* MFA_LAW_* (hyperelastic forms)                           */
  int32_t qdeg;            /* 0 = default.  Hex/quad: Gauss points per direction (default
                              p+1).  Tet/triangle: largest rule degree (default 2p;
                              hyperelastic 4 for p <= 2, 2p above); see MFA_RULE_*.     */
  int32_t precision;       /* MFA_PREC_*                                               */
  int32_t scatter;         /* MFA_SCATTER_*                                            */
  int32_t cells_per_block; /* 0 = automatic; else one of the default variant's choices
                              (mfa_form_list_configs), MFA_ERR_UNSUPPORTED otherwise   */
  double k2;               /* Helmholtz coefficient (paper: 1)                          */
  double lambda, mu;       /* Lame parameters (elasticity, hyperelasticity)             */
  double b[3];             /* body force of the hyperelastic residual                   */
  int32_t geometry;        /* MFA_GEOM_STORED (0, default) or MFA_GEOM_ONTHEFLY          */
  int32_t rule;            /* MFA_RULE_AUTO (0, default) or MFA_RULE_SYMMETRIC (simplices) */
} mfa_form_params;

typedef struct {
  int64_t ncell, ndof;
  int32_t nloc;            /* local nodes per cell                                      */
  int32_t nq;              /* quadrature points per cell used by the kernel              */
  int32_t ncolours;        /* colours of the deterministic scatter (0 if not built)     */
  int32_t scatter;         /* scatter actually used                                      */
  double flops;            /* algorithmic FP operations of one apply (hex: collocation sum
                              factorisation, 24 n^4 + pointwise physics per cell)       */
  double bytes;            /* algorithmic DRAM bytes of one apply                        */
  double setup_ms;         /* host+device time spent in mfa_form_create                  */
  double flops_executed;   /* FP operations the selected kernel executes: below `flops` for the
                              even-odd hex variant, which forms the 1D products from half-size
                              even and odd parts; equal to `flops` otherwise                */
} mfa_form_info;

typedef struct mfa_ctx mfa_ctx;
typedef struct mfa_mesh mfa_mesh;
typedef struct mfa_space mfa_space;
typedef struct mfa_form mfa_form;

/* Message of the calling thread's most recent failure ("" if none). */
MFA_API const char *mfa_last_error(void);
MFA_API int mfa_version(void);

/* Context bound to CUDA `device`; `stream` is a borrowed cudaStream_t (NULL =
 * the legacy default stream).  The stream must outlive the context. */
MFA_API int mfa_create(mfa_ctx **ctx, int device, void *stream);
MFA_API int mfa_set_stream(mfa_ctx *ctx, void *stream);
MFA_API int mfa_destroy(mfa_ctx *ctx);

/* Mesh: coords [nvert][3] (host, FP64), cell_vert [ncell][cell_type] (host,
 * int32).  Returns MFA_ERR_RANGE if a vertex index is outside [0, nvert).
 * Section 2.2: `coords(cell2vert, R)`. */
MFA_API int mfa_mesh_upload(mfa_ctx *ctx, int cell_type, int64_t ncell, int64_t nvert, const double *coords,
                    const int32_t *cell_vert, mfa_mesh **out);
MFA_API int mfa_mesh_destroy(mfa_mesh *mesh);

/* Continuous Lagrange space of `degree` (P1..P6 on tets and triangles, Q1..Q8 on
 * hexes and quads) with ncomp in {1, 3} (planar meshes: {1, 2}).  cell_node [ncell][nloc] (host, int32) is the cell->node
 * map of Section 2.2 (`cell2dof`); entries must lie in [0, nnode) and be
 * distinct within a cell.  cell_node = NULL: the library builds the map from
 * the mesh (mfa_build_cell_node; nnode is then ignored; read it back with
 * mfa_space_get_cell_node and the node count with mfa_space_ndof).  The mesh must outlive the space.  Local node order:
 * hex, the GLL tensor points with x fastest; P1/P2 tets, the vertices, then
 * the midpoints of edges (0,1), (0,2), (0,3), (1,2), (1,3), (2,3); P3..P6
 * tets, the equispaced lattice points (i, j, k)/p of the reference tet
 * (vertex 0 at the origin, vertex e+1 at the unit vector e), i fastest, then
 * j, then k; quads, the GLL tensor points with x fastest; triangles (every
 * degree), the lattice points (i, j)/p, i fastest. */
MFA_API int mfa_space_create(mfa_ctx *ctx, mfa_mesh *mesh, int degree, int ncomp, const int32_t *cell_node,
                     int64_t nnode, mfa_space **out);
/* The space's cell -> node map, copied to host memory [ncell][nloc]. */
MFA_API int mfa_space_get_cell_node(const mfa_space *space, int32_t *cell_node);

/* Cell -> node map of the continuous Q_p (hex and quad, p <= 8) or P_p (tet and triangle, p <= 6)
 * space from the vertex connectivity alone (host only, no device), in the
 * local node order of mfa_space_create.  A node on a vertex, edge or face is
 * the same global node in every cell that contains it, whatever the cells'
 * local vertex orders.  Nodes 0..nvert-1 are the mesh vertices; the others
 * follow in order of first appearance along the cells.  cell_node
 * [ncell][nloc] is caller-allocated; *nnode receives the node count.
 * mfa_space_create with cell_node = NULL calls this. */
MFA_API int mfa_build_cell_node(int cell_type, int degree, int64_t ncell, const int32_t *cell_vert, int64_t nvert,
                                int32_t *cell_node, int64_t *nnode);
/* The fully symmetric quadrature rule of degree `degree` (0..6) on the
 * reference triangle (cell_type MFA_CELL_TRI3; vertices (0,0), (1,0), (0,1)) or
 * tetrahedron (MFA_CELL_TET4; vertices 0, e1, e2, e3) that the forms use (host
 * only).  Table 2 gives the point counts: 1, 3, 6, 12 (triangle) and 1, 4, 14,
 * 24 (tetrahedron) for degree 0-1, 2, 3-4 / 3-5, 5-6 / 6.  Each rule is a union
 * of orbits of the barycentric permutations, with one weight per orbit, whose
 * weights and positions integrate every monomial of the rule's design degree
 * (triangle 1, 2, 4, 6; tet 1, 2, 5, 6) exactly; among the solutions with
 * positive weights and every point strictly inside, the one whose smallest
 * barycentric coordinate is largest.  Derived on first use (0.1-0.3 s for the
 * 24-point rule), then cached.  Outputs (caller-allocated, max_points entries):
 * pts [nq][2 or 3], w [nq] (summing to the reference area 1/2 or volume 1/6);
 * *nq receives the count.  MFA_ERR_ARG on a bad cell type, degree or a
 * max_points below the count; MFA_ERR_UNSUPPORTED if the derivation fails. */
MFA_API int mfa_simplex_rule(int cell_type, int degree, int max_points, double *pts, double *w, int *nq);
/* Physical positions of the nodes, out [nnode][3] (host only): the trilinear
 * (hex) or affine (tet) image of the reference nodes. */
MFA_API int mfa_node_coords(int cell_type, int degree, int64_t ncell, const int32_t *cell_vert, const double *coords,
                            const int32_t *cell_node, int64_t nnode, double *out);
MFA_API int mfa_space_ndof(const mfa_space *space, int64_t *ndof);
MFA_API int mfa_space_destroy(mfa_space *space);

/* Build a form on a space: quadrature tables, geometric factors (hex: stored
 * per quadrature point in FP64), and the cell colouring if the scatter is
 * coloured.  Synchronous.  The space must outlive the form. */
MFA_API int mfa_form_create(mfa_ctx *ctx, mfa_space *space, const mfa_form_params *params, mfa_form **out);
/* HYPER_JAC: linearisation point u (device, FP64, ndof entries, borrowed: it
 * must stay valid while the form is applied). */
MFA_API int mfa_form_set_coefficient(mfa_form *form, const double *u);
MFA_API int mfa_form_get_info(const mfa_form *form, mfa_form_info *info);
MFA_API int mfa_form_destroy(mfa_form *form);

/* Dirichlet constraints on `dofs` (host, n entries in [0, ndof); n = 0
 * removes them).  The form then acts as A_D x = R A R x + (I - R) x, R the
 * diagonal projection that zeroes the constrained dofs: the operator with
 * the constrained rows and columns replaced by the identity, symmetric
 * positive definite for elasticity with a clamped face (the rigid modes of
 * the unconstrained operator are gone).  mfa_apply, mfa_cg, mfa_cg_noalloc
 * and mfa_diagonal (1 at constrained dofs) follow it; a right-hand side for
 * zero prescribed values has zeros at the constrained dofs.  Allocates 17
 * bytes per dof on the device; synchronises the context stream.
 * mfa_apply_f32, mfa_fcg_mixed and mfa_fcg_learned return MFA_ERR_UNSUPPORTED
 * for constrained forms; set constraints before mfa_batch_create. */
MFA_API int mfa_form_set_dirichlet(mfa_form *form, const int32_t *dofs, int64_t n);

/* Launch configuration of a form and its autotuner.  The paper picks its
 * batch size (cells per SIMD vector) by the hardware's vector width
 * (Section 4.1); on the GPU the thread-to-data mapping, the number of cells a
 * thread block processes together and the scatter mode have no single best
 * value across degrees and forms, so they are chosen per form by timing.
 * Every configuration computes the same operator: the kernels differ only in
 * how the work is split, so results agree to rounding (bitwise for the same
 * variant and cells per block with the colour scatter).
 *  - variant: MFA_VARIANT_POINT  one thread per tensor point, a slab of n^3
 *                                threads per hex cell (FP64);
 *             MFA_VARIANT_EVEN_ODD one thread per 1D line with even-odd split
 *                                1D products (FP64 hex, n = p+1 = 5..9, p+1 points);
 *             MFA_VARIANT_LINE   one thread per 1D line, geometric factors read
 *                                from global memory (FP32/BF16 hex);
 *             MFA_VARIANT_LINE_STAGED as LINE with the factors staged in shared
 *                                memory by bulk copies (FP32/BF16 hex);
 *             MFA_VARIANT_CELL   one thread per cell (P1/P2 tets; P1..P4 triangles
 *                                whose rule has at most 25 points, but not the
 *                                P4 hyperelastic Jacobian action);
 *             MFA_VARIANT_CELL_WARP one warp per cell, dense tabulated basis (P3..P6 tets,
 *                                P1..P6 triangles).
 *  - cells_per_block: cells one thread block processes together (one thread
 *    per cell: threads per block); 0 in mfa_form_set_config = the variant's default.
 *  - scatter: MFA_SCATTER_ATOMIC, or (FP64 only) MFA_SCATTER_COLOUR or MFA_SCATTER_WARP.
 *  - geometry: stored factors or on-the-fly (the FP64 scalar point kernel; a
 *    form created with on-the-fly geometry has no stored factors to switch to).
 *  - max_blocks: 0 (default) sizes each persistent launch as one wave of
 *    resident blocks on every SM (fewer when there are fewer batches of
 *    cells); k > 0 caps the grid at k blocks, so that each block walks more
 *    batches.  The result does not depend on it (up to the rounding order of
 *    the atomic scatter).  It exists to exercise the multi-batch path of the
 *    persistent kernels on small meshes, and to leave SMs free for other work.
 *    mfa_form_list_configs lists 0; mfa_form_set_config keeps any k >= 0
 *    (MFA_ERR_ARG below 0); mfa_form_autotune times with 0 and leaves 0.
 *  - ms: mean time of one apply measured by mfa_form_autotune (else 0). */
enum {
  MFA_VARIANT_AUTO = 0,
  MFA_VARIANT_POINT = 1,
  MFA_VARIANT_EVEN_ODD = 2,
  MFA_VARIANT_LINE = 3,
  MFA_VARIANT_LINE_STAGED = 4,
  MFA_VARIANT_CELL = 5,
  MFA_VARIANT_CELL_WARP = 6
};
typedef struct {
  int32_t variant;
  int32_t cells_per_block;
  int32_t scatter;
  int32_t geometry;        /* MFA_GEOM_STORED or MFA_GEOM_ONTHEFLY (hex) */
  int32_t max_blocks;      /* grid cap, >= 0 (see above) */
  int32_t reserved;        /* 0 */
  double ms;
} mfa_launch_config;

/* All configurations the library has compiled for this form (the default
 * first).  Writes min(count, max) entries to `out` (may be NULL when max = 0)
 * and the full count to *count. */
MFA_API int mfa_form_list_configs(const mfa_form *form, mfa_launch_config *out, int max, int *count);
/* The configuration mfa_apply uses for this form. */
MFA_API int mfa_form_get_config(const mfa_form *form, mfa_launch_config *cfg);
/* Select a configuration; MFA_ERR_UNSUPPORTED if it is not one of
 * mfa_form_list_configs (MFA_VARIANT_AUTO selects the default).  Choosing the
 * colour scatter builds the space's colouring on first use (host work and a
 * device allocation). */
MFA_API int mfa_form_set_config(mfa_form *form, const mfa_launch_config *cfg);
/* Time every configuration of the form on the context stream (one untimed
 * apply, then `reps` >= 1 timed applies each, CUDA events) with y = A x on
 * the caller's device vectors x and y (y is overwritten), then select the
 * fastest.  `tried` receives min(count, max_tried) entries with their times,
 * in mfa_form_list_configs order (may be NULL when max_tried = 0); *ntried
 * the count.  Synchronises the context stream; do not call during stream
 * capture.  A configuration whose launch fails is reported with ms = -1 and
 * skipped; MFA_ERR_CUDA if all fail. */
MFA_API int mfa_form_autotune(mfa_ctx *ctx, mfa_form *form, const double *x, double *y, int reps,
                              mfa_launch_config *tried, int max_tried, int *ntried);

/* y = A(x) (accumulate = 0) or y += A(x) (accumulate = 1).  x, y: device,
 * ndof FP64 entries, must not overlap.  Asynchronous on the context stream.
 * Section 2.2 global assembly with the Section 2.1 local kernel. */
MFA_API int mfa_apply(mfa_ctx *ctx, mfa_form *form, const double *x, double *y, int accumulate);
/* The action of an FP32 or BF16 form on float vectors: x, y device, ndof
 * floats each.  Halves the vector traffic of mfa_apply and needs no
 * conversions; otherwise identical. */
MFA_API int mfa_apply_f32(mfa_ctx *ctx, mfa_form *form, const float *x, float *y, int accumulate);
/* Element-wise conversion of device vectors between FP64 and FP32, computed
 * on the integer pipe from the IEEE-754 bit fields: round to nearest, ties to
 * even; results below the smallest normal float become signed zero, above
 * the largest float infinity.  Asynchronous on the context stream. */
MFA_API int mfa_convert_f64_to_f32(mfa_ctx *ctx, const double *x, float *y, int64_t n);
MFA_API int mfa_convert_f32_to_f64(mfa_ctx *ctx, const float *x, double *y, int64_t n);
/* Same with host buffers: copies x to the device, applies, copies y back and
 * waits.  The device staging buffers are owned by the form. */
MFA_API int mfa_apply_host(mfa_ctx *ctx, mfa_form *form, const double *x_host, double *y_host);
/* y_host[i] = A_i x_host[i] for n forms, with the copies overlapped with the
 * applies: the copies in run ahead on one library-owned stream and the copies
 * out behind on another, so form i+1's x moves to the device and form i-1's y
 * to the host while form i computes (the applies stay in order on the context
 * stream).  Host buffers are best pinned (page-locked); they must stay valid
 * until the call returns, which is after everything finished.  Staging
 * buffers are owned by each form, as for mfa_apply_host, so a form may appear
 * only once per call (MFA_ERR_ARG otherwise). */
MFA_API int mfa_apply_host_many(mfa_ctx *ctx, int n, mfa_form *const *forms, const double *const *x_host,
                                double *const *y_host);
/* Wait for the context stream; MFA_ERR_DOMAIN if a kernel flagged det J <= 0
 * or a deformation with J <= 0, MFA_ERR_TIMEOUT if a kernel gave up a bounded
 * wait, since the last mfa_sync (the flag is cleared). */
MFA_API int mfa_sync(mfa_ctx *ctx);

/* d_i = A_ii (linear forms: mass, Laplace, Helmholtz, vector Laplace,
 * elasticity): the matrix-free diagonal, assembled per cell from the same
 * quadrature as mfa_apply, for every cell type and degree.  d: device, ndof
 * FP64.  MFA_ERR_UNSUPPORTED for the hyperelastic forms, FP32/BF16 forms and
 * forms without stored geometric factors (on-the-fly geometry). */
MFA_API int mfa_diagonal(mfa_ctx *ctx, mfa_form *form, double *d);

/* Conjugate gradients on a symmetric positive-definite linear form in FP64.
 * precond: MFA_PC_NONE or MFA_PC_JACOBI.  b, x: device (x is the initial guess
 * on entry and the solution on exit).  Stops when ||r||_2 <= rtol ||b||_2.
 * Returns MFA_ERR_NOT_CONVERGED at maxit, MFA_ERR_BREAKDOWN on p.Ap <= 0 or a
 * non-finite scalar.  iters and relres (nullable) receive the outcome. */
enum { MFA_PC_NONE = 0, MFA_PC_JACOBI = 1 };
MFA_API int mfa_cg(mfa_ctx *ctx, mfa_form *form, int precond, const double *b, double *x, double rtol, int maxit,
           int *iters, double *relres);

/* Mixed-precision flexible CG (spec solver; the paper has no solver).
 * Outer loop: flexible CG (Notay 2000, one stored direction) in FP64 with the
 * FP64 form `outer`, so convergence is decided on an FP64 residual
 * ||b - A x||_2 <= rtol ||b||_2.  Preconditioner: `inner_iters` steps of
 * Jacobi-PCG with the form `inner` (the same operator on the same space,
 * typically MFA_PREC_FP32), started from zero; inner_iters = 0 gives
 * Jacobi-preconditioned FCG.  The Jacobi diagonal comes from `outer`.
 * b, x: device FP64 (x: initial guess in, solution out).  Allocates its work
 * vectors (11 of ndof doubles) per call.  Returns MFA_ERR_NOT_CONVERGED at
 * maxit outer iterations, MFA_ERR_BREAKDOWN on p.Ap <= 0 or non-finite values. */
MFA_API int mfa_fcg_mixed(mfa_ctx *ctx, mfa_form *outer, mfa_form *inner, int inner_iters, const double *b,
                          double *x, double rtol, int maxit, int *outer_iters, int *inner_total, double *relres);

/* Learned element-wise preconditioner (spec component; the paper has
 * no solver).  For a residual r on a scalar Q1-Q4 hexahedral space,
 *   M(r) = D^{-1} r + sum_K R_K^T ( w_K * s_K * f(R_K r / s_K) ),
 *   f(z) = W2 relu(W1 z + b1),  s_K = ||R_K r||_2,
 * R_K gathers the cell's dofs, w_K = 1 / (cells sharing each node), D is the
 * diagonal of `form` (FP64).  W1 is 128 x nloc, b1 128, W2 nloc x 128; the
 * forward pass uses BF16 copies of W1 and W2 on the tensor cores with FP32
 * accumulation.  At creation W1 is seeded uniform in +-1/sqrt(nloc) from
 * SplitMix64(seed), b1 = W2 = 0, so the untrained M is Jacobi.
 * Vectors are device float arrays of ndof entries.
 *  - mfa_precond_apply: z = M(r).
 *  - mfa_precond_loss_grad: L = (M(r)-e)^T A (M(r)-e) / (e^T A e) with A the
 *    FP32/BF16 form `aform` on the same space, and (if grad_host != NULL) dL
 *    in the master layout of mfa_precond_get_weights, without updating.
 *  - mfa_precond_train: `steps` Adam steps (lr; beta 0.9/0.999) cycling over
 *    the (r, e) pairs; loss_first / loss_last receive the mean loss over the
 *    pairs before and after.
 *  - weights: FP32 master layout W1 [128][128] (columns >= nloc zero),
 *    b1 [128], W2 [128][128] (rows >= nloc zero): 32896 floats.
 *  - save/load: a 16-byte header ('MFAP', 1 for MLP / 2 for linear, nloc, 128)
 *    and the weights. */
typedef struct mfa_precond mfa_precond;
#define MFA_PRECOND_NPARAMS 32896
/* MFA_PRECOND_MLP: the network above (nonlinear; used by flexible CG).
 * MFA_PRECOND_LINEAR: no normalisation, bias or activation, W2 tied to W1^T:
 *   M(r) = D^{-1} r + sum_K R_K^T w_K W1^T W1 (w_K R_K r),
 * symmetric positive definite, so the inner loop is standard PCG; W1 starts
 * at +-0.01/sqrt(nloc) (b1 and W2 stay zero). */
enum { MFA_PRECOND_MLP = 0, MFA_PRECOND_LINEAR = 1 };
MFA_API int mfa_precond_create(mfa_ctx *ctx, mfa_form *form, int mode, uint64_t seed, mfa_precond **out);
MFA_API int mfa_precond_apply(mfa_ctx *ctx, mfa_precond *pc, const float *r, float *z);
MFA_API int mfa_precond_loss_grad(mfa_ctx *ctx, mfa_precond *pc, mfa_form *aform, const float *r, const float *e,
                                  double *loss, float *grad_host);
MFA_API int mfa_precond_train(mfa_ctx *ctx, mfa_precond *pc, mfa_form *aform, int npairs, const float *const *rs,
                              const float *const *es, int steps, double lr, double *loss_first, double *loss_last);
MFA_API int mfa_precond_get_weights(const mfa_precond *pc, float *host);
MFA_API int mfa_precond_set_weights(mfa_precond *pc, const float *host);
MFA_API int mfa_precond_save(const mfa_precond *pc, const char *path);
MFA_API int mfa_precond_load(mfa_precond *pc, const char *path);
MFA_API int mfa_precond_destroy(mfa_precond *pc);

/* Mixed-precision flexible CG whose inner loop is flexible CG (one stored
 * direction, float vectors, the FP32/BF16 form `inner`) preconditioned by the
 * learned M of `pc`; otherwise as mfa_fcg_mixed.  With fallback = 1 the
 * Jacobi inner loop of mfa_fcg_mixed takes over (a) for the rest of the solve
 * once the learned one stops reducing the FP64 residual (by less than 10%
 * over 30 outer steps): *used_fallback = 1; (b) from the initial guess if the
 * solve breaks down or reaches maxit: *used_fallback = 2.  With fallback = 0
 * the learned solver's own status is returned and *used_fallback = 0. */
MFA_API int mfa_fcg_learned(mfa_ctx *ctx, mfa_form *outer, mfa_form *inner, mfa_precond *pc, int inner_iters,
                            const double *b, double *x, double rtol, int maxit, int fallback, int *outer_iters,
                            int *inner_total, double *relres, int *used_fallback);

/* Many operators in one call (spec batching; the paper applies one
 * operator per parloop).  y_k = A_k(x_k) for k < n; each y_k is overwritten.
 * Hexahedral forms with the atomic scatter and p+1 points are grouped by
 * (degree, kind, precision) and each group runs as one persistent launch over
 * all its forms' cells; other forms get their own launch.  Synchronous: the
 * call returns when every y_k is complete.  x_k, y_k: device, FP64. */
MFA_API int mfa_apply_batched(mfa_ctx *ctx, int n, mfa_form *const *forms, const double *const *xs,
                              double *const *ys);

/* The same batch built once and recorded into a CUDA graph (zeroing of every
 * y_k, then the grouped and single launches).  mfa_batch_apply replays it
 * asynchronously on the context stream as one graph launch.  The forms and
 * vectors are borrowed and must outlive the batch; mfa_batch_create runs the
 * batch once eagerly and waits.  mfa_batch_info reports the number of grouped
 * launches and of single-form launches. */
typedef struct mfa_batch mfa_batch;
MFA_API int mfa_batch_create(mfa_ctx *ctx, int n, mfa_form *const *forms, const double *const *xs, double *const *ys,
                             mfa_batch **out);
MFA_API int mfa_batch_apply(mfa_ctx *ctx, mfa_batch *batch);
MFA_API int mfa_batch_info(const mfa_batch *batch, int *ngroups, int *nsingles);
MFA_API int mfa_batch_destroy(mfa_batch *batch);

/* Locality-restoring renumbering (host only, no device): reverse Cuthill-McKee
 * on the cell graph (cells adjacent when they share a vertex), then nodes
 * numbered by first touch along the new cell order.  Section 2.2's gather and
 * scatter go through the cell->node map; an arbitrary mesh order scatters
 * them over all of x and y, this brings consecutive cells' nodes together.
 * Inputs as for mfa_mesh_upload / mfa_space_create (nv = 4 or 8 vertices per
 * cell, nloc nodes per cell).  Outputs (caller-allocated): cell_order[ncell],
 * cell_order[new] = old cell; node_perm[nnode], node_perm[old] = new node.
 * Apply both to the maps (new cell_node[i] = node_perm[old cell_node[cell_order[i]]])
 * and to the node vectors before upload.  MFA_ERR_RANGE on an index outside
 * [0, nvert) or [0, nnode). */
MFA_API int mfa_order_rcm(int64_t ncell, int nv, const int32_t *cell_vert, int64_t nvert, int nloc,
                          const int32_t *cell_node, int64_t nnode, int32_t *cell_order, int32_t *node_perm);

/* Halo buffers of a cell-partitioned operator (Section 2.2's global assembly
 * with the cells split over ranks, one exchange per apply).  A rank applies
 * its cells over its local node numbering; a node that cells of several ranks
 * touch is owned by one rank and held as a ghost by the others.  Before the
 * apply, x at the ghosts is imported from the owners; after it, the ghosts'
 * partial sums are added into the owners' entries (the reverse exchange).
 * These calls move values between a node vector and the contiguous buffer a
 * rank sends or receives; the messages themselves are the caller's (NCCL).
 *  - ids: device int32 [n], local node ids in [0, nnode); v: device FP64
 *    [nnode][ncomp] (dof ncomp * node + c); buf: device FP64 [n][ncomp].
 *  - pack:   buf[k][c] = v[ids[k]][c].
 *  - unpack: v[ids[k]][c] = buf[k][c] (accumulate = 0) or += (accumulate = 1);
 *    ids must be distinct within one call.
 *  - Asynchronous on the context stream.  An id outside [0, nnode) is skipped
 *    (pack writes 0) and mfa_sync reports MFA_ERR_RANGE.
 * Not in the paper as a call: its runs are MPI-parallel with PyOP2's halo
 * exchange; this is the device side of that exchange. */
MFA_API int mfa_halo_pack(mfa_ctx *ctx, const int32_t *ids, int64_t n, int ncomp, int64_t nnode, const double *v,
                          double *buf);
MFA_API int mfa_halo_unpack(mfa_ctx *ctx, const int32_t *ids, int64_t n, int ncomp, int64_t nnode,
                            const double *buf, double *v, int accumulate);

/* FP64 FMA throughput of this GPU, measured: one wave of blocks on every SM,
 * each thread running 8 independent FMA chains for 2^15 steps, timed with
 * CUDA events (after one shorter warm-up launch).  *tflops = 2 flops per FMA
 * / elapsed time; *sm_mhz (may be NULL) = the median over blocks of SM clock
 * ticks per nanosecond of the global timer during the timed launch.  The
 * FP64 operator kernels are bound by this rate (their arithmetic intensity is
 * far above the FP64 ridge point), so it is the measured denominator of their
 * roofline.  Synchronous; allocates a few KB.  Not in the paper (the paper
 * quotes its CPUs' peak from clock and vector width, Table 1). */
MFA_API int mfa_probe_fp64_fma(mfa_ctx *ctx, double *tflops, double *sm_mhz);

/* mfa_cg without device allocation.  The paper has no counterpart: this is
 * for callers that cannot call cudaMalloc (an application whose memory pool
 * already holds the device memory, a solver step inside another framework's
 * stream pipeline where the implicit synchronisation of cudaMalloc/cudaFree
 * would stall other work, a loop that forbids allocation after start-up).
 * Same arguments, algorithm, kernels and status codes as mfa_cg.  The work
 * vectors live in one file-scope __device__ array of
 * 5 * MFA_CG_NOALLOC_MAX_NDOF + 1056 doubles (about 10 MiB), which every GPU
 * that loads the library holds until the process exits.
 *  - ndof above MFA_CG_NOALLOC_MAX_NDOF returns MFA_ERR_ARG, before any work.
 *  - The first call on a device looks up the array's device address (once per
 *    device, with that device current); make that first call before any
 *    stream capture.  Later calls made while the context stream is not
 *    capturing look it up again, so a reset of the device (after which every
 *    other handle must be created anew) leaves no stale address behind.
 *  - Errors: those of mfa_cg; a failure inside mfa_apply, mfa_diagonal or
 *    mfa_sync keeps that call's message in mfa_last_error().
 *  - All calls on a device share the array: calls that overlap on the GPU
 *    (other streams, other host threads) race.  Each call writes every part
 *    of the array it reads before reading it. */
#define MFA_CG_NOALLOC_MAX_NDOF 262144
MFA_API int mfa_cg_noalloc(mfa_ctx *ctx, mfa_form *form, int precond, const double *b, double *x, double rtol,
                           int maxit, int *iters, double *relres);

#ifdef __cplusplus
}
#endif
#endif /* MFA_H */
