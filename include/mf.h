/*
 * mf.h - C ABI of the GB300 (sm_103a) matrix-free Q1 finite-element library.
 *
 * The library applies the low-order finite-element operators of the paper "Performant low-order
 * matrix-free finite element kernels on GPU architectures" (Settgast et al.): the scalar Laplace
 * and isotropic linear-elasticity operators on trilinear hexahedra (Q1) with 2x2x2 Gauss
 * quadrature (Sec. 2, Eqs. 1, 3, 4, 6), matrix-free (Sec. 3, Eqs. 7 and 9, Algorithm 1) or through
 * an assembled CSR matrix (Sec. 3 and Table 1), and solves A x = b by conjugate gradient (the
 * operations of Table 4).  The same operators on linear tetrahedra (P1) and triquadratic
 * hexahedra (Q2), the elements Sec. 7 names as future work, are set up by mf_setup_mesh_elem.
 *
 * Conventions shared by every call:
 *   - All array arguments are DEVICE pointers on the current CUDA device, owned by the caller,
 *     unless marked "host".  The library never frees caller memory.
 *   - Node (i, j, k) of an nx x ny x nz box has id i + (nx+1)(j + (ny+1)k); element (ex, ey, ez)
 *     has id ex + nx(ey + ny ez).  Corner a = 0..7 of an element sits at reference coordinates
 *     (+-1, +-1, +-1) with bit 0 of a -> xi, bit 1 -> eta, bit 2 -> zeta (0 -> -1, 1 -> +1).
 *   - Vector problems interleave components: DoF 3*node + k (the 3(i-1)+k index of Eqs. 2-3).
 *   - Dirichlet DoFs: their columns are dropped and their rows are the identity, so
 *     (A x)_d = x_d for every constrained DoF d.
 *   - Calls taking a stream are asynchronous on it unless stated; NULL is the legacy default
 *     stream.  No call aborts or exits: every call returns an mf_status and, on failure, leaves a
 *     message for mf_last_error() in the calling thread.
 */
#ifndef MF_H_
#define MF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *mf_stream; /* identical to cudaStream_t */

typedef enum {
  MF_OK = 0,
  MF_NOT_CONVERGED = 1,    /* solver stopped at max_iter above the tolerance (x is still valid) */
  MF_ERR_ARG = -1,         /* invalid argument (null pointer, size, aliasing, bad option) */
  MF_ERR_CUDA = -2,        /* a CUDA runtime call failed (message names it) */
  MF_ERR_MESH = -3,        /* invalid mesh: det J <= 0, node id out of range, NaN, bad material */
  MF_ERR_OOM = -4,         /* device allocation failed */
  MF_ERR_BREAKDOWN = -5,   /* CG breakdown: p^T A p <= 0 or a NaN/Inf scalar */
  MF_ERR_TIMEOUT = -6,     /* wall-clock budget of a solve exhausted */
  MF_ERR_UNSUPPORTED = -7  /* operation not available for this mesh or physics */
} mf_status;

enum { MF_LAPLACE = 0, MF_ELASTICITY = 1, MF_VECTOR_LAPLACE = 2 };

typedef struct mf_mesh mf_mesh;
typedef struct mf_csr mf_csr;

/*
 * mf_setup_mesh - validate a Q1 hexahedral mesh and build the operator's device data.
 *
 * The inputs of Algorithm 1 (support-point coordinates) plus the cell constants of Table 2.
 *   physics    MF_LAPLACE (1 DoF per node), MF_ELASTICITY (3 DoFs per node) or MF_VECTOR_LAPLACE
 *              (3 DoFs per node: the vector Laplacian of Eqs. 2 and 5, the scalar operator acting
 *              on each component).
 *   n_nodes    N >= 8; n_cells E >= 1.  Indices are 32-bit: 3 N and 8 E (npe E for the element
 *              types of mf_setup_mesh_elem) must not exceed 2^31 - 1, about 715 M nodes and 268 M
 *              hexahedra (a 640^3 box); larger meshes are refused with MF_ERR_ARG.
 *   coords     device double[N][3], node coordinates.
 *   cells      device int32[E][8] element -> node map in the corner order above, or NULL for a
 *              structured nx x ny x nz box numbered as above (then E must equal nx*ny*nz and N
 *              must equal (nx+1)(ny+1)(nz+1); coordinates may still be arbitrary).
 *   mat        device double[E] (Laplace and vector Laplace: coefficient kappa_e > 0) or
 *              double[E][2] (elasticity: Young's modulus E_e > 0 and Poisson ratio
 *              -1 < nu_e < 0.5).
 *   dirichlet  device uint8[N] (nonzero = all DoFs of that node constrained) or NULL (none).
 * The library copies what it needs into its own layout; the caller's arrays may be freed after the
 * call returns.  Synchronises `stream`.  Errors: MF_ERR_ARG, MF_ERR_MESH (det J <= 0 at a Gauss
 * point or corner, node id out of range, non-finite coordinate or material), MF_ERR_OOM,
 * MF_ERR_CUDA.  *out is NULL on failure.
 */
mf_status mf_setup_mesh(int physics, int64_t n_nodes, int64_t n_cells, const double *coords,
                        const int32_t *cells, int32_t nx, int32_t ny, int32_t nz, const double *mat,
                        const uint8_t *dirichlet, mf_stream stream, mf_mesh **out);

/*
 * mf_setup_mesh_elem - mf_setup_mesh for an explicit connectivity of a given element type.
 *   element  MF_ELEM_HEX8: the Q1 hexahedron above (cells int32[E][8]; same as mf_setup_mesh with
 *            cells != NULL);
 *            MF_ELEM_TET4: the linear tetrahedron (P1), one of the simplex elements that Sec. 7
 *            lists as future work.  cells int32[E][4]; vertex 0 is phi_0 = 1 - xi - eta - zeta and
 *            vertices 1..3 follow xi, eta, zeta of the reference tetrahedron; the vertices must be
 *            positively oriented, det[x1 - x0, x2 - x0, x3 - x0] > 0.  The element integrals of
 *            Eqs. 1-3 have constant integrands and are evaluated exactly (one point, weight 1/6).
 *            MF_ELEM_HEX27: the triquadratic hexahedron (Q2), the higher-order element of Sec. 7.
 *            cells int32[E][27]; node a = i + 3j + 9k (i, j, k in {0, 1, 2}) at reference
 *            coordinates (i - 1, j - 1, k - 1); 3x3x3 Gauss quadrature; det J must be positive at
 *            the 27 Gauss points and the 8 vertices.
 *   Other arguments as mf_setup_mesh (cells is required).
 * Tetrahedral meshes run the reference kernel (one thread per element, colour-by-colour scatter,
 * FP64 or FP32) for every apply, the multi-RHS apply, CSR assembly, the operator diagonal and CG.
 * Q2 meshes do too for FP32 applies, the diagonal and CSR assembly; their FP64 applies (and CG) use a
 * partial assembly with sum factorisation when its data take at most a quarter of the device's total
 * memory (mf_mesh_query flag bit 3; MF_VARIANT_PARTIAL builds it on request, MF_VARIANT_REFERENCE
 * selects the reference kernel), one warp per element in double-word arithmetic with exact
 * power-of-two scalings (FP64 arithmetic if the Gauss-point data span more than 2^60).
 * MF_VARIANT_GENERAL, the batched solver and the learned preconditioner return
 * MF_ERR_UNSUPPORTED or MF_ERR_ARG for them.  Errors as mf_setup_mesh (MF_ERR_MESH for an element
 * with det <= 0).
 */
enum { MF_ELEM_HEX8 = 0, MF_ELEM_TET4 = 1, MF_ELEM_HEX27 = 2 };
mf_status mf_setup_mesh_elem(int element, int physics, int64_t n_nodes, int64_t n_cells, const double *coords,
                             const int32_t *cells, const double *mat, const uint8_t *dirichlet, mf_stream stream,
                             mf_mesh **out);

/* Frees every device buffer the handle owns (synchronises the device first).  NULL is a no-op. */
mf_status mf_destroy_mesh(mf_mesh *mesh);

/* Host outputs (any may be NULL): node, cell and DoF counts, free (unconstrained) DoFs, number of
 * element colours of the scatter, and flags (bit 0: structured, bit 1: every cell affine, bit 2:
 * tensor-product grid of axis-aligned cells, which enables the FP64-accurate tile kernels, bit 3:
 * partial-assembly data built, bit 4: tetrahedral mesh, bit 5: Q2 mesh, bit 6: structured mesh whose
 * cell constants or cell sizes span more than the double-word kernels cover, so that every apply
 * runs the FP64 reference kernel; bit 7: double-word data built from cell constants or coordinates
 * normalised by a power of two, which the kernels undo exactly on their results; see "Range"
 * below). */
mf_status mf_mesh_query(const mf_mesh *mesh, int64_t *n_nodes, int64_t *n_cells, int64_t *n_dof,
                        int64_t *n_free, int32_t *n_colours, int32_t *flags);

/*
 * Kernel variants for the operator apply (mf_set_apply_variant):
 *   MF_VARIANT_AUTO       fastest variant that meets FP64 accuracy for this mesh (default): on a
 *                         structured tensor-product grid the face-marching kernel (Walsh-Hadamard
 *                         form of the 2x2x2 Gauss sums, double-word FP32 arithmetic); on another
 *                         structured box the partial-assembly kernel when its data take at most
 *                         a quarter of the device's total memory (flag bit 3 of mf_mesh_query;
 *                         the choice depends on the mesh and the device model only), else the
 *                         general kernel; otherwise the reference kernel.  Results are bitwise
 *                         reproducible for a given variant
 *   MF_VARIANT_REFERENCE  Algorithm 1 as printed: one thread per element, FP64 arithmetic,
 *                         Jacobian at every quadrature point, colour-by-colour scatter
 *   MF_VARIANT_GENERAL    structured boxes that are not tensor-product grids: Jacobian, adjugate
 *                         and determinant at every quadrature point in double-word arithmetic
 *                         (MF_ERR_UNSUPPORTED on other meshes)
 *   MF_VARIANT_PARTIAL    the same meshes: partial assembly (Table 3), the quadrature-point data
 *                         computed once in FP64 and stored as float pairs (6 values per point for
 *                         Laplace, 10 for elasticity); built on first selection (MF_ERR_OOM if it
 *                         does not fit; synchronises the device)
 */
/*
 * Range of the double-word kernels (face-marching, general and partial-assembly; FP64 applies and
 * the FP64 CG on them).  Their arithmetic is pairs of floats: 48 significand bits, and FP32's
 * exponent range.  The library keeps FP64 accuracy (<= 1e-12 relative in the 2-norm against an FP64
 * evaluation) for every finite input as follows; all scalings are by powers of two, hence exact:
 *   - cell constants: when max |kappa| (or max(|lam|, mu)) is outside [2^-8, 2^9), the double-word
 *     data are built from constants scaled into that window; coordinates likewise when the largest
 *     det J at a Gauss point (~(h/2)^3) is outside [2^-40, 2^25); y is scaled back in the kernel;
 *   - x: every CTA records the largest |x| it reads; if that lies outside [2^-72, 2^41) the CTA
 *     computes its tile again with its inputs scaled into [1, 2) and y scaled back (the tile's
 *     inputs below 2^-74 of its largest one are then treated as zero).  The result does not depend
 *     on the scaling decision beyond rounding, and 2^k x gives exactly 2^k y.  Such applies take
 *     about twice the time of in-range ones;
 *   - meshes whose cell constants span a ratio above 2^80, or whose det J spans a ratio above 2^60
 *     (cell sizes over 2^20), do not build double-word data at all (mf_mesh_query flag bit 6): the
 *     auto variant runs the FP64 reference kernel and MF_VARIANT_GENERAL / MF_VARIANT_PARTIAL return
 *     MF_ERR_UNSUPPORTED.
 * The FP32 applies (mf_apply_f32, the inner solves of MF_PREC_MIXED_IR) have FP32's range.
 */
enum { MF_VARIANT_AUTO = 0, MF_VARIANT_REFERENCE = 1, MF_VARIANT_GENERAL = 2, MF_VARIANT_PARTIAL = 3 };
mf_status mf_set_apply_variant(mf_mesh *mesh, int variant);

/*
 * mf_apply_laplace - y = A x for the scalar Laplace operator, matrix-free (Eqs. 4 and 7 with the
 * per-cell factor kappa_e; Algorithm 1 with sigma replaced by the flux).
 *   x  device double[N], input; entries on Dirichlet nodes are ignored except that y_d = x_d.
 *   y  device double[N], output, overwritten.  Must not overlap x.
 * Asynchronous on `stream`, allocates nothing, deterministic (bitwise-reproducible: the scatter
 * uses no atomics).  FP64-accurate for every finite x (see "Range" above).  Errors: MF_ERR_ARG
 * (null, aliasing, mesh is not Laplace), MF_ERR_CUDA.
 */
mf_status mf_apply_laplace(const mf_mesh *mesh, const double *x, double *y, mf_stream stream);

/*
 * mf_apply_elasticity - y = A x for isotropic linear elasticity (Eqs. 6 and 9, Algorithm 1):
 * sigma = lam tr(eps) I + 2 mu eps, eps = sym grad u, (lam, mu) from each cell's (E, nu).
 *   x, y  device double[3N], xyz interleaved.  Same contract as mf_apply_laplace.
 */
mf_status mf_apply_elasticity(const mf_mesh *mesh, const double *x, double *y, mf_stream stream);

/*
 * mf_apply_vector_laplace - y = A x for the vector Laplace operator (Eq. 5: the element matrix is
 * the scalar one of Eq. 4, with the per-cell factor kappa_e, acting on each of the three components;
 * the vector form of Eq. 7).
 *   x, y  device double[3N], xyz interleaved.  Same contract as mf_apply_laplace; MF_ERR_ARG if
 *         the mesh was set up for another physics.
 */
mf_status mf_apply_vector_laplace(const mf_mesh *mesh, const double *x, double *y, mf_stream stream);

/*
 * mf_apply_f32 - the same operator (any physics) evaluated entirely in FP32: geometry from FP32
 * copies of the coordinates and cell constants, FP32 x and y.  Used by the mixed-precision solver.
 *   x, y  device float[N * ndof_per_node].  Same contract otherwise.
 */
mf_status mf_apply_f32(const mf_mesh *mesh, const float *x, float *y, mf_stream stream);

/*
 * mf_apply_multi - Y = A X for nrhs right-hand sides at once.  On tensor-product meshes one launch
 * of the face-marching kernel covers all right-hand sides (each column bitwise equal to the single
 * apply; the element coefficients are cheap there and are recomputed per right-hand side); on other
 * meshes the reference kernel evaluates the geometry (J, adj J, det J at every Gauss point) once per
 * element and reuses it for every right-hand side.
 *   X, Y  device double[N][nrhs][ndof_per_node] (node-major, then right-hand side, then
 *         component).  1 <= nrhs <= 16.  Same contract as the single apply.
 */
mf_status mf_apply_multi(const mf_mesh *mesh, int32_t nrhs, const double *X, double *Y, mf_stream stream);

/*
 * mf_assemble_csr - assemble the global matrix (Sec. 3, matrix-based operator): the element
 * matrices of Eqs. 4/6 are summed into a CSR matrix whose rows follow the DoF numbering; the fill
 * adds each element's rows without atomics (elements of one colour share no node).
 *   Rows of Dirichlet DoFs hold the single entry 1 on the diagonal; their columns are removed from
 *   the other rows.  Columns are sorted within each row.  Index types: int64 row pointers, int32
 *   column indices, double values (12 bytes per non-zero as in Table 1).
 * Synchronises `stream`.  Errors: MF_ERR_OOM, MF_ERR_CUDA, MF_ERR_ARG.
 */
mf_status mf_assemble_csr(const mf_mesh *mesh, mf_stream stream, mf_csr **out);

/* Host outputs (any may be NULL): rows, non-zeros and the DEVICE arrays (owned by the handle). */
mf_status mf_csr_query(const mf_csr *csr, int64_t *n_rows, int64_t *nnz, const int64_t **rowptr,
                       const int32_t **col, const double **val);

/* Copy the matrix into caller-owned device arrays: rowptr int64[n_rows+1], col int32[nnz],
 * val double[nnz].  Asynchronous on `stream`.  Errors: MF_ERR_ARG, MF_ERR_CUDA. */
mf_status mf_csr_export(const mf_csr *csr, int64_t *rowptr, int32_t *col, double *val, mf_stream stream);

/* y = A x with the assembled matrix.  x, y device double[n_rows], must not overlap.  Asynchronous,
 * allocates nothing, deterministic. */
mf_status mf_spmv_csr(const mf_csr *csr, const double *x, double *y, mf_stream stream);

/* Frees the matrix's device arrays (synchronises the device first).  NULL is a no-op.  CG graphs
 * captured for this matrix are never replayed for another one (they are keyed by a process-unique
 * matrix id). */
mf_status mf_destroy_csr(mf_csr *csr);

/* Solver options (mf_cg_solve). */
enum { MF_OP_MATFREE = 0, MF_OP_CSR = 1 };
enum { MF_PREC_FP64 = 0, MF_PREC_MIXED_IR = 1 };
enum { MF_PC_NONE = 0, MF_PC_JACOBI = 1, MF_PC_LEARNED = 2 };
/* CG recurrence (FP64 solves with MF_PC_NONE or MF_PC_JACOBI):
 *   MF_CG_CLASSIC    Hestenes-Stiefel as in Table 4.  On scalar Laplace tensor-product meshes with the
 *                    auto variant (without normalisation: mf_mesh_query flag bit 7 clear) the vector
 *                    updates are fused into the apply: its kernel forms p_k = z_k + beta p_{k-1} at
 *                    the nodes it stages, stores p_k and the deferred x += alpha p_{k-1} at the nodes
 *                    it owns, and returns A p_k with p_k^T A p_k; one vector kernel then updates r and
 *                    forms r^T z.  Elsewhere: the apply (p^T A p fused on tensor-product meshes), the
 *                    x/r update with r^T z, and the p update.
 *   MF_CG_PIPELINED  single-synchronisation recurrence of Chronopoulos and Gear (1989): w = A u
 *                    (u = M^-1 r) with u^T w fused into the apply, then one pass that updates p, s = A p,
 *                    x, r and u and forms r^T u; the same iterates in exact arithmetic.
 *   MF_CG_CLASSIC_SPLIT  the classic recurrence with the separate vector kernels everywhere.  Its
 *                    iterates, iteration count and solution are bitwise those of MF_CG_CLASSIC (the
 *                    fused kernels evaluate the same FP64 formulas on the same values).
 * PIPELINED and CLASSIC_SPLIT are not available for MIXED_IR, the learned preconditioner,
 * mf_cg_solve_noalloc or the batched solver (MF_ERR_ARG). */
enum { MF_CG_CLASSIC = 0, MF_CG_PIPELINED = 1, MF_CG_CLASSIC_SPLIT = 2 };
typedef struct mf_net mf_net;

typedef struct {
  int32_t op;            /* MF_OP_MATFREE or MF_OP_CSR (then `csr` must be set) */
  int32_t precision;     /* MF_PREC_FP64, or MF_PREC_MIXED_IR: FP32 inner CG, FP64 refinement */
  int32_t precond;       /* MF_PC_NONE, MF_PC_JACOBI (FP64 only) or MF_PC_LEARNED (flexible CG with
                            the network in `net`; FP64, matrix-free, structured Laplace meshes whose
                            node grid matches the network's; a stall or breakdown switches the
                            network off and the solve continues as Jacobi-PCG from the current
                            iterate; info->outer_iters reports the iteration of that switch, -1 if
                            never) */
  int32_t max_iter;      /* > 0; for MIXED_IR the total inner iterations */
  double rtol;           /* stop when ||r||_2 <= rtol ||b||_2 (FP64 residual for MIXED_IR) */
  int32_t check_every;   /* iterations per CUDA-graph launch between host convergence checks */
  int32_t use_graph;     /* 1: capture check_every iterations in a CUDA graph; 0: plain launches */
  double timeout_s;      /* wall-clock budget, <= 0 for none */
  double inner_rtol;     /* MIXED_IR: relative tolerance of each inner FP32 solve (e.g. 1e-4) */
  int32_t max_outer;     /* MIXED_IR: refinement steps */
  const mf_csr *csr;     /* operator when op == MF_OP_CSR */
  const mf_net *net;     /* network when precond == MF_PC_LEARNED (flexible CG, see mf_net_create) */
  int32_t recurrence;    /* MF_CG_CLASSIC (default), MF_CG_PIPELINED or MF_CG_CLASSIC_SPLIT */
} mf_solve_opts;

typedef struct {
  int32_t iters;          /* operator applies inside the Krylov loop(s) */
  int32_t outer_iters;    /* refinement steps (MIXED_IR); the switch-off iteration (LEARNED); else 0 */
  int32_t status;         /* same value as the return code */
  int32_t reserved;
  double rel_res;         /* ||r_k|| / ||b|| from the recurrence (inner FP64 residual for IR) */
  double rel_res_true;    /* ||b - A x|| / ||b|| recomputed with the FP64 operator after the solve */
  double seconds;         /* wall time of the call */
} mf_solve_info;

/* diag(A) of the FP64 operator (Eqs. 4/6; Dirichlet rows 1): device double[n_dof], asynchronous.
 * This is the Jacobi preconditioner's diagonal. */
mf_status mf_operator_diagonal(const mf_mesh *mesh, double *diag, mf_stream stream);

/* Fills *opts with defaults: matrix-free, FP64, no preconditioner, rtol 1e-8, max_iter 100000,
 * check_every 32, graphs on, no timeout, inner_rtol 1e-4, max_outer 50, classic recurrence. */
void mf_solve_opts_default(mf_solve_opts *opts);

/*
 * mf_cg_solve - solve A x = b by conjugate gradient (Table 4: per iteration one apply, the dots
 * p^T A p and r^T r, and the updates of x, r, p), starting from x0 = 0.
 *   b     device double[n_dof], right-hand side (Dirichlet entries are the prescribed values,
 *         normally 0).
 *   x     device double[n_dof], output solution (its input content is ignored).
 *   info  host, may be NULL.
 * The scalars alpha, beta and the residual norm stay on the device; the dots use a deterministic
 * two-level reduction fused into the update kernels; `check_every` iterations run per CUDA-graph
 * launch and the host reads a convergence flag between launches.  Synchronises `stream` before
 * returning.  Workspace (a few DoF vectors) is allocated on the first call per mesh and kept by the
 * handle.  Returns MF_OK, MF_NOT_CONVERGED, MF_ERR_BREAKDOWN, MF_ERR_TIMEOUT, MF_ERR_ARG,
 * MF_ERR_OOM or MF_ERR_CUDA.
 */
mf_status mf_cg_solve(mf_mesh *mesh, const mf_solve_opts *opts, const double *b, double *x,
                      mf_solve_info *info, mf_stream stream);

/*
 * CG checkpoint and resume.  The paper has no counterpart; this lets a long solve stop (iteration
 * limit, wall-clock budget, the process's own schedule) and continue later, in another process or
 * after the device was handed to other work.
 *
 * mf_cg_state_save copies the state of the last mf_cg_solve (or mf_cg_resume) on this mesh to host
 * memory: the iteration count k, the scalars of the recurrence (r.z, ||r||^2, ||b||^2, the
 * tolerance, beta) and the vectors x_k, r_k and the last search direction.  Only a solve that
 * stopped with MF_NOT_CONVERGED or MF_ERR_TIMEOUT in FP64 with MF_PC_NONE or MF_PC_JACOBI and the
 * classic recurrence (fused or MF_CG_CLASSIC_SPLIT) leaves a state; otherwise MF_ERR_ARG.  The call
 * synchronises the stream.
 *   host_state: mf_cg_state_bytes(mesh) bytes of host memory (caller-owned); bytes: its size.
 *
 * mf_cg_resume continues that solve: opts must name the same operator, preconditioner and
 * recurrence, and b must be the same right-hand side; opts->max_iter and rtol apply to the whole
 * solve (iterations count from the original start).  Then iterations, residual records and the
 * solution are bitwise those of a solve that was never interrupted (a state saved on one GPU resumes
 * on another of the same kind).  The state's vector length must equal the mesh's n_dof.
 *   Arguments and returns as for mf_cg_solve; MF_ERR_ARG for a state of another mesh size,
 *   preconditioner or recurrence, or a corrupt header.
 */
size_t mf_cg_state_bytes(const mf_mesh *mesh);
mf_status mf_cg_state_save(mf_mesh *mesh, void *host_state, size_t bytes, mf_stream stream);
mf_status mf_cg_resume(mf_mesh *mesh, const mf_solve_opts *opts, const void *host_state, size_t bytes, const double *b,
                       double *x, mf_solve_info *info, mf_stream stream);

/*
 * mf_cg_solve_noalloc - the unpreconditioned FP64 CG of mf_cg_solve for callers that cannot
 * allocate device memory while they run: for example an application that hands the whole device
 * to its own memory pool at start-up, or one whose memory budget is enforced outside CUDA, where a
 * cudaMalloc inside a solve would fail or is not allowed.  The paper has no counterpart to this
 * call; it is a deployment convenience.
 *
 * It calls no cudaMalloc, cudaFree or other allocating routine.  Its scratch (three DoF vectors,
 * the reduction partials and the device scalars) is a fixed array with static storage inside the
 * library, sized for MF_NOALLOC_MAX_DOF degrees of freedom (about 6 MB); every GPU that loads the
 * library holds that array until the process exits.  Larger problems are rejected with
 * MF_ERR_ARG.  The first call on each device looks up the array's device address (with that device
 * current); make that first call before any stream capture.
 *
 * All calls share the one array and it keeps the previous call's contents (each call clears what
 * must start at zero itself).  Calls whose work overlaps on the GPU - on two streams, or from two
 * host threads - race on the array: serialise them.
 *   mesh, b, x, info, stream: as for mf_cg_solve; x is used as the iterate and holds the solution.
 *   opts: op MF_OP_MATFREE or MF_OP_CSR (with opts->csr), precision MF_PREC_FP64, precond
 *   MF_PC_NONE; rtol, max_iter, check_every and timeout_s as for mf_cg_solve; use_graph is ignored.
 * Returns MF_OK, MF_NOT_CONVERGED, MF_ERR_BREAKDOWN, MF_ERR_TIMEOUT, MF_ERR_ARG or MF_ERR_CUDA.
 */
#define MF_NOALLOC_MAX_DOF 262144
mf_status mf_cg_solve_noalloc(const mf_mesh *mesh, const mf_solve_opts *opts, const double *b, double *x,
                              mf_solve_info *info, mf_stream stream);

/*
 * Batched solves (no counterpart in the paper, which solves one problem at a time): n independent
 * problems A_i x_i = b_i, one mesh each, solved by unpreconditioned FP64 CG in ONE persistent
 * cooperative kernel launch captured in a CUDA graph.  Every CTA of a co-resident grid loops over
 * the CG phases (tile apply, p.Ap, x/r update with r.r, p update) of all still-active problems,
 * separated by grid barriers whose waits are bounded (MF_ERR_TIMEOUT instead of a hang).  Each
 * problem has its own scalars and stops at its own tolerance.  Meshes must be Laplace on
 * tensor-product grids (MF_ERR_UNSUPPORTED otherwise); opts: MATFREE, FP64, no preconditioner;
 * rtol and max_iter apply per problem; timeout_s, when > 0, bounds each barrier wait instead of
 * the whole solve.
 *   mf_batch_create   allocates the batch workspace and captures the graph (synchronous).
 *   mf_batch_solve    b, x: HOST arrays of n DEVICE pointers (double[n_dof_i]); infos: host
 *                     array of n (rel_res_true is not recomputed: -1).  Synchronises `stream`.
 *   mf_batch_destroy  frees the workspace and the graph (synchronises the device); NULL is a no-op.
 *   mf_cg_solve_batched  create + solve + destroy in one call.
 */
typedef struct mf_batch mf_batch;
mf_status mf_batch_create(mf_mesh *const *meshes, int32_t n, const mf_solve_opts *opts, mf_batch **out);
mf_status mf_batch_solve(mf_batch *batch, const double *const *b, double *const *x, mf_solve_info *infos,
                         mf_stream stream);
mf_status mf_batch_destroy(mf_batch *batch);
mf_status mf_cg_solve_batched(mf_mesh *const *meshes, int32_t n, const mf_solve_opts *opts,
                              const double *const *b, double *const *x, mf_solve_info *infos, mf_stream stream);

/* z-segment length (node planes per tile work item) of the tile kernels for this mesh; 0 restores
 * the built-in choice.  Used by the autotuner of the batched solver; results do not depend on it. */
mf_status mf_set_tile_segment(mf_mesh *mesh, int32_t seg);

/*
 * Learned preconditioner (no counterpart in the paper, whose conclusions name matrix-free
 * preconditioners as future work).  A 3-level convolutional encoder-decoder on the node grid
 * (channels 16/32/64, 3x3x3 kernels, full-weighting restriction and trilinear prolongation between
 * (4m+1)^3, (2m+1)^3 and (m+1)^3 node grids, skip connections), BF16 weights and activations with
 * FP32 accumulation on the tensor cores, FP32 master weights and Adam.  Inputs: the residual
 * scaled by the diagonal and its RMS, and the node average of log kappa; output: the (scaled)
 * error.  In flexible CG it is the smooth-error correction of a two-level preconditioner between
 * damped-Jacobi smoothing steps: z1 = w D^-1 r; r1 = r - A z1; cn = D^-1/2 (s/c) NN(D^-1/2 r1 / s,
 * log kappa) with s = RMS(D^-1/2 r1); z2 = z1 + theta cn with the energy-norm step
 * theta = max(0, cn.r1 / cn.A cn); z = z2 + w D^-1 (r - A z2); w = 2/3, c the output scale.
 *   mf_net_create       node grid nx x ny x nz (each 4m+1 >= 5), seeded He initialisation.
 *   mf_net_destroy      frees the network (synchronises the device); NULL is a no-op.
 *   mf_net_set_output_scale  the factor c applied to the network's output (c > 0, else MF_ERR_ARG;
 *                       1 after mf_net_create); mf_cg_solve reads it once, when a solve starts.
 *   mf_net_forward      r, logk, out: device float[nx ny nz] (x fastest).  Asynchronous.
 *   mf_net_train_step   one Adam step on the relative squared error |out - target|^2 / |target|^2
 *                       (gradient norm clipped to 5x its moving average over earlier steps);
 *                       *loss (host, may be NULL) receives the loss before the step (synchronises).
 *   mf_net_gradients    loss and parameter gradients without an update (grads: host
 *                       float[mf_net_num_params], may be NULL).
 *   mf_net_get_params / mf_net_set_params   flat FP32 parameters (host arrays), for checkpoints and
 *                       for moving weights between networks of different grid sizes.
 *   mf_net_state_bytes / mf_net_state_save / mf_net_state_load   the whole training state in one
 *                       caller-owned host buffer: parameters, Adam's moments and step count, the
 *                       gradient-norm history of the clip, the output scale.  Training continued
 *                       after a load takes the same steps, bitwise, as training that was never
 *                       interrupted (the kernels are deterministic).  Save and load synchronise the
 *                       device; load returns MF_ERR_ARG for a buffer that is no state, is truncated,
 *                       holds another parameter count or a header out of range (negative step,
 *                       output scale not positive, clip values not finite), before it changes the
 *                       network.
 * Low-level kernels, exposed for parity tests (BF16 tensors as uint16 bit patterns, channels-last
 * [z][y][x][C]; weights [27][Cin][Cout] with tap t = dx + 3 dy + 9 dz for offsets (d - 1)):
 *   mf_conv3d_fwd   y = relu?(conv(x, w) + bias + skip); C in [1, 64].
 *   mf_conv3d_dgrad dx = conv^T(dy, w) (input gradient).
 *   mf_conv3d_wgrad dw[27][Cin][Cout] and db[Cout] (FP32); workspace of mf_conv3d_wgrad_workspace bytes.
 *   mf_grid_restrict / mf_grid_prolong   full weighting (2m+1)^3 -> (m+1)^3 and trilinear
 *                   (m+1)^3 -> (2m+1)^3, times `scale`.
 */
mf_status mf_net_create(int32_t nx, int32_t ny, int32_t nz, uint64_t seed, mf_net **out);
mf_status mf_net_destroy(mf_net *net);
int64_t mf_net_num_params(const mf_net *net);
mf_status mf_net_get_params(const mf_net *net, float *host);
mf_status mf_net_set_params(mf_net *net, const float *host);
int64_t mf_net_state_bytes(const mf_net *net);
mf_status mf_net_state_save(const mf_net *net, void *host, int64_t bytes);
mf_status mf_net_state_load(mf_net *net, const void *host, int64_t bytes);
mf_status mf_net_set_output_scale(mf_net *net, float scale);
mf_status mf_net_forward(mf_net *net, const float *r, const float *logk, float *out, mf_stream stream);
/* The network's second input for a scalar Laplace mesh on a structured box: out[node] (device
 * float[n_nodes]) = the mean of log kappa over the cells that touch the node (1 to 8 cells), computed
 * in FP64 and rounded to FP32; the flexible CG forms the same field.  Asynchronous.  Errors:
 * MF_ERR_ARG, MF_ERR_UNSUPPORTED (other meshes), MF_ERR_CUDA. */
mf_status mf_node_logk(const mf_mesh *mesh, float *out, mf_stream stream);
mf_status mf_net_train_step(mf_net *net, const float *r, const float *logk, const float *target, float lr,
                            float *loss, mf_stream stream);
mf_status mf_net_gradients(mf_net *net, const float *r, const float *logk, const float *target, float *grads,
                           float *loss, mf_stream stream);
mf_status mf_conv3d_fwd(const void *x, int32_t nx, int32_t ny, int32_t nz, int32_t cin, const void *w,
                        const float *bias, int32_t cout, const void *skip, int32_t relu, void *y_bf16,
                        float *y_f32, mf_stream stream);
mf_status mf_conv3d_dgrad(const void *dy, int32_t nx, int32_t ny, int32_t nz, int32_t cin, const void *w,
                          int32_t cout, void *dx_bf16, float *dx_f32, mf_stream stream);
int64_t mf_conv3d_wgrad_workspace(int32_t nx, int32_t ny, int32_t nz, int32_t cin, int32_t cout);
mf_status mf_conv3d_wgrad(const void *x, const void *dy, int32_t nx, int32_t ny, int32_t nz, int32_t cin,
                          int32_t cout, float *dw, float *db, float *workspace, int64_t ws_bytes, mf_stream stream);
mf_status mf_grid_restrict(const void *in, int32_t nfx, int32_t nfy, int32_t nfz, int32_t c, void *out,
                           float scale, mf_stream stream);
mf_status mf_grid_prolong(const void *in, int32_t ncx, int32_t ncy, int32_t ncz, int32_t c, void *out,
                          float scale, mf_stream stream);

/*
 * mf_training_pair - one (input, target) pair for training the learned preconditioner (the network's
 * workload; the paper has none).  Given b = A x* for an exact solution x* and an iterate x_k of a
 * solve of A x = b (device double[n_dof] each), forms in FP64 the residual r = b - A x_k and the
 * error e = x* - x_k (so that A e = r) in the variables of the symmetrically scaled system with
 * D = diag(A) (Eqs. 4/6, the Jacobi diagonal of mf_operator_diagonal): r~ = D^-1/2 r and
 * e~ = D^1/2 e, Dirichlet entries 0.
 *   r64, e64   device double[n_dof] outputs r~ and e~, or NULL.
 *   r32, e32   device float[n_dof] outputs r~ / s and e~ / s with s = RMS(r~) (network input and
 *              unscaled target).
 *   sums       host double[2] or NULL: sum of r~^2 and of e~^2.
 * Uses the mesh's solver workspace (allocated on first use, like mf_cg_solve).  Synchronises
 * `stream`.  Errors: MF_ERR_ARG, MF_ERR_OOM, MF_ERR_CUDA.
 */
mf_status mf_training_pair(mf_mesh *mesh, const double *b, const double *xs, const double *xk, double *r64,
                           double *e64, float *r32, float *e32, double *sums, mf_stream stream);

/* Message describing the last failure in the calling thread ("" if none).  Valid until the next
 * failing call in the same thread. */
const char *mf_last_error(void);

/* Index checks of the bounds-checked build (no counterpart in the paper: a debugging aid).  A
 * library built with -DMF_DEBUG_BOUNDS (`python -m paper_2308_09839_gb300.build --debug`, which
 * writes libmf_debug.so) checks the node, cell and column indices its kernels compute before they
 * use them; a failed check sets a bit (1 node index, 2 cell index, 4 CSR column index) in a device
 * status word and the access is redirected to index 0, so the kernel finishes in bounds.  This call
 * synchronises the device, returns the bits set since the last call in *bits (and clears them) and
 * *enabled = 1.  In a release build it touches no device: *bits = 0, *enabled = 0.  enabled may be
 * NULL.  Errors: MF_ERR_ARG (bits NULL), MF_ERR_CUDA. */
mf_status mf_debug_status(uint32_t *bits, int32_t *enabled);

/* Number of CUDA kernels this library has launched in the process so far (kernels replayed by a
 * CUDA graph count once per replay).  Host call, thread-safe; for accounting in benchmarks. */
int64_t mf_kernel_launches(void);

/* Library version string (host). */
const char *mf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MF_H_ */
