/*
 * fraclap.h -- C ABI of the GB300 library for the dense P1 finite element
 * matrix of the integral fractional Laplacian (-Δ)^s on a polygon (d = 2) or
 * interval (d = 1) with zero exterior data, and the dense linear algebra of its
 * iterative solvers.
 *
 * Method: Ainsworth & Glusa, "Towards an efficient finite element method for the
 * integral fractional Laplacian on polygonal domains" (arXiv:1708.03912).
 *   - operator, constant C(d,s), bilinear form a(u,v) with the boundary term:
 *     Section 2;
 *   - P1 space V_h, degree-of-freedom set I_h, A^s_ij = a(phi_i, phi_j): Section 3;
 *   - element-pair decomposition (eqs. elementPair, elementPairBoundary),
 *     singular quadrature of touching pairs, diagonal scaling and conjugate
 *     gradients: Section 5;
 *   - quadrature orders: Appendix B (here fixed per class, see fl_options).
 *
 * Conventions for every entry point:
 *   - return value: FL_OK (0) or one of the FL_E* codes below; a message is kept
 *     per handle and returned by fl_last_error().  No call aborts, throws across
 *     the ABI or traps on the device.
 *   - pointers named *_dev are device pointers (cudaMalloc / PyTorch memory on the
 *     current device); pointers named *_host are host pointers.  The caller owns
 *     every buffer it passes; the library never frees or keeps them after the call
 *     returns (work queued on `stream` may still read/write them until the stream
 *     reaches that point).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     All device work is enqueued on it; calls return without synchronising
 *     unless stated.
 *   - dense matrices are row-major with leading dimension `lda` (elements,
 *     lda >= n).  The stiffness matrix is symmetric and stored in full.
 *   - DOF order: increasing vertex index over the vertices in I_h (fl_dof_vertices).
 */
#ifndef FRACLAP_H
#define FRACLAP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define FL_OK        0
#define FL_EINVAL    1  /* bad argument, s outside (0,1), degenerate/inverted or non-conforming mesh */
#define FL_ENOMEM    2  /* device or host allocation failed */
#define FL_ECUDA     3  /* a CUDA runtime call or kernel launch failed */
#define FL_ENOTSPD   4  /* CG breakdown: p^T A p <= 0 */
#define FL_ENOTCONV  5  /* iteration limit reached before the tolerance */
#define FL_ETIMEOUT  6  /* a bounded device wait gave up */
#define FL_ENOTIMPL  7  /* combination of options not implemented */

/* degree-of-freedom rule (Section 3) */
#define FL_DOF_INTERIOR 0 /* interior vertices for every s (default) */
#define FL_DOF_PAPER    1 /* all vertices if s < 1/2, interior vertices otherwise */

/* arithmetic of the separated-pair quadrature */
#define FL_FP64  0 /* every step in float64 */
#define FL_MIXED 1 /* separated pairs (element/element and element/far facet) evaluated in
                      float32 and summed in float64; touching pairs, near facets and all
                      reductions in float64 */

/* storage types for matrices handed to fl_matvec / fl_convert */
#define FL_F64  0
#define FL_F32  1
#define FL_BF16 2
#define FL_F32X2 3  /* float32 hi + lo pair per entry (hi = fl32(a), lo = fl32(a - hi)), 8 bytes */

typedef struct fl_options {
    int k_far;    /* Gauss order per dimension, separated pairs at vertex-graph distance >= 2 (default 4) */
    int k_near;   /* separated pairs at vertex-graph distance 1 and near boundary facets (default 6) */
    int k_touch;  /* common-edge pairs (and 1D touching pairs), regular variables (default 8);
                     identical pairs use 2*k_touch angular points per piece */
    int k_bnd;    /* element/boundary-facet pairs that touch (default 8) */
    int regional; /* 1: drop the boundary term (regional fractional Laplacian, Section 2) */
    int k_vertex; /* common-vertex pairs, 3D regular variables (default 6) */
    int far_f64_pipe; /* FL_FP64 mode, 2D, k_far = 4, s in {1/4, 1/2, 3/4}: the separated pairs at
                         distance >= 2 are evaluated in double-word arithmetic on the float32 pipe
                         (about 2^-47 relative per operation; default 0); 1 evaluates them in
                         float64 on the float64 pipe instead.  Other cases always use float64. */
} fl_options;

typedef struct fl_ctx* fl_handle;

/* Fill *opt with the defaults listed above. */
void fl_default_options(fl_options* opt);

/*
 * Create a handle for a mesh (Section 3).  dim = 1 or 2; vertices_host is
 * [n_vertices][dim] float64; cells_host is [n_cells][dim+1] int32 vertex indices.
 * The arrays are copied.  Cells are re-oriented (counter-clockwise / left-to-right).
 * Boundary facets are the facets owned by exactly one cell.  The host planner runs
 * here (classification of element pairs, tables); device tables are uploaded lazily
 * by the first device call.  opt may be NULL (defaults).  A handle serves one host
 * thread at a time, and its device calls share the handle's workspace: calls on one
 * handle enqueued on different streams must not overlap on the GPU.
 * Errors: FL_EINVAL for dim not in {1,2}, indices out of range, degenerate cells,
 * edges shared by more than two triangles, dof_mode unknown, orders outside [1,32].
 */
int fl_create(fl_handle* h, int dim, int64_t n_vertices, const double* vertices_host,
              int64_t n_cells, const int32_t* cells_host, int dof_mode, const fl_options* opt);

/*
 * Symmetry reduction (Section 7, "Exploiting Symmetry"): Omega, f and hence u invariant under
 * the rotation B by 2 pi / K about the origin.  The caller meshes the sector
 * {0 <= phi <= 2 pi / K} (vertices_host [n_vertices][2], cells_host [n_cells][3], host arrays,
 * copied) so that the rotation maps the vertices on the ray phi = 0 onto those on the ray
 * phi = 2 pi / K; the handle holds the whole mesh, the K copies rotated by 2 pi l / K with
 * vertices closer than 1e-10 merged.  Its problem is the reduced one: one unknown per orbit
 * {B^l v} of interior vertices (numbered by the lowest sector vertex of the orbit, ascending;
 * fl_dof_vertices gives those sector vertices, fl_num_dofs their count n_red), the Galerkin
 * problem on the periodic subspace.  fl_assemble writes the n_red x n_red matrix: the
 * symmetric part of (|O_r| / K) sum_{j in O_c} A[rep_r, j], i.e. P^T A P / K with A the whole
 * mesh's matrix (the paper's bilinear form with the effective kernel
 * k_eff(x, y) = sum_l |x - B^l y|^{-d-2s}, over K); only the element pairs with a cell in a
 * representative's support are evaluated, about 2/K of the whole mesh's.  fl_load_vector
 * takes f_nodal_dev as [n_vertices (of the sector)][nrhs] and writes P^T b / K (n_red rows).
 * fl_solve / fl_matvec work on the reduced matrix as on any other (n = n_red).  Always interior
 * DOFs (dof_mode FL_DOF_INTERIOR).  Not available on such a handle (FL_ENOTIMPL): the
 * near-field CSR, heat-equation, adaptive, cluster-method, multigrid-prolongation and learned
 * preconditioner calls.
 * Errors: FL_EINVAL (NULL arrays, K outside [2, 64], index out of range, a copy that does not
 * close up into orbits), the errors of fl_create.
 */
int fl_create_sector(fl_handle* h, int64_t n_vertices, const double* vertices_host, int64_t n_cells,
                     const int32_t* cells_host, int K, const fl_options* opt);

/* Release the handle and every device buffer it owns (synchronises the device). */
void fl_destroy(fl_handle h);

/* Last error message of the handle ("" if none); valid until the next call on h.  With
 * h = NULL: the message of the calling thread's last failed fl_create or fl_refine. */
const char* fl_last_error(fl_handle h);

/* Number n of degrees of freedom for order s (depends on s only under FL_DOF_PAPER). */
int fl_num_dofs(fl_handle h, double s, int64_t* n);

/* vertex_of_dof_host[n]: the vertex index of each DOF (increasing). */
int fl_dof_vertices(fl_handle h, double s, int32_t* vertex_of_dof_host);

/*
 * Dense stiffness matrix A^s_ij = a(phi_i, phi_j) (Sections 2, 3, 5) into
 * A_dev[n][lda] (float64, full symmetric storage), by element-pair quadrature:
 * separated pairs with collapsed Gauss rules, touching pairs with regularised
 * rules whose radial integral is exact, boundary term over the boundary facets.
 * precision = FL_FP64 or FL_MIXED.  Deterministic: the same call on the same
 * device gives bitwise identical results (no floating-point atomics).
 * The handle owns a scratch workspace sized at the first call for this mesh.
 * Scheduling: the near, touching and boundary stages run on a second stream owned
 * by the handle (created at the first call), forked from and joined back into
 * `stream` by events, concurrently with the far-field stage; to the caller the
 * call behaves as work enqueued on `stream` alone, and it can be captured into a
 * CUDA graph once a first call has created that stream.  With profiling on
 * (fl_set_profiling) every stage runs on `stream`, one after another.
 * Errors: FL_EINVAL (s not in (0,1), lda < n, NULL A), FL_ENOTIMPL (2D with
 * FL_DOF_PAPER and s < 1/2 unless regional), FL_ENOMEM, FL_ECUDA.
 */
int fl_assemble(fl_handle h, double s, int precision, double* A_dev, int64_t lda, void* stream);

/*
 * Autotuner of the element-pair tile kernel (no counterpart in the paper).  In the FL_FP64
 * mode on 2D meshes with k_far = 4 and s in {1/4, 1/2, 3/4} the separated pairs at
 * distance >= 2 (Section 5's N_el^2 part) run in double-word arithmetic, one 4-warp block
 * per 32 x 32 tile of cells, in launch variants 1-4: the unroll of the loop over the column
 * cell's quadrature points and the minimum number of resident blocks per SM the kernel is
 * compiled for (which caps its registers per thread) are (4, 1), (1, 2), (2, 2), (1, 3).
 * fl_tune_assemble assembles A (A_dev, lda as for fl_assemble) once per variant plus
 * `reps` timed times with the stages in sequence, takes the median CUDA-event time of the
 * far stage, and records the fastest in the tuning table under ("far_tile_dw<PW>", number
 * of cells); later assemblies of any handle on a mesh with that cell count use it.
 * best_variant / best_ms (host, optional) receive the winner.  Synchronises `stream`.
 * Errors: FL_ENOTIMPL (the double-word kernel does not apply), FL_EINVAL, FL_ENOMEM,
 * FL_ECUDA.
 * fl_set_far_variant fixes the variant of h's later assemblies (1-4; 0: the tuning table,
 * else 3).  Errors: FL_EINVAL.
 */
int fl_tune_assemble(fl_handle h, double s, double* A_dev, int64_t lda, int reps, int* best_variant, double* best_ms,
                     void* stream);
int fl_set_far_variant(fl_handle h, int variant);

/*
 * Sparse near-field part N of A^s in CSR form, A = N + F (Sections 5 and 6): F holds
 * the off-diagonal blocks -C ∬ phi_i(x) phi_j(y) |x-y|^{-d-2s} of the separated
 * element pairs at vertex-graph distance >= 2 (the far field, where the kernel is
 * smooth); N holds everything else: touching pairs, separated pairs at distance 1,
 * identical pairs, the boundary term and the diagonal-block terms of every separated
 * pair.  Pattern: the (i, j) such that a cell of supp phi_i touches or lies at
 * distance 1 from a cell of supp phi_j; symmetric, columns ascending in each row.
 * Same quadrature, precision modes and determinism as fl_assemble (N_ij equals the
 * value fl_assemble would give for A_ij with F left out).
 * Two calls: with rowptr_dev == NULL only *nnz (host) is set, no device work; then
 * rowptr_dev[n + 1] and col_dev[nnz] (int32, device) and val_dev[nnz] (float64,
 * device), owned by the caller, are filled on `stream`.  The handle's workspace is
 * the one fl_assemble uses.
 * Errors: FL_EINVAL (s not in (0,1), NULL nnz, NULL col/val with rowptr_dev set),
 * FL_ENOTIMPL, FL_ENOMEM, FL_ECUDA as for fl_assemble.
 */
int fl_assemble_nearfield_csr(fl_handle h, double s, int precision, int64_t* nnz,
                              int32_t* rowptr_dev, int32_t* col_dev, double* val_dev,
                              void* stream);

/*
 * Load vector b = ∫ f phi_i (Section 5, system A u = b) into b_dev[n][ldb]
 * (column r at b_dev + r, row-major n x nrhs).  f_nodal_dev NULL: f = 1 (nrhs must
 * be 1); else f_nodal_dev is [n_vertices][nrhs] float64 nodal values and f is their
 * P1 interpolant, b = M f with the P1 mass matrix.
 */
int fl_load_vector(fl_handle h, double s, const double* f_nodal_dev, int nrhs,
                   double* b_dev, int64_t ldb, void* stream);

/*
 * Fractional heat equation d_t u + (-Delta)^s u = f (Section 2).  Implicit time steps give
 * systems (M + dt A^s) u = b with the P1 mass matrix M (Section 5); with implicit Euler,
 * (M + dt A^s) u^{k+1} = M u^k + dt F.  Both calls work on h's DOF set for order s.
 * fl_heat_matrix: H_dev = M + dt A_dev for the dense float64 A^s (n x n, row pitch lda) of
 * h's mesh at order s; H_dev (pitch ldh) may be A_dev itself (then ldh = lda) but must not
 * overlap it otherwise.  dt >= 0.  Deterministic (fixed summation order).
 * fl_mass_apply: Y = alpha M X + beta B for nrhs columns; X, B, Y float64 row-major
 * [n][ld*] (column r at +r); B may be NULL when beta = 0; Y must not be X.  With f the P1
 * interpolant of nodal values, the load vector F of fl_load_vector is M_full f.
 * Errors: FL_EINVAL (bad pointers, pitches, dt < 0, overlap), FL_ENOMEM, FL_ECUDA.
 */
int fl_heat_matrix(fl_handle h, double s, double dt, const double* A_dev, int64_t lda, double* H_dev, int64_t ldh,
                   void* stream);
int fl_mass_apply(fl_handle h, double s, int nrhs, double alpha, const double* X_dev, int64_t ldx, double beta,
                  const double* B_dev, int64_t ldb, double* Y_dev, int64_t ldy, void* stream);

/*
 * Adaptive refinement (Section 4 with Appendix A; the loop of Section 7: solve, estimate,
 * mark with the maximum strategy, refine without hanging nodes).
 *
 * Cell rule of order k_cell (the points where the strong form is evaluated): 1D Gauss-Legendre
 * on [x0, x1], q = k_cell points at x0 + t_a (x1 - x0); 2D the collapsed product rule,
 * q = k_cell^2 points at v0 + l1 (v1 - v0) + l2 (v2 - v0), l1 = t_a, l2 = t_b (1 - t_a), point
 * (a, b) at index a k_cell + b, weight w_a w_b (1 - t_a) 2|K|; (v0, v1, v2) the cell's vertices
 * in the given order, swapped to (v0, v2, v1) for a clockwise cell, as fl_create orients them.
 *
 * fl_strong_form: S_dev[K q + a] = (-Delta)^s u_h at point a of cell K (original cell order),
 *   u_h = sum_i u_i phi_i with u_dev the n float64 DOF values of h's DOF set at s (device).
 *   Lemma 4.1 turns the hypersingular integral into regular integrals over cell boundaries
 *   (eq. (8); eq. (9) for s = 1 - d/2, i.e. 1D with s = 1/2).  The three edges of the point's
 *   own cell are integrated by Gauss-Legendre of order k_near (the integrand is nearly
 *   singular there), every other edge by order k_edge (1D: the facets are points and neither
 *   order matters).  1 <= k_cell <= 16, 1 <= k_edge <= 32, 1 <= k_near <= 64.  Cost
 *   O(n_cells q n_edges k_edge): every point meets every edge.  Float64 accuracy; 2D with
 *   s in {1/4, 1/2, 3/4} runs in double-word arithmetic on the float32 pipe (unless the
 *   handle's options set far_f64_pipe), the rest on the float64 pipe.  Deterministic.  Uses
 *   a device workspace owned by h, grown on demand (the call may synchronise to grow it).
 * fl_br_indicators: eta_dev[n] = the Babuska-Rheinboldt indicators (eq. (BRindicators)),
 *   eta_i^2 = sum over the cells K around DOF i's vertex of h_K^{2s} ||f - (-Delta)^s u_h||^2
 *   on K, h_K the longest edge (1D: the length), the L2 norm by the cell rule above.
 *   f_nodal_dev NULL: f = 1; else n_vertices float64 nodal values, f their P1 interpolant.
 *   S_dev: NULL, or [n_cells q] float64 that receives the strong form.  Synchronises `stream`.
 * fl_mark_max: maximum marking with threshold theta, 0 < theta <= 1 (Section 7 uses 0.8):
 *   DOF i is marked when eta_i >= theta max_j eta_j (float64).  dof_marks_dev[n] (uint8,
 *   may be NULL) = 1 for marked DOFs, else 0; cell_marks_dev[n_cells] (uint8, may be NULL) = 1
 *   for the cells around a marked DOF's vertex (the patches S_i), else 0.  Not both NULL.
 * Errors: FL_EINVAL (s not in (0,1), NULL pointers, orders out of range, theta), FL_ENOMEM,
 *   FL_ECUDA.
 */
int fl_strong_form(fl_handle h, double s, const double* u_dev, int k_cell, int k_edge, int k_near, double* S_dev,
                   void* stream);
int fl_br_indicators(fl_handle h, double s, const double* u_dev, const double* f_nodal_dev, int k_cell, int k_edge,
                     int k_near, double* eta_dev, double* S_dev, void* stream);
int fl_mark_max(fl_handle h, double s, const double* eta_dev, double theta, uint8_t* dof_marks_dev,
                uint8_t* cell_marks_dev, void* stream);

/*
 * Conforming refinement of the cells with cell_marks[k] != 0 (host arrays; no handle, no
 * device work).  Input as fl_create: vertices [n_vertices][dim], cells [n_cells][dim+1].
 * 1D: a marked interval (a, b) becomes (a, m), (m, b).  2D: newest-vertex bisection; a cell
 * (v0, v1, v2) has newest vertex v0 and refinement edge {v1, v2}, and bisects into
 * (m, v0, v1), (m, v2, v0) with m the edge's midpoint.  Every marked cell is bisected, and
 * neighbours are bisected as far as needed to leave no hanging node: the set of halved edges
 * is the smallest that holds the marked cells' refinement edges and, with any edge of a cell,
 * that cell's refinement edge.  A cell thus becomes 1 to 4 cells; the result does not depend
 * on the order of the cells.  Numbering: old vertices keep their ids, midpoints follow in
 * order of creation (cells in input order; per cell the refinement edge's midpoint, then
 * those of its first and second child); each cell is replaced in place by its children.
 * Outputs (caller-owned host arrays): vertices_out [cap_vertices][dim], cells_out
 * [cap_cells][dim+1], and their counts.  n_vertices + 3 n_cells vertices and 4 n_cells cells
 * always suffice.  Errors: FL_EINVAL for bad arguments, an index out of range, an edge shared
 * by more than two cells, or a capacity below the result (the needed counts are still
 * stored); FL_ENOMEM.  fl_last_error(NULL) gives the message.
 */
int fl_refine(int dim, int64_t n_vertices, const double* vertices, int64_t n_cells, const int32_t* cells,
              const uint8_t* cell_marks, int64_t cap_vertices, int64_t cap_cells, double* vertices_out,
              int32_t* cells_out, int64_t* n_vertices_out, int64_t* n_cells_out);

/*
 * The dense matrix-vector product of the iterative solvers (Section 5: n^2 work per
 * product).  Y = A X for a dense n x n matrix stored as dtype (FL_F64 / FL_F32 / FL_BF16 /
 * FL_F32X2; the low-precision storages are not in the paper) with leading dimension lda
 * (in entries; an FL_F32X2 entry is a float2);
 * X_dev, Y_dev are [n][nrhs] float64 row-major with leading dimensions ldx, ldy
 * (>= nrhs).  Accumulation in float64 (FL_F64), float32 with float64 per-row totals
 * (FL_F32, FL_BF16), or double-float on the float32 pipe (FL_F32X2: x split into
 * float32 hi + lo, error about 2^-44 of sum_j |a_ij x_j|).  Streams A once per call;
 * stages x in shared memory (no allocation) while at least two 8-warp blocks per SM
 * fit with it (x up to about 12k entries for FL_F64 and FL_F32X2, 25k for FL_F32 and
 * FL_BF16); beyond that float32 / bfloat16 / hi + lo products allocate a copy of x.
 * Errors: FL_EINVAL (NULL pointers, n < 1, a leading dimension too small, an unknown
 * dtype, an FL_F32X2 matrix that is not 8-byte aligned), FL_ENOMEM, FL_ECUDA.
 */
int fl_matvec(int dtype, const void* A_dev, int64_t lda, int64_t n, int nrhs,
              const double* X_dev, int64_t ldx, double* Y_dev, int64_t ldy, void* stream);

/* A_lo_dev (dtype FL_F32 or FL_BF16, leading dimension ld_lo) = A_dev rounded to nearest;
 * FL_F32X2: the (hi, lo) float2 pairs hi = fl32(a), lo = fl32(a - hi), A_lo_dev 8-byte
 * aligned, ld_lo in pairs. */
int fl_convert(const double* A_dev, int64_t lda, int64_t n, int dtype, void* A_lo_dev,
               int64_t ld_lo, void* stream);

typedef struct fl_solve_opts {
    double tol;        /* stop at ||b - A u||_2 <= tol ||b||_2 (default 1e-8) */
    int maxit;         /* iteration limit of the outer solver (default 10000) */
    int inner_dtype;   /* FL_F64: plain Jacobi-PCG on A (Section 5); FL_F32: Jacobi-PCG on a
                          float32 copy inside float64 iterative refinement */
    const void* A_lo_dev; /* the float32 copy (required when inner_dtype = FL_F32) */
    int64_t ld_lo;
    double inner_tol;  /* relative tolerance of each inner solve (default 1e-4); a step
                          whose residual is already within a factor 1/inner_tol of the
                          target uses max(inner_tol, tol ||b|| / (2 ||b - A u||)) */
    int inner_maxit;   /* default 2000 */
    int barrier_timeout_us; /* bound of each grid-barrier wait of the cooperative solvers, in
                          microseconds (0: the default of 2 s); a wait that runs out makes
                          the call return FL_ETIMEOUT and leaves the handle usable */
} fl_solve_opts;

typedef struct fl_solve_info {
    int iterations;        /* total (inner) CG iterations */
    int outer_iterations;  /* refinement steps (1 for plain CG) */
    double rel_residual;   /* final ||b - A u|| / ||b|| computed in float64 with A */
    int status;            /* FL_OK, FL_ENOTCONV or FL_ENOTSPD */
} fl_solve_info;

void fl_default_solve_opts(fl_solve_opts* o);

/*
 * Solve A u = b for one right-hand side with diagonally preconditioned conjugate
 * gradients (Section 5; κ(D^-1 A) = O(n^{2s/d}), so O(n^{s/d}) iterations).
 * A_dev is the float64 matrix (n x n, lda); b_dev, u_dev are [n] float64 (u is
 * overwritten; the iteration starts from 0).  With inner_dtype = FL_F32 (or
 * FL_BF16) the Jacobi-PCG runs on the low-precision copy o->A_lo_dev inside float64
 * iterative refinement u += d, M d = b - A u, until ||b - A u|| <= tol ||b|| with
 * the float64 A.  Where cooperative launches are available the plain solve, and
 * with FL_F32 the whole refinement (float64 residual of each step, stop test,
 * float32 inner CG, update), run as one cooperative launch whose blocks own row
 * ranges; the host reads one result block at the end.  Otherwise (and for
 * FL_BF16) the iterations run as captured kernel batches with the scalars read
 * once per batch.  h supplies the workspace (grown on demand) and the error
 * message.  info (host) receives counts and the final residual ||b - A u|| /
 * ||b||, computed in float64 with A.  Synchronises `stream`.  Returns FL_OK,
 * FL_ENOTCONV, FL_ENOTSPD, FL_EINVAL, FL_ENOMEM, FL_ECUDA, or FL_ETIMEOUT when a
 * grid barrier of a cooperative launch waited longer than its bound
 * (o->barrier_timeout_us, default 2 s).
 */
int fl_solve(fl_handle h, int64_t n, const double* A_dev, int64_t lda, const double* b_dev, double* u_dev,
             const fl_solve_opts* o, fl_solve_info* info, void* stream);

/* ------------------------------------------------------------------------
 * Batched solves (no counterpart in the paper, which solves one system at a
 * time with the Jacobi-preconditioned CG of Section 5): several matrices A^s
 * (one per order s, or per mesh) with many right-hand sides each, solved
 * together.  The inner iteration is CG on the Jacobi-scaled matrix
 * Ã = D A D, D = diag(A)^{-1/2}, held as bfloat16 slices, whose product with
 * the block of search directions runs on the tensor cores; float64 iterative
 * refinement with the float64 residual B - A U decides convergence.
 * ------------------------------------------------------------------------ */
#define FL_BATCH_MAXPROB 8
#define FL_RESID_F64 0
#define FL_RESID_DF  1

/*
 * Bytes of the slice storage fl_split_bf16 writes for order n and nslices slices:
 * nslices * ceil(n/128) * ceil(n/64) * 16384 (0 for invalid arguments).
 */
int64_t fl_split_bf16_bytes(int64_t n, int nslices);

/*
 * d = diag(A)^{-1/2} into dscale_dev[n] (float64), and the bfloat16 slices of
 * Ã_ij = (d_i d_j) a_ij (exactly symmetric): S_0 = bf16(Ã), and for nslices = 2 also
 * S_1 = bf16(Ã - S_0), each rounded to nearest (ties to even) in one rounding
 * from float64; magnitudes below 2^-126 become zero.
 * Layout of S_dev (fl_split_bf16_bytes(n, nslices) bytes, 16-byte aligned): the
 * tiles the tensor cores read, one contiguous 16 KiB block per (slice k, row
 * tile t < ceil(n/128), column chunk c < ceil(n/64)) at byte offset
 * ((k ceil(n/128) + t) ceil(n/64) + c) 16384; inside a block, entry
 * (row r < 128, column q < 64) is at byte r 128 + 16 ((q/8) XOR (r mod 8))
 * + 2 (q mod 8) (the 128-byte swizzle); entries outside n x n are zero.
 * n <= 65536.  Errors: FL_EINVAL, FL_ECUDA.
 */
int fl_split_bf16(const double* A_dev, int64_t lda, int64_t n, int nslices, void* S_dev, double* dscale_dev,
                  void* stream);

/*
 * Y = S_0 (X_hi + X_lo) + S_1 X_hi on the tensor cores, where X_hi = bf16(X),
 * X_lo = bf16(X - X_hi) per entry, operands bfloat16 and float32
 * accumulation (relative accuracy about 2^-16 of |S||X| with two slices).
 * X_dev, Y_dev: float32, column j of X at X_dev + j*ldx (n entries), same for Y.
 * nrhs a multiple of 16 in [16, 128].  S_dev as written by fl_split_bf16.
 * Allocates its scratch on `stream` (stream-ordered) and synchronises it.
 * Errors: FL_EINVAL, FL_ENOMEM, FL_ECUDA, FL_ETIMEOUT (a bounded device wait
 * gave up).
 */
int fl_matmul_bf16(const void* S_dev, int64_t n, int nslices, int nrhs, const float* X_dev, int64_t ldx,
                   float* Y_dev, int64_t ldy, void* stream);

typedef struct fl_batch_problem {
    int64_t n;                 /* unknowns */
    const double* A_dev;       /* float64 matrix, n x n, row pitch lda: judges the residual */
    int64_t lda;
    const void* S_dev;         /* its bfloat16 slices and scaling from fl_split_bf16 */
    int nslices;               /* 1 or 2 */
    const double* dscale_dev;  /* [n] */
    int nrhs;                  /* right-hand sides, 1..128 */
    const double* B_dev;       /* [n][ldb] float64, right-hand side j in column j */
    int64_t ldb;
    double* U_dev;             /* [n][ldu] float64 solutions (overwritten; start from 0) */
    int64_t ldu;
} fl_batch_problem;

typedef struct fl_batch_opts {
    double tol;        /* stop column j at ||b_j - A u_j|| <= tol ||b_j|| (default 1e-8) */
    int max_outer;     /* refinement steps (default 8) */
    double inner_tol;  /* relative r.r reduction of each inner CG solve (default 1e-5) */
    int inner_maxit;   /* default 5000 */
    int ctas;          /* CTAs of the persistent kernel (0: one per SM) */
    int stages;        /* TMA pipeline depth (0: as many as shared memory holds) */
    int barrier_timeout_us; /* bound of each grid-barrier wait of the persistent kernel, in
                          microseconds (0: 2 s); a wait that runs out makes the call return
                          FL_ETIMEOUT.  The waits on the copy and tensor-core pipeline keep
                          their fixed 2 s bound: a CTA drains its own copies in flight with
                          that bound before it exits */
    int residual;      /* FL_RESID_DF (default): B - A U in double-float arithmetic on the float32
                          pipe (about 2^-47 relative per operand and operation, so each residual
                          entry is exact to about 2^-46 (|A||u|)_i); FL_RESID_F64: float64 FMA,
                          for tolerances near or below 2^-46 || |A||u| || / ||b|| */
} fl_batch_opts;

typedef struct fl_batch_info {
    int outer_iterations;  /* refinement steps taken */
    int inner_iterations;  /* CG steps summed over the refinement steps */
    int status;            /* FL_OK when every column converged */
    int ctas, stages;      /* launch shape used */
} fl_batch_info;

void fl_default_batch_opts(fl_batch_opts* o);

/*
 * Solve A_p U_p = B_p for p < nprob (nprob <= FL_BATCH_MAXPROB), all columns
 * together: each refinement step computes R = B - A U in float64, then runs one
 * persistent cooperative kernel that iterates CG on D R for every unfinished
 * column of every problem at once (per step: one tensor-core product
 * Ã [P_hi P_lo] per problem, then the vector updates), then U += D Z.
 * rel_residual_host / status_host (host, optional): per column, problems in
 * order, the final ||b - A u|| / ||b|| and FL_OK / FL_ENOTCONV / FL_ENOTSPD.
 * h supplies the workspace (grown on demand) and the error message; the
 * problems need not belong to h's mesh.  Synchronises `stream`.
 * Returns FL_OK if every column converged, else the first failing status;
 * FL_EINVAL, FL_ENOMEM, FL_ECUDA, FL_ETIMEOUT (a bounded device wait gave up),
 * FL_ENOTIMPL (no cooperative launch).
 */
int fl_batch_solve(fl_handle h, int nprob, const fl_batch_problem* probs, const fl_batch_opts* o,
                   fl_batch_info* info, double* rel_residual_host, int* status_host, void* stream);

/* ------------------------------------------------------------------------
 * Cluster method (Section 6): the stiffness matrix as an H-matrix.  The DOFs are
 * organised in a binary cluster tree (a cluster with more than `leaf` DOFs is split at the
 * middle of the longest side of its DOF vertices' bounding box); the cluster box is the
 * smallest cube containing the supports of its basis functions.  A pair of clusters is
 * admissible when eta dist >= max(diam, diam) (distance and diameters of the cubes); the
 * partition comes from the recursion over pairs from (root, root).  On admissible pairs
 * the kernel |x-y|^{-d-2s} is replaced by its tensor Chebyshev interpolant of order m, so
 * those blocks become -C U_sigma K_{sigma tau} U_tau^T with the basis far-field
 * coefficients (int phi_i L_alpha, Gauss order m + 1 per cell) moved through the tree by
 * the shift coefficients; inadmissible pairs of leaves keep their exact entries (near
 * field, CSR).  The product costs O(n log^{2d} n) instead of the dense n^2.
 * ------------------------------------------------------------------------ */
typedef struct fl_hm* fl_hmatrix;

/*
 * Host only (no device work): the cluster tree and partition of h's DOF set for order s.
 * sizes[0..2] receive the numbers of nodes, admissible pairs and near-field leaf pairs;
 * with non-NULL arrays also: perm [n] (DOFs in tree order), node [nodes][4] (range lo, hi
 * of the node in perm, first and second son or -1), far [2 * pairs] and near
 * [2 * pairs] (node ids sigma, tau in the order of the recursion).  Nodes are numbered
 * depth first, first son first.  Call once with NULL arrays to size them.
 * Errors: FL_EINVAL (leaf < 1, eta < 0, s not in (0, 1)).
 */
int fl_cluster_plan(fl_handle h, double s, double eta, int leaf, int64_t* sizes, int32_t* perm, int32_t* node,
                    int32_t* far, int32_t* near);
/*
 * Host only: the plan of fl_hmatrix_assemble_near for the same partition.  sizes[0..3] receive
 * the tiles, the facet-list entries, the facet-table size and the number of cells; with
 * non-NULL arrays also cell_perm [cells] (internal cell order -> cell index of the input),
 * ef_ptr [cells + 1], ef_fac and ef_cls [entries] (per internal cell with DOFs: the facets of the
 * boundary of N(K), ascending ids, and their classes: 2 / 3 = shares two / one vertex with K,
 * 1 = a vertex is a mesh neighbour of one of K, 0 = the rest), fac_vert [table * dim] (vertex
 * ids; ids below the number of boundary facets of Omega are those facets) and fac_normal
 * [table * dim] (unit normals pointing into N(K)).  Call once with NULL arrays to size them.
 * Errors: FL_EINVAL, FL_ENOMEM.
 */
int fl_near_region_plan(fl_handle h, double s, double eta, int leaf, int64_t* sizes, int32_t* cell_perm,
                        int32_t* ef_ptr, int32_t* ef_fac, int32_t* ef_cls, int32_t* fac_vert, double* fac_normal);
/*
 * Host only, no device work: the element-block tiles of the same plan (Section 6, the near field's
 * separated pairs at vertex-graph distance >= 2).  Blocks are 32 consecutive cells of the internal
 * order (cell_perm above); a tile (I, J), I <= J, is listed when some inadmissible leaf pair (A, B) has
 * a DOF of A in a cell of block I and a DOF of B in a cell of block J, or the other way round.
 * *ntiles receives their number; with non-NULL arrays also tiles [2 ntiles] (I, J, ordered by (I, J))
 * and rowmask [ntiles]: bit kk set when cell 32 I + kk has a DOF in a leaf that is near-paired with a
 * leaf holding a DOF of some cell of block J (the separated pairs of the other row cells feed no
 * near-field entry and are not computed).  Caller-owned host arrays.  Errors: FL_EINVAL, FL_ENOMEM.
 */
int fl_near_region_tiles(fl_handle h, double s, double eta, int leaf, int64_t* ntiles, int32_t* tiles,
                         uint32_t* rowmask);

/*
 * Builds the H-matrix of A^s on h's mesh: the plan above, then on the device the leaf
 * coefficients, the shift coefficients and the kernel matrices of the admissible pairs
 * (float64, m^{2d} per pair).  m in [1, 12].  The handle h must outlive the H-matrix.
 * Errors: FL_EINVAL, FL_ENOMEM, FL_ECUDA (message in h).
 */
int fl_hmatrix_create(fl_handle h, double s, int m, double eta, int leaf, fl_hmatrix* out, void* stream);
/* Near-field entries A_ij (i, j in inadmissible leaf pairs) gathered from the dense float64
 * A (row pitch lda) of the same mesh and order.  Errors: FL_EINVAL, FL_ECUDA. */
int fl_hmatrix_set_near(fl_hmatrix H, const double* A_dev, int64_t lda, void* stream);
/*
 * Near-field entries computed directly, by local computations only (Section 6: the near field
 * is assembled into a sparse matrix; its cost is that of the near field, O(n log^{2d} n), with
 * no dense matrix).  An entry a(phi_i, phi_j) gets
 *   - the separated pairs at vertex-graph distance >= 2 of a cell of supp phi_i and a cell of
 *     supp phi_j: only the 32 x 32 tiles of element blocks that near-field entries touch are
 *     computed (float64 rules of the dense assembly, double-word arithmetic where its float64
 *     mode uses it);
 *   - the touching, near (distance 1) and identical pairs as in the dense assembly;
 *   - the diagonal blocks, where the part that sums over the far cells and the boundary term
 *     is, for x in K, C/(2s) times the integral over the boundary of N(K) (K, its touching
 *     cells and the cells at distance 1) of n.(x - y)|x - y|^{-d-2s}, n pointing into N(K):
 *     by the divergence theorem the same quantity, integrated over fewer facets (its facets
 *     at distance 1 with the k_near rules, the others with k_far, the boundary facets of
 *     Omega that touch K with the singular rules of the boundary term).
 * precision FL_FP64: entries whose DOFs share no cell equal the dense float64 matrix's bit for bit;
 * the others differ from it by the quadrature error of the far part of the diagonal blocks.
 * FL_MIXED: the tiles, near and touching pairs and the identical pair in float32 as the mixed
 * dense assembly (the tile partials summed with compensation), the rest float64.  The first call
 * plans (host) and allocates the tiles' workspace; later calls recompute the values.  Not for
 * regional operators, symmetry-reduced handles or 2D boundary DOFs (FL_ENOTIMPL).
 * Errors: FL_EINVAL, FL_ENOMEM, FL_ENOTIMPL, FL_ECUDA.
 */
int fl_hmatrix_assemble_near(fl_hmatrix H, int precision, void* stream);
/* The near field as CSR over the DOFs (rows ascending, columns ascending in a row): *nnz
 * receives the entry count; non-NULL device arrays rowptr_dev [n + 1], col_dev [nnz] and
 * val_dev [nnz] (float64) receive the pattern and the values (the values need a near field,
 * else FL_EINVAL).  Copies on `stream`.  Errors: FL_EINVAL, FL_ECUDA. */
int fl_hmatrix_get_near(fl_hmatrix H, int64_t* nnz, int32_t* rowptr_dev, int32_t* col_dev, double* val_dev,
                        void* stream);
/*
 * The strong form (-Delta)^s u_h by the cluster method (Section 6), at the points of the cell rule
 * of order k_cell (S_dev [cells][k_cell^2], cells in input order, as fl_strong_form).  For a point
 * x0 of cell K0, with sigma the leaf of K0's DOF closest to x0 (ties: the lower DOF), u splits
 * into u_N, its part on the DOFs of sigma's inadmissible partners, and u_F, the rest: the strong
 * form of u_N is Lemma 4.1's (the facets of the cells touching a near DOF: those of K0 and through
 * its vertices in float64 with orders k_near / k_edge, the others in double-word arithmetic), that
 * of u_F is -C sum_alpha L_alpha^sigma(x0) yh_sigma[alpha] with yh the far-field coefficients of
 * u from the H-matrix product's upward pass, couplings and downward pass.  Points of cells without
 * a DOF vertex take the strong form of u itself.  Needs no near field.  2D, s in {1/4, 1/2, 3/4},
 * interior DOFs (else FL_ENOTIMPL).  The first call for a k_cell plans (host); a later call with another
 * k_cell plans again, the earlier plan's device memory staying with H until fl_hmatrix_destroy.  Calls on
 * one H must not overlap (they share its workspace).  Errors: FL_EINVAL, FL_ENOMEM, FL_ENOTIMPL, FL_ECUDA.
 */
int fl_hmatrix_strong_form(fl_hmatrix H, const double* u_dev, int k_cell, int k_edge, int k_near, double* S_dev,
                           void* stream);
/*
 * Host only: the plan of fl_hmatrix_strong_form for the partition (s, eta, leaf) and the cell rule
 * k_cell.  sizes[0..3] receive the points (cells x k_cell^2), the groups, the facet-list entries and
 * the facets of the strong form's facet table; with non-NULL arrays also pgroup [points] (the group
 * of point q of internal cell k at k k_cell^2 + q; internal order as in fl_near_region_plan's
 * cell_perm), gnode [groups] (the group's leaf node as numbered by fl_cluster_plan, -1 for the cells
 * without a DOF vertex), gf_ptr [groups + 1] and gf_fac [entries] (per group its facets, ascending)
 * and fac_vert [2 facets] (the facets' end vertices).  2D only (FL_ENOTIMPL).  Errors: FL_EINVAL,
 * FL_ENOMEM, FL_ENOTIMPL.
 */
int fl_strong_form_cluster_plan(fl_handle h, double s, double eta, int leaf, int k_cell, int64_t* sizes,
                                int32_t* pgroup, int32_t* gnode, int64_t* gf_ptr, int32_t* gf_fac,
                                int32_t* fac_vert);
/* The Babuska-Rheinboldt indicators (as fl_br_indicators, f_dev nodal or NULL for f = 1) from the
 * cluster method's strong form; S_dev [cells][k_cell^2] receives the strong form. */
int fl_hmatrix_br_indicators(fl_hmatrix H, const double* u_dev, const double* f_dev, int k_cell, int k_edge,
                             int k_near, double* eta_dev, double* S_dev, void* stream);
/* info[0..2] after fl_hmatrix_assemble_near: tiles computed, their partial-block entries,
 * device bytes of its plan and workspace (zeros before the first call). */
int fl_hmatrix_near_info(fl_hmatrix H, int64_t* info);
/* y_dev = H x_dev (float64 [n], y must not be x): near-field CSR product, upward pass,
 * couplings, downward pass; fixed summation orders.  Errors: FL_EINVAL (no near field
 * yet), FL_ECUDA. */
int fl_hmatrix_matvec(fl_hmatrix H, const double* x_dev, double* y_dev, void* stream);
/*
 * Solve A u = b with the cluster method's product in place of the dense one: Jacobi-PCG
 * (Section 5) on the H-matrix, the diagonal taken from the near field (exact entries), from
 * u = 0 until ||b - H u||_2 <= o->tol ||b||_2 (the H-matrix's own residual) or o->maxit steps
 * (the other fl_solve_opts fields are ignored; NULL: the defaults).  b_dev, u_dev: [n] float64,
 * DOF order (u overwritten, must not be b).  The scalars of each step are read back to the host
 * (the call synchronises `stream` every step).  The solution differs from the dense solve by the
 * interpolation error of the far field.  Returns FL_OK, FL_ENOTCONV, FL_ENOTSPD, or FL_EINVAL /
 * FL_ENOMEM / FL_ECUDA; *info (may be NULL) gets iterations and the final relative residual.
 */
int fl_hmatrix_solve(fl_hmatrix H, const double* b_dev, double* u_dev, const fl_solve_opts* o, fl_solve_info* info,
                     void* stream);
/* The same solver for (alpha M + beta A) u = b with M the P1 mass matrix on the DOFs (fl_mass_apply)
 * and A the H-matrix: the implicit time step of the fractional heat equation (Sections 2 and 5:
 * (M + dt A^s) u^{k+1} = M u^k + dt F with alpha = 1, beta = dt) without a dense matrix.  The Jacobi
 * diagonal is alpha M_ii + beta A_ii.  alpha >= 0, beta > 0 (else FL_EINVAL); alpha = 0, beta = 1 is
 * fl_hmatrix_solve. */
int fl_hmatrix_solve_shifted(fl_hmatrix H, double alpha, double beta, const double* b_dev, double* u_dev,
                             const fl_solve_opts* o, fl_solve_info* info, void* stream);
/* info[0..5] (host, 6 int64): nodes, admissible pairs, near-field leaf pairs, near-field entries,
 * device bytes held, tree depth.  Errors: FL_EINVAL (NULL H or info). */
int fl_hmatrix_info(fl_hmatrix H, int64_t* info);
/* The message of H's last failed call ("" if none; a fixed message for NULL H); owned by H, valid
 * until its next call. */
const char* fl_hmatrix_last_error(fl_hmatrix H);
/* Frees H's device memory after synchronising its device (work queued by its calls completes
 * first); NULL is a no-op.
 * The mesh handle H was made from is not touched. */
void fl_hmatrix_destroy(fl_hmatrix H);

/* ------------------------------------------------------------------------
 * Multigrid (Section 5 proposes multigrid for these dense systems; no algorithm is
 * given, this is the Galerkin V-cycle on nested meshes).
 * ------------------------------------------------------------------------ */

/*
 * Prolongation from the coarse mesh's DOFs to the fine mesh's DOFs for order s:
 * P_ij = (coarse hat function j)(fine DOF vertex i), exact when the fine mesh is a
 * refinement of the coarse one.  Host CSR (rows = fine DOFs): call first with
 * rowptr = col = val = NULL to get *nnz, then with arrays of n_fine + 1, nnz, nnz.
 * Errors: FL_EINVAL (dimensions differ, a fine vertex outside the coarse mesh).
 */
int fl_prolongation(fl_handle fine, fl_handle coarse, double s, int64_t* nnz, int32_t* rowptr, int32_t* col,
                    double* val);

typedef struct fl_mg* fl_mg_handle;

/* Start a hierarchy on the finest operator A_dev (float64, n x n, row pitch lda; not
   copied: it must outlive the handle). */
int fl_mg_create(fl_mg_handle* mg, const double* A_dev, int64_t lda, int64_t n);
/* Add a coarser level: P (host CSR, rows = DOFs of the current coarsest level, nc
   columns) from fl_prolongation; forms A_c = P^T A P on the device in float64.
   Synchronises `stream`. */
int fl_mg_add_level(fl_mg_handle mg, int64_t nc, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                    const double* val, void* stream);
/* Float32 level copies, Jacobi weights w = 4 / (3 lambda) (lambda: ten power-iteration
   steps on D^-1 A from (1, ..., 1), then |D^-1 A x| / |x|), the explicit inverse of the
   coarsest operator (Gauss-Jordan, float64); nu smoothing steps before and after the
   coarse correction.  Synchronises `stream`. */
int fl_mg_setup(fl_mg_handle mg, int nu, void* stream);
/* Order, float64 operator (device, owned by mg for level > 0) and its row pitch of a level. */
int fl_mg_level(fl_mg_handle mg, int level, int64_t* n, const double** A_dev, int64_t* lda);
/* Copy a level's float64 operator into dst_dev[n][ldd] (device). */
int fl_mg_level_copy(fl_mg_handle mg, int level, double* dst_dev, int64_t ldd, void* stream);
/* The Jacobi weight of a level (after fl_mg_setup). */
int fl_mg_omega(fl_mg_handle mg, int level, float* omega);
/* z = V(r): one V-cycle from zero on the finest level, float32 device vectors [n]. */
int fl_mg_vcycle(fl_mg_handle mg, const float* r_dev, float* z_dev, void* stream);
/* Conjugate gradients on the finest operator preconditioned by one V-cycle per step,
   from u = 0, until ||b - A u|| <= tol ||b|| (recursive residual, float64).
   Returns FL_OK, FL_ENOTCONV or FL_ENOTSPD; info as for fl_solve. */
int fl_mg_solve(fl_mg_handle mg, const double* b_dev, double* u_dev, double tol, int maxit, fl_solve_info* info,
                void* stream);
/* The message of mg's last failed call ("" if none or NULL mg); owned by mg. */
const char* fl_mg_last_error(fl_mg_handle mg);
/* Frees mg's device and pinned memory after synchronising its device; NULL is a no-op. */
void fl_mg_destroy(fl_mg_handle mg);

/* ------------------------------------------------------------------------
 * Learned patch preconditioner and flexible CG (not in the paper).  A linear
 * preconditioner whose stencil over each DOF's patch (the K = 12 nearest DOFs within
 * two mesh edges) a small network (hidden width 64, tanh) computes from the patch
 * geometry; applied as the symmetric part (M + M^T)/2; see learned.cu for the exact
 * definition.  The network starts as the Jacobi preconditioner.
 * ------------------------------------------------------------------------ */

/* Patch table of the mesh's DOFs at order s (host, 2D): nbr_host[n][K] DOF indices
   ordered by (distance, vertex index), -1 padded; hlen_host[n] mean edge length at the
   vertex; hop_host[n] mesh edges to the boundary (capped at 8).  Either of the last two
   may be NULL. */
int fl_patches(fl_handle h, double s, int K, int32_t* nbr_host, double* hlen_host, int32_t* hop_host);

typedef struct fl_lp* fl_lp_handle;
/* A network for the mesh's DOFs at order s: K = 12, hidden = 64 (FL_ENOTIMPL otherwise),
   hidden layers seeded (splitmix64 / Box-Muller, variance 1/fan-in), output layer zero
   (the Jacobi preconditioner).  `mesh` must outlive the handle. */
int fl_lp_create(fl_lp_handle* lp, fl_handle mesh, double s, int K, int hidden, uint64_t seed);
/* Sizes of lp (0 for NULL lp): float32 parameters (the layout below), floats per training sample
   row (G = 2K + 3 geometry features and the K + 1 stencil inputs: 40), samples collected so far. */
int64_t fl_lp_num_params(fl_lp_handle lp);
int fl_lp_num_features(fl_lp_handle lp);
int64_t fl_lp_num_samples(fl_lp_handle lp);
/* Parameters [W1 (G x H) | b1 | W2 (H x H) | b2 | W3 (H x (K+1)) | b3], G = 2K + 3, float32 host
   arrays; fl_lp_set_params also recomputes the stencil table. */
int fl_lp_get_params(fl_lp_handle lp, float* host);
int fl_lp_set_params(fl_lp_handle lp, const float* host);
/* Take the diagonal of A (device, float64) as the scale of the preconditioner. */
int fl_lp_bind(fl_lp_handle lp, const double* A_dev, int64_t lda, void* stream);
/* Training-sample rows X_dev[n][F] = [geometry (2K + 3) | residual patch / sigma (K + 1)] and
   sigma_dev[n] of a residual r_dev[n] (float64). */
int fl_lp_features(fl_lp_handle lp, const double* r_dev, float* X_dev, float* sigma_dev, void* stream);
/* Stencil table c [n][K + 1] (host) computed with the float16 network. */
int fl_lp_stencil(fl_lp_handle lp, float* host);
/* z = (M + M^T) r / 2, float64 device vectors. */
int fl_lp_apply(fl_lp_handle lp, const double* r_dev, double* z_dev, void* stream);
/* Loss mean (c(g) . x - t)^2 and its gradient (host, fl_lp_num_params floats) on a batch of
   sample rows X_dev[B][F] and targets T_dev[B] (float32, device). */
int fl_lp_loss_grad(fl_lp_handle lp, int64_t B, const float* X_dev, const float* T_dev, float* loss_host,
                    float* grad_host, void* stream);
/* Training pairs from error vectors E (column c at E_dev + c*lde): r = A e, features of r,
   targets e_i A_ii / sigma_i, appended to the handle's training set. */
int fl_lp_add_pairs(fl_lp_handle lp, const double* A_dev, int64_t lda, const double* E_dev, int64_t lde,
                    int count, void* stream);
/* Pairs from the method's own Jacobi-PCG: u = A^-1 b (to 1e-11), then for each k in ks
   the iterate x_k from 0 and the pair (A (u - x_k), u - x_k). */
int fl_lp_collect(fl_lp_handle lp, const double* A_dev, int64_t lda, const double* b_dev, int nk, const int* ks,
                  void* stream);
/* Pairs from Jacobi-PCG on A x = 0 started at seeded white noise x0 (splitmix64 / Box-Muller
   of (seed + c, i)), c < count: for each k in ks the iterate x_k (k = 0: x0) and the pair
   (A e, e) with the exact error e = -x_k.  For k = 0 the loss is the Frobenius fit of M to
   A^-1 on the stencil pattern; larger k weights the error components CG leaves behind. */
int fl_lp_collect_noise(fl_lp_handle lp, const double* A_dev, int64_t lda, int count, int nk, const int* ks,
                        uint64_t seed, void* stream);
/* Adam (0.9, 0.999, 1e-8) on mini-batches drawn from the training set with splitmix64(seed,
   step, slot); *loss_host = loss of the last batch. */
int fl_lp_train(fl_lp_handle lp, int steps, int64_t batch, float lr, uint64_t seed, float* loss_host, void* stream);
/* The message of lp's last failed call ("" if none or NULL lp); owned by lp. */
const char* fl_lp_last_error(fl_lp_handle lp);
/* Frees lp's device memory after synchronising its device; NULL is a no-op. */
void fl_lp_destroy(fl_lp_handle lp);

typedef struct fl_fcg_info {
    int iterations;
    int fallback_at;           /* iteration at which the fallback preconditioner took over, -1: none */
    int final_preconditioner;  /* 2 learned, 1 multigrid, 0 Jacobi */
    double rel_residual;       /* ||b - A u|| / ||b||, recomputed in float64 at the end */
    int status;
} fl_fcg_info;

/*
 * Flexible CG (one-step orthogonalisation, alpha = p.r / p.Ap) on the float64 matrix,
 * preconditioned by the learned map lp if given, else the multigrid V-cycle mg if
 * given, else Jacobi.  When the learned (or, after it, the multigrid) preconditioner
 * gives a non-descent direction or the residual falls by less than 10 % over 10 steps,
 * the next one in the order learned -> multigrid -> Jacobi takes over and the
 * directions restart.  Converged when the recursive residual meets tol and the
 * float64 residual recomputed at the end agrees.  h supplies the error message.
 */
int fl_fcg_solve(fl_handle h, int64_t n, const double* A_dev, int64_t lda, const double* b_dev, double* u_dev,
                 fl_lp_handle lp, fl_mg_handle mg, double tol, int maxit, fl_fcg_info* info, void* stream);

/* ------------------------------------------------------------------------
 * Autotuning (no counterpart in the paper): launch shapes measured on the
 * running device, kept in a process-wide table keyed by (kernel, n, nrhs,
 * nslices) and the device name, consulted when a launch parameter is left at
 * 0, persisted as JSON.
 * ------------------------------------------------------------------------ */

/*
 * Sweep the pipeline depth (2 .. what shared memory holds) and the CTA count
 * (the SM count and a few smaller grids) of the tensor-core product of
 * fl_batch_solve on these problems' slices (timed with CUDA events, median of
 * `reps` launches after one warm-up, inputs of zero), record the fastest as
 * kernel "batch_gemm" with p0 = stages, p1 = CTAs under key (max n, max nrhs
 * rounded up to 16, max nslices), and return it in *best (other fields at
 * their defaults) and its time in *best_ms.  Only S_dev, n, nslices and nrhs of
 * the problems are used.  Synchronous.  Errors: FL_EINVAL, FL_ENOMEM,
 * FL_ECUDA, FL_ETIMEOUT.
 */
int fl_tune_batch(fl_handle h, int nprob, const fl_batch_problem* probs, int reps, fl_batch_opts* best,
                  double* best_ms);

/* Add or replace a table entry for the current device (p0, p1: the kernel's two parameters). */
/*
 * Autotuner of the dense matvec (fl_matvec's shared-memory-staged products): times the one
 * fl_matvec uses on the caller's matrix (dtype FL_F64: the 8-warp staged product; FL_F32: the
 * 16-warp row-dot product; A aligned to its element size) for 1, 2, ... blocks per SM up to
 * what fits (at most 4 for FL_F32), median of reps CUDA-event timings after a warm-up, on
 * `stream`; records the fastest under ("gemv_smem_f64" | "gemv_rows_f32", n) for this device,
 * which fl_matvec then uses.  x_dev, y_dev: [n] float64 (y is overwritten).  *best_per_sm,
 * *best_ms (host, may be NULL) get the choice.  Errors: FL_EINVAL (bad arguments),
 * FL_ENOTIMPL (the staged product is not used at this size: x too large to stage, or for
 * FL_F64 fewer than two blocks per SM fit), FL_ECUDA.
 */
int fl_tune_matvec(int dtype, const void* A_dev, int64_t lda, int64_t n, const double* x_dev,
                   double* y_dev, int reps, int* best_per_sm, double* best_ms, void* stream);

/* Sets the entry (current device, kernel, n, nrhs, nslices) of the process-wide tuning table to
   (p0, p1, ms), replacing an earlier one.  Thread-safe.  FL_EINVAL for an empty kernel name or n < 1. */
int fl_tune_record(const char* kernel, int64_t n, int nrhs, int nslices, int p0, int p1, double ms);
/* FL_OK and the parameters if the current device has an entry, else FL_ENOTIMPL. */
int fl_tune_lookup(const char* kernel, int64_t n, int nrhs, int nslices, int* p0, int* p1);
/* Empty the table / the number of its entries (all devices). */
void fl_tune_clear(void);
int fl_tune_count(void);
/* Write / merge the table as JSON: {"entries": [{"device", "kernel", "n", "nrhs", "nslices",
   "p0", "p1", "ms"}, ...]}.  FL_EINVAL on I/O or format errors. */
int fl_tune_save(const char* path);
/* Merge a saved table: each entry replaces the one with the same key (device, kernel, n, nrhs,
   nslices).  FL_EINVAL if the file cannot be read or parsed (the table is then unchanged). */
int fl_tune_load(const char* path);

/* ------------------------------------------------------------------------
 * Measurement hooks (no counterpart in the paper): plan statistics, per-stage
 * device times of fl_assemble, and a count of kernel launches.
 * ------------------------------------------------------------------------ */
typedef struct fl_stats {
    int64_t n_cells, n_vertices, n_facets, n_dofs;
    int64_t n_tiles;            /* 32x32 cell tiles of the far-field kernel (upper triangle) */
    int64_t n_touch_pairs;      /* common edge / common vertex pairs with a DOF */
    int64_t n_near_pairs;       /* separated pairs at vertex-graph distance 1 with a DOF */
    int64_t n_far_pairs;        /* remaining unordered separated pairs with a DOF on either side */
    int64_t n_cells_with_dof;
    int64_t nnz_nearfield;      /* nonzeros of the sparse near-field part */
    int64_t h2d_bytes;          /* bytes of planner tables copied host -> device so far */
    int64_t workspace_bytes;    /* device bytes owned by the handle */
} fl_stats;

/* Fill *st for the DOF set of order s (plans it if needed). */
int fl_get_stats(fl_handle h, double s, fl_stats* st);

/* Stages of fl_assemble timed when profiling is on. */
#define FL_STAGE_PREP    0
#define FL_STAGE_FAR     1  /* separated pairs at distance >= 2 (the dominant kernel) */
#define FL_STAGE_NEAR    2
#define FL_STAGE_TOUCH   3
#define FL_STAGE_BND     4  /* element x far boundary facet sums */
#define FL_STAGE_ELEMENT 5
#define FL_STAGE_COMPOSE 6  /* sparse gather + dense compose */
#define FL_NSTAGES       7

/* enable = 1: record a CUDA event pair around every stage of each later fl_assemble
 * on its stream (events only, no synchronisation); the stages then run one after
 * another on that stream, so each pair times one stage alone.  enable = 2: only the far
 * stage (FL_STAGE_FAR) is bracketed, on the caller's stream, and the schedule is left as
 * without profiling (the other stages run beside it on the handle's second stream);
 * fl_stage_ms then reports the far stage and zeros.  enable = 0: off.  Errors: FL_EINVAL. */
int fl_set_profiling(fl_handle h, int enable);

/* Milliseconds of each stage of the last profiled fl_assemble (waits for its events). */
int fl_stage_ms(fl_handle h, double* ms_out /* [FL_NSTAGES] */);

/* Number of kernels this library has launched in the process so far. */
uint64_t fl_launch_count(void);

/*
 * Caching allocator.  Device tables, workspaces and pinned scalars of handles come from a
 * process-wide cache (per device, thread-safe): fl_destroy returns a handle's blocks to it
 * after synchronising the device, and a later handle reuses the smallest cached block of at
 * least the requested size and at most twice it.  When an allocation fails for lack of
 * memory the device's cached blocks are released and the allocation retried.
 * fl_pool_trim releases every cached block (cudaFree / cudaFreeHost) and returns the bytes
 * released; call it only while no handle's work is in flight.  fl_pool_stats reports the
 * cached bytes and the hit / miss counts of all requests (any argument may be NULL).
 */
int64_t fl_pool_trim(void);
void fl_pool_stats(int64_t* cached_device_bytes, int64_t* cached_host_bytes, int64_t* hits, int64_t* misses);

/* ------------------------------------------------------------------------
 * Allocation-free float32 matrix-vector product.  The paper has no counterpart;
 * this is a service for callers that cannot allocate device memory: code that
 * runs under a caller-owned memory budget or inside another allocator's arena,
 * real-time loops that must not enter the driver's allocator, and hosts that only
 * receive device pointers and own no allocator.  fl_matvec(FL_F32, ...) allocates
 * a float32 copy of x on every call; this entry point keeps that copy in a fixed
 * device array of FL_STATIC_MAX_N floats (256 KiB) that every GPU which loads the
 * library holds until the process exits.
 * ------------------------------------------------------------------------ */
#define FL_STATIC_MAX_N 65536

/*
 * y_dev[n] = A_dev x_dev for A_dev float32 (n x n, row-major, lda >= n), x_dev and
 * y_dev float64 device vectors (contiguous).  Same arithmetic as fl_matvec with
 * FL_F32: x rounded to float32, float32 lane sums, float64 row totals.
 * Returns FL_EINVAL for n < 1 or n > FL_STATIC_MAX_N (nothing is launched), for
 * NULL pointers or lda < n; FL_ECUDA if the device array cannot be located, if a
 * CUDA error was already pending on the calling thread when the call began (it is
 * reported, not cleared, and nothing is launched), or if one of the two launches
 * fails.  Calls no allocator.
 * The first call on each device looks up that device's copy of the array
 * (cudaGetSymbolAddress) with the device current and keeps the address for the rest
 * of the process; make that first call before any stream capture.  The kept address
 * does not survive cudaDeviceReset (or any other destruction of the device's
 * primary context): do not call this entry point on a device after resetting it.
 * All calls on a device share the one array and each call
 * rewrites the n entries it reads, so nothing has to be cleared between calls, but
 * calls that overlap on the GPU (different streams, or different host threads)
 * race on it: serialise them.
 */
int fl_matvec_f32_static(const float* A_dev, int64_t lda, int64_t n, const double* x_dev, double* y_dev,
                         void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FRACLAP_H */
