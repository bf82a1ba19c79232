/*
 * gofd.h -- C ABI of the GB300 grid-overlay finite-difference (GoFD) library.
 *
 * The library discretises the homogeneous Dirichlet problem for the
 * fractional Laplacian,
 *     (-Delta)^s u = f in Omega,  u = 0 outside Omega,   s = alpha/2 in (0,1)
 * (Huang & Shen, arXiv 2307.14437, Section 1, eq. (FL-1)) on an unstructured
 * simplicial mesh T_h overlaid by a uniform grid T_FD (Section 3.1).  Its hot
 * path is the stiffness product of the SPD system (GoFD-2),
 *     y = S u,   S = (I_h^FD)^T A_FD I_h^FD       (Section 3.2, eq. (GoFD-2))
 * where I_h^FD is piecewise-linear interpolation from mesh vertices to grid
 * nodes (eq. (IhFD-1)) and A_FD is the multilevel-Toeplitz FD matrix of
 * eqs. (T-1), (A-1), (AFD-1), applied by zero-padded circulant FFT
 * convolution (Section 2.2, eq. (AU-1)).
 *
 * Conventions shared by every call
 *  - Every call returns a gofd_status; nothing is thrown across the ABI.
 *    gofd_last_error() gives a message for the last failure on a handle
 *    (or, with a NULL handle, for the last failed handle-free call of the
 *    thread: gofd_build or gofd_afd_apply_noalloc).
 *  - Host inputs are copied; the caller keeps ownership of everything it
 *    passes.  A gofd_problem owns all of its device memory and frees it in
 *    gofd_destroy().  A handle is not thread safe: serialise calls on it.
 *  - Different handles may be used from different threads at once, with one
 *    restriction: the solvers capture their iterations as CUDA graphs on
 *    first use, and a capture fails if the device is synchronised meanwhile.
 *    gofd_destroy and gofd_group_destroy synchronise the device (they free
 *    device memory), so do not destroy a handle or group on a device while
 *    another thread is inside a solve on that device.
 *  - Device vectors are caller-owned device pointers, used in stream order on
 *    the caller's stream (`stream` is a cudaStream_t cast to void*; NULL is
 *    the legacy default stream).  The library allocates nothing per call on
 *    the device except where a function says so.
 *  - Vertex vectors have N_v entries in the caller's vertex order.  Boundary
 *    vertices (vertices of facets that belong to exactly one simplex) carry
 *    the Dirichlet value 0: their input entries are ignored and their output
 *    entries are written as 0 (Section 3.2, remark on interior unknowns).
 *  - Grid vectors have n_0*n_1*...*n_{d-1} entries, axis 0 fastest; node k has
 *    coordinates x_k = box_lo + k*h (one rounded product, one rounded sum).
 *  - The library runs only on a CUDA GPU of compute capability 10.3 (sm_103a).
 *    There is no CPU fallback: without such a GPU every call that needs the
 *    device returns GOFD_E_CUDA.
 */
#ifndef GOFD_H
#define GOFD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gofd_problem gofd_problem;

typedef enum {
    GOFD_OK = 0,
    GOFD_E_ARG = 1,                 /* invalid argument (NULL pointer, bad size, bad enum)      */
    GOFD_E_DEGENERATE_SIMPLEX = 2,  /* a simplex has zero volume (exact orientation test)        */
    GOFD_E_OUTSIDE_BOX = 3,         /* a mesh vertex lies outside [box_lo, box_hi]                */
    GOFD_E_GRID = 4,                /* (hi-lo)/h is not an integer, or the grid is too large      */
    GOFD_E_TOO_FEW_GRID_NODES = 5,  /* fewer grid nodes than mesh vertices (Remark 3.2)           */
    GOFD_E_ZERO_COLSUM = 6,         /* an interior column sum D_h,j is 0 (Theorem 3.1 hypothesis) */
    GOFD_E_PRECOND = 7,             /* the incomplete Cholesky factorisation broke down           */
    GOFD_E_NOT_CONVERGED = 8,       /* the solver hit maxit before reaching tol                   */
    GOFD_E_TIMEOUT = 9,             /* a bounded device-side wait ran out                          */
    GOFD_E_CUDA = 10,               /* a CUDA runtime error (message in gofd_last_error)          */
    GOFD_E_NOMEM = 11               /* device or host allocation failed                            */
} gofd_status;

/* GOFD_FP64_DF (2D and 3D, gofd_apply_interior only): FP64 inputs and outputs, the
 * gather and scatter in FP64, the FFT convolution in double-float arithmetic
 * (pairs of FP32 numbers, about 48 significant bits): the mixed solver's
 * residual product, within about 1e-13 of the FP64 product. */
typedef enum { GOFD_FP64 = 0, GOFD_FP32 = 1, GOFD_FP64_DF = 2 } gofd_precision;

typedef enum {
    GOFD_SOLVE_FP64 = 0,   /* PCG with FP64 operator, vectors and scalars                      */
    GOFD_SOLVE_MIXED = 1   /* FP64 residual refinement around an FP32-operator PCG (FP64 dots)  */
} gofd_solve_mode;

typedef enum {
    GOFD_OP_STIFFNESS = 0, /* y = S u                       (GoFD-2)                          */
    GOFD_OP_FRACLAP = 1    /* y = h^{-2s} D_h^{-1} S u      (Ah-1): the GoFD fractional Laplacian */
} gofd_op;

typedef enum {
    GOFD_RHS_GRID = 0,     /* f given on the grid (n^d values): b = h^{2s} I^T (f on located nodes), (GoFD-1)/(GoFD-2) */
    GOFD_RHS_VERTEX = 1    /* f given on the vertices (N_v values): b = h^{2s} D_h f, (GoFD-3)                    */
} gofd_rhs;

typedef struct {
    int precond;               /* 0: none; 5 or 9 (2D), 7 or 27 (3D), 3 (1D): IC(ic_level) of I^T A_FD^(k) I (Ah-4);
                                  1: the diagonal of S itself (Jacobi scaling; not in the paper, pays on graded
                                  meshes where the diagonal spans orders of magnitude);
                                  2 (2D): the circulant alternative of Section 3.3 (gofd_precond_apply)             */
    int ic_level;              /* level of fill of the incomplete Cholesky factor (paper: 1)                        */
    int64_t filon_M;           /* finest Filon panel count M; 0 = paper default (2^14 in 1D/2D, 2^11 in 3D), raised
                                  so that the coarsest Richardson level keeps M/2^(levels-1) >= n                      */
    int richardson_levels;     /* Filon levels M, M/2, ...; 0 = 4                                                     */
    uint64_t wait_budget_cycles; /* bound on one device-side wait (clock64 cycles); 0 = 2e9.  The persistent IC
                                    triangular solves (ic_solve = 0) wait on the rows a row depends on; a wait that
                                    runs out ends the solve and the call reports GOFD_E_TIMEOUT                    */
    double inner_tol;          /* mixed mode: relative reduction of each inner FP32 PCG (0 = 1e-4); a round that
                                  needs less (residual near tol) asks for half the remaining factor              */
    int check_every;           /* iterations between convergence checks (on the device); 0 = 8                      */
    int ordering;              /* IC unknown order: 0 natural vertex order, 1 multicolour (shorter dependency chains)  */
    int chunk_planes;          /* 3D: spectrum planes k_x0 per chunk of the axis-1/axis-2 stage; 0 = as many as fit a
                                  1 GiB middle buffer.  Bounds memory; results do not depend on it                    */
    int fp64_residual;         /* mixed mode, the FP64 residual b - S x of each refinement step: 0 = its convolution
                                  in double-float arithmetic in 2D and 3D (gather and scatter in FP64; FP64 in 1D),
                                  1 = plain FP64 throughout.  FP64 mode always uses plain FP64                     */
    int ic_solve;              /* IC triangular solves: 0 = one persistent launch per solve (rows claimed in level
                                  order, bounded per-row waits), 1 = one launch per level                           */
} gofd_options;

typedef struct {
    int outer_iters;           /* refinement steps (mixed) or 1 (fp64)                                   */
    int inner_iters;           /* total PCG iterations                                                   */
    double rel_res_fp64;       /* final ||b - S u||_2 / ||b||_2 with the FP64 operator                   */
    double ic_shift;           /* diagonal shift used by the IC factorisation (0 if none was needed)     */
    double a_h;                /* minimum element height                                                 */
    double min_colsum;         /* min over interior vertices of D_h,j                                    */
    int h_within_strict_bound; /* h <= a_h / ((d+1) sqrt(d))  (eq. (hFD-1))                               */
    int h_within_practical_bound; /* h <= a_h  (Remark 3.5)                                              */
    double t_setup_ms;         /* gofd_build wall time                                                   */
    double t_solve_ms;         /* this solve's wall time                                                 */
    int device_loop;           /* 1: the PCG iterations ran as a device-side CUDA graph loop, 0: host loop */
} gofd_solve_info;

typedef struct {
    int d;                     /* dimension 1..3                                         */
    int n[3];                  /* grid nodes per axis                                    */
    int P;                     /* circulant length per axis (power of two >= 2n-2)      */
    int64_t n_v, n_e;          /* mesh vertices, simplices                               */
    int64_t n_interior;        /* interior vertices (unknowns)                           */
    int64_t n_grid;            /* grid nodes                                             */
    int64_t n_loc;             /* located grid nodes (rows of the ELL form of I_h^FD)     */
    int64_t nnz_t;             /* stored entries of I^T over interior vertices           */
    int64_t n_runs;            /* runs of consecutive located nodes along axis 0         */
    int64_t filon_M;           /* finest Filon M used                                    */
    int richardson_levels;
    double alpha, s, h;
    double a_h, min_colsum;
    int64_t precond_nnz;       /* stored entries of the IC factor (0 without preconditioner) */
    int precond_levels;        /* dependency levels of the IC factor (the triangular solves' chain)   */
    double ic_shift;
    double t_setup_ms;
    int tune_lines_per_cta;    /* launch shapes in use (0 = built-in default; set by gofd_autotune):   */
    int tune_cols_per_cta;     /*   grid lines per CTA of the row FFTs, columns per CTA of the column */
    int tune_scatter_lanes;    /*   FFTs, lanes per row of the I^T scatter,                           */
    int tune_col_elems;        /*   elements per thread of the column FFTs,                           */
    int tune_batch_chunk;      /*   columns per sub-batch of the 2D batched product (0 = all),        */
    int tune_row_elems;        /*   elements per thread of the 2D row / 3D axis-1 FFTs (FP32)         */
    int warp_fft_path;         /* 1: the 2D FP32 product runs the one-warp-per-1024-point-FFT kernels
                                  (circulant 2048, default launch shapes); 0: the general kernels      */
} gofd_info;

/*
 * gofd_build -- set up the discrete problem (Sections 2.3, 3.1, 3.3).
 *   d            dimension, 1..3
 *   vertices     host, N_v*d doubles, row-major (vertex j at vertices[j*d .. j*d+d-1])
 *   simplices    host, N_e*(d+1) int32, 0-based vertex indices; either orientation
 *   alpha        = 2s, 0 < alpha < 2 (alpha = 2 is accepted: the standard Laplacian)
 *   h            overlay spacing h_FD > 0
 *   box_lo/hi    host, d doubles each; (hi_i-lo_i)/h must be an integer (1e-9 rel.)
 *   opt          options or NULL for defaults
 *   out          receives the new handle (NULL on failure)
 * Work done on the device: exact point location of every grid node (lowest
 * element index wins on shared facets), the ELL form of I_h^FD, boundary
 * detection and interior numbering, the transpose I^T, column sums D_h,
 * element heights and a_h, the FD coefficients T by Filon quadrature with
 * Richardson extrapolation (Section 2.3), the circulant symbol (Section 2.2),
 * and, if requested, the IC preconditioner (Section 3.3).
 * Grid limits: the same node count n on every axis, n <= 4097 in 1D and
 * 2D, n <= 513 in 3D (circulant length P <= 8192, resp. 1024); beyond them
 * GOFD_E_GRID.
 * Errors: GOFD_E_ARG, _DEGENERATE_SIMPLEX, _OUTSIDE_BOX, _GRID,
 * _TOO_FEW_GRID_NODES, _ZERO_COLSUM, _PRECOND, _CUDA, _NOMEM.
 */
gofd_status gofd_build(int d, const double* vertices, int64_t n_v,
                       const int32_t* simplices, int64_t n_e,
                       double alpha, double h,
                       const double* box_lo, const double* box_hi,
                       const gofd_options* opt, gofd_problem** out);

/*
 * gofd_apply -- y = S u (GOFD_OP_STIFFNESS, eq. (GoFD-2)) or
 * y = h^{-2s} D_h^{-1} S u (GOFD_OP_FRACLAP, eq. (Ah-1)).
 *   u_dev, y_dev  device, N_v values of double (GOFD_FP64) or float (GOFD_FP32);
 *                 they must not overlap.  The precision selects the arithmetic of
 *                 the gather, FFT convolution and scatter.
 * Boundary entries of u are ignored; boundary entries of y are set to 0.
 */
gofd_status gofd_apply(gofd_problem* p, gofd_op op, gofd_precision prec,
                       const void* u_dev, void* y_dev, void* stream);

/*
 * gofd_precond_apply -- z = M^{-1} r with the handle's preconditioner on
 * interior-compacted device vectors (r_dev: N_int+1 values, the last one 0;
 * z_dev receives N_int values and a 0 in slot N_int; r and z must differ).
 * The solver applies the same operator every PCG iteration.  For the
 * circulant preconditioner (precond = 2, 2D; Section 3.3 names circulant
 * preconditioners of A_FD as an alternative to its sparse ones):
 *   M^{-1} = D_h^{-1} I^T C^{-1} I D_h^{-1},
 * C the 2n-periodic circulant embedding of A_FD (symbol 1/lambda), one
 * stiffness product with the inverse symbol between two diagonal scalings.
 * GOFD_E_ARG if the problem was built without a preconditioner.  With the
 * IC factor's persistent solves (ic_solve = 0) the call synchronises the
 * stream and returns GOFD_E_TIMEOUT if a wait ran out (z is then undefined);
 * the other preconditioners only enqueue.
 */
gofd_status gofd_precond_apply(gofd_problem* p, gofd_precision prec, const void* r_dev, void* z_dev,
                               void* stream);

/*
 * gofd_apply_host -- gofd_apply on host buffers (N_v values each), and
 * synchronises the stream.  Pinned host buffers (cudaHostAlloc /
 * cudaMallocHost, or registered) are mapped into the device's address space:
 * the kernels read u and write y there directly.  Pageable buffers are
 * copied through two N_v device staging vectors that the first such call
 * allocates and the handle keeps.
 */
gofd_status gofd_apply_host(gofd_problem* p, gofd_op op, gofd_precision prec,
                            const void* u_host, void* y_host, void* stream);

/*
 * gofd_apply_interior -- the operator on interior-compacted device vectors:
 * x_dev holds N_int+1 values (interior unknowns in vertex order, then one
 * slot that must be 0), y_dev receives N_int values of S x.  This is the
 * product the solver iterates; it does no compaction.
 */
gofd_status gofd_apply_interior(gofd_problem* p, gofd_precision prec,
                                const void* x_dev, void* y_dev, void* stream);

/*
 * gofd_apply_interior_batch -- gofd_apply_interior on nb columns at once:
 * column c of x at x_dev + c*ld (N_int+1 values, the last one 0), of y at
 * y_dev + c*ld (N_int values written); ld >= N_int+1, x and y must not
 * overlap.  In 2D the product kernels run over all columns in one launch
 * each; other dimensions loop over the columns.  Results equal nb calls of
 * gofd_apply_interior.  Allocates the batch workspace (see gofd_solve_batch)
 * on first use.
 */
gofd_status gofd_apply_interior_batch(gofd_problem* p, gofd_precision prec, int nb, const void* x_dev,
                                      int64_t ld, void* y_dev, void* stream);

/*
 * gofd_apply_interior_profiled -- gofd_apply_interior with a CUDA event
 * recorded on `stream` after each kernel of the product; on return (the
 * stream is synchronised) stage_ms[i] holds the time of stage i in ms and
 * stage_names[i] (if stage_names is not NULL) a static name; *n_stages is the
 * number of stages written (at most cap; the first 32 kernels of a product are
 * marked).  One stage per kernel launch, so *n_stages counts the launches of a
 * product of up to 32 kernels.  For measurement only.
 */
gofd_status gofd_apply_interior_profiled(gofd_problem* p, gofd_precision prec, const void* x_dev,
                                         void* y_dev, void* stream, float* stage_ms,
                                         const char** stage_names, int cap, int* n_stages);

/*
 * gofd_solve -- solve (GoFD-2) S u = b for the interior unknowns.
 *   mode    GOFD_SOLVE_FP64 or GOFD_SOLVE_MIXED
 *   rhs     GOFD_RHS_GRID: f_dev holds n_grid doubles (values off the mesh are ignored);
 *           GOFD_RHS_VERTEX: f_dev holds N_v doubles
 *   tol     stop when ||b - S u||_2 <= tol ||b||_2 (FP64 operator)
 *   maxit   bound on the total number of PCG iterations
 *   u_dev   device, N_v doubles: initial guess on entry (ignored if init_zero),
 *           the solution on exit with boundary entries 0
 *   info    optional (may be NULL)
 * The solve runs on a stream of the handle, after the caller's pending work
 * on `stream`, and the caller's stream waits for it; the call returns when
 * the solve is done.  Each inner PCG runs as one CUDA graph launch: a
 * device-side loop whose control kernel tests the residual every
 * check_every iterations (info->device_loop says whether it was used).
 * Returns GOFD_E_NOT_CONVERGED (with u holding the last iterate) if maxit is
 * reached or the residual becomes non-finite, GOFD_E_ARG if the right-hand
 * side b (from the entries of f that reach it) or the initial guess has a
 * NaN or Inf, GOFD_E_TIMEOUT (u undefined) if a wait of the IC factor's
 * persistent triangular solves ran out of wait_budget_cycles.
 */
gofd_status gofd_solve(gofd_problem* p, gofd_solve_mode mode, gofd_rhs rhs,
                       const double* f_dev, double tol, int maxit, int init_zero,
                       double* u_dev, gofd_solve_info* info, void* stream);

/*
 * gofd_adjoint -- gradients of a loss L(u) through the solve with vertex data
 * (GoFD-3), u = S(X)^{-1} h^{2s} D_h(X) f, for the data f and the mesh vertex
 * coordinates X (the owner simplex of every grid node held fixed).
 *   f_dev      device, N_v doubles: the vertex data of the forward solve
 *   u_dev      device, N_v doubles: its solution (boundary entries are taken as 0)
 *   g_dev      device, N_v doubles: dL/du (boundary entries ignored)
 *   tol, maxit the adjoint solve S lambda = g (same modes as gofd_solve)
 *   grad_f_dev device, N_v doubles: dL/df = h^{2s} D_h lambda (0 on the boundary)
 *   grad_x_dev device, N_v*d doubles (row-major like the vertices): dL/dX
 * The adjoint state is one more solve; no iterate of the forward solve is
 * stored.  The first call allocates a vertex-major transpose of I_h^FD and
 * two grid vectors that the handle keeps.  The paper has no adjoint; this
 * differentiates its discrete system (Section 3.2).
 */
gofd_status gofd_adjoint(gofd_problem* p, gofd_solve_mode mode, const double* f_dev, const double* u_dev,
                         const double* g_dev, double tol, int maxit, double* grad_f_dev,
                         double* grad_x_dev, gofd_solve_info* info, void* stream);

/*
 * gofd_solve_batch -- solve (GoFD-2) S u_c = b_c for nb right-hand sides on
 * one mesh and grid, in lock step (block PCG: one batched product of S per
 * iteration for all columns, per-column scalars and stopping).
 *   f_dev   device, column c at f_dev + c*ldf (ldf >= n_grid for
 *           GOFD_RHS_GRID, >= N_v for GOFD_RHS_VERTEX)
 *   u_dev   device, N_v*nb doubles, column c at u_dev + c*N_v; the solutions
 *           (boundary entries 0).  Always started from zero.
 *   infos   optional, nb entries (iteration counts are those of the columns'
 *           active rounds; t_solve_ms is the batch's wall time)
 * Every column meets ||b_c - S u_c|| <= tol ||b_c|| with the FP64 operator,
 * else GOFD_E_NOT_CONVERGED (also when a residual becomes non-finite); a
 * column b_c with a NaN or Inf gives GOFD_E_ARG; GOFD_E_TIMEOUT as gofd_solve.
 * Allocates on the first call (or a larger nb)
 * about (12 n_int + n_grid) * 8 bytes per column, plus (2D) a batch spectrum
 * of (P/2+1) * round16(n) complex per column, and keeps it in the handle.
 * The paper solves one right-hand side at a time; the batch is ours (many
 * data f on one mesh share every set-up product).
 */
gofd_status gofd_solve_batch(gofd_problem* p, gofd_solve_mode mode, gofd_rhs rhs, int nb,
                             const double* f_dev, int64_t ldf, double tol, int maxit,
                             double* u_dev, gofd_solve_info* infos, void* stream);

/*
 * Groups -- several 2D problems (meshes, alpha) on ONE overlay grid (same box
 * and h, hence the same n and circulant), each with nb right-hand sides,
 * solved together: the np*nb columns advance in lock step through one block
 * PCG (per-column scalars and convergence, as gofd_solve_batch), whose
 * iterations run as one CUDA graph launch with a device-side loop; every
 * product kernel covers the columns of all problems in one launch, each
 * column taking its problem's ELL, runs, symbol and I^T from a device table.
 * Problems with equal alpha, Filon M and Richardson levels share one symbol.
 * The paper has no counterpart: this is the batching of many instances.
 *
 * gofd_group_create -- np >= 1 problems (each 2D, all on one grid and one
 *   device; they must outlive the group), nb >= 1 columns each.  Allocates the
 *   group's workspace: 12 vectors of the largest N_int + 1 per column, one
 *   grid vector and one half spectrum per column (FP64 size).  GOFD_E_ARG if
 *   the problems do not share a grid.  The launch shapes are those of the
 *   first problem (gofd_group_autotune tunes them on the whole group).
 * gofd_group_autotune -- gofd_autotune for the group's product of np*nb
 *   columns; sets the first problem's launch shapes.  *best_ms may be NULL.
 * gofd_group_solve -- f_dev[i] (device, np pointers in a host array): the nb
 *   columns of problem i at f_dev[i] + c*ldf[i] (n_grid doubles each for grid
 *   data, N_v of problem i for vertex data); u_dev[i] receives nb x N_v(i)
 *   doubles, row-major.  infos: np*nb entries, column c of problem i at
 *   i*nb + c (may be NULL).  Modes, tolerance and errors as gofd_solve_batch.
 *   Synchronises `stream`.  Messages go to gofd_last_error(NULL).
 * gofd_group_destroy -- free the group (NULL is a no-op); the problems stay.
 */
typedef struct gofd_group gofd_group;
gofd_status gofd_group_create(int np, gofd_problem* const* problems, int nb, gofd_group** out);
gofd_status gofd_group_autotune(gofd_group* g, void* stream, double* best_ms);
gofd_status gofd_group_solve(gofd_group* g, gofd_solve_mode mode, gofd_rhs rhs, const double* const* f_dev,
                             const int64_t* ldf, double tol, int maxit, double* const* u_dev,
                             gofd_solve_info* infos, void* stream);
void gofd_group_destroy(gofd_group* g);

/*
 * gofd_autotune -- time the batched FP32 product with nb columns for each
 * launch shape (elements per thread of the column FFTs and of the 2D row /
 * 3D axis-1 FFTs, grid lines per CTA in the row FFTs, columns per CTA in the column
 * FFTs, lanes per row in the scatter; one choice at a time with the others
 * at their best so far) and
 * keep the fastest in the handle for all later products; with nb > 1 in 2D
 * also the number of columns per sub-batch of the batched product.  *best_ms (may be
 * NULL) receives its time per product of nb columns.  CTA shapes leave every
 * result bit unchanged; the elements per thread of the FFTs (their radix
 * plans) and the scatter's lanes per row change the rounding order, so
 * products may differ in the last bits between choices (each choice is
 * reproducible run to run).  Uses the batch workspace of gofd_solve_batch
 * and drops the solvers' captured CUDA graphs.
 */
gofd_status gofd_autotune(gofd_problem* p, int nb, void* stream, double* best_ms);

/*
 * gofd_set_launch_shapes -- set the launch shapes gofd_autotune chooses
 * from, e.g. to reuse a tuned set on a new handle or to test one shape.
 * Each argument is 0 (the built-in default) or one of:
 *   lines_per_cta  1, 2, 4        grid lines per CTA of the 2D row FFTs
 *   cols_per_cta   1, 2, 4        spectrum columns per CTA of the 2D column FFTs
 *   scatter_lanes  4, 8, 16, 32   lanes per row of the I^T scatter
 *   col_elems      8, 16, 32      elements per thread of the column (2D) / axis-2 (3D) FFTs
 *   row_elems      8, 16          elements per thread of the 2D row / 3D axis-1 FFTs
 *   batch_chunk    >= 0           columns per sub-batch of the 2D batched product
 * A value that does not apply to the problem's sizes or precision is
 * replaced by the default at launch (as for tuned values).  Any other value:
 * GOFD_E_ARG and nothing changes.  Drops the solvers' captured CUDA graphs.
 * gofd_get_info reports the shapes in use.
 */
gofd_status gofd_set_launch_shapes(gofd_problem* p, int lines_per_cta, int cols_per_cta, int scatter_lanes,
                                   int col_elems, int row_elems, int batch_chunk);

/* gofd_get_info -- sizes and set-up results (host struct). */
gofd_status gofd_get_info(const gofd_problem* p, gofd_info* info);

/*
 * gofd_export_transfer -- the canonical ELL form of I_h^FD, copied to host:
 *   owner    n_grid int32: owner simplex of each grid node, or -1
 *   ell_idx  (d+1)*n_loc int32, slot-major: slot a of located node r (rows in
 *            increasing grid index) is ell_idx[a*n_loc + r] = simplices[owner][a]
 *   ell_w    (d+1)*n_loc doubles, same layout: phi of that vertex at the node
 * Any output pointer may be NULL.
 */
gofd_status gofd_export_transfer(const gofd_problem* p, int32_t* owner,
                                 int32_t* ell_idx, double* ell_w);

/*
 * gofd_export_vertex_data -- per-vertex set-up results, copied to host:
 *   interior_index  N_v int32: index among the unknowns, or -1 on the boundary
 *   colsum          N_v doubles: D_h,j for interior vertices (0 on the boundary)
 */
gofd_status gofd_export_vertex_data(const gofd_problem* p, int32_t* interior_index,
                                    double* colsum);

/*
 * gofd_export_precond -- the incomplete Cholesky factor L (L L^T ~ P A_h^(k) P^T,
 * Section 3.3) copied to host: perm (n_interior int32, perm[new] = old interior
 * index), lptr (n_interior+1 int32), lcol/lval (precond_nnz entries; columns
 * ascending, the diagonal last in each row).  Any pointer may be NULL.
 * GOFD_E_ARG if the problem was built without a preconditioner.  With the
 * IC factor's persistent solves (ic_solve = 0) the call synchronises the
 * stream and returns GOFD_E_TIMEOUT if a wait ran out (z is then undefined);
 * the other preconditioners only enqueue.
 */
gofd_status gofd_export_precond(const gofd_problem* p, int32_t* perm, int32_t* lptr, int32_t* lcol,
                                double* lval);

/*
 * gofd_export_diagonal -- the diagonal of S over the interior unknowns
 * (n_interior doubles, host), S_jj = sum over the grid nodes k, m of the
 * support of phi_j of phi_j(x_k) T_{|k-m|} phi_j(x_m) (products in FP32, sums
 * in FP64).  Available when the problem was built with precond = 1
 * (GOFD_E_ARG otherwise).  Not in the paper.
 */
gofd_status gofd_export_diagonal(const gofd_problem* p, double* diag);

/* gofd_get_coefficients -- T_p for p in [0,n)^d (FP64, axis 0 fastest), to host. */
gofd_status gofd_get_coefficients(const gofd_problem* p, double* T);

/* gofd_get_symbol -- the real circulant symbol on [0,P/2]^d (FP64, unscaled), to host. */
gofd_status gofd_get_symbol(const gofd_problem* p, double* lambda);

/*
 * gofd_afd_apply -- w = A_FD v on the grid (device, n_grid values each, no
 * overlap), by the library's FFT convolution (Section 2.2).
 */
gofd_status gofd_afd_apply(gofd_problem* p, gofd_precision prec,
                           const void* v_dev, void* w_dev, void* stream);

/*
 * gofd_afd_apply_noalloc -- w = A_FD v in FP32 on an n^d grid (d = 1..3)
 * without allocating any memory.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc at the moment they
 * need the product: plug-ins inside a framework that owns all device memory
 * through its own allocator (a cudaMalloc behind its back can fail or break
 * its accounting), real-time loops that must not risk an allocation failure
 * or its latency, and code whose device memory is fixed up front.
 *   d, n        grid dimension and nodes per axis (no handle is needed)
 *   lambda_dev  device, (P/2+1)^d floats, axis 0 fastest: the real circulant
 *               symbol divided by P^d, lambda_k / P^d for k in [0, P/2]^d, with
 *               P = max(32, smallest power of two >= 2n-2); gofd_get_symbol
 *               returns lambda_k (unscaled, FP64) for a built problem
 *   v_dev       device, n^d floats (input grid vector)
 *   w_dev       device, n^d floats (output), must not overlap v_dev
 * The spectrum scratch is a file-scope device array of 1,064,960 complex
 * floats (8.1 MiB, plus 32 KiB of twiddle tables, one per circulant length
 * from 32 to 2048) that every GPU loading the library holds until the process
 * exits.  A grid whose spectrum does not fit
 * (a 2D grid needs n*pitch, a 3D grid n^2*pitch + n*P*pitch complex values,
 * pitch = P/2+1 rounded up to a multiple of 16; so 2D n <= 1024) is rejected
 * with GOFD_E_ARG before any device work.  The first call on each device
 * looks up the arrays' device addresses (cudaGetSymbolAddress), raises the
 * kernels' shared-memory limit and fills the twiddle tables (one launch on
 * `stream`, then a wait for that stream), so make that first call before any
 * stream capture.  Every call uses the same array and it keeps the last call's
 * contents; calls that overlap on the GPU (several streams or threads) race
 * and give wrong results.  No cudaMalloc, cudaFree or allocating library
 * routine is called.  Messages go to gofd_last_error(NULL).
 */
gofd_status gofd_afd_apply_noalloc(int d, int n, const float* lambda_dev, const float* v_dev,
                                   float* w_dev, void* stream);

/*
 * gofd_fma_rates -- measured fused multiply-add throughput of the current
 * device in GFLOP/s (2 flops per FMA), FP64 and FP32 (either pointer may be
 * NULL): independent FMA chains on every SM, timed with CUDA events on
 * `stream` (synchronised).  A measurement utility with no counterpart in the
 * paper: the FP64 product is bound by FP64 arithmetic, and its roofline
 * needs this peak.  Takes about a tenth of a second.
 */
gofd_status gofd_fma_rates(void* stream, double* fp64_gflops, double* fp32_gflops);

/* gofd_destroy -- free the handle and all of its device memory (NULL is a no-op). */
void gofd_destroy(gofd_problem* p);

/* gofd_last_error -- message of the last failure (never NULL). */
const char* gofd_last_error(const gofd_problem* p);

#ifdef __cplusplus
}
#endif

#endif /* GOFD_H */
