/*
 * air.h -- C ABI of the GB300 AIR-preconditioned GMRES library (libair.so).
 *
 * Solves the block-scaled, statically condensed space-time HDG trace system
 *     A x = b,   A = D_b^{-1} S,  b = D_b^{-1} H
 * (arXiv:2010.11130, Section 2.5 eq. systemLambda with the facet
 * block-diagonal left scaling of the Section 4 solver settings) by GMRES
 * accelerated with l-AIR algebraic multigrid (Section 3).
 *
 * Conventions for every entry point:
 *  - Matrices are CSR: row_ptr int64 [n_rows+1] (row_ptr[0] = 0), col int32
 *    [nnz] strictly ascending within each row, val float64 [nnz].  Square,
 *    with a stored nonzero diagonal in every row.
 *  - Vectors are float64.  "Device" pointers are CUDA global memory of the
 *    current device; "host" pointers are ordinary (preferably pinned) memory.
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  All work is ordered on that stream.
 *  - The caller owns every pointer it passes.  The library owns the
 *    hierarchy and its workspace and frees them in air_free.
 *  - Every function returns a status (AIR_OK = 0, > 0 informational,
 *    < 0 error).  Nothing throws across the ABI and nothing is printed.
 */
#ifndef AIR_H
#define AIR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define AIR_OK                    0
#define AIR_NOT_CONVERGED         1   /* solve stopped at max_iter; info filled in */
#define AIR_ERR_INVALID_ARG      -1   /* NULL pointer, bad size or option */
#define AIR_ERR_CSR_MALFORMED    -2   /* unsorted/out-of-range column, missing or zero
                                         diagonal, non-finite value, bad row_ptr */
#define AIR_ERR_OOM              -3   /* device allocation failed */
#define AIR_ERR_CUDA             -4   /* a CUDA runtime call failed */
#define AIR_ERR_SINGULAR_COARSE  -5   /* coarsest operator singular to working precision */
#define AIR_ERR_DEVICE_TIMEOUT   -6   /* a bounded device loop hit its iteration cap */
#define AIR_ERR_COARSE_TOO_LARGE -7   /* coarsening stalled above max_dense rows */
#define AIR_ERR_UNSUPPORTED      -8   /* option value not implemented on the GPU path */
#define AIR_ERR_NOALLOC_LIMIT    -9   /* problem too large for the fixed workspace of
                                         air_gmres_solve_noalloc */

/* precision in which the hierarchy is stored and the V-cycle is applied */
#define AIR_PREC_F64  0
#define AIR_PREC_F32  1
#define AIR_PREC_BF16 2   /* off-diagonal values of A_l and R_l in BF16, diagonals and vectors FP32 */

typedef struct {
    int64_t n_rows, n_cols, nnz;
    const int64_t *row_ptr;
    const int32_t *col;
    const double *val;
    int on_device;       /* 1: the three arrays are device pointers, 0: host pointers */
} air_csr;

typedef struct {
    double theta;        /* classical strength threshold (Section 4: 0.3 for R, 0.2 for C/F) */
    int distance;        /* l-AIR neighbourhood distance (Section 4: 1); 1 or 2 on the GPU */
    char relax[16];      /* relaxation sweeps after the interpolation, one per character: 'F', 'C',
                            'A' a Jacobi sweep over the F, C or all points ("FCF" by default); 'f',
                            'c', 'a' a forward Gauss-Seidel sweep (ascending point order, the
                            values already updated; Section 4 post-relaxes with "fa") over the
                            same sets, level-scheduled (FP64 and FP32 hierarchies; the many
                            right-hand-side calls take 'F' and 'C' only) */
    double omega;        /* Jacobi weight */
    int max_coarse;      /* stop coarsening at or below this many rows */
    int max_levels;      /* hard cap on levels (<= 32) */
    int max_dense;       /* largest coarsest level inverted densely */
    int precision;       /* AIR_PREC_F64, AIR_PREC_F32 or AIR_PREC_BF16 */
    int restart;         /* GMRES restart length m (<= 32) */
    int max_iter;        /* total inner GMRES steps */
    int validate;        /* 1: check the CSR before setup (one extra pass) */
    double theta_r;      /* strength threshold of R's l-AIR neighbourhoods; < 0: theta (Section 4
                            uses 0.3 for R with 0.2 for the coarsening) */
    int falgout_block;   /* 0: C/F splitting by the first pass of Ruge-Stueben over the whole level
                            (default); a multiple of 1024 up to 8192: Falgout-style splitting
                            (Section 4 names Falgout coarsening): the first pass runs in every
                            block of that many consecutive points at once, on the strength graph
                            restricted to the block, and interface points left F without a strong
                            C point are fixed by rounds of a parallel independent set (weight
                            |S^T_i| plus a SplitMix64 fraction of i) */
    int block_size;      /* 0: every level stored entry by entry; b in {2, 3, 4, 6, 10}: when every
                            row of the finest operator is whole aligned b-blocks of consecutive
                            columns plus at most its diagonal (the facet blocks of the trace
                            system), its relaxation sweeps and the Krylov matrix products use a
                            block form (one column index per block, the block's values read as
                            runs); otherwise, or for other b, the entry form */
    int autotune;        /* lanes per row of the entry-form sweeps and restriction on each level:
                            0: by a rule on the stored row width; 1: the fastest of 1, 2, 4, ..., 32
                            lanes, timed with CUDA events at the end of air_setup (about a hundred
                            launches; the choice can differ between runs, and the V-cycle's
                            results with it in the last bits) */
} air_options;

typedef struct {
    int iters;           /* total inner GMRES steps */
    int restarts;        /* completed restart cycles */
    int vcycles;         /* preconditioner applications */
    int status;          /* AIR_OK or AIR_NOT_CONVERGED */
    double relres;       /* final true relative residual ||b - A x|| / ||b|| */
} air_solve_info;

typedef struct {
    int64_t n, nnz;      /* rows and stored entries of A_l */
    int64_t nnz_s;       /* strength graph entries (0 on the coarsest level) */
    int64_t nc;          /* C points = rows of A_{l+1} (0 on the coarsest level) */
    int64_t nnz_r;       /* entries of R_l */
    int64_t n_singular;  /* l-AIR local systems treated as singular (injection rows) */
    int32_t max_m;       /* largest l-AIR local system */
    int32_t coarsest;    /* 1 on the last level */
    int32_t block_size;  /* b when the level's relaxation uses the block form, else 0 */
    int32_t lanes_f;     /* lanes per row of the F sweep, the C sweep and the restriction */
    int32_t lanes_c;     /* (entry form; 1 = one thread per row) */
    int32_t lanes_r;
} air_level_info;

typedef struct air_hierarchy air_hierarchy;   /* opaque, library-owned */

/* Fill *opt with the defaults: theta 0.25, distance 1, relax "FCF", omega 1,
 * max_coarse 1000, max_levels 25, max_dense 4096, AIR_PREC_F64, restart 30,
 * max_iter 1000, validate 1, theta_r -1 (same as theta), falgout_block 0, block_size 0,
 * autotune 0. */
void air_default_options(air_options *opt);

/* Build the l-AIR hierarchy of A (Section 3; Section 4 solver settings):
 * classical strength of connection, first-pass Ruge-Stueben C/F splitting,
 * restriction R ~ R_ideal = [-A_cf A_ff^{-1}, I] from one dense local solve
 * per C point over its distance-1 or distance-2 neighbourhood of strongly
 * connected F points (at most 2048 points at distance 2, else UNSUPPORTED),
 * one-point interpolation P = [W; I],
 * Galerkin A_c = R A P;
 * repeated until max_coarse, then the coarsest operator is inverted densely.
 * theta and distance override the fields of opt (opt may be NULL for the
 * defaults).  If A is on the device and precision is F64, the hierarchy keeps
 * A's pointers as its finest level: the caller must keep A alive and
 * unchanged until air_free.  A host A is copied to the device.
 * Synchronises the stream (level sizes are read back).
 * Errors: INVALID_ARG, CSR_MALFORMED (validate = 1), OOM, CUDA,
 * DEVICE_TIMEOUT, COARSE_TOO_LARGE, SINGULAR_COARSE, UNSUPPORTED. */
int air_setup(const air_csr *A, double theta, int distance, const air_options *opt,
              void *stream, air_hierarchy **out);

/* One V-cycle x = M^{-1} b (Section 3, x <- x + P (RAP)^{-1} R r, applied
 * recursively from a zero guess, followed by the relax sweeps).  b and x are
 * device float64 vectors of length n; an F32 or BF16 hierarchy converts
 * at the finest level.  The first call captures the V-cycle into a CUDA
 * graph (replayed by later calls).  Asynchronous on stream. */
int air_vcycle(const air_hierarchy *H, const double *b, double *x, void *stream);

/* y = A x for device CSR A and device vectors.  Asynchronous. */
int air_spmv(const air_csr *A, const double *x, double *y, void *stream);

/* y = A x with the FP64 copy of the finest operator that the hierarchy keeps
 * for the Krylov solves (the block layout when opt->block_size was set, else
 * SELL-32): the matrix product inside air_gmres_solve (Section 5.1).  x and y
 * are device float64 vectors of length n, distinct.  Asynchronous on stream.
 * INVALID_ARG for a NULL argument. */
int air_hierarchy_spmv(const air_hierarchy *H, const double *x, double *y, void *stream);

/* BiCGSTAB preconditioned on the right by one V-cycle of H (van der Vorst,
 * 1992): the Krylov method of the paper's experiments (Section 5.1, Table 2,
 * stopping at relative residual 1e-12).  x0 = 0, shadow residual r0 = b.  It
 * stops when the recursive residual and then the true residual ||b - A x|| /
 * ||b|| are <= rtol; a true residual above rtol restarts the iteration from
 * it.  A breakdown ((r^, r) = 0, (r^, v) = 0) or omega = 0 ends it.  Same
 * arguments, buffers, ownership and status as air_gmres_solve; info->iters
 * counts BiCGSTAB iterations (two V-cycles each), info->restarts the
 * restarts from the true residual.  Synchronises the stream four times per
 * iteration (the scalar recurrence runs on the host). */
int air_bicgstab_solve(const air_csr *A, const air_hierarchy *H, const double *b, double *x, double rtol,
                       void *stream, air_solve_info *info);

/* Many right-hand sides through one hierarchy.  b and x are device arrays
 * of n x k doubles, row-major (the k values of row i are contiguous), k in
 * 1 .. 32.  The matrix traffic of a V-cycle is shared by the k systems: one
 * warp per matrix row, one lane per system.
 *
 * air_vcycle_multi: x = M^{-1} b column by column, the FP64 V-cycle of H
 * (whatever H's storage precision), summed in the same order as air_vcycle's
 * FP64 form.  Asynchronous on the stream.
 *
 * air_vcycle_multi_f32: the same with float b and x on round-to-nearest
 * FP32 copies of the hierarchy's operators (made on first use), summed in the
 * order of air_vcycle's FP32 form.  The FP32 FMA rate of GB300 is many times
 * its FP64 rate, and k systems per matrix entry make the FP64 form ALU-bound.
 *
 * air_bicgstab_solve_multi: air_bicgstab_solve on the k systems A x_j = b_j
 * in lockstep, preconditioned by the multi V-cycle in H's precision (FP64 for
 * an FP64 hierarchy, FP32 for FP32 and BF16 storage): each column has its own
 * scalars and stopping test and is frozen once converged; info[j] (k entries)
 * reports column j.  Returns AIR_NOT_CONVERGED if any column did not
 * converge.  Device buffers only.  The paper solves one right-hand side at a
 * time. */
int air_vcycle_multi(const air_hierarchy *H, int k, const double *b, double *x, void *stream);
int air_vcycle_multi_f32(const air_hierarchy *H, int k, const float *b, float *x, void *stream);
int air_bicgstab_solve_multi(const air_csr *A, const air_hierarchy *H, int k, const double *b, double *x,
                             double rtol, void *stream, air_solve_info *info);

/* Independent problems at once.  The paper solves one system at a time;
 * these run count independent setups (or solves) together and return when
 * all are done.  Each problem works on its own stream (streams[k], or a
 * library-created stream when streams is NULL or streams[k] is NULL).
 *
 * air_setup_batch builds the hierarchies level by level in lockstep: every
 * problem's strength, transpose and C/F splitting of level l run on its own
 * host thread and stream (the one-warp first passes of different problems
 * run side by side), then the local l-AIR solves of level l of all problems
 * run as one kernel launch over the union of their C points (Section 3), then
 * each problem builds P and A_{l+1}.  theta, distance and opt apply to every
 * problem.
 *
 * air_gmres_solve_batch runs every problem's flexible GMRES(m) in lockstep
 * rounds on one host thread: in each round the V-cycles of all problems in an
 * Arnoldi step are one CUDA graph launch (a gather of the vectors into the
 * hierarchies, their V-cycles as parallel branches, a scatter back; the
 * graph is rebuilt only when a problem finishes), then each problem's
 * matrix product, CGS2 and Givens update run on its stream, with one host
 * synchronisation per round for all problems.  Hierarchies of different
 * precisions may be mixed.
 *
 * Each problem's result is exactly that of the single-problem call (the same
 * kernels on the same data).  A is an array of count air_csr; out / H / b / x
 * / info / status are arrays of count.  status[k] (if status is not NULL)
 * receives problem k's status; the return value is the first negative
 * status, else AIR_OK (a solve that stops at max_iter reports
 * AIR_NOT_CONVERGED in status[k] and info[k] only).  A hierarchy may appear
 * only once in a solve batch (AIR_ERR_INVALID_ARG): its Krylov workspace
 * serves one solve at a time. */
int air_setup_batch(int count, const air_csr *A, double theta, int distance, const air_options *opt,
                    void *const *streams, air_hierarchy **out, int *status);
int air_gmres_solve_batch(int count, const air_csr *A, const air_hierarchy *const *H, const double *const *b,
                          double *const *x, double rtol, void *const *streams, air_solve_info *info,
                          int *status);

/* Adjoint support.  The paper solves only the forward system S Lambda = H
 * (Section 2.5) and has no adjoint; these two calls serve the gradient of a
 * loss L(u) through u = A^{-1} b: with lambda = A^{-T} dL/du (an l-AIR solve on
 * the transpose, whose unit diagonal blocks and reversed upwind structure suit
 * the same setup), dL/db = lambda and dL/da_ij = -lambda_i u_j.
 *
 * air_csr_transpose: A^T of a device CSR (n_rows x n_cols) into caller-owned
 * device arrays row_ptr_t (n_cols + 1), col_t (nnz), val_t (nnz); columns
 * ascending in every row, values moved bit for bit.  Returns
 * AIR_ERR_CSR_MALFORMED if a column index is out of range, AIR_ERR_INVALID_ARG
 * for a host CSR or NULL pointers.  Synchronises the stream once. */
int air_csr_transpose(const air_csr *A, int64_t *row_ptr_t, int32_t *col_t, double *val_t, void *stream);

/* The adjoint operator in the block-scaled form that l-AIR expects.  A is the
 * block-scaled system D_b^{-1} S (facet blocks of b unknowns, diag = the n/b
 * diagonal blocks D_b of S, row-major b x b each, as air_hdg_assemble returns
 * them).  A^T = S^T D_b^{-T} is scaled on the right, not on the left; the
 * similar matrix D_b^{-T} A^T D_b^T = D_b^{-T} S^T has identity diagonal
 * blocks again, like A (Section 4: the left block-diagonal scaling the AIR
 * solver settings prescribe).  With nu = D_b^{-T} lambda, A^T lambda = g
 * becomes (D_b^{-T} A^T D_b^T) nu = D_b^{-T} g and lambda = D_b^T nu.
 *
 * air_csr_transpose_scaled writes D_b^{-T} A^T D_b^T into caller-owned device
 * arrays sized like air_csr_transpose's.  Every row of a facet must hold
 * whole b x b blocks in the same layout with the diagonal block stored as its
 * b ones (the layout air_hdg_assemble produces); otherwise CSR_MALFORMED.
 * b <= 11.  Synchronises the stream.
 *
 * air_block_diag_apply: y_k = op(D_k) x_k for the nblocks b-blocks of device
 * vectors x, y (op 0: D, 1: D^T, 2: D^{-1}, 3: D^{-T}); b <= 11.
 * SINGULAR_COARSE if a block is singular.  Synchronises the stream. */
int air_csr_transpose_scaled(const air_csr *A, int b, const double *diag, int64_t *row_ptr_t, int32_t *col_t,
                             double *val_t, void *stream);
int air_block_diag_apply(int64_t nblocks, int b, const double *diag, int op, const double *x, double *y,
                         void *stream);

/* out[e] = alpha * u[i] * w[j] for every stored entry e = (i, j) of the device
 * CSR A (the gradient of L over A's values with alpha = -1, u = lambda,
 * w = the forward solution).  out has nnz entries, device, caller-owned; an
 * entry whose column is out of range gets NaN.  Asynchronous on the stream. */
int air_csr_outer(const air_csr *A, const double *u, const double *w, double alpha, double *out, void *stream);

/* Right-preconditioned flexible GMRES(restart) with classical Gram-Schmidt
 * applied twice, x0 = 0, until ||b - A x|| / ||b|| <= rtol (the paper's
 * Krylov method is BiCGSTAB; GMRES is named as an alternative in Section 5.1).
 * A must be the matrix H was built from.  If A->on_device is 1, b and x are
 * device vectors; if 0, b and x are host vectors and the library copies b in
 * and x out (A's values are then taken from the hierarchy's device copy).
 * Synchronises the stream once per inner step (8-byte residual read).
 * info may be NULL.  Returns AIR_OK or AIR_NOT_CONVERGED, or an error. */
int air_gmres_solve(const air_csr *A, const air_hierarchy *H, const double *b, double *x,
                    double rtol, void *stream, air_solve_info *info);

/* The same flexible GMRES solve as air_gmres_solve, for callers that must
 * not have the library allocate device memory during the solve: memory
 * fully pre-assigned by a pool or budget, or a host framework that forbids
 * allocation inside its solve phase.  (The paper has no counterpart; this is
 * a deployment variant.)  Build H beforehand with air_setup; this call then
 * allocates nothing -- no cudaMalloc, no pinned host buffer.
 * The Krylov workspace is one fixed 32 MiB array of device memory that every
 * GPU loading the library reserves until the process exits; it must hold
 * (2 restart + 1) n + O(restart^2) doubles, so with restart 30 n can reach
 * about 68,000; larger problems return AIR_ERR_NOALLOC_LIMIT before any work.
 * A, b and x must be on the device (A->on_device = 1).  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) and
 * keeps it for the life of the process; make that first call before any
 * stream capture, and do not call this function again after a
 * cudaDeviceReset of that device (the reset reloads the module, and the kept
 * address would no longer be the array's).  All calls share the array and it keeps the
 * previous call's contents (the solve clears what must start at zero):
 * calls that overlap on the GPU -- from two streams or two host threads --
 * race on it.  Synchronises the stream once per inner step. */
int air_gmres_solve_noalloc(const air_csr *A, const air_hierarchy *H, const double *b, double *x,
                            double rtol, void *stream, air_solve_info *info);

/* ------------------------------------------------ HDG assembly on the GPU
 * The space-time HDG discretisation of advection-diffusion (Section 2.3,
 * eqs. st-hdg and bilin with the upwind flux sigma_a and the interior-penalty
 * flux sigma_d of eq. IPpenalty, alpha = 10 p^2 in Section 4), its static
 * condensation S = D - C A^{-1} B, H = G - C A^{-1} F (Section 2.5,
 * eqs. linsys and systemLambda) and the left scaling by the facet
 * block-diagonal inverse (Section 4 settings), assembled on the device into
 * the CSR trace system that air_setup / air_gmres_solve take.
 *
 * Mesh: simplices of a D-dimensional space-time domain (D = 2 for 1D+time,
 * 3 for 2D+time); coordinates ordered (t, x[, y]).  Facet k of an element is
 * the one opposite its local vertex k.  Every facet is interior (two
 * elements), Dirichlet (spatial boundary: its trace is the L2 projection of
 * the Dirichlet data and is not an unknown) or Neumann (the t = t0 and t = T
 * faces).  Facet basis: Lagrange on the equispaced lattice of the facet's
 * canonical frame (its global vertex ids ascending); unknown m of free facet
 * r is row r b + m, free facets numbered in ascending facet id.  Within a row
 * the columns ascend; the scaled diagonal block is stored as its b ones.
 *
 * All arrays in these three structures are device pointers owned by the
 * caller.  The reference tables (quadrature, bases on the reference element
 * and the canonical facet frames; see paper_2010_11130_gb300/hdg_ref.py for
 * their definitions) are per (D, p) and independent of the mesh. */
typedef struct {
    int D;                        /* 2 or 3 */
    int64_t n_verts, n_elems, n_facets;
    const double *verts;          /* n_verts x D coordinates */
    const int32_t *elems;         /* n_elems x (D+1) vertex ids */
    const int32_t *elem_facets;   /* n_elems x (D+1) facet opposite local vertex k */
    const int32_t *facets;        /* n_facets x D vertex ids, ascending */
    const int32_t *facet_elems;   /* n_facets x 2 adjacent elements, ascending, -1 if none */
    const int8_t *facet_kind;     /* 0 interior, 1 Dirichlet, 2 Neumann */
} air_hdg_mesh;

typedef struct {
    int p;                        /* 1, 2 or 3 */
    int nb, b, nq, nqf, nperm;    /* element / facet basis sizes, volume / facet points, D! */
    const double *wq;             /* nq volume weights (sum 1/D!) */
    const double *xq;             /* nq x D volume points */
    const double *phi, *gphi;     /* nq x nb element basis, nq x nb x D its reference gradient */
    const double *wf;             /* nqf facet weights (sum 1/(D-1)!) */
    const double *sq;             /* nqf x (D-1) facet points, canonical frame */
    const double *psi;            /* nqf x b trace basis */
    const double *xi_f;           /* (D+1) x nperm x nqf x D facet points in element coordinates */
    const double *phi_f, *gphi_f; /* (D+1) x nperm x nqf x nb [x D] element basis there */
    const int32_t *perms;         /* nperm x D: canonical vertex m = local facet vertex perms[s][m] */
    const double *dir_proj;       /* b x nqf: L2 projection of point values onto the trace basis */
} air_hdg_ref;

typedef struct {
    double nu;                    /* diffusion coefficient */
    double alpha;                 /* interior-penalty parameter (Section 4: 10 p^2) */
    const double *vel_vol;        /* n_elems x nq x (D-1): spatial velocity at the volume points */
    const double *src;            /* n_elems x nq: source f at the volume points */
    const double *vel_face;       /* n_elems x (D+1) x nqf x (D-1): velocity at the facet points */
    const double *u0_face;        /* n_elems x (D+1) x nqf: data u on Neumann facets; the inflow flux
                                     g = -a_hat_n u where a_hat_n < 0 (NULL: zero) */
    const double *g_dir;          /* n_facets x nqf: Dirichlet data at the canonical facet points
                                     (read on Dirichlet facets only; NULL: zero) */
} air_hdg_data;

/* Physical coordinates of the quadrature points, for evaluating the data of
 * air_hdg_data: x_vol n_elems x nq x D, x_face n_elems x (D+1) x nqf x D (the
 * facet points as each element sees them, in the order of vel_face and
 * u0_face), x_facet n_facets x nqf x D (canonical facet points, the order of
 * g_dir).  Any output may be NULL.  Asynchronous on the stream. */
int air_hdg_points(const air_hdg_mesh *M, const air_hdg_ref *R, double *x_vol, double *x_face, double *x_facet,
                   void *stream);

/* Rows (= free facets x b) and stored entries of the assembled trace system
 * (scale = 1: diagonal blocks stored as b ones; 0: full diagonal blocks).
 * Synchronises the stream.  Errors: INVALID_ARG (D, p or the table sizes). */
int air_hdg_size(const air_hdg_mesh *M, const air_hdg_ref *R, int scale, int64_t *n_rows, int64_t *nnz,
                 void *stream);

/* Assemble, condense and (scale = 1) block-scale: row_ptr (n_rows + 1),
 * col (nnz), val (nnz) and rhs (n_rows), caller-allocated device arrays sized
 * by air_hdg_size.  diag (optional, n_rows x b) receives the unscaled
 * diagonal block of every free facet row-major (the D_b of A = D_b^{-1} S),
 * lam_dir (optional, n_facets x b) the Dirichlet trace values.  One warp per
 * element builds the local matrices by quadrature, condenses them in shared
 * memory and writes its off-diagonal blocks; one warp per facet sums the two
 * diagonal contributions, inverts and scales its row.  Synchronises the
 * stream.  Errors: INVALID_ARG, CUDA, SINGULAR_COARSE (a singular element
 * matrix A_K or diagonal block). */
int air_hdg_assemble(const air_hdg_mesh *M, const air_hdg_ref *R, const air_hdg_data *data, int scale,
                     int64_t *row_ptr, int32_t *col, double *val, double *rhs, double *diag, double *lam_dir,
                     void *stream);

/* Gradient of a loss L(Lambda) with respect to a velocity perturbation that
 * is constant on each element (the element velocities of a piecewise-constant
 * field).  The trace system S Lambda = H (unscaled) depends on the velocity
 * through the element matrices; with mu = S^{-T} dL/dLambda,
 *   dL/da_e = sum over the element's facets and volume of
 *             mu_K^T (dH_K/da_e - dS_K/da_e Lambda_K),
 * evaluated without forming dS_K as -(dB_h/da_e)((U, Lambda), (-y, mu)):
 * U = A_K^{-1}(F_K - B_K Lambda_K) is the element solution and
 * y = A_K^{-T} C_K^T mu_K.  lam (n_rows) is the solution of the scaled system
 * A x = b of air_hdg_assemble (the trace unknowns), adj (n_rows) the adjoint
 * solution of A^T adj = dL/dLambda; mu = D_b^{-T} adj is formed here from
 * diag (air_hdg_assemble's output) and lam_dir gives Lambda on Dirichlet
 * facets.  grad (n_elems x (D-1), device) is overwritten.  The source is
 * taken as independent of the velocity.  Synchronises the stream. */
int air_hdg_velocity_gradient(const air_hdg_mesh *M, const air_hdg_ref *R, const air_hdg_data *data,
                              const double *diag, const double *lam_dir, const double *lam, const double *adj,
                              double *grad, void *stream);

/* Device time of air_setup's phases in milliseconds, summed over levels:
 * ms[0] strength, [1] transpose, [2] C/F splitting, [3] l-AIR restriction,
 * [4] one-point P, [5] Galerkin RAP, [6] coarsest inverse, [7] diagonals,
 * precision copies and vectors; then counters of the C/F splitting kernel
 * (filled by the default cursor kernel, zero for the other variants):
 * ms[8] picks, [9] cursor refills (a bucket's cached 512-point line ran
 * empty and the global bitmaps were searched), [10] bitmap lines read by
 * those searches.  Copies min(count, 11) values.  Measured
 * with CUDA events on the setup stream; the paper reports only wall-clock
 * stage totals (Section 5.1: setup, assembly, solve, reconstruction). */
int air_setup_timings(const air_hierarchy *H, double *ms, int count);

/* Number of levels of H (>= 1). */
int air_hierarchy_levels(const air_hierarchy *H);

/* Sizes of level l. */
int air_hierarchy_info(const air_hierarchy *H, int level, air_level_info *info);

/* Copy one array of level l to host memory dst (caller-sized from
 * air_hierarchy_info).  what: 0 A.row_ptr (int64 n+1), 1 A.col (int32 nnz),
 * 2 A.val (float64 nnz), 3 S.row_ptr (int64 n+1), 4 S.col (int32 nnz_s),
 * 5 cf (int8 n, 1 = C), 6 coarse id (int32 n, -1 for F), 7 R.row_ptr (int64
 * nc+1), 8 R.col (int32 nnz_r), 9 R.val (float64 nnz_r), 10 P column (int32
 * n, -1 = empty row; the one-point weight is 1).  Synchronous. */
int air_hierarchy_export(const air_hierarchy *H, int level, int what, void *dst);

/* Free the hierarchy and its workspace (NULL is a no-op). */
void air_free(air_hierarchy *H);

/* Number of CUDA kernels this library has launched in the process so far
 * (diagnostic counter, all threads and devices). */
unsigned long long air_kernel_launches(void);

/* Static description of a status code. */
const char *air_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* AIR_H */
