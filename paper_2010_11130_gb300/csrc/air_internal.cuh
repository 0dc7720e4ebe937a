// Internal declarations of libair: device data layout and kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/air.h"

#define AIR_MAX_LEVELS 32
#define AIR_MAX_RESTART 64

// Return a library status from a CUDA call.
#define AIR_CUDA(call)                                                        \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) {                                              \
            (void)cudaGetLastError();                                         \
            return e_ == cudaErrorMemoryAllocation ? AIR_ERR_OOM : AIR_ERR_CUDA; \
        }                                                                     \
    } while (0)

#define AIR_TRY(expr)                  \
    do {                               \
        int s_ = (expr);               \
        if (s_ != AIR_OK) return s_;   \
    } while (0)

#define AIR_LAUNCH() AIR_CUDA(cudaGetLastError())

// Every kernel launch passes its grid size through air_counted(), which
// counts the launch (host-side, for diagnostics) and returns the size.
unsigned long long air_launch_counter_add(unsigned long long k);
void air_launch_counter_sub(unsigned long long k);
inline dim3 air_counted(dim3 g) {
    air_launch_counter_add(1);
    return g;
}

// Device memory of the library call in progress on this host thread.  While
// an AirCallStream guard is alive, air_dmalloc / air_dfree are stream-ordered
// (cudaMallocAsync / cudaFreeAsync on the call's stream) and never synchronise
// the device, so calls on different streams from different host threads run
// concurrently; outside a call they fall back to cudaMalloc / cudaFree.
struct AirCallSlot {
    cudaStream_t s = nullptr;
    bool active = false;
};
AirCallSlot &air_call_slot();
struct AirCallStream {
    AirCallSlot prev;
    explicit AirCallStream(cudaStream_t s) : prev(air_call_slot()) {
        air_call_slot().s = s;
        air_call_slot().active = true;
    }
    ~AirCallStream() { air_call_slot() = prev; }
};
cudaError_t air_dmalloc(void **p, size_t bytes);
void air_dfree(void *p);

// Every kernel with more than 48 KB of dynamic shared memory is opted in to
// this one size (each launch checks its own need against it).  One value for
// all calls: the attribute is per function, and setups running concurrently on
// several host threads must not lower it under one another's launches.
#define AIR_SMEM_OPTIN (200 * 1024)
// Opts kernel f in to AIR_SMEM_OPTIN bytes once per device and process: the
// attribute is set by the first caller only, so that concurrent setups on
// several host threads do not keep setting it while instances of the kernel run.
cudaError_t air_smem_optin_impl(const void *f);
template <typename F>
inline cudaError_t air_smem_optin(F *f) { return air_smem_optin_impl((const void *)f); }

// device error flags written by bounded kernels
#define AIR_DEVERR_RS_CAP 1
#define AIR_DEVERR_CSR 2
#define AIR_DEVERR_SINGULAR 4
#define AIR_DEVERR_CAP 8        // a fixed per-warp buffer was too small (reported as UNSUPPORTED)

// SELL-32 storage of a set of CSR rows: slice s holds rows 32s .. 32s+31 of
// the set (in the order of `rows`); entry k of the slice's lane l sits at
// ptr[s] + 32 k + l.  A slice is as wide as its longest row; shorter rows are
// padded with zero values (column = the row itself).  Values are in the
// V-cycle's storage type.
//
// Block form (b > 0): rows made of whole aligned b-blocks of consecutive
// columns plus at most a standalone diagonal entry (the level-0 trace matrix:
// facet blocks, the scaled diagonal block stored as its ones).  Then ptr
// counts stored blocks: slot t of lane l holds the block's first column
// bc[ptr[s] + 32 t + l] and its b values at v + (ptr[s] + 32 t + l) b; dv[pos]
// is the standalone diagonal in the vector type (0 when the diagonal sits in
// a block; for BF16 storage the diagonal is always zeroed in the blocks and
// kept in dv in FP32).  Padding slots: column 0 with zero values.
struct Sell {
    int64_t m = 0;              // rows
    int32_t *rows = nullptr;    // pos -> row id (rows sorted by length inside windows of 1024)
    int64_t *ptr = nullptr;     // m / 32 + 1 slice offsets
    int32_t *ci = nullptr;
    void *v = nullptr;
    int64_t stored = 0;         // entries (block form: blocks) including padding
    int b = 0;                  // block size of the block form, 0 for entries
    int32_t *bc = nullptr;      // block form: first column of each stored block
    void *dv = nullptr;         // block form: standalone diagonal per position
};

struct AirLevel {
    int64_t n = 0, nnz = 0;
    int32_t maxrow = 0, maxrow_r = 0; // longest row of A_l and of R_l
    const int64_t *rp = nullptr;      // A_l (level 0 may alias the caller)
    const int32_t *ci = nullptr;
    const double *v = nullptr;
    int owns_A = 0;
    float *diag32 = nullptr;          // a_ii in FP32 (BF16 storage)
    double *dinv = nullptr;           // 1 / a_ii
    float *dinv32 = nullptr;
    // strength graph
    int64_t nnz_s = 0;
    int64_t *srp = nullptr;
    int32_t *sci = nullptr;
    // splitting
    int8_t *cf = nullptr;             // 1 = C, 0 = F
    int32_t *cid = nullptr;           // coarse id or -1
    int64_t nc = 0;
    int32_t *crows = nullptr;         // C points ascending (nc)
    int32_t *frows = nullptr;         // F points ascending (nf)
    int64_t nf = 0;
    // restriction
    int64_t nnz_r = 0;
    int64_t *rrp = nullptr;
    int32_t *rci = nullptr;
    double *rv = nullptr;

    int64_t n_singular = 0;
    int32_t max_m = 0;
    // one-point interpolation
    int32_t *pcol = nullptr;
    // SELL-32 copies for the V-cycle: the rows of A_l split by point set
    // (0 = F, 1 = C) for the relaxation sweeps, and R_l for the restriction
    Sell sset[2];
    Sell sr;
    // lanes per row of the entry-form kernels: F sweep, C sweep, restriction
    // (1: one thread per row; more: the row's entries split over that many lanes)
    int lanes[3] = {1, 1, 1};
    // forward Gauss-Seidel level schedules of the F points, the C points and
    // all points: rows grouped by their depth in the graph of lower-index
    // couplings (dev_rows, device), group k = dev_rows[ptr[k] .. ptr[k+1])
    // with ptr on the host
    struct GsSchedule {
        int64_t m = 0;
        int32_t depth = 0;
        int32_t *dev_rows = nullptr;
        int64_t *ptr = nullptr;      // host, depth + 1
    } gs[3];
    float *v32 = nullptr;            // FP32 copy of A_l's values (Gauss-Seidel on an FP32 hierarchy)
    // V-cycle work vectors (precision of the hierarchy)
    void *b = nullptr, *x = nullptr, *x2 = nullptr;
};

struct air_hierarchy {
    int nlev = 0;
    AirLevel lev[AIR_MAX_LEVELS];
    air_options opt;
    int dev = 0;
    // coarsest: explicit inverse (row major)
    int64_t nco = 0;
    double *cinv = nullptr;
    float *cinv32 = nullptr;
    // device scalars and scratch
    int *d_err = nullptr;
    unsigned long long *d_stats = nullptr;   // 8 first-pass counters: picks, refills, lines searched, long lists, cursor moves
    // SELL-32 FP64 copy of the finest operator for the GMRES matrix products
    Sell a0;
    // V-cycle body captured as a CUDA graph on first use
    cudaGraphExec_t vgraph = nullptr;
    int vgraph_failed = 0;
    long long vgraph_kernels = 0;
    // setup phase times (ms): strength, transpose, splitting, l-AIR, P, RAP, coarsest, other
    double phase_ms[12] = {0};
    // GMRES workspace (allocated on first solve)
    int64_t ws_n = 0;
    int ws_m = 0;
    double *V = nullptr, *Z = nullptr, *w = nullptr, *r = nullptr;
    double *partials = nullptr;       // (m+2) x nblk_reduce
    double *hcol = nullptr;           // small device arrays for the Arnoldi step
    double *Hm = nullptr;             // (m+1) x m Hessenberg (column major), rotated
    double *gvec = nullptr, *cs = nullptr, *sn = nullptr, *y = nullptr;
    double *scal = nullptr;           // [0] norm, [1] estimate, ...
    double *h_est = nullptr;          // pinned host mirror of scalars
    double *xd = nullptr, *bd = nullptr;  // device b and x when the caller passes host vectors
    // many right-hand sides (allocated on first use): per level, b, x and a
    // compact sweep buffer of n_l x mk row-major FP64; the Krylov vectors of
    // the lockstep solve
    int mk = 0;
    double *mb[AIR_MAX_LEVELS] = {}, *mx[AIR_MAX_LEVELS] = {}, *mt[AIR_MAX_LEVELS] = {};
    double *mkry = nullptr;
    size_t mkry_n = 0;
    // FP32 copies for the FP32 multi V-cycle: A_l values, 1 / a_ii, R_l values, coarsest inverse
    int m32 = 0;
    float *mv32[AIR_MAX_LEVELS] = {}, *md32[AIR_MAX_LEVELS] = {}, *mr32[AIR_MAX_LEVELS] = {};
    float *mc32 = nullptr;
};

// Scratch carried between the halves of one coarsening step (air_api.cu):
// the splitting half leaves the local l-AIR solves of LS ready to run.
struct AirCoarsen {
    int stop = 0;                    // level l is the coarsest; nothing is kept
    int32_t *cnt = nullptr, *dmax = nullptr, *rsci = nullptr;
    int64_t *scanw = nullptr, *rsrp = nullptr, *dsing = nullptr;
    AirLevel LS;                     // level l with R's strength graph
};
int air_check_options(double theta, int distance, const air_options *opt, air_options *out);
int air_setup_begin(const air_csr *A, const air_options *opt, cudaStream_t s, air_hierarchy *H);
bool air_setup_is_coarsest(const air_hierarchy *H, int l);
int air_coarsen_split(air_hierarchy *H, int l, cudaStream_t s, AirCoarsen *c);
int air_coarsen_lair(air_hierarchy *H, int l, cudaStream_t s, AirCoarsen *c);
int air_coarsen_finish(air_hierarchy *H, int l, cudaStream_t s, AirCoarsen *c);
int air_setup_end(air_hierarchy *H, cudaStream_t s);
void air_add_phase_ms(air_hierarchy *H, int phase, double ms);
// The local l-AIR solves of several levels (of independent hierarchies) in one
// launch; levels[k] with R's strength graph, max_m[k] its largest
// neighbourhood, d_nsing[k] its count of singular systems.
int air_lair_solve_batch(int count, const AirLevel *const *levels, const int32_t *max_m, int distance,
                         int64_t *const *d_nsing, cudaStream_t s);

// One flexible GMRES solve split at its host reads (air_api.cu).
struct AirGmres {
    enum Phase { OPENED, CYCLE, STEP, DONE };
    air_hierarchy *H = nullptr;
    const AirLevel *A0 = nullptr;
    const double *b = nullptr;
    double *x = nullptr;
    double rtol = 0.0, bnorm = 0.0;
    cudaStream_t s = nullptr;
    air_solve_info *info = nullptr;
    int64_t n = 0;
    int m = 0, nblk = 0, it = 0, j = 0, k = 0;
    Phase phase = OPENED;
};
int air_gmres_open(AirGmres &g, const AirLevel &A0, const air_hierarchy *H, const double *b, double *x,
                   double rtol, cudaStream_t s, air_solve_info *info);
void air_gmres_after_open(AirGmres &g);
int air_gmres_cycle(AirGmres &g);
int air_gmres_after_cycle(AirGmres &g);
double *air_gmres_vj(const AirGmres &g);
double *air_gmres_zj(const AirGmres &g);
int air_gmres_step(AirGmres &g);
int air_gmres_after_step(AirGmres &g);
int air_gmres_close(AirGmres &g);
// The V-cycle from lev[0].b to lev[0].x (the hierarchy's own precision, no graph).
int air_vcycle_staged(air_hierarchy *H, cudaStream_t s);
// Conversions between caller vectors (FP64) and hierarchies' lev[0] buffers, several at once.
struct AirConvJob {
    const void *src;
    void *dst;
    int64_t n;       // 0: skip
    int mode;        // 0 FP64 copy, 1 FP64 -> FP32, 2 FP32 -> FP64
};
int air_convert_batch(int count, const AirConvJob *d_jobs, cudaStream_t s);


// ------------------------------------------------------------------ launchers
// scan.cu
int air_exclusive_scan_i32(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s);
int air_exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s);
int air_reduce_max_i32(const int32_t *in, int64_t n, int32_t *d_out, cudaStream_t s);

// setup_kernels.cu
int air_validate_csr(int64_t n, int64_t nnz, const int64_t *rp, const int32_t *ci, const double *v,
                     int *d_err, cudaStream_t s);
int air_strength(const AirLevel &L, double theta, int64_t *srp, int32_t *sci, int32_t *cnt, int fill,
                 cudaStream_t s);
int air_transpose_pattern(int64_t n, int64_t nnz, const int64_t *srp, const int32_t *sci, int64_t *strp,
                          int32_t *stci, int32_t *work, cudaStream_t s);
int air_rs_first_pass(int64_t n, const int64_t *srp, const int32_t *sci, const int64_t *strp,
                      const int32_t *stci, int32_t max_st, int32_t max_s, int8_t *cf, int *d_err, int cached,
                      unsigned long long *stats, cudaStream_t s);
// first_pass.cu: the cursor first pass (AIR_ERR_UNSUPPORTED: outside its limits, nothing launched)
int air_rs_first_pass_cursor(int64_t n, const int64_t *srp, const int32_t *sci, const int64_t *strp,
                             const int32_t *stci, int32_t max_st, int8_t *cf, int *d_err,
                             unsigned long long *stats, cudaStream_t s);
// falgout.cu: Falgout-style splitting with index blocks of `block` points (a multiple of 1024, <= 8192)
int air_falgout_split(int64_t n, int64_t block, const int64_t *srp, const int32_t *sci, const int64_t *strp,
                      const int32_t *stci, int8_t *cf, int *d_err, cudaStream_t s);
int air_coarse_ids(int64_t n, const int8_t *cf, int32_t *cid, int32_t *crows, int64_t *work, int64_t *nc,
                   cudaStream_t s);
// distance 1: N_i = S_i intersect F; distance 2 adds S_k intersect F for k in it
// (at most 2048 distinct points per C point: more sets AIR_DEVERR_CAP in d_err)
int air_lair_counts(int64_t nc, const int32_t *crows, const int64_t *srp, const int32_t *sci, const int8_t *cf,
                    int32_t *cnt, int distance, int *d_err, cudaStream_t s);
int air_lair_solve(const AirLevel &L, int32_t max_m, int distance, int64_t *d_nsing, cudaStream_t s);
int air_onepoint_P(const AirLevel &L, double theta, cudaStream_t s);
// terms: RAP terms per coarse row (air_rap_terms); rows with more than 2048
// use a global-memory hash table
int air_rap(const AirLevel &L, int64_t *acrp, int32_t *acci, double *acv, int32_t *cnt, int fill,
            int32_t max_terms, const int32_t *terms, int *d_err, cudaStream_t s);
int air_rap_terms(const AirLevel &L, int32_t *terms, cudaStream_t s);
int air_coarse_inverse(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, double *inv,
                       double *work, int *d_err, cudaStream_t s);

// adjoint.cu
int air_csr_transpose_impl(int64_t n, int64_t ncols, int64_t nnz, const int64_t *rp, const int32_t *ci,
                           const double *v, int64_t *rpt, int32_t *cit, double *vt, int *d_err, cudaStream_t s);
// adjoint.cu: A^T with block b x b scaling D_f^{-T} (.) D_g^T, and block-diagonal products
int air_block_scale_transpose_impl(int64_t n, int b, const double *diag, const int64_t *rpt, const int32_t *cit,
                                   double *vt, int *d_err, cudaStream_t s);
int air_block_apply_impl(int64_t nblk, int b, const double *diag, int op, const double *x, double *y, int *d_err,
                         cudaStream_t s);
int air_csr_outer_impl(int64_t n, int64_t ncols, const int64_t *rp, const int32_t *ci, const double *u,
                       const double *w, double alpha, double *out, cudaStream_t s);

// multi_rhs.cu: k <= 32 right-hand sides, row-major n x k FP64
int air_vcycle_multi_run(const air_hierarchy *H, int k, const double *b, double *x, cudaStream_t s);
int air_vcycle_multi_run_f32(const air_hierarchy *H, int k, const float *b, float *x, cudaStream_t s);
int air_bicgstab_multi_impl(const air_hierarchy *H, int k, const double *b, double *x, double rtol,
                            cudaStream_t s, air_solve_info *info);
void air_free_multi(air_hierarchy *H);

// gauss_seidel.cu: level schedules of the forward Gauss-Seidel sweeps the
// relaxation string asks for ('f', 'c', 'a'), built at the end of setup, and
// one sweep x <- GS(x) over set which (0 F, 1 C, 2 all); xn is n scratch
int air_gs_build(air_hierarchy *H, cudaStream_t s);
void air_gs_free(AirLevel &L);
template <typename T>
int air_gs_sweep(const AirLevel &L, int which, T omega, const T *b, T *x, T *xn, cudaStream_t s);

// solve_kernels.cu
// y = A x, or y = b - A x if b != NULL; nnz < 0 / maxrow <= 0 when unknown
int air_spmv_f64(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const double *x,
                 double *y, const double *b, cudaStream_t s, int64_t nnz = -1, int32_t maxrow = 0);
int air_max_row(int64_t n, const int64_t *rp, int32_t *out_max, cudaStream_t s);
int air_vcycle_run(const air_hierarchy *H, const double *b, double *x, cudaStream_t s, int use_graph = 1);
int air_point_list(int64_t n, const int8_t *cf, int which, int32_t *list, int64_t *work, cudaStream_t s);
int air_cast_d2f(const double *in, float *out, int64_t n, cudaStream_t s);
int air_lincomb(int64_t n, double *out, const double *a, double ca, const double *b, double cb, const double *c,
                double cc, cudaStream_t s);
int air_cast_bf16(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, void *out16, float *diag32,
                  cudaStream_t s);
int air_build_sell(int64_t m, const int32_t *rows, const int64_t *rp, const int32_t *ci, const double *v,
                   int precision, int zero_diag, Sell *out, cudaStream_t s);
// The block form of the same rows with block size b (2, 3, 4, 6 or 10).
// AIR_ERR_UNSUPPORTED (out left empty, nothing else changed) when a row is not
// whole aligned blocks plus at most its diagonal.
int air_build_sell_blocks(int64_t m, const int32_t *rows, const int64_t *rp, const int32_t *ci, const double *v,
                          int precision, int b, Sell *out, cudaStream_t s);
void air_free_sell(Sell &S);
int air_sell_spmv_f64(const Sell &S, const double *x, double *y, const double *b, cudaStream_t s);
// Lanes per row for every level's sweeps and restriction: a rule on the
// stored row width, or (timed = 1) the fastest of 1, 2, 4, 8, 16, 32 lanes
// timed with CUDA events on the level's own data.
int air_tune_lanes(air_hierarchy *H, int timed, cudaStream_t s);
int air_diag_inverse(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, double *dinv,
                     float *dinv32, cudaStream_t s);

// gmres kernels
int air_dot_partials(int64_t n, const double *V, int64_t ldv, int k, const double *w, double *partials,
                     int nblk, cudaStream_t s);
int air_update_dot_partials(int64_t n, const double *V, int64_t ldv, int k, const double *h, double *w,
                            double *partials, int nblk, int dots, cudaStream_t s);
int air_reduce_partials(int k, const double *partials, int nblk, double *out, cudaStream_t s);
int air_scale_vec(int64_t n, const double *in, double *out, const double *d_norm, int sqrt_of, cudaStream_t s);
int air_arnoldi_givens(int j, int m, const double *h1, const double *h2, const double *nrm2, double *Hm,
                       double *cs, double *sn, double *g, double *scal, double bnorm, cudaStream_t s);
int air_hessenberg_solve(int k, int m, const double *Hm, const double *g, double *y, cudaStream_t s);
int air_axpy_multi(int64_t n, const double *Z, int64_t ldz, int k, const double *y, double *x, cudaStream_t s);
int air_fill_zero(double *x, int64_t n, cudaStream_t s);
int air_set_scalar(double *p, double v, cudaStream_t s);
int air_norm_init(int64_t n, const double *r, double *partials, int nblk, cudaStream_t s);

int air_reduce_nblk(int64_t n);
