// C ABI of libair: hierarchy setup (arXiv:2010.11130, Section 3 with the
// Section 4 solver settings), V-cycle application and flexible GMRES.
// Host code only orchestrates: every arithmetic step runs in the kernels of
// setup_kernels.cu, solve_kernels.cu and scan.cu.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <new>
#include <set>
#include <utility>

#include "air_internal.cuh"

static std::atomic<unsigned long long> g_launches{0};

unsigned long long air_launch_counter_add(unsigned long long k) { return g_launches.fetch_add(k) + k; }
void air_launch_counter_sub(unsigned long long k) { g_launches.fetch_sub(k); }

AirCallSlot &air_call_slot() {
    thread_local AirCallSlot slot;
    return slot;
}

cudaError_t air_smem_optin_impl(const void *f) {
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({dev, f})) return cudaSuccess;
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, AIR_SMEM_OPTIN);
    if (e == cudaSuccess) done.insert({dev, f});
    return e;
}

cudaError_t air_dmalloc(void **p, size_t bytes) {
    const AirCallSlot &c = air_call_slot();
    return c.active ? cudaMallocAsync(p, bytes, c.s) : cudaMalloc(p, bytes);
}

void air_dfree(void *p) {
    if (!p) return;
    const AirCallSlot &c = air_call_slot();
    if (c.active) cudaFreeAsync(p, c.s); else cudaFree(p);
}

namespace {

template <typename T>
int dalloc(T **p, int64_t count) {
    *p = nullptr;
    if (count <= 0) count = 1;
    AIR_CUDA(air_dmalloc((void **)p, (size_t)count * sizeof(T)));
    return AIR_OK;
}

template <typename T>
void dfree(T *&p) {
    air_dfree((void *)p);
    p = nullptr;
}

// Small reads into pageable host memory wait for the stream first, so that the
// copy itself never waits on a long kernel (other host threads keep launching).
int read_i64(const int64_t *d, int64_t *h, cudaStream_t s) {
    AIR_CUDA(cudaStreamSynchronize(s));
    AIR_CUDA(cudaMemcpyAsync(h, d, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    AIR_CUDA(cudaStreamSynchronize(s));
    return AIR_OK;
}

int check_err(air_hierarchy *H, cudaStream_t s) {
    int e = 0;
    AIR_CUDA(cudaStreamSynchronize(s));
    AIR_CUDA(cudaMemcpyAsync(&e, H->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    AIR_CUDA(cudaStreamSynchronize(s));
    if (e & AIR_DEVERR_CSR) return AIR_ERR_CSR_MALFORMED;
    if (e & AIR_DEVERR_RS_CAP) return AIR_ERR_DEVICE_TIMEOUT;
    if (e & AIR_DEVERR_SINGULAR) return AIR_ERR_SINGULAR_COARSE;
    if (e & AIR_DEVERR_CAP) return AIR_ERR_UNSUPPORTED;
    return AIR_OK;
}

void free_level(AirLevel &L) {
    if (L.owns_A) {
        dfree(L.rp);
        dfree(L.ci);
        dfree(L.v);
    }
    L.rp = nullptr; L.ci = nullptr; L.v = nullptr;
    dfree(L.dinv); dfree(L.dinv32); dfree(L.diag32);
    dfree(L.srp); dfree(L.sci);
    dfree(L.cf); dfree(L.cid); dfree(L.crows); dfree(L.frows);
    dfree(L.rrp); dfree(L.rci); dfree(L.rv);
    dfree(L.pcol);
    air_free_sell(L.sset[0]);
    air_free_sell(L.sset[1]);
    air_free_sell(L.sr);
    air_gs_free(L);
    dfree(L.b); dfree(L.x); dfree(L.x2);
}

void free_workspace(air_hierarchy *H) {
    dfree(H->V); dfree(H->Z); dfree(H->w); dfree(H->r); dfree(H->partials); dfree(H->hcol);
    dfree(H->Hm); dfree(H->gvec); dfree(H->cs); dfree(H->sn); dfree(H->y); dfree(H->scal);
    if (H->h_est) cudaFreeHost(H->h_est);
    H->h_est = nullptr;
    H->ws_n = 0;
    H->ws_m = 0;
}

// First-pass kernel variant: 4 (default, fastest measured) per-bucket
// cursors in shared memory, deduplicated neighbourhood blocks and
// fire-and-forget bitmap updates, two dependent round trips per pick (levels
// outside its limits take 2); 2 exact bitmaps, two-hop lists and int8 measures
// with warp-combined read-modify-writes (measures up to 124); 1 lazy bitmaps
// with L1-cached loads and 0 lazy bitmaps with L2-only loads (int32 measures,
// the fallback for any level).  All give the same splitting.  Set by the
// environment variable AIR_RS_VARIANT (read once).
int rs_cached() {
    static const int v = [] {
        const char *e = getenv("AIR_RS_VARIANT");
        return (e && (e[0] == '0' || e[0] == '1' || e[0] == '2' || e[0] == '4')) ? e[0] - '0' : 4;
    }();
    return v;
}

// CUDA-event phase timer accumulated into H->phase_ms (read after setup's syncs).
struct PhaseTimer {
    air_hierarchy *H;
    cudaStream_t s;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int cur = -1;
    PhaseTimer(air_hierarchy *h, cudaStream_t st) : H(h), s(st) {
        cudaEventCreate(&ev[0]);
        cudaEventCreate(&ev[1]);
    }
    ~PhaseTimer() {
        stop();
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
    }
    void start(int phase) {
        stop();
        cur = phase;
        cudaEventRecord(ev[0], s);
    }
    void stop() {
        if (cur < 0) return;
        cudaEventRecord(ev[1], s);
        cudaEventSynchronize(ev[1]);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess) H->phase_ms[cur] += ms;
        cur = -1;
    }
};

}  // namespace

// First half of building level l+1 from level l: strength, transpose, C/F
// splitting, coarse ids, the l-AIR neighbourhood sizes and R's arrays.  Sets
// c->stop = 1 (and keeps nothing) when level l is the coarsest; otherwise the
// local l-AIR solves of c->LS are ready to run.
int air_coarsen_split(air_hierarchy *H, int l, cudaStream_t s, AirCoarsen *c) {
    AirLevel &L = H->lev[l];
    const air_options &o = H->opt;
    int64_t n = L.n;
    *c = AirCoarsen{};
    PhaseTimer T(H, s);
    T.start(0);
    // a1 strength
    int32_t *&cnt = c->cnt;
    AIR_TRY(dalloc(&cnt, n + 1));
    AIR_TRY(dalloc(&L.srp, n + 1));
    AIR_TRY(air_strength(L, o.theta, nullptr, nullptr, cnt, 0, s));
    AIR_TRY(air_exclusive_scan_i32(cnt, L.srp, n, s));
    int32_t *&dmax = c->dmax;
    AIR_TRY(dalloc(&dmax, 1));
    AIR_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int32_t), s));
    AIR_TRY(air_reduce_max_i32(cnt, n, dmax, s));
    int32_t max_s = 0;
    AIR_CUDA(cudaMemcpyAsync(&max_s, dmax, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AIR_TRY(read_i64(L.srp + n, &L.nnz_s, s));
    AIR_TRY(dalloc(&L.sci, L.nnz_s));
    AIR_TRY(air_strength(L, o.theta, L.srp, L.sci, nullptr, 1, s));
    // a2 transpose
    T.start(1);
    int64_t *strp = nullptr;
    int32_t *stci = nullptr;
    AIR_TRY(dalloc(&strp, n + 1));
    AIR_TRY(dalloc(&stci, L.nnz_s));
    AIR_TRY(air_transpose_pattern(n, L.nnz_s, L.srp, L.sci, strp, stci, cnt, s));
    // largest |S^T_i| (the transposed counts are still in cnt after the scatter)
    AIR_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int32_t), s));
    AIR_TRY(air_reduce_max_i32(cnt, n, dmax, s));
    int32_t max_st = 0;
    AIR_CUDA(cudaMemcpyAsync(&max_st, dmax, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AIR_CUDA(cudaStreamSynchronize(s));
    // a3 C/F splitting
    T.start(2);
    AIR_TRY(dalloc(&L.cf, n));
    if (o.falgout_block > 0)
        AIR_TRY(air_falgout_split(n, o.falgout_block, L.srp, L.sci, strp, stci, L.cf, H->d_err, s));
    else
        AIR_TRY(air_rs_first_pass(n, L.srp, L.sci, strp, stci, max_st, max_s, L.cf, H->d_err, rs_cached(),
                                  H->d_stats, s));
    AIR_TRY(check_err(H, s));
    dfree(strp);
    dfree(stci);
    int64_t *&scanw = c->scanw;
    AIR_TRY(dalloc(&scanw, n + 1));
    AIR_TRY(dalloc(&L.cid, n));
    int64_t nc = 0;
    AIR_TRY(air_coarse_ids(n, L.cf, L.cid, nullptr, scanw, &nc, s));
    if (nc == 0 || (double)nc > 0.9 * (double)n) {
        dfree(cnt); dfree(dmax); dfree(scanw);
        dfree(L.srp); dfree(L.sci); dfree(L.cf); dfree(L.cid);
        L.nnz_s = 0;
        *c = AirCoarsen{};
        c->stop = 1;
        return AIR_OK;
    }
    L.nc = nc;
    AIR_TRY(dalloc(&L.crows, nc));
    AIR_TRY(air_coarse_ids(n, L.cf, L.cid, L.crows, scanw, &nc, s));
    L.nf = n - nc;
    AIR_TRY(dalloc(&L.frows, L.nf));
    AIR_TRY(air_point_list(n, L.cf, 0, L.frows, scanw, s));
    // a4 l-AIR restriction, from its own strength graph when its threshold differs
    T.start(3);
    int64_t *&rsrp = c->rsrp;
    int32_t *&rsci = c->rsci;
    if (o.theta_r >= 0.0 && o.theta_r != o.theta) {
        AIR_TRY(dalloc(&rsrp, n + 1));
        AIR_TRY(air_strength(L, o.theta_r, nullptr, nullptr, cnt, 0, s));
        AIR_TRY(air_exclusive_scan_i32(cnt, rsrp, n, s));
        int64_t nnz_sr = 0;
        AIR_TRY(read_i64(rsrp + n, &nnz_sr, s));
        AIR_TRY(dalloc(&rsci, nnz_sr));
        AIR_TRY(air_strength(L, o.theta_r, rsrp, rsci, nullptr, 1, s));
    }
    AIR_TRY(air_lair_counts(nc, L.crows, rsrp ? rsrp : L.srp, rsrp ? rsci : L.sci, L.cf, cnt, o.distance, H->d_err,
                            s));
    if (o.distance >= 2) AIR_TRY(check_err(H, s));
    AIR_TRY(dalloc(&L.rrp, nc + 1));
    AIR_TRY(air_exclusive_scan_i32(cnt, L.rrp, nc, s));
    AIR_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int32_t), s));
    AIR_TRY(air_reduce_max_i32(cnt, nc, dmax, s));
    int32_t max_m1 = 0;
    AIR_CUDA(cudaMemcpyAsync(&max_m1, dmax, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AIR_TRY(read_i64(L.rrp + nc, &L.nnz_r, s));
    L.max_m = max_m1 - 1;
    AIR_TRY(dalloc(&L.rci, L.nnz_r));
    AIR_TRY(dalloc(&L.rv, L.nnz_r));
    AIR_TRY(dalloc(&c->dsing, 1));
    AIR_CUDA(cudaMemsetAsync(c->dsing, 0, sizeof(int64_t), s));
    c->LS = L;                  // the level with R's strength graph in place of the coarsening one
    if (rsrp) {
        c->LS.srp = rsrp;
        c->LS.sci = rsci;
    }
    AIR_CUDA(cudaStreamSynchronize(s));
    return AIR_OK;
}

// Second half, after the local l-AIR solves of c->LS have run: the count of
// singular local systems, one-point P and the Galerkin product A_{l+1}.
int air_coarsen_finish(air_hierarchy *H, int l, cudaStream_t s, AirCoarsen *c) {
    AirLevel &L = H->lev[l];
    const air_options &o = H->opt;
    const int64_t n = L.n, nc = L.nc;
    int32_t *cnt = c->cnt, *dmax = c->dmax;
    int64_t *scanw = c->scanw;
    PhaseTimer T(H, s);
    AIR_TRY(read_i64(c->dsing, &L.n_singular, s));
    dfree(c->dsing);
    dfree(c->rsrp);
    dfree(c->rsci);
    c->dsing = nullptr;
    c->rsrp = nullptr;
    c->rsci = nullptr;
    // a5 one-point interpolation
    T.start(4);
    AIR_TRY(dalloc(&L.pcol, n));
    AIR_TRY(air_onepoint_P(L, o.theta, s));
    // a6 Galerkin product
    T.start(5);
    int32_t *terms = nullptr;
    AIR_TRY(dalloc(&terms, nc));
    AIR_TRY(air_rap_terms(L, terms, s));
    AIR_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int32_t), s));
    AIR_TRY(air_reduce_max_i32(terms, nc, dmax, s));
    int32_t max_terms = 0;
    AIR_CUDA(cudaMemcpyAsync(&max_terms, dmax, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AIR_CUDA(cudaStreamSynchronize(s));
    AirLevel &C = H->lev[l + 1];
    C.n = nc;
    C.owns_A = 1;
    int64_t *acrp = nullptr;
    int32_t *acci = nullptr;
    double *acv = nullptr;
    AIR_TRY(air_rap(L, nullptr, nullptr, nullptr, cnt, 0, max_terms, terms, H->d_err, s));
    AIR_TRY(dalloc(&acrp, nc + 1));
    AIR_TRY(air_exclusive_scan_i32(cnt, acrp, nc, s));
    AIR_TRY(read_i64(acrp + nc, &C.nnz, s));
    AIR_TRY(dalloc(&acci, C.nnz));
    AIR_TRY(dalloc(&acv, C.nnz));
    AIR_TRY(air_rap(L, acrp, acci, acv, nullptr, 1, max_terms, terms, H->d_err, s));
    dfree(terms);
    AIR_TRY(check_err(H, s));
    C.rp = acrp;
    C.ci = acci;
    C.v = acv;
    dfree(cnt); dfree(dmax); dfree(scanw);
    *c = AirCoarsen{};
    AIR_CUDA(cudaStreamSynchronize(s));
    return AIR_OK;
}

// The local l-AIR solves of one level, timed as the l-AIR phase.
int air_coarsen_lair(air_hierarchy *H, int l, cudaStream_t s, AirCoarsen *c) {
    PhaseTimer T(H, s);
    T.start(3);
    return air_lair_solve(c->LS, H->lev[l].max_m, H->opt.distance, c->dsing, s);
}

// Adds a batched launch's time to a hierarchy's l-AIR phase.
void air_add_phase_ms(air_hierarchy *H, int phase, double ms) { H->phase_ms[phase] += ms; }

namespace {

// Build level l+1 from level l.  Returns AIR_OK with *stop = 1 when level l
// is the coarsest.
int coarsen(air_hierarchy *H, int l, cudaStream_t s, int *stop) {
    AirCoarsen c;
    AIR_TRY(air_coarsen_split(H, l, s, &c));
    *stop = c.stop;
    if (c.stop) return AIR_OK;
    AIR_TRY(air_coarsen_lair(H, l, s, &c));
    return air_coarsen_finish(H, l, s, &c);
}

}  // namespace

// Level 0 of a new hierarchy: options, the finest operator (borrowed when it
// is on the device and FP64), validation.
int air_setup_begin(const air_csr *A, const air_options *opt, cudaStream_t s, air_hierarchy *H) {
    H->opt = *opt;
    AIR_CUDA(cudaGetDevice(&H->dev));
    AIR_TRY(dalloc(&H->d_err, 1));
    AIR_CUDA(cudaMemsetAsync(H->d_err, 0, sizeof(int), s));
    AIR_TRY(dalloc(&H->d_stats, 8));
    AIR_CUDA(cudaMemsetAsync(H->d_stats, 0, 8 * sizeof(unsigned long long), s));
    AirLevel &L0 = H->lev[0];
    L0.n = A->n_rows;
    L0.nnz = A->nnz;
    if (A->on_device && opt->precision == AIR_PREC_F64) {
        L0.rp = A->row_ptr; L0.ci = A->col; L0.v = A->val;
        L0.owns_A = 0;
    } else {
        int64_t *rp; int32_t *ci; double *v;
        AIR_TRY(dalloc(&rp, A->n_rows + 1));
        AIR_TRY(dalloc(&ci, A->nnz));
        AIR_TRY(dalloc(&v, A->nnz));
        L0.rp = rp; L0.ci = ci; L0.v = v;
        L0.owns_A = 1;
        cudaMemcpyKind k = A->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        AIR_CUDA(cudaMemcpyAsync(rp, A->row_ptr, (size_t)(A->n_rows + 1) * sizeof(int64_t), k, s));
        AIR_CUDA(cudaMemcpyAsync(ci, A->col, (size_t)A->nnz * sizeof(int32_t), k, s));
        AIR_CUDA(cudaMemcpyAsync(v, A->val, (size_t)A->nnz * sizeof(double), k, s));
    }
    if (opt->validate) {
        int64_t last = -1;
        AIR_TRY(read_i64(L0.rp + L0.n, &last, s));
        if (last != L0.nnz) return AIR_ERR_CSR_MALFORMED;
        AIR_TRY(air_validate_csr(L0.n, L0.nnz, L0.rp, L0.ci, L0.v, H->d_err, s));
        AIR_TRY(check_err(H, s));
    }
    H->nlev = 1;
    return AIR_OK;
}

// True when level l (the last built) is to be the coarsest without trying to coarsen it.
bool air_setup_is_coarsest(const air_hierarchy *H, int l) {
    return H->lev[l].n <= H->opt.max_coarse || l == H->opt.max_levels - 1;
}

// Everything after the last level: coarsest inverse, smoother diagonals,
// precision copies, the FP64 copy of A for GMRES, tuning and schedules.
int air_setup_end(air_hierarchy *H, cudaStream_t s) {
    const air_options *opt = &H->opt;
    // coarsest level: dense inverse
    AirLevel &Lc = H->lev[H->nlev - 1];
    H->nco = Lc.n;
    if (Lc.n > opt->max_dense) return AIR_ERR_COARSE_TOO_LARGE;
    PhaseTimer T(H, s);
    T.start(6);
    {
        double *work = nullptr;
        int64_t n = Lc.n;
        AIR_TRY(dalloc(&H->cinv, n * n));
        AIR_CUDA(cudaMallocAsync((void **)&work, (size_t)(2 * n * n + n + 1) * sizeof(double), s));
        AIR_TRY(air_coarse_inverse(n, Lc.rp, Lc.ci, Lc.v, H->cinv, work, H->d_err, s));
        cudaFreeAsync(work, s);
        AIR_TRY(check_err(H, s));
    }
    {
        unsigned long long st[4] = {0, 0, 0, 0};
        AIR_CUDA(cudaMemcpyAsync(st, H->d_stats, sizeof(st), cudaMemcpyDeviceToHost, s));
        AIR_CUDA(cudaStreamSynchronize(s));
        H->phase_ms[8] = (double)st[0];
        H->phase_ms[9] = (double)st[1];
        H->phase_ms[10] = (double)st[2];
    }
    // smoother diagonals, precision copies, V-cycle vectors
    T.start(7);
    int f32 = opt->precision != AIR_PREC_F64;      // FP32 vectors (F32 and BF16 storage)
    int bf16 = opt->precision == AIR_PREC_BF16;
    for (int q = 0; q < H->nlev; ++q) {
        AirLevel &L = H->lev[q];
        AIR_TRY(air_max_row(L.n, L.rp, &L.maxrow, s));
        if (q + 1 < H->nlev) AIR_TRY(air_max_row(L.nc, L.rrp, &L.maxrow_r, s));
        if (q + 1 < H->nlev) {
            AIR_TRY(dalloc(&L.dinv, L.n));
            if (f32) AIR_TRY(dalloc(&L.dinv32, L.n));
            AIR_TRY(air_diag_inverse(L.n, L.rp, L.ci, L.v, L.dinv, L.dinv32, s));
            if (bf16) {
                AIR_TRY(dalloc(&L.diag32, L.n));
                AIR_TRY(air_cast_bf16(L.n, L.rp, L.ci, L.v, nullptr, L.diag32, s));
            }
            // level 0 of a matrix made of b x b blocks: the block form, else entries
            bool blocked = false;
            if (q == 0 && opt->block_size > 0) {
                Sell bf, bcs;
                int s0 = air_build_sell_blocks(L.nf, L.frows, L.rp, L.ci, L.v, opt->precision, opt->block_size, &bf, s);
                int s1 = s0 == AIR_OK ? air_build_sell_blocks(L.nc, L.crows, L.rp, L.ci, L.v, opt->precision,
                                                              opt->block_size, &bcs, s)
                                      : s0;
                if (s0 == AIR_OK && s1 == AIR_OK) {
                    L.sset[0] = bf;
                    L.sset[1] = bcs;
                    blocked = true;
                } else {
                    air_free_sell(bf);
                    air_free_sell(bcs);
                    if ((s0 != AIR_OK && s0 != AIR_ERR_UNSUPPORTED) || (s1 != AIR_OK && s1 != AIR_ERR_UNSUPPORTED))
                        return s0 != AIR_OK ? s0 : s1;
                }
            }
            if (!blocked) {
                AIR_TRY(air_build_sell(L.nf, L.frows, L.rp, L.ci, L.v, opt->precision, bf16, &L.sset[0], s));
                AIR_TRY(air_build_sell(L.nc, L.crows, L.rp, L.ci, L.v, opt->precision, bf16, &L.sset[1], s));
            }
            AIR_TRY(air_build_sell(L.nc, nullptr, L.rrp, L.rci, L.rv, opt->precision, 0, &L.sr, s));
        }
        size_t es = f32 ? sizeof(float) : sizeof(double);
        AIR_CUDA(air_dmalloc(&L.b, (size_t)(L.n > 0 ? L.n : 1) * es));
        AIR_CUDA(air_dmalloc(&L.x, (size_t)(L.n > 0 ? L.n : 1) * es));
        AIR_CUDA(air_dmalloc(&L.x2, (size_t)(L.n > 0 ? L.n : 1) * es));
    }
    {
        AirLevel &L0 = H->lev[0];
        int sb = opt->block_size > 0
                     ? air_build_sell_blocks(L0.n, nullptr, L0.rp, L0.ci, L0.v, AIR_PREC_F64, opt->block_size, &H->a0, s)
                     : AIR_ERR_UNSUPPORTED;
        if (sb != AIR_OK) {
            air_free_sell(H->a0);
            if (sb != AIR_ERR_UNSUPPORTED) return sb;
            AIR_TRY(air_build_sell(L0.n, nullptr, L0.rp, L0.ci, L0.v, AIR_PREC_F64, 0, &H->a0, s));
        }
    }
    if (f32) {
        AIR_TRY(dalloc(&H->cinv32, H->nco * H->nco));
        AIR_TRY(air_cast_d2f(H->cinv, H->cinv32, H->nco * H->nco, s));
    }
    AIR_TRY(air_tune_lanes(H, opt->autotune, s));
    AIR_TRY(air_gs_build(H, s));
    AIR_CUDA(cudaStreamSynchronize(s));
    return AIR_OK;
}

namespace {

int setup_impl(const air_csr *A, const air_options *opt, cudaStream_t s, air_hierarchy *H) {
    AIR_TRY(air_setup_begin(A, opt, s, H));
    int l = 0;
    for (;;) {
        H->nlev = l + 1;
        if (air_setup_is_coarsest(H, l)) break;
        int stop = 0;
        AIR_TRY(coarsen(H, l, s, &stop));
        if (stop) break;
        ++l;
    }
    return air_setup_end(H, s);
}

int ensure_workspace(air_hierarchy *H, int64_t n, int m) {
    if (H->ws_n == n && H->ws_m >= m) return AIR_OK;
    free_workspace(H);
    int nblk = air_reduce_nblk(n);
    AIR_TRY(dalloc(&H->V, (int64_t)(m + 1) * n));
    AIR_TRY(dalloc(&H->Z, (int64_t)m * n));
    AIR_TRY(dalloc(&H->partials, (int64_t)(m + 2) * nblk));
    AIR_TRY(dalloc(&H->hcol, 2 * (m + 2)));
    AIR_TRY(dalloc(&H->Hm, (int64_t)(m + 1) * m));
    AIR_TRY(dalloc(&H->gvec, m + 1));
    AIR_TRY(dalloc(&H->cs, m));
    AIR_TRY(dalloc(&H->sn, m));
    AIR_TRY(dalloc(&H->y, m));
    AIR_TRY(dalloc(&H->scal, 8));
    AIR_CUDA(cudaMallocHost((void **)&H->h_est, 8 * sizeof(double)));
    H->ws_n = n;
    H->ws_m = m;
    return AIR_OK;
}

// ||v||^2 into dst (device), via block partials
int norm2(int64_t n, const double *v, double *partials, int nblk, double *dst, cudaStream_t s) {
    AIR_TRY(air_dot_partials(n, v, 0, 1, v, partials, nblk, s));
    AIR_TRY(air_reduce_partials(1, partials, nblk, dst, s));
    return AIR_OK;
}

}  // namespace

// Flexible GMRES(m) with classical Gram-Schmidt applied twice and Givens
// rotations on the device (Section 5.1), split at its host reads so that
// independent problems can step in lockstep (batch.cu).  Every phase enqueues
// its work on g.s and ends with a device-to-host copy; the matching air_gmres_after_*
// runs once the stream has been synchronised and decides the next phase.
int air_gmres_open(AirGmres &g, const AirLevel &A0, const air_hierarchy *Hc, const double *b, double *x,
                   double rtol, cudaStream_t s, air_solve_info *info) {
    g.H = const_cast<air_hierarchy *>(Hc);
    g.A0 = &A0;
    g.b = b;
    g.x = x;
    g.rtol = rtol;
    g.s = s;
    g.info = info;
    g.n = A0.n;
    g.m = g.H->opt.restart;
    AIR_TRY(ensure_workspace(g.H, g.n, g.m));
    g.nblk = air_reduce_nblk(g.n);
    g.it = 0;
    g.j = 0;
    g.k = 0;
    info->iters = 0;
    info->restarts = 0;
    info->vcycles = 0;
    info->relres = 0.0;
    info->status = AIR_NOT_CONVERGED;
    double *sc = g.H->scal;   // [0] ||b||^2, [1] estimate, [2] h_{j+1,j}, [3] ||r||^2
    AIR_TRY(air_fill_zero(x, g.n, s));
    AIR_TRY(norm2(g.n, b, g.H->partials, g.nblk, sc, s));
    AIR_CUDA(cudaMemcpyAsync(g.H->h_est, sc, sizeof(double), cudaMemcpyDeviceToHost, s));
    g.phase = AirGmres::OPENED;
    return AIR_OK;
}

void air_gmres_after_open(AirGmres &g) {
    g.bnorm = sqrt(g.H->h_est[0]);
    if (g.bnorm == 0.0) {
        g.info->status = AIR_OK;
        g.phase = AirGmres::DONE;
    } else {
        g.phase = AirGmres::CYCLE;
    }
}

// Start of a restart cycle: r = b - A x into V_0 and its norm.
int air_gmres_cycle(AirGmres &g) {
    air_hierarchy *H = g.H;
    AIR_TRY(air_sell_spmv_f64(H->a0, g.x, H->V, g.b, g.s));
    AIR_TRY(norm2(g.n, H->V, H->partials, g.nblk, H->scal + 3, g.s));
    AIR_CUDA(cudaMemcpyAsync(H->h_est + 3, H->scal + 3, sizeof(double), cudaMemcpyDeviceToHost, g.s));
    return AIR_OK;
}

int air_gmres_after_cycle(AirGmres &g) {
    air_hierarchy *H = g.H;
    const double beta = sqrt(H->h_est[3]);
    g.info->relres = beta / g.bnorm;
    if (g.info->relres <= g.rtol) {
        g.info->status = AIR_OK;
        g.phase = AirGmres::DONE;
        return AIR_OK;
    }
    if (g.it >= H->opt.max_iter) {
        g.phase = AirGmres::DONE;
        return AIR_OK;
    }
    AIR_TRY(air_scale_vec(g.n, H->V, H->V, H->scal + 3, 1, g.s));
    AIR_CUDA(cudaMemsetAsync(H->gvec, 0, (size_t)(g.m + 1) * sizeof(double), g.s));
    AIR_TRY(air_set_scalar(H->gvec, beta, g.s));
    g.j = 0;
    g.k = 0;
    g.phase = AirGmres::STEP;
    return AIR_OK;
}

// The vectors of Arnoldi step j: z_j = M^{-1} v_j is the V-cycle's part.
double *air_gmres_vj(const AirGmres &g) { return g.H->V + (int64_t)g.j * g.n; }
double *air_gmres_zj(const AirGmres &g) { return g.H->Z + (int64_t)g.j * g.n; }

// Step j after its V-cycle: w = A z_j, CGS2 against V_0..V_j, Givens, v_{j+1}.
int air_gmres_step(AirGmres &g) {
    air_hierarchy *H = g.H;
    const int64_t n = g.n;
    const int j = g.j, m = g.m, nblk = g.nblk;
    double *h1 = H->hcol, *h2 = H->hcol + (m + 2), *sc = H->scal;
    double *zj = air_gmres_zj(g), *w = H->V + (int64_t)(j + 1) * n;
    g.info->vcycles++;
    AIR_TRY(air_sell_spmv_f64(H->a0, zj, w, nullptr, g.s));
    AIR_TRY(air_dot_partials(n, H->V, n, j + 1, w, H->partials, nblk, g.s));
    AIR_TRY(air_reduce_partials(j + 1, H->partials, nblk, h1, g.s));
    AIR_TRY(air_update_dot_partials(n, H->V, n, j + 1, h1, w, H->partials, nblk, j + 1, g.s));
    AIR_TRY(air_reduce_partials(j + 1, H->partials, nblk, h2, g.s));
    AIR_TRY(air_update_dot_partials(n, H->V, n, j + 1, h2, w, H->partials, nblk, -1, g.s));
    AIR_TRY(air_reduce_partials(1, H->partials, nblk, sc + 4, g.s));
    AIR_TRY(air_arnoldi_givens(j, m, h1, h2, sc + 4, H->Hm, H->cs, H->sn, H->gvec, sc, g.bnorm, g.s));
    AIR_TRY(air_scale_vec(n, w, w, sc + 2, 0, g.s));
    AIR_CUDA(cudaMemcpyAsync(H->h_est + 1, sc + 1, 2 * sizeof(double), cudaMemcpyDeviceToHost, g.s));
    return AIR_OK;
}

// After step j: end the cycle (solve the Hessenberg system, update x) when the
// estimate meets the tolerance, on breakdown, after m steps or at max_iter.
int air_gmres_after_step(AirGmres &g) {
    air_hierarchy *H = g.H;
    ++g.it;
    g.k = g.j + 1;
    const double est = H->h_est[1], hn = H->h_est[2];
    if (est <= g.rtol || hn == 0.0 || !(est == est) || g.k >= g.m || g.it >= H->opt.max_iter) {
        AIR_TRY(air_hessenberg_solve(g.k, g.m, H->Hm, H->gvec, H->y, g.s));
        AIR_TRY(air_axpy_multi(g.n, H->Z, g.n, g.k, H->y, g.x, g.s));
        g.info->restarts++;
        g.phase = AirGmres::CYCLE;
    } else {
        ++g.j;
    }
    return AIR_OK;
}

int air_gmres_close(AirGmres &g) {
    g.info->iters = g.it;
    AIR_CUDA(cudaStreamSynchronize(g.s));
    return g.info->status;
}

namespace {

int gmres_impl(const AirLevel &A0, const air_hierarchy *Hc, const double *b, double *x, double rtol,
               cudaStream_t s, air_solve_info *info) {
    AirGmres g;
    AIR_TRY(air_gmres_open(g, A0, Hc, b, x, rtol, s, info));
    AIR_CUDA(cudaStreamSynchronize(s));
    air_gmres_after_open(g);
    while (g.phase != AirGmres::DONE) {
        if (g.phase == AirGmres::CYCLE) {
            AIR_TRY(air_gmres_cycle(g));
            AIR_CUDA(cudaStreamSynchronize(s));
            AIR_TRY(air_gmres_after_cycle(g));
        } else {
            AIR_TRY(air_vcycle_run(g.H, air_gmres_vj(g), air_gmres_zj(g), s));
            AIR_TRY(air_gmres_step(g));
            AIR_CUDA(cudaStreamSynchronize(s));
            AIR_TRY(air_gmres_after_step(g));
        }
    }
    return air_gmres_close(g);
}

// Right-preconditioned BiCGSTAB (van der Vorst, 1992), the Krylov method the
// paper pairs with AIR (Section 5.1): the same iteration, restarts and stopping
// test as the oracle's, with dot products reduced on the device and the scalar
// recurrence (rho, alpha, omega) on the host, four small reads per iteration.
int bicgstab_impl(const AirLevel &A0, const air_hierarchy *Hc, const double *b, double *x, double rtol,
                  cudaStream_t s, air_solve_info *info) {
    air_hierarchy *H = const_cast<air_hierarchy *>(Hc);
    const int64_t n = A0.n;
    AIR_TRY(ensure_workspace(H, n, H->opt.restart > 8 ? H->opt.restart : 8));
    const int nblk = air_reduce_nblk(n);
    double *r = H->V, *rh = H->V + n, *p = H->V + 2 * n, *v = H->V + 3 * n;
    double *sv = H->V + 4 * n, *t = H->V + 5 * n, *ph = H->V + 6 * n, *sh = H->V + 7 * n;   // s, t adjacent
    double *sc = H->scal;
    auto fetch = [&](int k) -> int {
        AIR_CUDA(cudaMemcpyAsync(H->h_est, sc, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, s));
        AIR_CUDA(cudaStreamSynchronize(s));
        return AIR_OK;
    };
    auto dots = [&](const double *V, int k, const double *w) -> int {   // sc[i] = V_i . w, i < k
        AIR_TRY(air_dot_partials(n, V, n, k, w, H->partials, nblk, s));
        AIR_TRY(air_reduce_partials(k, H->partials, nblk, sc, s));
        return fetch(k);
    };
    info->iters = 0;
    info->restarts = 0;
    info->vcycles = 0;
    info->relres = 0.0;
    info->status = AIR_NOT_CONVERGED;
    AIR_TRY(air_fill_zero(x, n, s));
    AIR_TRY(dots(b, 1, b));
    const double bn = sqrt(H->h_est[0]);
    if (bn == 0.0) {
        info->status = AIR_OK;
        return AIR_OK;
    }
    AIR_CUDA(cudaMemcpyAsync(r, b, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    AIR_CUDA(cudaMemcpyAsync(rh, b, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    AIR_TRY(air_fill_zero(p, n, s));
    AIR_TRY(air_fill_zero(v, n, s));
    double rho_prev = 1.0, alpha = 1.0, omega = 1.0;
    info->relres = 1.0;
    bool conv = false;
    int it = 0;
    while (it < H->opt.max_iter) {
        AIR_TRY(dots(rh, 1, r));
        const double rho = H->h_est[0];
        if (rho == 0.0) break;
        const double beta = (rho / rho_prev) * (alpha / omega);
        AIR_TRY(air_lincomb(n, p, r, 1.0, p, beta, v, -beta * omega, s));        // p = r + beta (p - omega v)
        AIR_TRY(air_vcycle_run(H, p, ph, s));
        AIR_TRY(air_sell_spmv_f64(H->a0, ph, v, nullptr, s));
        AIR_TRY(dots(rh, 1, v));
        const double den = H->h_est[0];
        if (den == 0.0) break;
        alpha = rho / den;
        AIR_TRY(air_lincomb(n, sv, r, 1.0, v, -alpha, nullptr, 0.0, s));          // s = r - alpha v
        AIR_TRY(air_vcycle_run(H, sv, sh, s));
        AIR_TRY(air_sell_spmv_f64(H->a0, sh, t, nullptr, s));
        AIR_TRY(dots(sv, 2, t));                                                  // (s, t), (t, t)
        const double ts = H->h_est[0], tt = H->h_est[1];
        omega = tt > 0.0 ? ts / tt : 0.0;
        AIR_TRY(air_lincomb(n, x, x, 1.0, ph, alpha, sh, omega, s));              // x += alpha p^ + omega s^
        AIR_TRY(air_lincomb(n, r, sv, 1.0, t, -omega, nullptr, 0.0, s));          // r = s - omega t
        info->vcycles += 2;
        rho_prev = rho;
        ++it;
        AIR_TRY(dots(r, 1, r));
        if (sqrt(H->h_est[0]) / bn <= rtol) {
            AIR_TRY(air_sell_spmv_f64(H->a0, x, r, b, s));                       // true residual b - A x
            AIR_TRY(dots(r, 1, r));
            info->relres = sqrt(H->h_est[0]) / bn;
            if (info->relres <= rtol) { conv = true; break; }
            AIR_CUDA(cudaMemcpyAsync(rh, r, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s));
            AIR_TRY(air_fill_zero(p, n, s));
            AIR_TRY(air_fill_zero(v, n, s));
            rho_prev = alpha = omega = 1.0;
            info->restarts++;
            continue;
        }
        if (omega == 0.0) break;
    }
    if (!conv) {
        AIR_TRY(air_sell_spmv_f64(H->a0, x, r, b, s));
        AIR_TRY(dots(r, 1, r));
        info->relres = sqrt(H->h_est[0]) / bn;
    }
    info->iters = it;
    info->status = conv ? AIR_OK : AIR_NOT_CONVERGED;
    return info->status;
}

}  // namespace

// The options of one setup (opt, or the defaults when null, with theta and
// distance from the call), checked.
int air_check_options(double theta, int distance, const air_options *opt, air_options *out) {
    air_options &o = *out;
    if (opt) o = *opt; else air_default_options(&o);
    o.theta = theta;
    o.distance = distance;
    o.relax[sizeof(o.relax) - 1] = 0;
    bool gs = false;
    for (const char *c = o.relax; *c; ++c) {
        if (!strchr("FCAfca", *c)) return AIR_ERR_INVALID_ARG;
        gs = gs || (*c >= 'a');
    }
    if (gs && o.precision == AIR_PREC_BF16) return AIR_ERR_UNSUPPORTED;
    if (!(theta >= 0.0) || !(theta <= 1.0) || !(o.theta_r <= 1.0) || o.max_levels < 1 || o.max_levels > AIR_MAX_LEVELS ||
        o.max_dense < 1 || o.restart < 1 || o.restart > 32 || o.max_iter < 0 || o.falgout_block < 0 ||
        (o.falgout_block > 0 && (o.falgout_block % 1024 != 0 || o.falgout_block > 8192)) || o.block_size < 0 ||
        o.block_size > 16 ||
        (o.precision != AIR_PREC_F64 && o.precision != AIR_PREC_F32 && o.precision != AIR_PREC_BF16))
        return AIR_ERR_INVALID_ARG;
    if (distance < 1) return AIR_ERR_INVALID_ARG;
    if (distance > 2) return AIR_ERR_UNSUPPORTED;
    return AIR_OK;
}

extern "C" {

void air_default_options(air_options *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->theta = 0.25;
    o->distance = 1;
    strcpy(o->relax, "FCF");
    o->omega = 1.0;
    o->max_coarse = 1000;
    o->max_levels = 25;
    o->max_dense = 4096;
    o->precision = AIR_PREC_F64;
    o->restart = 30;
    o->max_iter = 1000;
    o->validate = 1;
    o->theta_r = -1.0;
    o->falgout_block = 0;
    o->block_size = 0;
    o->autotune = 0;
}

int air_setup(const air_csr *A, double theta, int distance, const air_options *opt, void *stream,
              air_hierarchy **out) {
    if (!out) return AIR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!A || !A->row_ptr || !A->col || !A->val || A->n_rows <= 0 || A->n_rows != A->n_cols || A->nnz < A->n_rows ||
        A->n_rows > INT32_MAX)
        return AIR_ERR_INVALID_ARG;
    air_options o;
    const int oc = air_check_options(theta, distance, opt, &o);
    if (oc != AIR_OK) return oc;
    air_hierarchy *H = new (std::nothrow) air_hierarchy();
    if (!H) return AIR_ERR_OOM;
    AirCallStream call((cudaStream_t)stream);
    int st = setup_impl(A, &o, (cudaStream_t)stream, H);
    if (st != AIR_OK) {
        cudaStreamSynchronize((cudaStream_t)stream);
        air_free(H);
        return st;
    }
    *out = H;
    return AIR_OK;
}

int air_vcycle(const air_hierarchy *H, const double *b, double *x, void *stream) {
    AirCallStream call((cudaStream_t)stream);
    if (!H || !b || !x) return AIR_ERR_INVALID_ARG;
    return air_vcycle_run(H, b, x, (cudaStream_t)stream);
}

int air_spmv(const air_csr *A, const double *x, double *y, void *stream) {
    if (!A || !x || !y || !A->on_device || A->n_rows <= 0) return AIR_ERR_INVALID_ARG;
    return air_spmv_f64(A->n_rows, A->row_ptr, A->col, A->val, x, y, nullptr, (cudaStream_t)stream, A->nnz, 0);
}

int air_hierarchy_spmv(const air_hierarchy *H, const double *x, double *y, void *stream) {
    if (!H || !x || !y || x == y) return AIR_ERR_INVALID_ARG;
    return air_sell_spmv_f64(H->a0, x, y, nullptr, (cudaStream_t)stream);
}

int air_bicgstab_solve(const air_csr *A, const air_hierarchy *H, const double *b, double *x, double rtol,
                       void *stream, air_solve_info *info) {
    if (!A || !H || !b || !x || !(rtol > 0.0) || A->n_rows != H->lev[0].n) return AIR_ERR_INVALID_ARG;
    AirCallStream call((cudaStream_t)stream);
    air_solve_info local;
    if (!info) info = &local;
    cudaStream_t s = (cudaStream_t)stream;
    air_hierarchy *Hm = const_cast<air_hierarchy *>(H);
    const int64_t n = A->n_rows;
    if (A->on_device) return bicgstab_impl(H->lev[0], H, b, x, rtol, s, info);
    if (!H->lev[0].owns_A || H->lev[0].v == nullptr) return AIR_ERR_INVALID_ARG;
    if (!Hm->bd) AIR_TRY(dalloc(&Hm->bd, n));
    if (!Hm->xd) AIR_TRY(dalloc(&Hm->xd, n));
    AIR_CUDA(cudaMemcpyAsync(Hm->bd, b, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, s));
    const int st = bicgstab_impl(H->lev[0], H, Hm->bd, Hm->xd, rtol, s, info);
    if (st < 0) return st;
    AIR_CUDA(cudaMemcpyAsync(x, Hm->xd, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s));
    AIR_CUDA(cudaStreamSynchronize(s));
    return st;
}

namespace {
bool fc_jacobi_only(const air_hierarchy *H) {
    for (const char *c = H->opt.relax; *c; ++c)
        if (*c != 'F' && *c != 'C') return false;
    return true;
}
}  // namespace

int air_vcycle_multi(const air_hierarchy *H, int k, const double *b, double *x, void *stream) {
    if (!H || !b || !x || k < 1 || k > 32) return AIR_ERR_INVALID_ARG;
    if (!fc_jacobi_only(H)) return AIR_ERR_UNSUPPORTED;
    AirCallStream call((cudaStream_t)stream);
    return air_vcycle_multi_run(H, k, b, x, (cudaStream_t)stream);
}

int air_vcycle_multi_f32(const air_hierarchy *H, int k, const float *b, float *x, void *stream) {
    if (!H || !b || !x || k < 1 || k > 32) return AIR_ERR_INVALID_ARG;
    if (!fc_jacobi_only(H)) return AIR_ERR_UNSUPPORTED;
    AirCallStream call((cudaStream_t)stream);
    return air_vcycle_multi_run_f32(H, k, b, x, (cudaStream_t)stream);
}

int air_bicgstab_solve_multi(const air_csr *A, const air_hierarchy *H, int k, const double *b, double *x,
                             double rtol, void *stream, air_solve_info *info) {
    if (!A || !H || !b || !x || !info || k < 1 || k > 32 || !(rtol > 0.0) || !A->on_device ||
        A->n_rows != H->lev[0].n)
        return AIR_ERR_INVALID_ARG;
    if (!fc_jacobi_only(H)) return AIR_ERR_UNSUPPORTED;
    AirCallStream call((cudaStream_t)stream);
    return air_bicgstab_multi_impl(H, k, b, x, rtol, (cudaStream_t)stream, info);
}

int air_csr_transpose(const air_csr *A, int64_t *row_ptr_t, int32_t *col_t, double *val_t, void *stream) {
    if (!A || !row_ptr_t || !A->on_device || A->n_rows < 0 || A->n_cols < 0 || A->nnz < 0 || !A->row_ptr)
        return AIR_ERR_INVALID_ARG;
    if (A->nnz > 0 && (!A->col || !A->val || !col_t || !val_t)) return AIR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int *d_err = nullptr;
    AIR_CUDA(cudaMallocAsync(&d_err, sizeof(int), s));
    AIR_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), s));
    int st = air_csr_transpose_impl(A->n_rows, A->n_cols, A->nnz, A->row_ptr, A->col, A->val, row_ptr_t, col_t,
                                    val_t, d_err, s);
    int herr = 0;
    if (st == AIR_OK) {
        cudaError_t e = cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = AIR_ERR_CUDA;
    }
    cudaFreeAsync(d_err, s);
    if (st == AIR_OK && herr) st = AIR_ERR_CSR_MALFORMED;
    return st;
}

int air_csr_transpose_scaled(const air_csr *A, int b, const double *diag, int64_t *row_ptr_t, int32_t *col_t,
                             double *val_t, void *stream) {
    if (!A || !diag || !row_ptr_t || !col_t || !val_t || !A->on_device || !A->row_ptr || !A->col || !A->val ||
        b < 1 || b > 11 || A->n_rows <= 0 || A->n_rows != A->n_cols || A->n_rows % b != 0)
        return AIR_ERR_INVALID_ARG;
    AirCallStream call((cudaStream_t)stream);
    cudaStream_t s = (cudaStream_t)stream;
    int *d_err = nullptr;
    AIR_CUDA(cudaMallocAsync(&d_err, sizeof(int), s));
    AIR_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), s));
    int st = air_csr_transpose_impl(A->n_rows, A->n_cols, A->nnz, A->row_ptr, A->col, A->val, row_ptr_t, col_t,
                                    val_t, d_err, s);
    if (st == AIR_OK) st = air_block_scale_transpose_impl(A->n_rows, b, diag, row_ptr_t, col_t, val_t, d_err, s);
    int herr = 0;
    if (st == AIR_OK) {
        cudaError_t e = cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = AIR_ERR_CUDA;
    }
    cudaFreeAsync(d_err, s);
    if (st == AIR_OK && (herr & AIR_DEVERR_SINGULAR)) st = AIR_ERR_SINGULAR_COARSE;
    else if (st == AIR_OK && herr) st = AIR_ERR_CSR_MALFORMED;
    return st;
}

int air_block_diag_apply(int64_t nblocks, int b, const double *diag, int op, const double *x, double *y,
                         void *stream) {
    if (nblocks < 0 || b < 1 || b > 11 || op < 0 || op > 3 || (nblocks > 0 && (!diag || !x || !y)))
        return AIR_ERR_INVALID_ARG;
    if (nblocks == 0) return AIR_OK;
    AirCallStream call((cudaStream_t)stream);
    cudaStream_t s = (cudaStream_t)stream;
    int *d_err = nullptr;
    AIR_CUDA(cudaMallocAsync(&d_err, sizeof(int), s));
    AIR_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), s));
    int st = air_block_apply_impl(nblocks, b, diag, op, x, y, d_err, s);
    int herr = 0;
    if (st == AIR_OK) {
        cudaError_t e = cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = AIR_ERR_CUDA;
    }
    cudaFreeAsync(d_err, s);
    if (st == AIR_OK && herr) st = AIR_ERR_SINGULAR_COARSE;
    return st;
}

int air_csr_outer(const air_csr *A, const double *u, const double *w, double alpha, double *out, void *stream) {
    if (!A || !A->on_device || A->n_rows < 0 || A->nnz < 0 || !A->row_ptr) return AIR_ERR_INVALID_ARG;
    if (A->nnz > 0 && (!A->col || !u || !w || !out)) return AIR_ERR_INVALID_ARG;
    return air_csr_outer_impl(A->n_rows, A->n_cols, A->row_ptr, A->col, u, w, alpha, out, (cudaStream_t)stream);
}

int air_gmres_solve(const air_csr *A, const air_hierarchy *H, const double *b, double *x, double rtol, void *stream,
                    air_solve_info *info) {
    if (!A || !H || !b || !x || !(rtol > 0.0) || A->n_rows != H->lev[0].n) return AIR_ERR_INVALID_ARG;
    AirCallStream call((cudaStream_t)stream);
    air_solve_info local;
    if (!info) info = &local;
    cudaStream_t s = (cudaStream_t)stream;
    air_hierarchy *Hm = const_cast<air_hierarchy *>(H);
    int64_t n = A->n_rows;
    if (A->on_device) {
        AirLevel A0 = H->lev[0];
        A0.rp = A->row_ptr; A0.ci = A->col; A0.v = A->val; A0.nnz = A->nnz;
        return gmres_impl(A0, H, b, x, rtol, s, info);
    }
    if (!H->lev[0].owns_A || H->lev[0].v == nullptr) return AIR_ERR_INVALID_ARG;
    if (!Hm->bd) AIR_TRY(dalloc(&Hm->bd, n));
    if (!Hm->xd) AIR_TRY(dalloc(&Hm->xd, n));
    AIR_CUDA(cudaMemcpyAsync(Hm->bd, b, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, s));
    int st = gmres_impl(H->lev[0], H, Hm->bd, Hm->xd, rtol, s, info);
    if (st < 0) return st;
    AIR_CUDA(cudaMemcpyAsync(x, Hm->xd, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s));
    AIR_CUDA(cudaStreamSynchronize(s));
    return st;
}

int air_hierarchy_levels(const air_hierarchy *H) { return H ? H->nlev : 0; }

int air_setup_timings(const air_hierarchy *H, double *ms, int count) {
    if (!H || !ms || count < 0) return AIR_ERR_INVALID_ARG;
    for (int i = 0; i < count && i < 11; ++i) ms[i] = H->phase_ms[i];
    return AIR_OK;
}

int air_hierarchy_info(const air_hierarchy *H, int level, air_level_info *info) {
    if (!H || !info || level < 0 || level >= H->nlev) return AIR_ERR_INVALID_ARG;
    const AirLevel &L = H->lev[level];
    info->n = L.n;
    info->nnz = L.nnz;
    info->nnz_s = L.nnz_s;
    info->nc = L.nc;
    info->nnz_r = L.nnz_r;
    info->n_singular = L.n_singular;
    info->max_m = L.max_m;
    info->coarsest = level == H->nlev - 1;
    info->block_size = L.sset[0].b > 0 ? L.sset[0].b : L.sset[1].b;
    info->lanes_f = L.lanes[0];
    info->lanes_c = L.lanes[1];
    info->lanes_r = L.lanes[2];
    return AIR_OK;
}

int air_hierarchy_export(const air_hierarchy *H, int level, int what, void *dst) {
    if (!H || !dst || level < 0 || level >= H->nlev) return AIR_ERR_INVALID_ARG;
    const AirLevel &L = H->lev[level];
    const void *src = nullptr;
    size_t bytes = 0;
    switch (what) {
    case 0: src = L.rp; bytes = (size_t)(L.n + 1) * 8; break;
    case 1: src = L.ci; bytes = (size_t)L.nnz * 4; break;
    case 2: src = L.v; bytes = (size_t)L.nnz * 8; break;
    case 3: src = L.srp; bytes = (size_t)(L.n + 1) * 8; break;
    case 4: src = L.sci; bytes = (size_t)L.nnz_s * 4; break;
    case 5: src = L.cf; bytes = (size_t)L.n; break;
    case 6: src = L.cid; bytes = (size_t)L.n * 4; break;
    case 7: src = L.rrp; bytes = (size_t)(L.nc + 1) * 8; break;
    case 8: src = L.rci; bytes = (size_t)L.nnz_r * 4; break;
    case 9: src = L.rv; bytes = (size_t)L.nnz_r * 8; break;
    case 10: src = L.pcol; bytes = (size_t)L.n * 4; break;
    default: return AIR_ERR_INVALID_ARG;
    }
    if (!src) return AIR_ERR_INVALID_ARG;
    if (bytes == 0) return AIR_OK;
    AIR_CUDA(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
    return AIR_OK;
}

void air_free(air_hierarchy *H) {
    if (!H) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != H->dev) cudaSetDevice(H->dev);
    cudaDeviceSynchronize();
    for (int l = 0; l < AIR_MAX_LEVELS; ++l) free_level(H->lev[l]);
    air_free_multi(H);
    air_free_sell(H->a0);
    if (H->vgraph) cudaGraphExecDestroy(H->vgraph);
    H->vgraph = nullptr;
    dfree(H->cinv);
    dfree(H->cinv32);
    dfree(H->d_err);
    dfree(H->d_stats);
    dfree(H->xd);
    dfree(H->bd);
    free_workspace(H);
    if (cur != H->dev) cudaSetDevice(cur);
    delete H;
}

unsigned long long air_kernel_launches(void) { return g_launches.load(); }

const char *air_status_string(int s) {
    switch (s) {
    case AIR_OK: return "ok";
    case AIR_NOT_CONVERGED: return "not converged within max_iter";
    case AIR_ERR_INVALID_ARG: return "invalid argument";
    case AIR_ERR_CSR_MALFORMED: return "malformed CSR matrix";
    case AIR_ERR_OOM: return "device out of memory";
    case AIR_ERR_CUDA: return "CUDA runtime error";
    case AIR_ERR_SINGULAR_COARSE: return "coarsest operator singular";
    case AIR_ERR_DEVICE_TIMEOUT: return "device loop hit its iteration cap";
    case AIR_ERR_COARSE_TOO_LARGE: return "coarsening stalled above max_dense";
    case AIR_ERR_UNSUPPORTED: return "option not supported on the GPU path";
    case AIR_ERR_NOALLOC_LIMIT: return "problem exceeds the fixed workspace of the allocation-free solve";
    default: return "unknown status";
    }
}

}  // extern "C"
