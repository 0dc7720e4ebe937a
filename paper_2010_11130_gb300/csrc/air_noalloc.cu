// air_gmres_solve_noalloc: the flexible GMRES solve of air_gmres_solve with
// its Krylov workspace in a fixed, file-scope device array instead of memory
// the library allocates.
//
// Why: some callers cannot let a library call cudaMalloc -- an application
// whose memory is fully pre-assigned by a pool or budget it must not exceed,
// or a host framework that forbids device allocation inside its solve phase
// (allocation there can synchronise the device or fail under memory pressure
// at a point the caller cannot recover from).  They build the hierarchy up
// front with air_setup and then solve without any further allocation.
//
// The array below is reserved on every GPU that loads the library and stays
// there until the process exits.  In host code its name only stands for the
// device symbol: the device address is obtained once per device with
// cudaGetSymbolAddress and passed to the kernels.
#include <math.h>
#include <string.h>

#include <mutex>

#include "air_internal.cuh"

namespace {

// 32 MiB of FP64 words: V (m+1) x n, Z m x n, reduction partials and the
// small Arnoldi arrays must fit (restart 30 -> n up to about 68,000).
constexpr int64_t kWsDoubles = (int64_t)4 * 1024 * 1024;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_ws[kWsDoubles];

std::mutex g_mu;
double *g_ws_addr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_ws on the current device, looked up on the
// first call on each device and kept: a cudaDeviceReset of that device
// reloads the module and invalidates it (the header tells callers so).
int workspace_address(double **out) {
    int dev = 0;
    AIR_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return AIR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ws_addr[dev]) {
        void *p = nullptr;
        AIR_CUDA(cudaGetSymbolAddress(&p, g_noalloc_ws));
        g_ws_addr[dev] = (double *)p;
    }
    *out = g_ws_addr[dev];
    return AIR_OK;
}

struct Ws {
    double *V, *Z, *partials, *h1, *h2, *Hm, *g, *cs, *sn, *y, *sc;
};

int64_t ws_need(int64_t n, int m, int nblk) {
    return (int64_t)(m + 1) * n + (int64_t)m * n + (int64_t)(m + 2) * nblk + 2 * (m + 2) +
           (int64_t)(m + 1) * m + (m + 1) + 3 * m + 8 + 64;
}

Ws carve(double *base, int64_t n, int m, int nblk) {
    Ws w;
    double *p = base;
    auto take = [&](int64_t k) { double *q = p; p += k; return q; };
    w.V = take((int64_t)(m + 1) * n);
    w.Z = take((int64_t)m * n);
    w.partials = take((int64_t)(m + 2) * nblk);
    w.h1 = take(m + 2);
    w.h2 = take(m + 2);
    w.Hm = take((int64_t)(m + 1) * m);
    w.g = take(m + 1);
    w.cs = take(m);
    w.sn = take(m);
    w.y = take(m);
    w.sc = take(8);
    return w;
}

int read_scalars(const double *d, double *h, int count, cudaStream_t s) {
    AIR_CUDA(cudaMemcpyAsync(h, d, (size_t)count * sizeof(double), cudaMemcpyDeviceToHost, s));
    AIR_CUDA(cudaStreamSynchronize(s));
    return AIR_OK;
}

int norm2(int64_t n, const double *v, double *partials, int nblk, double *dst, cudaStream_t s) {
    AIR_TRY(air_dot_partials(n, v, 0, 1, v, partials, nblk, s));
    AIR_TRY(air_reduce_partials(1, partials, nblk, dst, s));
    return AIR_OK;
}

}  // namespace

extern "C" int air_gmres_solve_noalloc(const air_csr *A, const air_hierarchy *H, const double *b, double *x,
                                       double rtol, void *stream, air_solve_info *info) {
    if (!A || !H || !b || !x || !(rtol > 0.0) || !A->on_device || A->n_rows != H->lev[0].n)
        return AIR_ERR_INVALID_ARG;
    const int64_t n = A->n_rows;
    const int m = H->opt.restart;
    const int nblk = air_reduce_nblk(n);
    if (ws_need(n, m, nblk) > kWsDoubles) return AIR_ERR_NOALLOC_LIMIT;
    air_solve_info local;
    if (!info) info = &local;
    cudaStream_t s = (cudaStream_t)stream;
    double *base = nullptr;
    AIR_TRY(workspace_address(&base));
    Ws w = carve(base, n, m, nblk);
    AirLevel A0 = H->lev[0];
    A0.rp = A->row_ptr;
    A0.ci = A->col;
    A0.v = A->val;
    A0.nnz = A->nnz;
    double hs[8] = {0};
    info->iters = 0;
    info->restarts = 0;
    info->vcycles = 0;
    info->relres = 0.0;
    info->status = AIR_NOT_CONVERGED;
    // the array keeps the previous call's contents: clear the scalar block
    AIR_CUDA(cudaMemsetAsync(w.sc, 0, 8 * sizeof(double), s));
    AIR_TRY(air_fill_zero(x, n, s));
    AIR_TRY(norm2(n, b, w.partials, nblk, w.sc, s));
    AIR_TRY(read_scalars(w.sc, hs, 1, s));
    double bnorm = sqrt(hs[0]);
    if (bnorm == 0.0) {
        info->status = AIR_OK;
        return AIR_OK;
    }
    int it = 0;
    for (;;) {
        AIR_TRY(air_spmv_f64(n, A0.rp, A0.ci, A0.v, x, w.V, b, s, A0.nnz, A0.maxrow));
        AIR_TRY(norm2(n, w.V, w.partials, nblk, w.sc + 3, s));
        AIR_TRY(read_scalars(w.sc + 3, hs + 3, 1, s));
        double beta = sqrt(hs[3]);
        info->relres = beta / bnorm;
        if (info->relres <= rtol) { info->status = AIR_OK; break; }
        if (it >= H->opt.max_iter) break;
        AIR_TRY(air_scale_vec(n, w.V, w.V, w.sc + 3, 1, s));
        AIR_CUDA(cudaMemsetAsync(w.g, 0, (size_t)(m + 1) * sizeof(double), s));
        AIR_TRY(air_set_scalar(w.g, beta, s));
        int k = 0;
        for (int j = 0; j < m && it < H->opt.max_iter; ++j) {
            double *vj = w.V + (int64_t)j * n, *zj = w.Z + (int64_t)j * n, *wj = w.V + (int64_t)(j + 1) * n;
            AIR_TRY(air_vcycle_run(H, vj, zj, s, 0));   // no graph: instantiating one may allocate
            info->vcycles++;
            AIR_TRY(air_spmv_f64(n, A0.rp, A0.ci, A0.v, zj, wj, nullptr, s, A0.nnz, A0.maxrow));
            AIR_TRY(air_dot_partials(n, w.V, n, j + 1, wj, w.partials, nblk, s));
            AIR_TRY(air_reduce_partials(j + 1, w.partials, nblk, w.h1, s));
            AIR_TRY(air_update_dot_partials(n, w.V, n, j + 1, w.h1, wj, w.partials, nblk, j + 1, s));
            AIR_TRY(air_reduce_partials(j + 1, w.partials, nblk, w.h2, s));
            AIR_TRY(air_update_dot_partials(n, w.V, n, j + 1, w.h2, wj, w.partials, nblk, -1, s));
            AIR_TRY(air_reduce_partials(1, w.partials, nblk, w.sc + 4, s));
            AIR_TRY(air_arnoldi_givens(j, m, w.h1, w.h2, w.sc + 4, w.Hm, w.cs, w.sn, w.g, w.sc, bnorm, s));
            AIR_TRY(air_scale_vec(n, wj, wj, w.sc + 2, 0, s));
            AIR_TRY(read_scalars(w.sc + 1, hs + 1, 2, s));
            ++it;
            k = j + 1;
            double est = hs[1], hn = hs[2];
            if (est <= rtol || hn == 0.0 || !(est == est)) break;
        }
        AIR_TRY(air_hessenberg_solve(k, m, w.Hm, w.g, w.y, s));
        AIR_TRY(air_axpy_multi(n, w.Z, n, k, w.y, x, s));
        info->restarts++;
    }
    info->iters = it;
    AIR_CUDA(cudaStreamSynchronize(s));
    return info->status;
}
