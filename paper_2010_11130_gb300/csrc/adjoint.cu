// Operations for the adjoint of the condensed system.
//
// A solve u = A^{-1} b of the block-scaled trace system (Section 2.5) has the
// adjoint lambda = A^{-T} g for a loss gradient g = dL/du: then dL/db = lambda
// and dL/da_ij = -lambda_i u_j on the stored entries of A.  A^T keeps the unit
// diagonal blocks of A and is the upwind operator of the reversed flow, so the
// same l-AIR setup applies to it.  This file holds the two operations the
// adjoint needs beyond setup and solve: the transpose of A with its values and
// the outer product restricted to A's pattern.
#include "air_internal.cuh"
#include "warp_dense.cuh"

namespace {

unsigned blocks_for(int64_t items, int threads) {
    int64_t b = (items + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)b;
}

__global__ void col_count_kernel(int64_t nnz, const int32_t *ci, int64_t ncols, int32_t *cnt, int *err) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = ci[e];
        if (c < 0 || c >= ncols) { atomicOr(err, AIR_DEVERR_CSR); continue; }
        atomicAdd(&cnt[c], 1);
    }
}

// Entries of row i go to row ci[e] of the transpose at a claimed slot.
__global__ void scatter_t_kernel(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, int64_t ncols,
                                 const int64_t *rpt, int32_t *fill, int32_t *cit, double *vt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            const int32_t c = ci[e];
            if (c < 0 || c >= ncols) continue;
            const int64_t p = rpt[c] + atomicAdd(&fill[c], 1);
            cit[p] = (int32_t)i;
            vt[p] = v[e];
        }
    }
}

// The slots were claimed in any order: sort each row of the transpose by
// column (an insertion sort; rows hold a few dozen entries).
__global__ void sort_rows_kernel(int64_t m, const int64_t *rpt, int32_t *cit, double *vt) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = rpt[r], e = rpt[r + 1];
        for (int64_t p = b + 1; p < e; ++p) {
            const int32_t c = cit[p];
            const double x = vt[p];
            int64_t q = p - 1;
            while (q >= b && cit[q] > c) {
                cit[q + 1] = cit[q];
                vt[q + 1] = vt[q];
                --q;
            }
            cit[q + 1] = c;
            vt[q + 1] = x;
        }
    }
}

__global__ void outer_kernel(int64_t n, int64_t ncols, const int64_t *rp, const int32_t *ci, const double *u,
                             const double *w, double alpha, double *out) {
    // one warp per row: u_i once, w gathered along the row
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        const double ai = alpha * u[i];
        for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += 32) {
            const int32_t c = ci[e];
            out[e] = (c >= 0 && c < ncols) ? ai * w[c] : __longlong_as_double(0x7ff8000000000000ll);   // NaN marks a bad column
        }
    }
}

// One warp per block row f of A^T (rows f b .. f b + b - 1): every
// off-diagonal block B (columns g b .. g b + b - 1) becomes D_f^{-T} B D_g^T,
// the diagonal block (stored as its b ones) stays the identity.  Rows of a
// block row must share one layout of whole blocks; otherwise err gets
// AIR_DEVERR_CSR and the block row is left unscaled.
__global__ void __launch_bounds__(128) block_scale_t_kernel(int64_t nblk, int b, const double *diag,
                                                            const int64_t *rpt, const int32_t *cit, double *vt,
                                                            int *err) {
    extern __shared__ double bsm[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t f = (int64_t)blockIdx.x * 4 + w;
    if (f >= nblk) return;
    const int bb = b * b;
    double *Dt = bsm + (size_t)w * 6 * bb, *Di = Dt + bb, *W = Di + bb, *T = W + 2 * bb, *G = T + bb;
    const int64_t r0 = f * b;
    const int64_t len = rpt[r0 + 1] - rpt[r0];
    bool ok = len >= 1 && (len - 1) % b == 0;
    for (int i = 1; i < b && ok; ++i) ok = rpt[r0 + i + 1] - rpt[r0 + i] == len;
    if (!ok) {
        if (lane == 0) atomicOr(err, AIR_DEVERR_CSR);
        return;
    }
    for (int t = lane; t < bb; t += 32) Dt[t] = diag[f * bb + (t % b) * b + t / b];   // D_f^T
    __syncwarp();
    if (!warp_inverse(Dt, b, W, Di)) {                                               // Di = D_f^{-T}
        if (lane == 0) atomicOr(err, AIR_DEVERR_SINGULAR);
        return;
    }
    const int64_t nb = (len - 1) / b;
    int64_t p = 0;                      // position within the row
    for (int64_t k = 0; k < nb; ++k) {
        // skip the diagonal entry if it comes first
        const int32_t c0 = cit[rpt[r0] + p];
        if (c0 / b == f) ++p;
        const int64_t off = p;
        const int32_t cs = cit[rpt[r0] + off];
        const int64_t g = cs / b;
        bool good = cs % b == 0 && g != f;
        for (int i = 0; i < b && good; ++i)
            for (int j = 0; j < b && good; ++j) good = cit[rpt[r0 + i] + off + j] == (int32_t)(g * b + j);
        if (!good) {
            if (lane == 0) atomicOr(err, AIR_DEVERR_CSR);
            return;
        }
        for (int t = lane; t < bb; t += 32) {
            const int i = t / b, j = t % b;
            T[t] = vt[rpt[r0 + i] + off + j];
            G[t] = diag[g * bb + t];                                                  // D_g
        }
        __syncwarp();
        // T <- Di T G^T
        double res[4];
        int cntr = 0;
        for (int t = lane; t < bb; t += 32) {
            const int i = t / b, j = t % b;
            double acc = 0.0;
            for (int a = 0; a < b; ++a) {
                double inner = 0.0;
                for (int c = 0; c < b; ++c) inner += T[a * b + c] * G[j * b + c];
                acc += Di[i * b + a] * inner;
            }
            res[cntr++] = acc;
        }
        __syncwarp();
        cntr = 0;
        for (int t = lane; t < bb; t += 32) {
            const int i = t / b, j = t % b;
            vt[rpt[r0 + i] + off + j] = res[cntr++];
        }
        __syncwarp();
        p = off + b;
    }
}

// y_k = op(D_k) x_k over the b-blocks: op 0 D, 1 D^T, 2 D^{-1}, 3 D^{-T}.  One warp per block.
__global__ void __launch_bounds__(128) block_apply_kernel(int64_t nblk, int b, const double *diag, int op,
                                                          const double *x, double *y, int *err) {
    extern __shared__ double bsm[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t k = (int64_t)blockIdx.x * 4 + w;
    if (k >= nblk) return;
    const int bb = b * b;
    double *M = bsm + (size_t)w * 5 * bb, *Mi = M + bb, *W = Mi + bb, *xs = W + 2 * bb;
    const bool tr = op == 1 || op == 3;
    for (int t = lane; t < bb; t += 32) M[t] = tr ? diag[k * bb + (t % b) * b + t / b] : diag[k * bb + t];
    for (int t = lane; t < b; t += 32) xs[t] = x[k * b + t];
    __syncwarp();
    const double *Op = M;
    if (op >= 2) {
        if (!warp_inverse(M, b, W, Mi)) {
            if (lane == 0) atomicOr(err, AIR_DEVERR_SINGULAR);
            return;
        }
        Op = Mi;
    }
    for (int i = lane; i < b; i += 32) {
        double acc = 0.0;
        for (int j = 0; j < b; ++j) acc += Op[i * b + j] * xs[j];
        y[k * b + i] = acc;
    }
}

}  // namespace

int air_csr_transpose_impl(int64_t n, int64_t ncols, int64_t nnz, const int64_t *rp, const int32_t *ci,
                           const double *v, int64_t *rpt, int32_t *cit, double *vt, int *d_err, cudaStream_t s) {
    int32_t *cnt = nullptr;
    AIR_CUDA(cudaMallocAsync(&cnt, (size_t)(ncols > 0 ? ncols : 1) * sizeof(int32_t), s));
    AIR_CUDA(cudaMemsetAsync(cnt, 0, (size_t)(ncols > 0 ? ncols : 1) * sizeof(int32_t), s));
    if (nnz > 0) {
        col_count_kernel<<<air_counted(blocks_for(nnz, 256)), 256, 0, s>>>(nnz, ci, ncols, cnt, d_err);
        AIR_LAUNCH();
    }
    int st = air_exclusive_scan_i32(cnt, rpt, ncols, s);
    if (st == AIR_OK) {
        AIR_CUDA(cudaMemsetAsync(cnt, 0, (size_t)(ncols > 0 ? ncols : 1) * sizeof(int32_t), s));
        scatter_t_kernel<<<air_counted(blocks_for(n, 256)), 256, 0, s>>>(n, rp, ci, v, ncols, rpt, cnt, cit, vt);
        AIR_LAUNCH();
        sort_rows_kernel<<<air_counted(blocks_for(ncols, 256)), 256, 0, s>>>(ncols, rpt, cit, vt);
        AIR_LAUNCH();
    }
    cudaFreeAsync(cnt, s);
    return st;
}

int air_csr_outer_impl(int64_t n, int64_t ncols, const int64_t *rp, const int32_t *ci, const double *u,
                       const double *w, double alpha, double *out, cudaStream_t s) {
    if (n <= 0) return AIR_OK;
    outer_kernel<<<air_counted(blocks_for(n * 32, 256)), 256, 0, s>>>(n, ncols, rp, ci, u, w, alpha, out);
    AIR_LAUNCH();
    return AIR_OK;
}

int air_block_scale_transpose_impl(int64_t n, int b, const double *diag, const int64_t *rpt, const int32_t *cit,
                                   double *vt, int *d_err, cudaStream_t s) {
    const int64_t nblk = n / b;
    const size_t smem = (size_t)4 * 6 * b * b * sizeof(double);
    if (nblk <= 0) return AIR_OK;
    block_scale_t_kernel<<<air_counted((unsigned)((nblk + 3) / 4)), 128, smem, s>>>(nblk, b, diag, rpt, cit, vt,
                                                                                     d_err);
    AIR_LAUNCH();
    return AIR_OK;
}

int air_block_apply_impl(int64_t nblk, int b, const double *diag, int op, const double *x, double *y, int *d_err,
                         cudaStream_t s) {
    const size_t smem = (size_t)4 * 5 * b * b * sizeof(double);
    if (nblk <= 0) return AIR_OK;
    block_apply_kernel<<<air_counted((unsigned)((nblk + 3) / 4)), 128, smem, s>>>(nblk, b, diag, op, x, y, d_err);
    AIR_LAUNCH();
    return AIR_OK;
}
