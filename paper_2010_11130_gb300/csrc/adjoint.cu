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
