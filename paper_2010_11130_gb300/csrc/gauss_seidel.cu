// Forward Gauss-Seidel relaxation, the paper's post-relaxation (Section 4
// settings: forward Gauss-Seidel on the F points, then on all points), in
// ascending point order on every level, as sweeps the relaxation string
// selects with 'f' (F points), 'c' (C points) and 'a' (all points).
//
// A sweep over a point set S updates i in S in ascending order with the
// values already updated: x_i <- x_i + omega (b_i - sum_j a_ij x_j) / a_ii,
// where x_j is new for j < i and old for j >= i.  Rows with no coupling to a
// lower-index row of S depend on nothing; grouping every row by its depth in
// the graph of lower-index couplings inside S gives groups whose rows are
// independent, and processing the groups in depth order reproduces the
// sequential sweep exactly.  The schedule is built once at setup by a
// frontier traversal (one launch per depth); a sweep copies x to a second
// vector xn, runs one launch per group that reads x_j from xn for j < i and
// from x otherwise and writes xn_i, then copies xn back.
#include <string.h>

#include <type_traits>
#include <vector>

#include "air_internal.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;

unsigned grid_for(int64_t items, int threads) {
    int64_t b = (items + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)b;
}

__device__ __forceinline__ bool in_set(const int8_t *cf, int which, int64_t j) {
    return which == 2 || cf[j] == which;
}

// in-degree (lower-index couplings inside the set) and the out-degree counts of the transposed graph
__global__ void gs_degree_kernel(int64_t n, const int64_t *rp, const int32_t *ci, const int8_t *cf, int which,
                                 int32_t *indeg, int32_t *outdeg) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (!in_set(cf, which, i)) { indeg[i] = -1; continue; }
        int d = 0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
            const int32_t j = ci[k];
            if (j < i && in_set(cf, which, j)) { ++d; atomicAdd(&outdeg[j], 1); }
        }
        indeg[i] = d;
    }
}

__global__ void gs_succ_kernel(int64_t n, const int64_t *rp, const int32_t *ci, const int8_t *cf, int which,
                               const int64_t *optr, int32_t *fill, int32_t *succ) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (!in_set(cf, which, i)) continue;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
            const int32_t j = ci[k];
            if (j < i && in_set(cf, which, j)) succ[optr[j] + atomicAdd(&fill[j], 1)] = (int32_t)i;
        }
    }
}

__global__ void gs_roots_kernel(int64_t n, const int32_t *indeg, int32_t *rows, unsigned long long *tail) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (indeg[i] == 0) rows[atomicAdd(tail, 1ull)] = (int32_t)i;
}

// one depth step: successors whose last lower-index coupling was just placed join the next group
__global__ void gs_advance_kernel(int64_t a, int64_t b, const int64_t *optr, const int32_t *succ, int32_t *indeg,
                                  int32_t *rows, unsigned long long *tail) {
    for (int64_t t = a + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < b; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = rows[t];
        for (int64_t k = optr[i]; k < optr[i + 1]; ++k) {
            const int32_t sx = succ[k];
            if (atomicSub(&indeg[sx], 1) == 1) rows[atomicAdd(tail, 1ull)] = sx;
        }
    }
}

// one group: VL lanes per row
template <int VL, typename TV, typename T>
__global__ void __launch_bounds__(256) gs_group_kernel(int64_t cnt, const int32_t *rows, const int64_t *rp,
                                                       const int32_t *ci, const TV *v, const T *xo, T *xn,
                                                       const T *b, const T *dinv, T omega) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t g = t / VL;
    const int j0 = (int)(t % VL);
    const bool valid = g < cnt;
    T acc = 0;
    int64_t i = 0;
    if (valid) {
        i = rows[g];
        for (int64_t k = rp[i] + j0; k < rp[i + 1]; k += VL) {
            const int32_t j = ci[k];
            const T xj = j < i ? xn[j] : xo[j];
            acc += (T)v[k] * xj;
        }
    }
#pragma unroll
    for (int o = VL / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o, VL);
    if (valid && j0 == 0) xn[i] = xo[i] + omega * (b[i] - acc) * dinv[i];
}

template <typename TV, typename T>
void launch_group(int vl, int64_t cnt, const int32_t *rows, const int64_t *rp, const int32_t *ci, const TV *v,
                  const T *xo, T *xn, const T *b, const T *dinv, T omega, cudaStream_t s) {
    const unsigned g = (unsigned)((cnt * vl + 255) / 256);
    switch (vl) {
    case 1: gs_group_kernel<1, TV, T><<<air_counted(g), 256, 0, s>>>(cnt, rows, rp, ci, v, xo, xn, b, dinv, omega); break;
    case 2: gs_group_kernel<2, TV, T><<<air_counted(g), 256, 0, s>>>(cnt, rows, rp, ci, v, xo, xn, b, dinv, omega); break;
    case 4: gs_group_kernel<4, TV, T><<<air_counted(g), 256, 0, s>>>(cnt, rows, rp, ci, v, xo, xn, b, dinv, omega); break;
    case 8: gs_group_kernel<8, TV, T><<<air_counted(g), 256, 0, s>>>(cnt, rows, rp, ci, v, xo, xn, b, dinv, omega); break;
    case 16: gs_group_kernel<16, TV, T><<<air_counted(g), 256, 0, s>>>(cnt, rows, rp, ci, v, xo, xn, b, dinv, omega); break;
    default: gs_group_kernel<32, TV, T><<<air_counted(g), 256, 0, s>>>(cnt, rows, rp, ci, v, xo, xn, b, dinv, omega); break;
    }
}

int lanes_for(const AirLevel &L) {
    const double avg = L.n > 0 ? (double)L.nnz / (double)L.n : 1.0;
    int vl = 1;
    while (vl < 32 && avg / vl > 8.0) vl *= 2;
    return vl;
}

int build_one(AirLevel &L, int which, cudaStream_t s) {
    AirLevel::GsSchedule &G = L.gs[which];
    const int64_t n = L.n;
    int32_t *indeg = nullptr, *outdeg = nullptr, *fill = nullptr, *succ = nullptr;
    int64_t *optr = nullptr;
    unsigned long long *tail = nullptr;
    AIR_CUDA(cudaMallocAsync(&indeg, (size_t)n * sizeof(int32_t), s));
    AIR_CUDA(cudaMallocAsync(&outdeg, (size_t)n * sizeof(int32_t), s));
    AIR_CUDA(cudaMemsetAsync(outdeg, 0, (size_t)n * sizeof(int32_t), s));
    gs_degree_kernel<<<air_counted(grid_for(n, 256)), 256, 0, s>>>(n, L.rp, L.ci, L.cf, which, indeg, outdeg);
    AIR_LAUNCH();
    AIR_CUDA(cudaMallocAsync(&optr, (size_t)(n + 1) * sizeof(int64_t), s));
    AIR_TRY(air_exclusive_scan_i32(outdeg, optr, n, s));
    int64_t ne = 0;
    AIR_CUDA(cudaMemcpyAsync(&ne, optr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    AIR_CUDA(cudaStreamSynchronize(s));
    AIR_CUDA(cudaMallocAsync(&succ, (size_t)(ne > 0 ? ne : 1) * sizeof(int32_t), s));
    AIR_CUDA(cudaMallocAsync(&fill, (size_t)n * sizeof(int32_t), s));
    AIR_CUDA(cudaMemsetAsync(fill, 0, (size_t)n * sizeof(int32_t), s));
    gs_succ_kernel<<<air_counted(grid_for(n, 256)), 256, 0, s>>>(n, L.rp, L.ci, L.cf, which, optr, fill, succ);
    AIR_LAUNCH();
    const int64_t m = which == 2 ? n : (which == 1 ? L.nc : L.nf);
    G.m = m;
    AIR_CUDA(air_dmalloc((void **)&G.dev_rows, (size_t)(m > 0 ? m : 1) * sizeof(int32_t)));
    AIR_CUDA(cudaMallocAsync(&tail, sizeof(unsigned long long), s));
    AIR_CUDA(cudaMemsetAsync(tail, 0, sizeof(unsigned long long), s));
    gs_roots_kernel<<<air_counted(grid_for(n, 256)), 256, 0, s>>>(n, indeg, G.dev_rows, tail);
    AIR_LAUNCH();
    std::vector<int64_t> ptr(1, 0);
    unsigned long long h = 0;
    AIR_CUDA(cudaMemcpyAsync(&h, tail, sizeof(h), cudaMemcpyDeviceToHost, s));
    AIR_CUDA(cudaStreamSynchronize(s));
    int64_t a = 0, b = (int64_t)h;
    while (b > a) {
        ptr.push_back(b);
        if ((int64_t)ptr.size() > m + 2) break;      // cannot happen: the graph is acyclic
        gs_advance_kernel<<<air_counted(grid_for(b - a, 256)), 256, 0, s>>>(a, b, optr, succ, indeg, G.dev_rows, tail);
        AIR_LAUNCH();
        AIR_CUDA(cudaMemcpyAsync(&h, tail, sizeof(h), cudaMemcpyDeviceToHost, s));
        AIR_CUDA(cudaStreamSynchronize(s));
        a = b;
        b = (int64_t)h;
    }
    cudaFreeAsync(indeg, s);
    cudaFreeAsync(outdeg, s);
    cudaFreeAsync(fill, s);
    cudaFreeAsync(succ, s);
    cudaFreeAsync(optr, s);
    cudaFreeAsync(tail, s);
    if (b != m) return AIR_ERR_CUDA;                  // every row of the set must be placed
    G.depth = (int32_t)(ptr.size() - 1);
    G.ptr = (int64_t *)malloc(ptr.size() * sizeof(int64_t));
    if (!G.ptr) return AIR_ERR_OOM;
    memcpy(G.ptr, ptr.data(), ptr.size() * sizeof(int64_t));
    return AIR_OK;
}

__global__ void d2f_values_kernel(int64_t n, const double *in, float *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

}  // namespace

int air_gs_build(air_hierarchy *H, cudaStream_t s) {
    bool need[3] = {false, false, false};
    for (const char *c = H->opt.relax; *c; ++c) {
        if (*c == 'f') need[0] = true;
        if (*c == 'c') need[1] = true;
        if (*c == 'a') need[2] = true;
    }
    if (!need[0] && !need[1] && !need[2]) return AIR_OK;
    for (int q = 0; q + 1 < H->nlev; ++q) {
        AirLevel &L = H->lev[q];
        for (int w = 0; w < 3; ++w)
            if (need[w]) AIR_TRY(build_one(L, w, s));
        if (H->opt.precision == AIR_PREC_F32) {
            AIR_CUDA(air_dmalloc((void **)&L.v32, (size_t)(L.nnz > 0 ? L.nnz : 1) * sizeof(float)));
            d2f_values_kernel<<<air_counted(grid_for(L.nnz, 256)), 256, 0, s>>>(L.nnz, L.v, L.v32);
            AIR_LAUNCH();
        }
    }
    return AIR_OK;
}

void air_gs_free(AirLevel &L) {
    for (auto &G : L.gs) {
        air_dfree(G.dev_rows);
        free(G.ptr);
        G = AirLevel::GsSchedule();
    }
    air_dfree(L.v32);
    L.v32 = nullptr;
}

template <typename T>
int air_gs_sweep(const AirLevel &L, int which, T omega, const T *b, T *x, T *xn, cudaStream_t s) {
    const AirLevel::GsSchedule &G = L.gs[which];
    if (G.m == 0) return AIR_OK;
    const T *dinv = std::is_same<T, double>::value ? (const T *)L.dinv : (const T *)L.dinv32;
    const int vl = lanes_for(L);
    AIR_CUDA(cudaMemcpyAsync(xn, x, (size_t)L.n * sizeof(T), cudaMemcpyDeviceToDevice, s));
    for (int k = 0; k < G.depth; ++k) {
        const int64_t a = G.ptr[k], cnt = G.ptr[k + 1] - a;
        if (std::is_same<T, double>::value)
            launch_group<double, double>(vl, cnt, G.dev_rows + a, L.rp, L.ci, L.v, (const double *)x, (double *)xn,
                                         (const double *)b, (const double *)dinv, (double)omega, s);
        else
            launch_group<float, float>(vl, cnt, G.dev_rows + a, L.rp, L.ci, L.v32, (const float *)x, (float *)xn,
                                       (const float *)b, (const float *)dinv, (float)omega, s);
    }
    AIR_LAUNCH();
    AIR_CUDA(cudaMemcpyAsync(x, xn, (size_t)L.n * sizeof(T), cudaMemcpyDeviceToDevice, s));
    return AIR_OK;
}

template int air_gs_sweep<double>(const AirLevel &, int, double, const double *, double *, double *, cudaStream_t);
template int air_gs_sweep<float>(const AirLevel &, int, float, const float *, float *, float *, cudaStream_t);
