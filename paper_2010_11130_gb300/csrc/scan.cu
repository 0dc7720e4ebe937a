// Exclusive prefix sums and max-reductions used by the setup phase
// (row counts -> row pointers, C markers -> coarse ids).
//
// Three launches: per-tile sums, one-block scan of the tile sums, per-tile
// rescan plus offset.  A tile is 1024 threads x 8 items; out has n+1 entries
// and out[n] is the total.
#include "air_internal.cuh"

namespace {

constexpr int kThreads = 1024;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;

template <typename T>
__device__ int64_t block_sum(int64_t v) {
    __shared__ int64_t warp_sums[kThreads / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) warp_sums[wid] = v;
    __syncthreads();
    int64_t t = 0;
    if (wid == 0) {
        t = lane < kThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    return t;   // valid in thread 0
}

template <typename T>
__global__ void tile_sums(const T *in, int64_t n, int64_t *sums) {
    int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    int64_t v = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k)
        if (base + k < n) v += (int64_t)in[base + k];
    int64_t t = block_sum<T>(v);
    if (threadIdx.x == 0) sums[blockIdx.x] = t;
}

// inclusive-to-exclusive block scan of per-thread values; returns the exclusive prefix
__device__ int64_t block_exclusive(int64_t v, int64_t *total) {
    __shared__ int64_t warp_tot[kThreads / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int64_t w = lane < kThreads / 32 ? warp_tot[lane] : 0;
        int64_t winc = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(0xffffffffu, winc, o);
            if (lane >= o) winc += t;
        }
        if (lane < kThreads / 32) warp_tot[lane] = winc - w;   // exclusive warp offsets
        if (lane == kThreads / 32 - 1) *total = winc;
    }
    __syncthreads();
    int64_t r = warp_tot[wid] + inc - v;
    __syncthreads();
    return r;
}

__global__ void scan_sums(int64_t *sums, int64_t nt) {
    __shared__ int64_t tot;
    int64_t carry = 0;
    for (int64_t base = 0; base < nt; base += kThreads) {
        int64_t i = base + threadIdx.x;
        int64_t v = i < nt ? sums[i] : 0;
        int64_t ex = block_exclusive(v, &tot);
        if (i < nt) sums[i] = carry + ex;
        __syncthreads();
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[nt] = carry;
}

template <typename T>
__global__ void tile_scan(const T *in, int64_t n, const int64_t *sums, int64_t *out, int64_t nt) {
    __shared__ int64_t tot;
    int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    int64_t vals[kItems];
    int64_t v = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        vals[k] = base + k < n ? (int64_t)in[base + k] : 0;
        v += vals[k];
    }
    int64_t ex = block_exclusive(v, &tot) + sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        if (base + k < n) out[base + k] = ex;
        ex += vals[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = sums[nt];
}

template <typename T>
int scan_impl(const T *in, int64_t *out, int64_t n, cudaStream_t s) {
    if (n == 0) {
        AIR_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return AIR_OK;
    }
    int64_t nt = (n + kTile - 1) / kTile;
    int64_t *sums = nullptr;
    AIR_CUDA(cudaMallocAsync(&sums, (nt + 1) * sizeof(int64_t), s));
    tile_sums<T><<<air_counted((unsigned)nt), kThreads, 0, s>>>(in, n, sums);
    scan_sums<<<air_counted(1), kThreads, 0, s>>>(sums, nt);
    tile_scan<T><<<air_counted((unsigned)nt), kThreads, 0, s>>>(in, n, sums, out, nt);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(sums, s);
    if (e != cudaSuccess) return AIR_ERR_CUDA;
    return AIR_OK;
}

__global__ void max_i32_kernel(const int32_t *in, int64_t n, int32_t *out) {
    int32_t m = INT32_MIN;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, in[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

__global__ void max_row_kernel(const int64_t *rp, int64_t n, int32_t *out) {
    int32_t m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (int32_t)(rp[i + 1] - rp[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

}  // namespace

// Longest row of a CSR row pointer (synchronises the stream to read it).
int air_max_row(int64_t n, const int64_t *rp, int32_t *out_max, cudaStream_t s) {
    *out_max = 0;
    if (n <= 0) return AIR_OK;
    int32_t *d = nullptr;
    AIR_CUDA(cudaMallocAsync(&d, sizeof(int32_t), s));
    AIR_CUDA(cudaMemsetAsync(d, 0, sizeof(int32_t), s));
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    max_row_kernel<<<air_counted((unsigned)blocks), 256, 0, s>>>(rp, n, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_max, d, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return AIR_ERR_CUDA;
    return AIR_OK;
}

int air_exclusive_scan_i32(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s) {
    return scan_impl<int32_t>(in, out, n, s);
}

int air_exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) {
    return scan_impl<int64_t>(in, out, n, s);
}

// *d_out must be initialised by the caller (e.g. to INT32_MIN or 0).
int air_reduce_max_i32(const int32_t *in, int64_t n, int32_t *d_out, cudaStream_t s) {
    if (n == 0) return AIR_OK;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    max_i32_kernel<<<air_counted((unsigned)blocks), 256, 0, s>>>(in, n, d_out);
    AIR_LAUNCH();
    return AIR_OK;
}
