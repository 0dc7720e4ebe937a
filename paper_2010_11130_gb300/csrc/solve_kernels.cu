// Solve-phase kernels: CSR SpMV, the V-cycle (restriction, coarsest dense
// solve, one-point interpolation fused into the first relaxation sweep,
// masked Jacobi sweeps) and the GMRES building blocks (block-partial multi-dot
// products fused with the Gram-Schmidt updates, device-side Givens rotations).
//
// The V-cycle is x = 0 on every level, b_{l+1} = R_l b_l, x_L = A_L^{-1} b_L,
// x_l = P_l x_{l+1} followed by Jacobi sweeps over the point sets of the
// relaxation pattern (arXiv:2010.11130, Section 3; FCF-Jacobi replaces the
// paper's forward Gauss-Seidel of Section 4).  All of it is sparse or
// bandwidth-bound: no tensor cores.
#include <math.h>
#include <string.h>

#include <type_traits>

#include <cuda_bf16.h>

#include "air_internal.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;

unsigned grid_cap(int64_t items, int threads, int64_t cap = 152 * 16) {
    int64_t b = (items + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

template <typename T>
struct Acc;
template <>
struct Acc<double> { using type = double; };
template <>
struct Acc<float> { using type = float; };

template <typename A, typename TV>
__device__ __forceinline__ A to_acc(TV v) { return (A)v; }
template <>
__device__ __forceinline__ float to_acc<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <int VL, typename A>
__device__ __forceinline__ A seg_sum(A s) {
#pragma unroll
    for (int o = VL / 2; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o, VL);
    return s;
}

// Row kernels (SpMV and masked Jacobi).  VL lanes share a row; each lane
// owns U entries of it, so all column / value loads of the row and then all
// x gathers are in flight together (the short HDG rows are otherwise
// latency-bound).  Entries beyond U*VL fall to a remainder loop.  The loop
// runs over blocks of rows with a trip count that is uniform across the
// warp, so every lane reaches the segment shuffles.
// ROW_JACOBI writes a sweep's new values compactly (y[pos], scattered
// afterwards); ROW_JACOBI_FULL writes them in place of the rows (y[row]) of a
// second full vector, and the launch's extra blocks copy the rows the sweep
// leaves unchanged (crows), so that the sweeps alternate between two vectors.
enum { ROW_SPMV = 0, ROW_JACOBI = 1, ROW_JACOBI_FULL = 2 };

// Block blk of the copy part of a ROW_JACOBI_FULL launch.
template <typename TX>
__device__ __forceinline__ void copy_rows(int64_t mc, const int32_t *__restrict__ crows, const TX *__restrict__ x,
                                          TX *__restrict__ y, int64_t blk) {
    const int64_t p = blk * blockDim.x + threadIdx.x;
    if (p < mc) {
        const int32_t r = crows[p];
        y[r] = x[r];
    }
}

template <typename TV, typename TX>
struct RowArgs {
    int64_t n;
    const int64_t *rp;
    const int32_t *ci;
    const TV *v;
    const TX *x;        // input vector (gathered)
    TX *y;              // output
    const TX *b;        // SpMV: optional (y = b - A x); Jacobi: right-hand side
    const TX *dinv;     // Jacobi: 1 / a_ii
    const int32_t *rows;  // Jacobi: the rows of the relaxed point set (ascending); n = their count
    const TX *diag;       // if set, the stored values hold no diagonal: a_ii x_i is added from here
    TX omega;
};

template <int VL, int U, typename TV, typename TX, int MODE>
__global__ void __launch_bounds__(256) row_kernel(RowArgs<TV, TX> a) {
    using A = typename Acc<TX>::type;
    const int lane = threadIdx.x & (VL - 1);
    const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / VL;
    const int64_t ng = ((int64_t)gridDim.x * blockDim.x) / VL;
    const int64_t gw = g0 - (threadIdx.x & 31) / VL;            // first group of this warp
    for (int64_t base = gw; base < a.n; base += ng) {
        const int64_t pos = base + (g0 - gw);
        const bool valid = pos < a.n;
        int64_t row = pos;
        if (MODE == ROW_JACOBI && valid) row = a.rows[pos];
        A acc = 0;
        if (valid) {
            const int64_t rs = a.rp[row], re = a.rp[row + 1];
            int32_t cols[U];
            TV vals[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t e = rs + lane + (int64_t)u * VL;
                const bool ok = e < re;
                cols[u] = ok ? __ldg(a.ci + e) : 0;
                vals[u] = ok ? a.v[e] : (TV)0;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) acc += to_acc<A, TV>(vals[u]) * (A)__ldg(a.x + cols[u]);
            for (int64_t e = rs + lane + (int64_t)U * VL; e < re; e += VL)
                acc += to_acc<A, TV>(a.v[e]) * (A)a.x[a.ci[e]];
            if (a.diag && lane == 0) acc += (A)a.diag[row] * (A)a.x[row];
        }
        acc = seg_sum<VL, A>(acc);
        if (lane == 0 && valid) {
            if (MODE == ROW_SPMV) {
                a.y[row] = a.b ? (TX)((A)a.b[row] - acc) : (TX)acc;
            } else {
                // the new value goes to the compact buffer y[pos]; scatter_kernel writes it back
                a.y[pos] = (TX)(a.x[row] + a.omega * ((TX)((A)a.b[row] - acc)) * a.dinv[row]);
            }
        }
    }
}

// x[rows[pos]] = t[pos]: finishes one Jacobi sweep in place.
template <typename T>
__global__ void scatter_kernel(int64_t m, const int32_t *__restrict__ rows, const T *__restrict__ t, T *__restrict__ x) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x)
        x[rows[p]] = t[p];
}

template <typename T>
__global__ void interp_kernel(int64_t n, const int32_t *pcol, const T *xc, T *x) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t pc = pcol[i];
        x[i] = pc >= 0 ? xc[pc] : (T)0;
    }
}

// x = Cinv b, dense row-major, one warp per row
template <typename T>
__global__ void dense_gemv_kernel(int64_t n, const T *__restrict__ Ci, const T *__restrict__ b, T *__restrict__ x) {
    int lane = threadIdx.x & 31;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w; r < n; r += nw) {
        T s = 0;
        for (int64_t c = lane; c < n; c += 32) s += Ci[r * n + c] * b[c];
        s = seg_sum<32, T>(s);
        if (lane == 0) x[r] = s;
    }
}

__global__ void d2f_kernel(const double *in, float *out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

// BF16 copy of CSR values with the diagonal entries set to zero (the
// diagonal is kept separately in FP32); diag32 may be NULL (rectangular R).
__global__ void d2bf_offdiag_kernel(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                                    __nv_bfloat16 *out, float *diag32) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
            bool d = diag32 && ci[k] == i;
            if (out) out[k] = __double2bfloat16(d ? 0.0 : v[k]);
            if (d) diag32[i] = (float)v[k];
        }
    }
}

// -------------------------------------------------------------- SELL-32
// sigma-sorting: inside each window of 1024 rows, order the rows by
// decreasing length (ties by position) so each 32-row slice is nearly
// uniform and carries little padding.
constexpr int SIGMA = 1024;

__global__ void __launch_bounds__(SIGMA / 2) sell_sort_kernel(int64_t m, const int32_t *rows, const int64_t *rp,
                                                              int32_t *out) {
    __shared__ unsigned long long key[SIGMA];
    const int64_t w0 = (int64_t)blockIdx.x * SIGMA;
    for (int t = threadIdx.x; t < SIGMA; t += blockDim.x) {
        const int64_t p = w0 + t;
        if (p < m) {
            const int64_t r = rows ? rows[p] : p;
            const unsigned len = (unsigned)(rp[r + 1] - rp[r]);
            key[t] = ((unsigned long long)(0xffffffffu - len) << 32) | (unsigned)t;   // longest first
        } else {
            key[t] = ~0ull;
        }
    }
    __syncthreads();
    for (int size = 2; size <= SIGMA; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int idx = threadIdx.x; idx < SIGMA / 2; idx += blockDim.x) {
                const int a = 2 * stride * (idx / stride) + (idx % stride), b = a + stride;
                const bool up = (a & size) == 0;
                const unsigned long long ka = key[a], kb = key[b];
                if ((ka > kb) == up) { key[a] = kb; key[b] = ka; }
            }
            __syncthreads();
        }
    for (int t = threadIdx.x; t < SIGMA; t += blockDim.x) {
        const int64_t p = w0 + t;
        if (p < m) {
            const int64_t src = w0 + (int64_t)(key[t] & 0xffffffffu);
            out[p] = rows ? rows[src] : (int32_t)src;
        }
    }
}

__global__ void sell_width_kernel(int64_t m, const int32_t *rows, const int64_t *rp, int32_t *wid) {
    const int64_t ns = (m + 31) / 32;
    for (int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; sl < ns; sl += (int64_t)gridDim.x * blockDim.x) {
        int32_t w = 0;
        for (int64_t p = sl * 32; p < m && p < sl * 32 + 32; ++p) {
            const int64_t r = rows[p];
            w = max(w, (int32_t)(rp[r + 1] - rp[r]));
        }
        wid[sl] = w * 32;
    }
}

template <typename TV, bool ZERO_DIAG>
__global__ void sell_fill_kernel(int64_t m, const int32_t *rows, const int64_t *rp, const int32_t *ci,
                                 const double *v, const int64_t *ptr, int32_t *sci, TV *sv) {
    const int64_t ns32 = ((m + 31) / 32) * 32;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < ns32; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sl = p >> 5, l = p & 31;
        const int64_t base = ptr[sl], w = (ptr[sl + 1] - base) >> 5;
        if (p < m) {
            const int64_t r = rows[p];
            const int64_t b = rp[r], len = rp[r + 1] - b;
            for (int64_t k = 0; k < w; ++k) {
                const int64_t dst = base + 32 * k + l;
                if (k < len) {
                    const int32_t c = ci[b + k];
                    sci[dst] = c;
                    sv[dst] = (TV)((ZERO_DIAG && c == r) ? 0.0 : v[b + k]);
                } else {
                    sci[dst] = (int32_t)r;
                    sv[dst] = (TV)0.0;
                }
            }
        } else {
            for (int64_t k = 0; k < w; ++k) {   // lanes past the last row: harmless zeros
                sci[base + 32 * k + l] = 0;
                sv[base + 32 * k + l] = (TV)0.0;
            }
        }
    }
}

template <typename TV, typename TX>
struct SellArgs {
    int64_t m;
    const int64_t *ptr;
    const int32_t *ci;
    const TV *v;
    const int32_t *rows;   // pos -> row id of the vectors
    const TX *x;
    TX *y;                 // SpMV: y[row]; Jacobi: y[pos] (compact, scattered afterwards)
    const TX *b;
    const TX *dinv;
    const TX *diag;        // FP32 diagonal when the stored values hold none
    TX omega;
    int64_t mc;            // ROW_JACOBI_FULL: rows copied unchanged from x to y, and the blocks before them
    const int32_t *crows;
    int64_t sweep_blocks;
};

// One thread per row: entry k of the 32 rows of a slice is one coalesced
// load; UN entries are loaded before their x gathers.
template <int UN, typename TV, typename TX, int MODE>
__global__ void __launch_bounds__(256) sell_kernel(SellArgs<TV, TX> a) {
    using A = typename Acc<TX>::type;
    if (MODE == ROW_JACOBI_FULL && (int64_t)blockIdx.x >= a.sweep_blocks) {
        copy_rows(a.mc, a.crows, a.x, a.y, (int64_t)blockIdx.x - a.sweep_blocks);
        return;
    }
    const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= a.m) return;
    const int64_t sl = pos >> 5;
    const int l = (int)(pos & 31);
    const int64_t base = a.ptr[sl];
    const int w = (int)((a.ptr[sl + 1] - base) >> 5);
    const int32_t *cp = a.ci + base + l;
    const TV *vp = a.v + base + l;
    A acc = 0;
    int k = 0;
    for (; k + UN <= w; k += UN) {
        int32_t c[UN];
        TV vv[UN];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            c[u] = __ldg(cp + 32 * (k + u));
            vv[u] = vp[32 * (k + u)];
        }
#pragma unroll
        for (int u = 0; u < UN; ++u) acc += to_acc<A, TV>(vv[u]) * (A)__ldg(a.x + c[u]);
    }
    for (; k < w; ++k) acc += to_acc<A, TV>(vp[32 * k]) * (A)__ldg(a.x + cp[32 * k]);
    const int64_t row = a.rows[pos];
    if (MODE == ROW_SPMV) {
        a.y[row] = a.b ? (TX)((A)a.b[row] - acc) : (TX)acc;
    } else {
        if (a.diag) acc += (A)a.diag[row] * (A)a.x[row];
        const TX nv = (TX)(a.x[row] + a.omega * ((TX)((A)a.b[row] - acc)) * a.dinv[row]);
        a.y[MODE == ROW_JACOBI ? pos : row] = nv;
    }
}

// ------------------------------------------------------- block SELL-32
// Loads of b consecutive values: pairs when b is even and the start is
// aligned to a pair (2 b-element rows of float / double / bf16 keep that
// alignment when the base is aligned), scalars otherwise.
template <typename T>
struct Pair;
template <>
struct Pair<double> { using type = double2; };
template <>
struct Pair<float> { using type = float2; };
template <>
struct Pair<__nv_bfloat16> { using type = __nv_bfloat162; };

template <typename A, typename T>
__device__ __forceinline__ void pair_to(const typename Pair<T>::type &p, A &a0, A &a1) {
    a0 = (A)p.x;
    a1 = (A)p.y;
}
template <>
__device__ __forceinline__ void pair_to<float, __nv_bfloat16>(const __nv_bfloat162 &p, float &a0, float &a1) {
    a0 = __bfloat162float(p.x);
    a1 = __bfloat162float(p.y);
}

template <int B, bool PAIRS, typename A, typename T>
__device__ __forceinline__ void load_run(const T *__restrict__ p, A (&out)[B]) {
    if constexpr (PAIRS && B % 2 == 0) {
        const typename Pair<T>::type *q = reinterpret_cast<const typename Pair<T>::type *>(p);
#pragma unroll
        for (int j = 0; j < B / 2; ++j) pair_to<A, T>(__ldg(q + j), out[2 * j], out[2 * j + 1]);
    } else {
#pragma unroll
        for (int j = 0; j < B; ++j) out[j] = to_acc<A, T>(__ldg(p + j));
    }
}

template <typename TV, typename TX>
struct BSellArgs {
    int64_t m;
    const int64_t *ptr;
    const int32_t *bc;
    const TV *v;
    const TX *dv;
    const int32_t *rows;
    const TX *x;
    TX *y;
    const TX *b;
    const TX *dinv;
    TX omega;
    int64_t mc;            // as in SellArgs
    const int32_t *crows;
    int64_t sweep_blocks;
};

// One thread per row: the row's blocks two at a time, each block's b values
// and b entries of x as runs of consecutive elements.
template <int B, bool PAIRS, typename TV, typename TX, int MODE>
__global__ void __launch_bounds__(256) bsell_kernel(BSellArgs<TV, TX> a) {
    using A = typename Acc<TX>::type;
    if (MODE == ROW_JACOBI_FULL && (int64_t)blockIdx.x >= a.sweep_blocks) {
        copy_rows(a.mc, a.crows, a.x, a.y, (int64_t)blockIdx.x - a.sweep_blocks);
        return;
    }
    const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= a.m) return;
    const int64_t sl = pos >> 5;
    const int l = (int)(pos & 31);
    const int64_t base = a.ptr[sl];
    const int w = (int)((a.ptr[sl + 1] - base) >> 5);
    const int64_t row = a.rows[pos];
    A acc = (A)a.dv[pos] * (A)a.x[row];
    int t = 0;
    for (; t + 2 <= w; t += 2) {
        const int64_t i0 = base + 32 * t + l, i1 = i0 + 32;
        const int32_t c0 = __ldg(a.bc + i0), c1 = __ldg(a.bc + i1);
        A v0[B], v1[B], x0[B], x1[B];
        load_run<B, PAIRS>(a.v + i0 * B, v0);
        load_run<B, PAIRS>(a.v + i1 * B, v1);
        load_run<B, PAIRS>(a.x + c0, x0);
        load_run<B, PAIRS>(a.x + c1, x1);
#pragma unroll
        for (int j = 0; j < B; ++j) acc += v0[j] * x0[j];
#pragma unroll
        for (int j = 0; j < B; ++j) acc += v1[j] * x1[j];
    }
    if (t < w) {
        const int64_t i0 = base + 32 * t + l;
        const int32_t c0 = __ldg(a.bc + i0);
        A v0[B], x0[B];
        load_run<B, PAIRS>(a.v + i0 * B, v0);
        load_run<B, PAIRS>(a.x + c0, x0);
#pragma unroll
        for (int j = 0; j < B; ++j) acc += v0[j] * x0[j];
    }
    if (MODE == ROW_SPMV) {
        a.y[row] = a.b ? (TX)((A)a.b[row] - acc) : (TX)acc;
    } else {
        const TX nv = (TX)(a.x[row] + a.omega * ((TX)((A)a.b[row] - acc)) * a.dinv[row]);
        a.y[MODE == ROW_JACOBI ? pos : row] = nv;
    }
}

template <int B, typename TV, typename TX, int MODE>
void bsell_launch_b(const BSellArgs<TV, TX> &a0, bool pairs, cudaStream_t s) {
    BSellArgs<TV, TX> a = a0;
    a.sweep_blocks = (a.m + 255) / 256;
    const unsigned g = (unsigned)(a.sweep_blocks + (MODE == ROW_JACOBI_FULL ? (a.mc + 255) / 256 : 0));
    if (pairs) bsell_kernel<B, true, TV, TX, MODE><<<air_counted(g), 256, 0, s>>>(a);
    else bsell_kernel<B, false, TV, TX, MODE><<<air_counted(g), 256, 0, s>>>(a);
}

// pairs are safe when x starts on a pair boundary (the values always do)
template <typename TV, typename TX, int MODE>
void bsell_launch(int b, const BSellArgs<TV, TX> &a, cudaStream_t s) {
    if (a.m <= 0) return;
    const bool pairs = ((uintptr_t)a.x % (2 * sizeof(TX))) == 0;
    switch (b) {
    case 2: bsell_launch_b<2, TV, TX, MODE>(a, pairs, s); break;
    case 3: bsell_launch_b<3, TV, TX, MODE>(a, pairs, s); break;
    case 4: bsell_launch_b<4, TV, TX, MODE>(a, pairs, s); break;
    case 6: bsell_launch_b<6, TV, TX, MODE>(a, pairs, s); break;
    default: bsell_launch_b<10, TV, TX, MODE>(a, pairs, s); break;
    }
}

// VL lanes per row (VL divides 32): lane j of a row takes the row's stored
// entries j, j + VL, ..., four at a time, then the lanes sum their partial
// results.  For levels whose rows are long (Galerkin fill) and few, the row's
// latency chain is VL times shorter.
template <int VL, typename TV, typename TX, int MODE>
__global__ void __launch_bounds__(256) sell_lanes_kernel(SellArgs<TV, TX> a) {
    using A = typename Acc<TX>::type;
    if (MODE == ROW_JACOBI_FULL && (int64_t)blockIdx.x >= a.sweep_blocks) {   // whole blocks: no lane is left in a shuffle
        copy_rows(a.mc, a.crows, a.x, a.y, (int64_t)blockIdx.x - a.sweep_blocks);
        return;
    }
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t pos = t / VL;
    const int j = (int)(t % VL);
    const bool valid = pos < a.m;                 // whole groups of VL lanes share validity
    A acc = 0;
    int64_t row = 0;
    if (valid) {
        const int64_t sl = pos >> 5;
        const int l = (int)(pos & 31);
        const int64_t base = a.ptr[sl];
        const int w = (int)((a.ptr[sl + 1] - base) >> 5);
        const int32_t *cp = a.ci + base + l;
        const TV *vp = a.v + base + l;
        int k = j;
        for (; k + 3 * VL < w; k += 4 * VL) {
            int32_t c[4];
            TV vv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                c[u] = __ldg(cp + 32 * (k + u * VL));
                vv[u] = vp[32 * (k + u * VL)];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) acc += to_acc<A, TV>(vv[u]) * (A)__ldg(a.x + c[u]);
        }
        for (; k < w; k += VL) acc += to_acc<A, TV>(vp[32 * k]) * (A)__ldg(a.x + cp[32 * k]);
        row = a.rows[pos];
    }
#pragma unroll
    for (int o = VL / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o, VL);
    if (!valid || j != 0) return;
    if (MODE == ROW_SPMV) {
        a.y[row] = a.b ? (TX)((A)a.b[row] - acc) : (TX)acc;
    } else {
        if (a.diag) acc += (A)a.diag[row] * (A)a.x[row];
        const TX nv = (TX)(a.x[row] + a.omega * ((TX)((A)a.b[row] - acc)) * a.dinv[row]);
        a.y[MODE == ROW_JACOBI ? pos : row] = nv;
    }
}

// Blocks of the copy part of a ROW_JACOBI_FULL launch.
inline int64_t copy_blocks(int64_t mc) { return (mc + 255) / 256; }

template <int VL, typename TV, typename TX, int MODE>
void sell_lanes_launch(const SellArgs<TV, TX> &a0, cudaStream_t s) {
    SellArgs<TV, TX> a = a0;
    a.sweep_blocks = (a.m * VL + 255) / 256;
    const int64_t g = a.sweep_blocks + (MODE == ROW_JACOBI_FULL ? copy_blocks(a.mc) : 0);
    sell_lanes_kernel<VL, TV, TX, MODE><<<air_counted((unsigned)g), 256, 0, s>>>(a);
}

template <typename TV, typename TX, int MODE>
void sell_launch(const SellArgs<TV, TX> &a, cudaStream_t s, int lanes = 1) {
    if (a.m <= 0) return;
    switch (lanes) {
    case 2: sell_lanes_launch<2, TV, TX, MODE>(a, s); return;
    case 4: sell_lanes_launch<4, TV, TX, MODE>(a, s); return;
    case 8: sell_lanes_launch<8, TV, TX, MODE>(a, s); return;
    case 16: sell_lanes_launch<16, TV, TX, MODE>(a, s); return;
    case 32: sell_lanes_launch<32, TV, TX, MODE>(a, s); return;
    default: break;
    }
    SellArgs<TV, TX> b = a;
    b.sweep_blocks = (a.m + 255) / 256;
    const int64_t g = b.sweep_blocks + (MODE == ROW_JACOBI_FULL ? copy_blocks(a.mc) : 0);
    sell_kernel<8, TV, TX, MODE><<<air_counted((unsigned)g), 256, 0, s>>>(b);
}

__global__ void f2d_kernel(const float *in, double *out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

__global__ void diag_inverse_kernel(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, double *dinv,
                                    float *dinv32) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
            if (ci[k] == i) { d = v[k]; break; }
        double r = 1.0 / d;
        dinv[i] = r;
        if (dinv32) dinv32[i] = (float)r;
    }
}

// ------------------------------------------------------------------ GMRES
constexpr int RT = 256;          // threads of the reduction kernels
constexpr int MAXK = AIR_MAX_RESTART + 1;

// partials[i * nblk + blk] = sum over this block's slice of V_i . w   (i < k)
template <int KB>
__global__ void __launch_bounds__(RT) dot_partials_kernel(int64_t n, const double *__restrict__ V, int64_t ldv,
                                                          int k0, int k, const double *__restrict__ w,
                                                          double *__restrict__ partials, int nblk) {
    __shared__ double red[RT / 32][KB];
    double acc[KB];
#pragma unroll
    for (int i = 0; i < KB; ++i) acc[i] = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * RT + threadIdx.x; t < n; t += (int64_t)gridDim.x * RT) {
        double wt = w[t];
#pragma unroll
        for (int i = 0; i < KB; ++i)
            if (k0 + i < k) acc[i] += V[(int64_t)(k0 + i) * ldv + t] * wt;
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < KB; ++i) {
        double s = acc[i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
        if (lane == 0) red[wid][i] = s;
    }
    __syncthreads();
    if (threadIdx.x < KB && k0 + (int)threadIdx.x < k) {
        double s = 0.0;
        for (int q = 0; q < RT / 32; ++q) s += red[q][threadIdx.x];
        partials[(int64_t)(k0 + threadIdx.x) * nblk + blockIdx.x] = s;
    }
}

// w -= sum_i h_i V_i (i < k); then partial dots of the updated w with V_i
// (i < dots) or, if dots == -1, the partial squared norm of w into row 0.
template <int KB>
__global__ void __launch_bounds__(RT) update_dot_kernel(int64_t n, const double *__restrict__ V, int64_t ldv, int k,
                                                        const double *__restrict__ h, double *__restrict__ w,
                                                        double *__restrict__ partials, int nblk, int dots) {
    __shared__ double red[RT / 32][KB];
    __shared__ double hs[KB];
    if (threadIdx.x < KB) hs[threadIdx.x] = (int)threadIdx.x < k ? h[threadIdx.x] : 0.0;
    __syncthreads();
    double acc[KB];
#pragma unroll
    for (int i = 0; i < KB; ++i) acc[i] = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * RT + threadIdx.x; t < n; t += (int64_t)gridDim.x * RT) {
        double vt[KB];
        double wt = w[t];
#pragma unroll
        for (int i = 0; i < KB; ++i) {
            vt[i] = i < k ? V[(int64_t)i * ldv + t] : 0.0;
            wt -= hs[i] * vt[i];
        }
        w[t] = wt;
        if (dots < 0) {
            acc[0] += wt * wt;
        } else {
#pragma unroll
            for (int i = 0; i < KB; ++i) acc[i] += vt[i] * wt;
        }
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int nd = dots < 0 ? 1 : dots;
#pragma unroll
    for (int i = 0; i < KB; ++i) {
        double s = acc[i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
        if (lane == 0) red[wid][i] = s;
    }
    __syncthreads();
    if ((int)threadIdx.x < nd && (int)threadIdx.x < KB) {
        double s = 0.0;
        for (int q = 0; q < RT / 32; ++q) s += red[q][threadIdx.x];
        partials[(int64_t)threadIdx.x * nblk + blockIdx.x] = s;
    }
}

__global__ void reduce_partials_kernel(const double *partials, int nblk, double *out) {
    __shared__ double red[32];
    const double *p = partials + (int64_t)blockIdx.x * nblk;
    double s = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += p[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
        if (threadIdx.x == 0) out[blockIdx.x] = t;
    }
}

// out = in / d, with d = *dn (or sqrt(*dn) if sqrt_of)
__global__ void scale_kernel(int64_t n, const double *in, double *out, const double *dn, int sqrt_of) {
    double d = sqrt_of ? sqrt(*dn) : *dn;
    double r = d != 0.0 ? 1.0 / d : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i] * r;
}

// Column j of the Hessenberg matrix from the two Gram-Schmidt passes, the
// rotations, and the residual estimate |g_{j+1}| / ||b||.
__global__ void givens_kernel(int j, int m, const double *h1, const double *h2, const double *nrm2, double *Hm,
                              double *cs, double *sn, double *g, double *scal, double bnorm) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double *col = Hm + (int64_t)j * (m + 1);
    for (int i = 0; i <= j; ++i) col[i] = h1[i] + h2[i];
    double hn = sqrt(*nrm2);
    col[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
        double a = col[i], c = col[i + 1];
        col[i] = cs[i] * a + sn[i] * c;
        col[i + 1] = -sn[i] * a + cs[i] * c;
    }
    double a = col[j], c = col[j + 1];
    double r = hypot(a, c);
    cs[j] = r > 0.0 ? a / r : 1.0;
    sn[j] = r > 0.0 ? c / r : 0.0;
    col[j] = r;
    col[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    scal[1] = fabs(g[j + 1]) / bnorm;
    scal[2] = hn;
}

__global__ void hessenberg_solve_kernel(int k, int m, const double *Hm, const double *g, double *y) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int c = i + 1; c < k; ++c) s -= Hm[(int64_t)c * (m + 1) + i] * y[c];
        y[i] = s / Hm[(int64_t)i * (m + 1) + i];
    }
}

__global__ void axpy_multi_kernel(int64_t n, const double *__restrict__ Z, int64_t ldz, int k,
                                  const double *__restrict__ y, double *__restrict__ x) {
    __shared__ double ys[MAXK];
    for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = y[i];
    __syncthreads();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        double s = x[t];
        for (int i = 0; i < k; ++i) s += ys[i] * Z[(int64_t)i * ldz + t];
        x[t] = s;
    }
}

__global__ void set_scalar_kernel(double *p, double v) { *p = v; }

// out = ca a + cb b (+ cc c when c != NULL); out may alias any input (elementwise)
__global__ void lincomb_kernel(int64_t n, double *out, const double *a, double ca, const double *b, double cb,
                               const double *c, double cc) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = ca * a[i] + cb * b[i];
        if (c) v += cc * c[i];
        out[i] = v;
    }
}

template <int U, typename TV, typename TX, int MODE>
void launch_row(const RowArgs<TV, TX> &a, cudaStream_t s) {
    unsigned g = grid_cap(a.n * 4, 256, 152 * 16);
    row_kernel<4, U, TV, TX, MODE><<<air_counted(g), 256, 0, s>>>(a);
}

// Entries per lane: enough for the longest row when rows are at most 64
// long, else for the average row with the remainder loop taking the rest.
template <typename TV, typename TX, int MODE>
void row_dispatch(const RowArgs<TV, TX> &a, int64_t nnz, int32_t maxrow, cudaStream_t s) {
    double avg = a.n > 0 ? (double)nnz / (double)a.n : 0.0;
    int want = maxrow > 0 && maxrow <= 64 ? (maxrow + 3) / 4 : (int)((avg * 1.25 + 3.0) / 4.0);
    if (want <= 1) launch_row<1, TV, TX, MODE>(a, s);
    else if (want <= 2) launch_row<2, TV, TX, MODE>(a, s);
    else if (want <= 4) launch_row<4, TV, TX, MODE>(a, s);
    else if (want <= 6) launch_row<6, TV, TX, MODE>(a, s);
    else if (want <= 8) launch_row<8, TV, TX, MODE>(a, s);
    else if (want <= 10) launch_row<10, TV, TX, MODE>(a, s);
    else if (want <= 12) launch_row<12, TV, TX, MODE>(a, s);
    else launch_row<16, TV, TX, MODE>(a, s);
}

template <typename TV, typename TX>
void spmv_dispatch(int64_t n, int64_t nnz, int32_t maxrow, const int64_t *rp, const int32_t *ci, const TV *v,
                   const TX *x, TX *y, const TX *b, cudaStream_t s) {
    RowArgs<TV, TX> a{};
    a.n = n; a.rp = rp; a.ci = ci; a.v = v; a.x = x; a.y = y; a.b = b;
    row_dispatch<TV, TX, ROW_SPMV>(a, nnz, maxrow, s);
}

// One Jacobi sweep over the point set `which` (0 = F, 1 = C), in place on x:
// new values of the set's rows go to tmp, then are scattered back.
template <typename TV, typename T>
void jacobi_dispatch(const AirLevel &L, const T *diag, const T *dinv, int which, T omega, const T *b, T *x, T *tmp,
                     cudaStream_t s, bool scatter = true) {
    const Sell &S = L.sset[which];
    if (S.m == 0) return;
    if (S.b > 0) {
        BSellArgs<TV, T> ba{};
        ba.m = S.m; ba.ptr = S.ptr; ba.bc = S.bc; ba.v = (const TV *)S.v; ba.dv = (const T *)S.dv; ba.rows = S.rows;
        ba.x = x; ba.y = tmp; ba.b = b; ba.dinv = dinv; ba.omega = omega;
        bsell_launch<TV, T, ROW_JACOBI>(S.b, ba, s);
        if (scatter) scatter_kernel<T><<<air_counted(grid_cap(S.m, 256)), 256, 0, s>>>(S.m, S.rows, tmp, x);
        return;
    }
    SellArgs<TV, T> a{};
    a.m = S.m; a.ptr = S.ptr; a.ci = S.ci; a.v = (const TV *)S.v; a.rows = S.rows;
    a.x = x; a.y = tmp; a.b = b; a.dinv = dinv; a.diag = diag; a.omega = omega;
    sell_launch<TV, T, ROW_JACOBI>(a, s, L.lanes[which]);
    if (scatter) scatter_kernel<T><<<air_counted(grid_cap(S.m, 256)), 256, 0, s>>>(S.m, S.rows, tmp, x);
}

// One Jacobi sweep over the point set `which` from x into the full vector y:
// the set's rows get their new values, the other set's rows (when copy) their
// values in x, in the same launch.
template <typename TV, typename T>
void jacobi_full_dispatch(const AirLevel &L, const T *diag, const T *dinv, int which, T omega, const T *b,
                          const T *x, T *y, bool copy, cudaStream_t s) {
    const Sell &S = L.sset[which], &O = L.sset[1 - which];
    const int64_t mc = copy ? O.m : 0;
    if (S.m == 0) {
        if (mc > 0) {
            SellArgs<TV, T> a{};
            a.m = 0; a.x = x; a.y = y; a.mc = mc; a.crows = O.rows; a.sweep_blocks = 0;
            sell_kernel<8, TV, T, ROW_JACOBI_FULL><<<air_counted((unsigned)copy_blocks(mc)), 256, 0, s>>>(a);
        }
        return;
    }
    if (S.b > 0) {
        BSellArgs<TV, T> ba{};
        ba.m = S.m; ba.ptr = S.ptr; ba.bc = S.bc; ba.v = (const TV *)S.v; ba.dv = (const T *)S.dv; ba.rows = S.rows;
        ba.x = x; ba.y = y; ba.b = b; ba.dinv = dinv; ba.omega = omega; ba.mc = mc; ba.crows = O.rows;
        bsell_launch<TV, T, ROW_JACOBI_FULL>(S.b, ba, s);
        return;
    }
    SellArgs<TV, T> a{};
    a.m = S.m; a.ptr = S.ptr; a.ci = S.ci; a.v = (const TV *)S.v; a.rows = S.rows;
    a.x = x; a.y = y; a.b = b; a.dinv = dinv; a.diag = diag; a.omega = omega; a.mc = mc; a.crows = O.rows;
    sell_launch<TV, T, ROW_JACOBI_FULL>(a, s, L.lanes[which]);
}

// One Jacobi sweep over all points: both point sets from the same old x into
// the two halves of tmp, then both scatters.
template <typename TV, typename T>
void jacobi_all_dispatch(const AirLevel &L, const T *diag, const T *dinv, T omega, const T *b, T *x, T *tmp,
                         cudaStream_t s) {
    T *tf = tmp, *tc = tmp + L.sset[0].m;
    jacobi_dispatch<TV, T>(L, diag, dinv, 0, omega, b, x, tf, s, false);
    jacobi_dispatch<TV, T>(L, diag, dinv, 1, omega, b, x, tc, s, false);
    for (int w = 0; w < 2; ++w) {
        const Sell &S = L.sset[w];
        if (S.m > 0)
            scatter_kernel<T><<<air_counted(grid_cap(S.m, 256)), 256, 0, s>>>(S.m, S.rows, w == 0 ? tf : tc, x);
    }
}

// The separate FP32 diagonal (BF16 storage only) and 1/a_ii in the vector
// type T.
template <typename T> const T *lvl_dinv(const AirLevel &L);
template <> const double *lvl_dinv<double>(const AirLevel &L) { return L.dinv; }
template <> const float *lvl_dinv<float>(const AirLevel &L) { return L.dinv32; }
template <typename TV> const float *lvl_diag(const AirLevel &L) { return nullptr; }
template <> const float *lvl_diag<__nv_bfloat16>(const AirLevel &L) { return L.diag32; }

// V-cycle with values stored as TV and vectors in T.  b0: finest right-hand
// side, x0: finest output.
template <typename TV, typename T>
int vcycle_t(const air_hierarchy *H, const T *b0, T *x0, cudaStream_t s) {
    int L = H->nlev;
    const char *relax = H->opt.relax;
    int ns = (int)strnlen(relax, sizeof(H->opt.relax));
    T omega = (T)H->opt.omega;
    // restriction down to the coarsest level
    for (int l = 0; l + 1 < L; ++l) {
        const AirLevel &A = H->lev[l];
        const T *bl = l == 0 ? b0 : (const T *)A.b;
        SellArgs<TV, T> ra{};
        ra.m = A.sr.m; ra.ptr = A.sr.ptr; ra.ci = A.sr.ci; ra.v = (const TV *)A.sr.v; ra.rows = A.sr.rows;
        ra.x = bl; ra.y = (T *)H->lev[l + 1].b;
        sell_launch<TV, T, ROW_SPMV>(ra, s, A.lanes[2]);
    }
    // coarsest: x = A_L^{-1} b
    {
        const AirLevel &C = H->lev[L - 1];
        const T *bl = L == 1 ? b0 : (const T *)C.b;
        T *xl = L == 1 ? x0 : (T *)C.x;
        const T *Ci = std::is_same<T, double>::value ? (const T *)H->cinv : (const T *)H->cinv32;
        unsigned g = grid_cap(C.n * 32, 256, 152 * 8);
        dense_gemv_kernel<T><<<air_counted(g), 256, 0, s>>>(C.n, Ci, bl, xl);
    }
    // interpolation and relaxation back up
    for (int l = L - 2; l >= 0; --l) {
        const AirLevel &A = H->lev[l];
        const T *bl = l == 0 ? b0 : (const T *)A.b;
        T *out = l == 0 ? x0 : (T *)A.x;
        T *alt = (T *)A.x2;
        const T *xc = (const T *)H->lev[l + 1].x;
        const T *diag = (const T *)lvl_diag<TV>(A);
        const T *dinv = lvl_dinv<T>(A);
        bool gs = false;
        for (int q = 0; q < ns; ++q) gs = gs || relax[q] >= 'a';
        if (!gs) {
            // x = P x_c, then Jacobi sweeps alternating between out and alt,
            // starting in whichever of the two makes the last sweep end in out
            T *cur = ns % 2 == 1 ? alt : out, *nxt = ns % 2 == 1 ? out : alt;
            interp_kernel<T><<<air_counted(grid_cap(A.n, 256)), 256, 0, s>>>(A.n, A.pcol, xc, cur);
            for (int q = 0; q < ns; ++q) {
                const char c = relax[q];
                if (c == 'A') {
                    jacobi_full_dispatch<TV, T>(A, diag, dinv, 0, omega, bl, cur, nxt, false, s);
                    jacobi_full_dispatch<TV, T>(A, diag, dinv, 1, omega, bl, cur, nxt, false, s);
                } else {
                    jacobi_full_dispatch<TV, T>(A, diag, dinv, c == 'C' ? 1 : 0, omega, bl, cur, nxt, true, s);
                }
                T *t = cur;
                cur = nxt;
                nxt = t;
            }
            continue;
        }
        // x = P x_c, then the sweeps in place
        interp_kernel<T><<<air_counted(grid_cap(A.n, 256)), 256, 0, s>>>(A.n, A.pcol, xc, out);
        for (int q = 0; q < ns; ++q) {
            const char c = relax[q];
            if (c == 'F' || c == 'C') {
                jacobi_dispatch<TV, T>(A, diag, dinv, c == 'C' ? 1 : 0, omega, bl, out, alt, s);
            } else if (c == 'A') {
                jacobi_all_dispatch<TV, T>(A, diag, dinv, omega, bl, out, alt, s);
            } else {                                   // 'f', 'c', 'a': forward Gauss-Seidel
                AIR_TRY(air_gs_sweep<T>(A, c == 'f' ? 0 : (c == 'c' ? 1 : 2), omega, bl, out, alt, s));
            }
        }
    }
    AIR_LAUNCH();
    return AIR_OK;
}

}  // namespace

int air_spmv_f64(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const double *x, double *y,
                 const double *b, cudaStream_t s, int64_t nnz, int32_t maxrow) {
    if (nnz < 0) nnz = 40 * n;      // unknown: sized for the 2D+time p = 2 rows, remainder loop for longer ones
    spmv_dispatch<double, double>(n, nnz, maxrow, rp, ci, v, x, y, b, s);
    AIR_LAUNCH();
    return AIR_OK;
}

// The V-cycle body (from the finest-level buffers lev[0].b to lev[0].x) is
// captured once into a CUDA graph on a private stream and replayed on the
// caller's stream; only the conversion in and out of lev[0] runs outside it.
template <typename TV, typename T>
int vcycle_graph(air_hierarchy *H, cudaStream_t s) {
    const AirLevel &L0 = H->lev[0];
    if (!H->vgraph && !H->vgraph_failed) {
        cudaStream_t cs = nullptr;
        AIR_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        unsigned long long c0 = air_launch_counter_add(0);
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            int st = vcycle_t<TV, T>(H, (const T *)L0.b, (T *)L0.x, cs);
            e = cudaStreamEndCapture(cs, &g);
            if (st != AIR_OK && e == cudaSuccess) e = cudaErrorUnknown;
        }
        unsigned long long c1 = air_launch_counter_add(0);
        air_launch_counter_sub(c1 - c0);   // captured, not yet run
        if (e == cudaSuccess) e = cudaGraphInstantiate(&H->vgraph, g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            H->vgraph = nullptr;
            H->vgraph_failed = 1;
        } else {
            H->vgraph_kernels = (long long)(c1 - c0);
        }
    }
    if (H->vgraph) {
        AIR_CUDA(cudaGraphLaunch(H->vgraph, s));
        air_launch_counter_add((unsigned long long)H->vgraph_kernels);
        return AIR_OK;
    }
    return vcycle_t<TV, T>(H, (const T *)L0.b, (T *)L0.x, s);
}

int air_vcycle_staged(air_hierarchy *H, cudaStream_t s) {
    const AirLevel &L0 = H->lev[0];
    if (H->opt.precision == AIR_PREC_F64) return vcycle_t<double, double>(H, (const double *)L0.b, (double *)L0.x, s);
    if (H->opt.precision == AIR_PREC_BF16)
        return vcycle_t<__nv_bfloat16, float>(H, (const float *)L0.b, (float *)L0.x, s);
    return vcycle_t<float, float>(H, (const float *)L0.b, (float *)L0.x, s);
}

namespace {

// Job blockIdx.y: the same element conversions as d2f_kernel / f2d_kernel, or a copy.
__global__ void convert_batch_kernel(const AirConvJob *jobs) {
    const AirConvJob J = jobs[blockIdx.y];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < J.n; i += (int64_t)gridDim.x * blockDim.x) {
        if (J.mode == 1) ((float *)J.dst)[i] = (float)((const double *)J.src)[i];
        else if (J.mode == 2) ((double *)J.dst)[i] = (double)((const float *)J.src)[i];
        else ((double *)J.dst)[i] = ((const double *)J.src)[i];
    }
}

}  // namespace

int air_convert_batch(int count, const AirConvJob *d_jobs, cudaStream_t s) {
    if (count <= 0) return AIR_OK;
    if (count > 65535) return AIR_ERR_INVALID_ARG;
    unsigned bx = (unsigned)((152 * 8 + count - 1) / count);
    dim3 grid(bx < 1 ? 1 : bx, (unsigned)count);
    convert_batch_kernel<<<air_counted(grid), 256, 0, s>>>(d_jobs);
    AIR_LAUNCH();
    return AIR_OK;
}

int air_vcycle_run(const air_hierarchy *Hc, const double *b, double *x, cudaStream_t s, int use_graph) {
    air_hierarchy *H = const_cast<air_hierarchy *>(Hc);
    const AirLevel &L0 = H->lev[0];
    if (H->opt.precision == AIR_PREC_F64) {
        if (!use_graph) return vcycle_t<double, double>(H, b, x, s);
        AIR_CUDA(cudaMemcpyAsync(L0.b, b, (size_t)L0.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        AIR_TRY((vcycle_graph<double, double>(H, s)));
        AIR_CUDA(cudaMemcpyAsync(x, L0.x, (size_t)L0.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        return AIR_OK;
    }
    float *b32 = (float *)L0.b, *x32 = (float *)L0.x;
    d2f_kernel<<<air_counted(grid_cap(L0.n, 256)), 256, 0, s>>>(b, b32, L0.n);
    AIR_LAUNCH();
    const bool bf16 = H->opt.precision == AIR_PREC_BF16;
    if (use_graph) {
        if (bf16) AIR_TRY((vcycle_graph<__nv_bfloat16, float>(H, s)));
        else AIR_TRY((vcycle_graph<float, float>(H, s)));
    } else {
        if (bf16) AIR_TRY((vcycle_t<__nv_bfloat16, float>(H, b32, x32, s)));
        else AIR_TRY((vcycle_t<float, float>(H, b32, x32, s)));
    }
    f2d_kernel<<<air_counted(grid_cap(L0.n, 256)), 256, 0, s>>>(x32, x, L0.n);
    AIR_LAUNCH();
    return AIR_OK;
}

int air_build_sell(int64_t m, const int32_t *rows_in, const int64_t *rp, const int32_t *ci, const double *v,
                   int precision, int zero_diag, Sell *out, cudaStream_t s) {
    air_free_sell(*out);
    out->m = m;
    const int64_t ns = (m + 31) / 32;
    AIR_CUDA(air_dmalloc((void **)&out->rows, (size_t)(m > 0 ? m : 1) * sizeof(int32_t)));
    if (m > 0) {
        sell_sort_kernel<<<air_counted((unsigned)((m + SIGMA - 1) / SIGMA)), SIGMA / 2, 0, s>>>(m, rows_in, rp,
                                                                                              out->rows);
        AIR_LAUNCH();
    }
    const int32_t *rows = out->rows;
    int32_t *wid = nullptr;
    AIR_CUDA(air_dmalloc((void **)&out->ptr, (size_t)(ns + 1) * sizeof(int64_t)));
    AIR_CUDA(cudaMallocAsync(&wid, (size_t)(ns > 0 ? ns : 1) * sizeof(int32_t), s));
    sell_width_kernel<<<air_counted(grid_cap(ns, 256)), 256, 0, s>>>(m, rows, rp, wid);
    AIR_LAUNCH();
    AIR_TRY(air_exclusive_scan_i32(wid, out->ptr, ns, s));
    AIR_CUDA(cudaMemcpyAsync(&out->stored, out->ptr + ns, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    AIR_CUDA(cudaStreamSynchronize(s));
    cudaFreeAsync(wid, s);
    const int64_t cnt = out->stored > 0 ? out->stored : 1;
    const size_t vb = precision == AIR_PREC_F64 ? 8 : (precision == AIR_PREC_F32 ? 4 : 2);
    AIR_CUDA(air_dmalloc((void **)&out->ci, (size_t)cnt * sizeof(int32_t)));
    AIR_CUDA(air_dmalloc(&out->v, (size_t)cnt * vb));
    unsigned g = grid_cap(ns * 32, 256, 152 * 32);
    if (precision == AIR_PREC_F64)
        sell_fill_kernel<double, false><<<air_counted(g), 256, 0, s>>>(m, rows, rp, ci, v, out->ptr, out->ci,
                                                                       (double *)out->v);
    else if (precision == AIR_PREC_F32)
        sell_fill_kernel<float, false><<<air_counted(g), 256, 0, s>>>(m, rows, rp, ci, v, out->ptr, out->ci,
                                                                      (float *)out->v);
    else if (zero_diag)
        sell_fill_kernel<__nv_bfloat16, true><<<air_counted(g), 256, 0, s>>>(m, rows, rp, ci, v, out->ptr, out->ci,
                                                                             (__nv_bfloat16 *)out->v);
    else
        sell_fill_kernel<__nv_bfloat16, false><<<air_counted(g), 256, 0, s>>>(m, rows, rp, ci, v, out->ptr, out->ci,
                                                                              (__nv_bfloat16 *)out->v);
    AIR_LAUNCH();
    return AIR_OK;
}

void air_free_sell(Sell &S) {
    air_dfree(S.rows);
    air_dfree(S.ptr);
    air_dfree(S.ci);
    air_dfree(S.v);
    air_dfree(S.bc);
    air_dfree(S.dv);
    S = Sell();
}

// Blocks of each row (pos order of rows_in, or rows 0.. when NULL) into nb[pos];
// a row that is not whole aligned b-blocks plus at most its diagonal sets *err.
__global__ void block_count_kernel(int64_t m, const int32_t *rows, const int64_t *rp, const int32_t *ci, int b,
                                   int32_t *nb, int *err) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = rows ? rows[p] : p;
        int64_t k = rp[r];
        const int64_t e = rp[r + 1];
        int cnt = 0;
        while (k < e) {
            const int32_t c = ci[k];
            if (c % b == 0 && k + b <= e && ci[k + b - 1] == c + b - 1) { ++cnt; k += b; }
            else if (c == r) { ++k; }
            else { atomicOr(err, 1); break; }
        }
        nb[p] = cnt;
    }
}

__global__ void block_width_kernel(int64_t m, const int32_t *sorted, const int32_t *pos_of, const int32_t *nb,
                                   int32_t *wid) {
    const int64_t ns = (m + 31) / 32;
    for (int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; sl < ns; sl += (int64_t)gridDim.x * blockDim.x) {
        int32_t w = 0;
        for (int64_t p = sl * 32; p < m && p < sl * 32 + 32; ++p) w = max(w, nb[pos_of[p]]);
        wid[sl] = w * 32;
    }
}

// position in the unsorted set of every sorted position (rows are distinct)
__global__ void block_posmap_kernel(int64_t m, const int32_t *rows_in, const int32_t *sorted, int32_t *inv_row,
                                    int32_t *pos_of) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x)
        pos_of[p] = inv_row[sorted[p]];
}

__global__ void block_invrow_kernel(int64_t m, const int32_t *rows_in, int32_t *inv_row) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x)
        inv_row[rows_in ? rows_in[p] : p] = (int32_t)p;
}

template <typename TV, typename TD, bool ZERO_DIAG>
__global__ void block_fill_kernel(int64_t m, const int32_t *rows, const int64_t *rp, const int32_t *ci,
                                  const double *v, int b, const int64_t *ptr, int32_t *bc, TV *bv, TD *dv) {
    const int64_t ns32 = ((m + 31) / 32) * 32;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < ns32; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sl = p >> 5, l = p & 31;
        const int64_t base = ptr[sl], w = (ptr[sl + 1] - base) >> 5;
        int64_t t = 0;
        if (p < m) {
            const int64_t r = rows[p];
            int64_t k = rp[r];
            const int64_t e = rp[r + 1];
            double dstand = 0.0, dall = 0.0;    // standalone diagonal; the diagonal wherever it is
            while (k < e && t < w) {
                const int32_t c = ci[k];
                if (c % b == 0 && k + b <= e && ci[k + b - 1] == c + b - 1) {
                    const int64_t slot = base + 32 * t + l;
                    bc[slot] = c;
                    for (int j = 0; j < b; ++j) {
                        const bool dg = c + j == r;
                        if (dg) dall = v[k + j];
                        bv[slot * b + j] = (TV)((ZERO_DIAG && dg) ? 0.0 : v[k + j]);
                    }
                    ++t;
                    k += b;
                } else {                         // the standalone diagonal (the structure check passed)
                    dstand = v[k];
                    dall = v[k];
                    ++k;
                }
            }
            if (k < e && ci[k] == r) {           // a standalone diagonal after the last block
                dstand = v[k];
                dall = v[k];
            }
            dv[p] = (TD)(ZERO_DIAG ? dall : dstand);
        }
        for (; t < w; ++t) {
            const int64_t slot = base + 32 * t + l;
            bc[slot] = 0;
            for (int j = 0; j < b; ++j) bv[slot * b + j] = (TV)0.0;
        }
    }
}

namespace {

// Lanes per row by rule: double the lanes while the grid holds fewer than
// about two waves of threads (or rows longer than 32 stored entries per lane)
// and each lane keeps more than four entries.
int lanes_rule(const Sell &S) {
    if (S.m <= 0 || S.b > 0) return 1;
    const double avg = (double)S.stored / (double)S.m;
    int L = 1;
    while (L < 32 && avg / L > 4.0 && ((double)S.m * L < 152.0 * 2048.0 || avg / L > 32.0)) L *= 2;
    return L;
}

// Times the candidate lanes per row on the launch the V-cycle makes: a sweep
// (into the full vector y, with the other point set's rows copied, `other`)
// or a restriction.
template <typename TV, typename T>
int tune_set(const AirLevel &Lv, const Sell &S, const Sell *other, bool jacobi, const T *x, const T *b, T *y,
             const T *dinv, const T *diag, int *out, cudaStream_t s) {
    SellArgs<TV, T> a{};
    a.m = S.m; a.ptr = S.ptr; a.ci = S.ci; a.v = (const TV *)S.v; a.rows = S.rows;
    a.x = x; a.y = y; a.b = b; a.dinv = dinv; a.diag = diag; a.omega = (T)1;
    if (other) {
        a.mc = other->m;
        a.crows = other->rows;
    }
    const int cand_all[6] = {1, 2, 4, 8, 16, 32};
    const double avg = S.m > 0 ? (double)S.stored / (double)S.m : 0.0;
    cudaEvent_t e0, e1;
    AIR_CUDA(cudaEventCreate(&e0));
    AIR_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int pick = 1;
    for (int c : cand_all) {
        if (c > 1 && (avg / c < 1.0 || (S.m >= 2000000 && c > 2))) continue;
        for (int rep = 0; rep < 4; ++rep) {
            if (rep == 1) cudaEventRecord(e0, s);
            if (jacobi) sell_launch<TV, T, ROW_JACOBI_FULL>(a, s, c);
            else sell_launch<TV, T, ROW_SPMV>(a, s, c);
        }
        cudaEventRecord(e1, s);
        AIR_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        AIR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) { best = ms; pick = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    AIR_LAUNCH();
    *out = pick;
    return AIR_OK;
}

template <typename TV, typename T>
int tune_levels(air_hierarchy *H, cudaStream_t s) {
    for (int q = 0; q + 1 < H->nlev; ++q) {
        AirLevel &L = H->lev[q];
        const size_t es = sizeof(T);
        AIR_CUDA(cudaMemsetAsync(L.b, 0, (size_t)L.n * es, s));
        AIR_CUDA(cudaMemsetAsync(L.x, 0, (size_t)L.n * es, s));
        const T *dinv = lvl_dinv<T>(L);
        const T *diag = (const T *)lvl_diag<TV>(L);
        for (int which = 0; which < 2; ++which)
            if (L.sset[which].b == 0 && L.sset[which].m > 0)
                AIR_TRY((tune_set<TV, T>(L, L.sset[which], &L.sset[1 - which], true, (const T *)L.x, (const T *)L.b,
                                         (T *)L.x2, dinv, diag, &L.lanes[which], s)));
        if (L.sr.m > 0)
            AIR_TRY((tune_set<TV, T>(L, L.sr, nullptr, false, (const T *)L.b, nullptr, (T *)H->lev[q + 1].b, nullptr,
                                     nullptr, &L.lanes[2], s)));
    }
    return AIR_OK;
}

}  // namespace

int air_tune_lanes(air_hierarchy *H, int timed, cudaStream_t s) {
    for (int q = 0; q + 1 < H->nlev; ++q) {
        AirLevel &L = H->lev[q];
        L.lanes[0] = lanes_rule(L.sset[0]);
        L.lanes[1] = lanes_rule(L.sset[1]);
        L.lanes[2] = lanes_rule(L.sr);
    }
    if (!timed) return AIR_OK;
    if (H->opt.precision == AIR_PREC_F64) return tune_levels<double, double>(H, s);
    if (H->opt.precision == AIR_PREC_F32) return tune_levels<float, float>(H, s);
    return tune_levels<__nv_bfloat16, float>(H, s);
}

int air_build_sell_blocks(int64_t m, const int32_t *rows_in, const int64_t *rp, const int32_t *ci, const double *v,
                          int precision, int b, Sell *out, cudaStream_t s) {
    if (b != 2 && b != 3 && b != 4 && b != 6 && b != 10) return AIR_ERR_UNSUPPORTED;
    *out = Sell();
    if (m <= 0) return AIR_ERR_UNSUPPORTED;
    int32_t *nb = nullptr, *inv = nullptr, *pos_of = nullptr, *wid = nullptr;
    int *err = nullptr;
    const int64_t ns = (m + 31) / 32;
    // rows_in are row ids of the level; inverse map sized by the largest id + 1 (<= the level's rows)
    int64_t idmax = m;
    if (rows_in) {
        int32_t hmax = 0;
        int32_t *dmax = nullptr;
        AIR_CUDA(cudaMallocAsync(&dmax, sizeof(int32_t), s));
        AIR_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int32_t), s));
        AIR_TRY(air_reduce_max_i32(rows_in, m, dmax, s));
        AIR_CUDA(cudaMemcpyAsync(&hmax, dmax, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        AIR_CUDA(cudaStreamSynchronize(s));
        cudaFreeAsync(dmax, s);
        idmax = (int64_t)hmax + 1;
    }
    AIR_CUDA(cudaMallocAsync(&nb, (size_t)m * sizeof(int32_t), s));
    AIR_CUDA(cudaMallocAsync(&err, sizeof(int), s));
    AIR_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    block_count_kernel<<<air_counted(grid_cap(m, 256)), 256, 0, s>>>(m, rows_in, rp, ci, b, nb, err);
    AIR_LAUNCH();
    int herr = 0;
    AIR_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    AIR_CUDA(cudaStreamSynchronize(s));
    cudaFreeAsync(err, s);
    if (herr) {
        cudaFreeAsync(nb, s);
        return AIR_ERR_UNSUPPORTED;
    }
    out->m = m;
    out->b = b;
    AIR_CUDA(air_dmalloc((void **)&out->rows, (size_t)m * sizeof(int32_t)));
    sell_sort_kernel<<<air_counted((unsigned)((m + SIGMA - 1) / SIGMA)), SIGMA / 2, 0, s>>>(m, rows_in, rp, out->rows);
    AIR_LAUNCH();
    AIR_CUDA(cudaMallocAsync(&inv, (size_t)idmax * sizeof(int32_t), s));
    AIR_CUDA(cudaMallocAsync(&pos_of, (size_t)m * sizeof(int32_t), s));
    block_invrow_kernel<<<air_counted(grid_cap(m, 256)), 256, 0, s>>>(m, rows_in, inv);
    block_posmap_kernel<<<air_counted(grid_cap(m, 256)), 256, 0, s>>>(m, rows_in, out->rows, inv, pos_of);
    AIR_CUDA(air_dmalloc((void **)&out->ptr, (size_t)(ns + 1) * sizeof(int64_t)));
    AIR_CUDA(cudaMallocAsync(&wid, (size_t)ns * sizeof(int32_t), s));
    block_width_kernel<<<air_counted(grid_cap(ns, 256)), 256, 0, s>>>(m, out->rows, pos_of, nb, wid);
    AIR_LAUNCH();
    AIR_TRY(air_exclusive_scan_i32(wid, out->ptr, ns, s));
    AIR_CUDA(cudaMemcpyAsync(&out->stored, out->ptr + ns, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    AIR_CUDA(cudaStreamSynchronize(s));
    cudaFreeAsync(wid, s);
    cudaFreeAsync(inv, s);
    cudaFreeAsync(pos_of, s);
    cudaFreeAsync(nb, s);
    const int64_t cnt = out->stored > 0 ? out->stored : 1;
    const size_t vb = precision == AIR_PREC_F64 ? 8 : (precision == AIR_PREC_F32 ? 4 : 2);
    const size_t db = precision == AIR_PREC_F64 ? 8 : 4;
    AIR_CUDA(air_dmalloc((void **)&out->bc, (size_t)cnt * sizeof(int32_t)));
    AIR_CUDA(air_dmalloc(&out->v, (size_t)cnt * b * vb));
    AIR_CUDA(air_dmalloc(&out->dv, (size_t)m * db));
    unsigned g = grid_cap(ns * 32, 256, 152 * 32);
    if (precision == AIR_PREC_F64)
        block_fill_kernel<double, double, false><<<air_counted(g), 256, 0, s>>>(m, out->rows, rp, ci, v, b, out->ptr,
                                                                                 out->bc, (double *)out->v,
                                                                                 (double *)out->dv);
    else if (precision == AIR_PREC_F32)
        block_fill_kernel<float, float, false><<<air_counted(g), 256, 0, s>>>(m, out->rows, rp, ci, v, b, out->ptr,
                                                                               out->bc, (float *)out->v,
                                                                               (float *)out->dv);
    else
        block_fill_kernel<__nv_bfloat16, float, true><<<air_counted(g), 256, 0, s>>>(
            m, out->rows, rp, ci, v, b, out->ptr, out->bc, (__nv_bfloat16 *)out->v, (float *)out->dv);
    AIR_LAUNCH();
    return AIR_OK;
}

int air_sell_spmv_f64(const Sell &S, const double *x, double *y, const double *b, cudaStream_t s) {
    if (S.b > 0) {
        BSellArgs<double, double> ba{};
        ba.m = S.m; ba.ptr = S.ptr; ba.bc = S.bc; ba.v = (const double *)S.v; ba.dv = (const double *)S.dv;
        ba.rows = S.rows; ba.x = x; ba.y = y; ba.b = b;
        bsell_launch<double, double, ROW_SPMV>(S.b, ba, s);
        AIR_LAUNCH();
        return AIR_OK;
    }
    SellArgs<double, double> a{};
    a.m = S.m; a.ptr = S.ptr; a.ci = S.ci; a.v = (const double *)S.v; a.rows = S.rows; a.x = x; a.y = y; a.b = b;
    sell_launch<double, double, ROW_SPMV>(a, s);
    AIR_LAUNCH();
    return AIR_OK;
}

int air_cast_bf16(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, void *out16, float *diag32,
                  cudaStream_t s) {
    d2bf_offdiag_kernel<<<air_counted(grid_cap(n, 256)), 256, 0, s>>>(n, rp, ci, v, (__nv_bfloat16 *)out16, diag32);
    AIR_LAUNCH();
    return AIR_OK;
}

int air_cast_d2f(const double *in, float *out, int64_t n, cudaStream_t s) {
    d2f_kernel<<<air_counted(grid_cap(n, 256)), 256, 0, s>>>(in, out, n);
    AIR_LAUNCH();
    return AIR_OK;
}

int air_diag_inverse(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, double *dinv, float *dinv32,
                     cudaStream_t s) {
    diag_inverse_kernel<<<air_counted(grid_cap(n, 256)), 256, 0, s>>>(n, rp, ci, v, dinv, dinv32);
    AIR_LAUNCH();
    return AIR_OK;
}

int air_reduce_nblk(int64_t n) {
    int64_t b = (n + RT * 8 - 1) / (RT * 8);
    if (b > 152 * 4) b = 152 * 4;
    if (b < 1) b = 1;
    return (int)b;
}

int air_dot_partials(int64_t n, const double *V, int64_t ldv, int k, const double *w, double *partials, int nblk,
                     cudaStream_t s) {
    for (int k0 = 0; k0 < k; k0 += 16) {
        if (k - k0 <= 4) dot_partials_kernel<4><<<air_counted(nblk), RT, 0, s>>>(n, V, ldv, k0, k, w, partials, nblk);
        else if (k - k0 <= 8) dot_partials_kernel<8><<<air_counted(nblk), RT, 0, s>>>(n, V, ldv, k0, k, w, partials, nblk);
        else dot_partials_kernel<16><<<air_counted(nblk), RT, 0, s>>>(n, V, ldv, k0, k, w, partials, nblk);
    }
    AIR_LAUNCH();
    return AIR_OK;
}

int air_update_dot_partials(int64_t n, const double *V, int64_t ldv, int k, const double *h, double *w,
                            double *partials, int nblk, int dots, cudaStream_t s) {
    if (k <= 4) update_dot_kernel<4><<<air_counted(nblk), RT, 0, s>>>(n, V, ldv, k, h, w, partials, nblk, dots);
    else if (k <= 8) update_dot_kernel<8><<<air_counted(nblk), RT, 0, s>>>(n, V, ldv, k, h, w, partials, nblk, dots);
    else if (k <= 16) update_dot_kernel<16><<<air_counted(nblk), RT, 0, s>>>(n, V, ldv, k, h, w, partials, nblk, dots);
    else if (k <= 32) update_dot_kernel<32><<<air_counted(nblk), RT, 0, s>>>(n, V, ldv, k, h, w, partials, nblk, dots);
    else return AIR_ERR_UNSUPPORTED;
    AIR_LAUNCH();
    return AIR_OK;
}

int air_reduce_partials(int k, const double *partials, int nblk, double *out, cudaStream_t s) {
    if (k <= 0) return AIR_OK;
    reduce_partials_kernel<<<air_counted(k), 256, 0, s>>>(partials, nblk, out);
    AIR_LAUNCH();
    return AIR_OK;
}

int air_scale_vec(int64_t n, const double *in, double *out, const double *d_norm, int sqrt_of, cudaStream_t s) {
    scale_kernel<<<air_counted(grid_cap(n, 256)), 256, 0, s>>>(n, in, out, d_norm, sqrt_of);
    AIR_LAUNCH();
    return AIR_OK;
}

int air_arnoldi_givens(int j, int m, const double *h1, const double *h2, const double *nrm2, double *Hm, double *cs,
                       double *sn, double *g, double *scal, double bnorm, cudaStream_t s) {
    givens_kernel<<<air_counted(1), 32, 0, s>>>(j, m, h1, h2, nrm2, Hm, cs, sn, g, scal, bnorm);
    AIR_LAUNCH();
    return AIR_OK;
}

int air_hessenberg_solve(int k, int m, const double *Hm, const double *g, double *y, cudaStream_t s) {
    hessenberg_solve_kernel<<<air_counted(1), 32, 0, s>>>(k, m, Hm, g, y);
    AIR_LAUNCH();
    return AIR_OK;
}

int air_axpy_multi(int64_t n, const double *Z, int64_t ldz, int k, const double *y, double *x, cudaStream_t s) {
    axpy_multi_kernel<<<air_counted(grid_cap(n, 256)), 256, 0, s>>>(n, Z, ldz, k, y, x);
    AIR_LAUNCH();
    return AIR_OK;
}

int air_fill_zero(double *x, int64_t n, cudaStream_t s) {
    AIR_CUDA(cudaMemsetAsync(x, 0, (size_t)n * sizeof(double), s));
    return AIR_OK;
}

int air_lincomb(int64_t n, double *out, const double *a, double ca, const double *b, double cb, const double *c,
                double cc, cudaStream_t s) {
    if (n <= 0) return AIR_OK;
    lincomb_kernel<<<air_counted(grid_cap(n, 256)), 256, 0, s>>>(n, out, a, ca, b, cb, c, cc);
    AIR_LAUNCH();
    return AIR_OK;
}

int air_set_scalar(double *p, double v, cudaStream_t s) {
    set_scalar_kernel<<<air_counted(1), 1, 0, s>>>(p, v);
    AIR_LAUNCH();
    return AIR_OK;
}
