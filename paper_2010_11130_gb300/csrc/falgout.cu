// Falgout-style C/F splitting (the coarsening named in the paper's Section 4
// settings, whose details the paper leaves to its library): the points are cut
// into consecutive index blocks of `block` points; the first pass of
// Ruge-Stueben runs in every block at once on the strength graph restricted to
// the block, one warp per block with the block's measures in shared memory;
// then the interface points that ended F with strong connections but no
// strong C point are fixed by rounds of a parallel independent set.
//
// Local pass (the single-warp first pass of first_pass.cu, restricted): the
// measure of i is the number of points of its block that depend strongly on
// it; a point with no strong connection inside its block starts F.  Pick the
// undecided point of largest measure, ties to the smallest index; it becomes
// C, its undecided strong dependants in the block become F, every undecided
// point of the block in S_j of a new F point j gains one, every undecided
// point of the block in S_i loses one; stop when the largest measure is 0 (the
// rest become F).  The maximum is found through two levels of upper bounds
// (per 32 points and per 1024 points) that increments raise and searches
// repair when they meet a stale one.
//
// Interface rounds: U = F points with S_i non-empty, no C point in S_i and a
// strong connection (either way) to another block.  Weight
// w_i = |S^T_i| + frac(i), frac from the SplitMix64 hash of i (Steele, Lea and
// Flood, 2014).  A point of U whose weight beats every point of U in S_i and
// S^T_i (ties -> smaller index) becomes C; points of U with a C point in S_i
// leave U; repeat until U is empty.
#include "air_internal.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int FWARPS = 4;            // blocks of points (warps) per CTA
constexpr int NEWF_CAP = 1024;       // new F points of one pick
constexpr int LAM_F = -1, LAM_C = -2;
constexpr int8_t CF_F = 0, CF_C = 1;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int warp_max_i(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

unsigned grid_for(int64_t items, int threads) {
    int64_t b = (items + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)b;
}

// Shared memory of one warp: lam[block] (int32), g1[block / 32], g2[block / 1024], newF[NEWF_CAP].
__global__ void __launch_bounds__(FWARPS * 32) local_pass_kernel(int64_t n, int64_t block, const int64_t *srp,
                                                                 const int32_t *sci, const int64_t *strp,
                                                                 const int32_t *stci, int8_t *cf, int *err) {
    extern __shared__ int32_t fsm[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nblk = (n + block - 1) / block;
    const int64_t b = (int64_t)blockIdx.x * FWARPS + w;
    if (b >= nblk) return;
    const int64_t lo = b * block, hi = lo + block < n ? lo + block : n;
    const int m = (int)(hi - lo);
    const int ng1 = (int)((block + 31) / 32), ng2 = (int)((block + 1023) / 1024);
    int32_t *lam = fsm + (size_t)w * (block + ng1 + ng2 + NEWF_CAP);
    int32_t *g1 = lam + block, *g2 = g1 + ng1, *newF = g2 + ng2;
    // measures inside the block
    for (int t = lane; t < (int)block; t += 32) {
        int v = LAM_F;
        if (t < m) {
            const int64_t i = lo + t;
            int cnt = 0, ns = 0;
            for (int64_t a = strp[i]; a < strp[i + 1]; ++a) cnt += (stci[a] >= lo && stci[a] < hi);
            for (int64_t a = srp[i]; a < srp[i + 1]; ++a) ns += (sci[a] >= lo && sci[a] < hi);
            v = (cnt == 0 && ns == 0) ? LAM_F : cnt;
        }
        lam[t] = v;
    }
    __syncwarp();
    for (int gidx = lane; gidx < ng1; gidx += 32) {
        int mx = LAM_C;
        for (int t = 0; t < 32; ++t) mx = max(mx, lam[gidx * 32 + t]);
        g1[gidx] = mx;
    }
    __syncwarp();
    for (int h = lane; h < ng2; h += 32) {
        int mx = LAM_C;
        for (int t = 0; t < 32 && h * 32 + t < ng1; ++t) mx = max(mx, g1[h * 32 + t]);
        g2[h] = mx;
    }
    __syncwarp();
    const int64_t cap = 64 * (int64_t)m + 1024;  // picks plus repairs of stale bounds (a safety net)
    for (int64_t step = 0;; ++step) {
        if (step > cap) {
            if (lane == 0) atomicOr(err, AIR_DEVERR_RS_CAP);
            break;
        }
        // level 2: the largest bound and its first 1024-point range
        int v2 = lane < ng2 ? g2[lane] : LAM_C;
        for (int h = lane + 32; h < ng2; h += 32) v2 = max(v2, g2[h]);
        const int top = warp_max_i(v2);
        if (top < 1) break;
        int h = -1;
        for (int h0 = 0; h0 < ng2 && h < 0; h0 += 32) {
            const unsigned bal = __ballot_sync(FULL, h0 + lane < ng2 && g2[h0 + lane] == top);
            if (bal) h = h0 + __ffs(bal) - 1;
        }
        // level 1: the first 32-point group of that range with the bound
        const int gi = h * 32 + lane;
        const int b1 = gi < ng1 ? g1[gi] : LAM_C;
        const unsigned bal1 = __ballot_sync(FULL, b1 == top);
        if (!bal1) {                                   // stale range bound: repair it
            const int mx = warp_max_i(b1);
            if (lane == 0) g2[h] = mx;
            __syncwarp();
            continue;
        }
        const int g = h * 32 + __ffs(bal1) - 1;
        const int lv = lam[g * 32 + lane];
        const unsigned bal0 = __ballot_sync(FULL, lv == top);
        if (!bal0) {                                   // stale group bound: repair it
            const int mx = warp_max_i(lv);
            if (lane == 0) g1[g] = mx;
            __syncwarp();
            continue;
        }
        const int li = g * 32 + __ffs(bal0) - 1;
        const int64_t i = lo + li;
        if (lane == 0) lam[li] = LAM_C;
        __syncwarp();
        // undecided strong dependants of i in the block become F
        int nf = 0;
        for (int64_t a0 = strp[i]; a0 < strp[i + 1]; a0 += 32) {
            const int64_t a = a0 + lane;
            int32_t j = a < strp[i + 1] ? stci[a] : -1;
            const bool f = j >= lo && j < hi && lam[j - lo] >= 0;
            const unsigned bal = __ballot_sync(FULL, f);
            if (f) {
                const int p = nf + __popc(bal & lanemask_lt());
                if (p < NEWF_CAP) newF[p] = j;
                lam[j - lo] = LAM_F;
            }
            nf += __popc(bal);
        }
        if (nf > NEWF_CAP) {
            if (lane == 0) atomicOr(err, AIR_DEVERR_CAP);
            break;
        }
        __syncwarp();
        // every undecided point of the block in S_j of a new F point j gains one
        for (int q = 0; q < nf; ++q) {
            const int32_t j = newF[q];
            for (int64_t a = srp[j] + lane; a < srp[j + 1]; a += 32) {
                const int32_t k = sci[a];
                if (k >= lo && k < hi && lam[k - lo] >= 0) {
                    const int nv = atomicAdd(&lam[k - lo], 1) + 1;
                    atomicMax(&g1[(k - lo) >> 5], nv);
                    atomicMax(&g2[(k - lo) >> 10], nv);
                }
            }
        }
        __syncwarp();
        // every undecided point of the block in S_i loses one (bounds stay upper bounds)
        for (int64_t a = srp[i] + lane; a < srp[i + 1]; a += 32) {
            const int32_t k = sci[a];
            if (k >= lo && k < hi && lam[k - lo] >= 0) atomicSub(&lam[k - lo], 1);
        }
        __syncwarp();
    }
    __syncwarp();
    for (int t = lane; t < m; t += 32) cf[lo + t] = lam[t] == LAM_C ? CF_C : CF_F;
}

__device__ __forceinline__ double hash_frac(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ double weight(const int64_t *strp, int64_t i) {
    return __dadd_rn((double)(strp[i + 1] - strp[i]), hash_frac((uint64_t)i));
}

__device__ __forceinline__ bool has_c(const int64_t *srp, const int32_t *sci, const int8_t *cf, int64_t i) {
    for (int64_t a = srp[i]; a < srp[i + 1]; ++a)
        if (cf[sci[a]] == CF_C) return true;
    return false;
}

__global__ void interface_init_kernel(int64_t n, int64_t block, const int64_t *srp, const int32_t *sci,
                                      const int64_t *strp, const int32_t *stci, const int8_t *cf, int8_t *inU,
                                      unsigned long long *count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int8_t u = 0;
        if (cf[i] == CF_F && srp[i + 1] > srp[i] && !has_c(srp, sci, cf, i)) {
            const int64_t bi = i / block;
            bool cross = false;
            for (int64_t a = srp[i]; a < srp[i + 1] && !cross; ++a) cross = sci[a] / block != bi;
            for (int64_t a = strp[i]; a < strp[i + 1] && !cross; ++a) cross = stci[a] / block != bi;
            u = cross ? 1 : 0;
        }
        inU[i] = u;
        if (u) atomicAdd(count, 1ull);
    }
}

__global__ void interface_select_kernel(int64_t n, const int64_t *srp, const int32_t *sci, const int64_t *strp,
                                        const int32_t *stci, const int8_t *inU, int8_t *sel) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int8_t s = 0;
        if (inU[i]) {
            const double wi = weight(strp, i);
            bool best = true;
            for (int64_t a = srp[i]; a < srp[i + 1] && best; ++a) {
                const int32_t j = sci[a];
                if (!inU[j]) continue;
                const double wj = weight(strp, j);
                if (wj > wi || (wj == wi && j < i)) best = false;
            }
            for (int64_t a = strp[i]; a < strp[i + 1] && best; ++a) {
                const int32_t j = stci[a];
                if (!inU[j]) continue;
                const double wj = weight(strp, j);
                if (wj > wi || (wj == wi && j < i)) best = false;
            }
            s = best ? 1 : 0;
        }
        sel[i] = s;
    }
}

__global__ void interface_apply_kernel(int64_t n, const int8_t *sel, int8_t *cf, int8_t *inU) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (sel[i]) {
            cf[i] = CF_C;
            inU[i] = 0;
        }
}

__global__ void interface_leave_kernel(int64_t n, const int64_t *srp, const int32_t *sci, const int8_t *cf,
                                       int8_t *inU, unsigned long long *count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (!inU[i]) continue;
        if (has_c(srp, sci, cf, i)) inU[i] = 0;
        else atomicAdd(count, 1ull);
    }
}

}  // namespace

int air_falgout_split(int64_t n, int64_t block, const int64_t *srp, const int32_t *sci, const int64_t *strp,
                      const int32_t *stci, int8_t *cf, int *d_err, cudaStream_t s) {
    if (block < 32 || block % 1024 != 0) return AIR_ERR_INVALID_ARG;
    const int64_t nblk = (n + block - 1) / block;
    const int64_t ng1 = (block + 31) / 32, ng2 = (block + 1023) / 1024;
    const size_t per_warp = (size_t)(block + ng1 + ng2 + NEWF_CAP) * sizeof(int32_t);
    if (per_warp * FWARPS > AIR_SMEM_OPTIN) return AIR_ERR_UNSUPPORTED;     // block <= 8192 points
    AIR_CUDA(air_smem_optin(local_pass_kernel));
    local_pass_kernel<<<air_counted((unsigned)((nblk + FWARPS - 1) / FWARPS)), FWARPS * 32, per_warp * FWARPS, s>>>(
        n, block, srp, sci, strp, stci, cf, d_err);
    AIR_LAUNCH();
    int8_t *inU = nullptr, *sel = nullptr;
    unsigned long long *count = nullptr;
    AIR_CUDA(air_dmalloc((void **)&inU, (size_t)n));
    AIR_CUDA(air_dmalloc((void **)&sel, (size_t)n));
    AIR_CUDA(air_dmalloc((void **)&count, sizeof(unsigned long long)));
    int st = AIR_OK;
    unsigned long long left = 0;
    if (cudaMemsetAsync(count, 0, sizeof(unsigned long long), s) != cudaSuccess) st = AIR_ERR_CUDA;
    if (st == AIR_OK) {
        interface_init_kernel<<<air_counted(grid_for(n, 256)), 256, 0, s>>>(n, block, srp, sci, strp, stci, cf, inU,
                                                                            count);
        if (cudaMemcpyAsync(&left, count, sizeof(left), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            st = AIR_ERR_CUDA;
    }
    // every round makes the heaviest remaining point of each component of U a C point
    for (int64_t round = 0; st == AIR_OK && left > 0; ++round) {
        if (round > n) { st = AIR_ERR_DEVICE_TIMEOUT; break; }
        interface_select_kernel<<<air_counted(grid_for(n, 256)), 256, 0, s>>>(n, srp, sci, strp, stci, inU, sel);
        interface_apply_kernel<<<air_counted(grid_for(n, 256)), 256, 0, s>>>(n, sel, cf, inU);
        if (cudaMemsetAsync(count, 0, sizeof(unsigned long long), s) != cudaSuccess) { st = AIR_ERR_CUDA; break; }
        interface_leave_kernel<<<air_counted(grid_for(n, 256)), 256, 0, s>>>(n, srp, sci, cf, inU, count);
        if (cudaMemcpyAsync(&left, count, sizeof(left), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            st = AIR_ERR_CUDA;
    }
    air_dfree(inU);
    air_dfree(sel);
    air_dfree(count);
    return st;
}
