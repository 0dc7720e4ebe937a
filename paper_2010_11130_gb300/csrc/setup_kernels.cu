// Setup-phase kernels of the l-AIR hierarchy (arXiv:2010.11130, Section 3 and
// the Section 4 solver settings).  Every floating-point step here that decides
// an integer result or feeds a coarser level is written with explicit
// round-to-nearest intrinsics (__dmul_rn, __dadd_rn, __dsub_rn, __ddiv_rn) so
// that no multiply-add is contracted: strength tests, local LU solves and the
// Galerkin sums reproduce a plain sequential FP64 evaluation bit for bit.
#include <cooperative_groups.h>
#include <float.h>
#include <math.h>

#include <vector>

#include "air_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int64_t global_warp() {
    return ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
}

__device__ __forceinline__ int64_t warp_count() { return ((int64_t)gridDim.x * blockDim.x) >> 5; }

unsigned grid_for(int64_t work_items, int threads, int64_t cap = 152 * 32) {
    int64_t b = (work_items + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

// ------------------------------------------------------------- validation
__global__ void validate_kernel(int64_t n, int64_t nnz, const int64_t *rp, const int32_t *ci,
                                const double *v, int *err) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t b = rp[i], e = rp[i + 1];
        bool bad = (i == 0 && b != 0) || b < 0 || e < b || e > nnz;
        bool diag = false;
        if (!bad) {
            int32_t prev = -1;
            for (int64_t k = b; k < e; ++k) {
                int32_t c = ci[k];
                double a = v[k];
                if (c < 0 || c >= n || c <= prev || !isfinite(a)) { bad = true; break; }
                if (c == i) diag = (a != 0.0);
                prev = c;
            }
        }
        if (bad || !diag) atomicOr(err, AIR_DEVERR_CSR);
    }
}

// ---------------------------------------------------------------- strength
// j in S_i iff j != i and |a_ij| >= theta * max_{k != i} |a_ik|; empty if the max is 0.
template <bool FILL>
__global__ void strength_kernel(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, double theta,
                                int32_t *cnt, const int64_t *srp, int32_t *sci) {
    int lane = threadIdx.x & 31;
    for (int64_t i = global_warp(); i < n; i += warp_count()) {
        int64_t b = rp[i], e = rp[i + 1];
        double m = 0.0;
        for (int64_t k = b + lane; k < e; k += 32)
            if (ci[k] != i) m = fmax(m, fabs(v[k]));
        m = warp_max_d(m);
        if (m == 0.0) {
            if (!FILL && lane == 0) cnt[i] = 0;
            continue;
        }
        double thr = __dmul_rn(theta, m);
        int64_t pos = FILL ? srp[i] : 0;
        int c = 0;
        for (int64_t k0 = b; k0 < e; k0 += 32) {
            int64_t k = k0 + lane;
            bool s = k < e && ci[k] != i && fabs(v[k]) >= thr;
            unsigned bal = __ballot_sync(FULL, s);
            if (FILL && s) sci[pos + __popc(bal & lanemask_lt())] = ci[k];
            pos += __popc(bal);
            c += __popc(bal);
        }
        if (!FILL && lane == 0) cnt[i] = c;
    }
}

// -------------------------------------------------------------- transpose
__global__ void col_count_kernel(int64_t nnz, const int32_t *sci, int32_t *cnt) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[sci[k]], 1);
}

__global__ void transpose_scatter_kernel(int64_t n, const int64_t *srp, const int32_t *sci, const int64_t *strp,
                                         int32_t *fill, int32_t *stci) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int64_t k = srp[i]; k < srp[i + 1]; ++k) {
            int32_t j = sci[k];
            int32_t p = atomicAdd(&fill[j], 1);
            stci[strp[j] + p] = (int32_t)i;
        }
}

__global__ void sort_rows_kernel(int64_t n, const int64_t *rp, int32_t *ci) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t b = rp[i], e = rp[i + 1];
        for (int64_t k = b + 1; k < e; ++k) {          // insertion sort (rows are short)
            int32_t key = ci[k];
            int64_t t = k - 1;
            while (t >= b && ci[t] > key) { ci[t + 1] = ci[t]; --t; }
            ci[t + 1] = key;
        }
    }
}

// ------------------------------------------------- first-pass C/F splitting
// Sequential Ruge-Stueben first pass (largest measure first, ties to the
// smallest index), run exactly by ONE warp.  lam[k] holds the measure of an
// undecided point (>= 0) or its decision (-1 = F, -2 = C), so one load
// answers both questions.  Undecided points with measure >= 1 live in bucket
// lambda of a three-level bitmap (64-bit words; level 2 of every bucket sits
// in shared memory).  Bits are removed lazily: the search validates a
// candidate (lam equal to the bucket) and clears stale bits it meets.
// Only this warp touches lam and the bitmaps while it runs, so it uses plain
// loads and stores (L1-cached when CACHED) and no atomics on global memory:
// concurrent updates of one point or one bitmap word inside a 32-lane chunk
// are combined with __match_any_sync / __reduce_*_sync first.
constexpr int32_t LAM_F = -1, LAM_C = -2;
constexpr int8_t CF_F = 0, CF_C = 1;   // values of the cf marker

struct RSArgs {
    int64_t n;
    const int64_t *srp, *strp;
    const int32_t *sci, *stci;
    int32_t *lam;
    int8_t *cf;
    uint64_t *L0, *L1, *L2;
    int64_t w0, w1, w2;
    int nb;            // buckets 0 .. nb-1 (bucket 0 unused)
    int top;           // largest bucket that may be non-empty
    int max_st, touch_cap;
    int64_t cap;       // bound on search iterations
    int *err;
};

__global__ void rs_init_kernel(RSArgs a) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t lam = (int32_t)(a.strp[i + 1] - a.strp[i]);
        bool isolated = (a.srp[i + 1] == a.srp[i]) && lam == 0;
        a.lam[i] = isolated ? LAM_F : lam;
        if (!isolated && lam > 0) {
            uint64_t o0 = atomicOr((unsigned long long *)&a.L0[(int64_t)lam * a.w0 + (i >> 6)],
                                   (unsigned long long)(1ull << (i & 63)));
            if (o0 == 0) {
                int64_t i1 = i >> 6;
                uint64_t o1 = atomicOr((unsigned long long *)&a.L1[(int64_t)lam * a.w1 + (i1 >> 6)],
                                       (unsigned long long)(1ull << (i1 & 63)));
                if (o1 == 0) {
                    int64_t i2 = i1 >> 6;
                    atomicOr((unsigned long long *)&a.L2[(int64_t)lam * a.w2 + (i2 >> 6)],
                             (unsigned long long)(1ull << (i2 & 63)));
                }
            }
        }
    }
}

template <bool CACHED, typename T>
__device__ __forceinline__ T rs_ld(const T *p) {
    if (CACHED) return *p;
    return __ldcg(p);
}

// Lane 0 walks level 1 and level 0 of bucket b after the warp found a
// non-empty level-2 word.  Returns the point or -3 (retry after clearing a
// stale bit).
template <bool CACHED>
__device__ int64_t rs_probe(const RSArgs &a, uint64_t *L2s, int b, int64_t w) {
    uint64_t *p2 = &L2s[(int64_t)b * a.w2 + w];
    uint64_t l2 = *p2;
    int bit2 = __ffsll((long long)l2) - 1;
    int64_t i1 = w * 64 + bit2;
    uint64_t *p1 = &a.L1[(int64_t)b * a.w1 + i1];
    uint64_t l1 = rs_ld<CACHED>((const unsigned long long *)p1);
    if (l1 == 0ull) {
        *p2 = l2 & ~(1ull << bit2);
        return -3;
    }
    int bit1 = __ffsll((long long)l1) - 1;
    int64_t i0 = i1 * 64 + bit1;
    uint64_t *p0 = &a.L0[(int64_t)b * a.w0 + i0];
    uint64_t l0 = rs_ld<CACHED>((const unsigned long long *)p0);
    bool clear0 = false;
    if (l0 == 0ull) {
        clear0 = true;
    } else {
        int bit0 = __ffsll((long long)l0) - 1;
        int64_t k = i0 * 64 + bit0;
        if (rs_ld<CACHED>(&a.lam[k]) == b) return k;
        uint64_t n0 = l0 & ~(1ull << bit0);
        *p0 = n0;
        clear0 = (n0 == 0ull);
    }
    if (clear0) {
        uint64_t n1 = l1 & ~(1ull << bit1);
        *p1 = n1;
        if (n1 == 0ull) *p2 = l2 & ~(1ull << bit2);
    }
    return -3;
}

// The undecided point of largest measure (ties -> smallest index); -1 when
// the largest measure is 0, -2 when the iteration cap is hit.
template <bool CACHED>
__device__ int64_t rs_search(const RSArgs &a, uint64_t *L2s, int *top, int64_t *iters) {
    int lane = threadIdx.x & 31;
    int b = *top;
    while (true) {
        if (b < 1) { *top = 0; return -1; }
        if (++(*iters) > a.cap) return -2;
        int64_t w = -1;
        for (int64_t base = 0; base < a.w2; base += 32) {
            uint64_t val = (base + lane < a.w2) ? L2s[(int64_t)b * a.w2 + base + lane] : 0ull;
            unsigned bal = __ballot_sync(FULL, val != 0ull);
            if (bal) { w = base + __ffs(bal) - 1; break; }
        }
        if (w < 0) { --b; continue; }
        int64_t res = -3;
        if (lane == 0) res = rs_probe<CACHED>(a, L2s, b, w);
        res = __shfl_sync(FULL, res, 0);
        __syncwarp();
        if (res >= 0) { *top = b; return res; }
    }
}

// Add dlt to the measure of every still undecided point k given by the
// active lanes (duplicates within the chunk are combined), recording the
// points it changed in touched[].
template <bool CACHED>
__device__ __forceinline__ void rs_bump(const RSArgs &a, int32_t k, bool active, int dlt, int32_t *touched,
                                        int &nt) {
    int lane = threadIdx.x & 31;
    unsigned m = __match_any_sync(FULL, active ? k : -1);
    bool leader = active && (__ffs(m) - 1) == lane;
    bool changed = false;
    if (leader) {
        int32_t v = rs_ld<CACHED>(&a.lam[k]);
        if (v >= 0) {
            a.lam[k] = v + dlt * __popc(m);
            changed = true;
        }
    }
    unsigned bal = __ballot_sync(FULL, changed);
    if (changed) {
        int p = nt + __popc(bal & lanemask_lt());
        if (p < a.touch_cap) touched[p] = k;
    }
    nt += __popc(bal);
}

template <bool CACHED>
__global__ void __launch_bounds__(32) rs_warp_kernel(RSArgs a) {
    extern __shared__ uint64_t smem[];
    uint64_t *L2s = smem;                                            // nb * w2 words
    int32_t *newF = (int32_t *)(smem + (int64_t)a.nb * a.w2);        // max_st
    int32_t *touched = newF + a.max_st + 1;                          // touch_cap
    int lane = threadIdx.x & 31;
    for (int64_t t = lane; t < (int64_t)a.nb * a.w2; t += 32) L2s[t] = a.L2[t];
    int top = a.top;
    int64_t iters = 0;
    __syncwarp();
    for (int64_t pick_no = 0; pick_no <= a.n; ++pick_no) {
        int64_t i = rs_search<CACHED>(a, L2s, &top, &iters);
        if (i < 0) {
            if (i == -2 && lane == 0) atomicOr(a.err, AIR_DEVERR_RS_CAP);
            break;
        }
        if (lane == 0) a.lam[i] = LAM_C;
        __syncwarp();
        // undecided strong dependants of i become F
        int nf = 0;
        int64_t qb = a.strp[i], qe = a.strp[i + 1];
        for (int64_t q0 = qb; q0 < qe; q0 += 32) {
            int64_t q = q0 + lane;
            int32_t j = q < qe ? a.stci[q] : -1;
            bool u = j >= 0 && rs_ld<CACHED>(&a.lam[j]) >= 0;
            if (u) a.lam[j] = LAM_F;
            unsigned bal = __ballot_sync(FULL, u);
            if (u) newF[nf + __popc(bal & lanemask_lt())] = j;
            nf += __popc(bal);
        }
        __syncwarp();
        // measure updates: +1 on S_j of each new F point, -1 on S_i
        int nt = 0;
        for (int f = 0; f < nf; ++f) {
            int32_t j = newF[f];
            int64_t sb = a.srp[j], se = a.srp[j + 1];
            for (int64_t q0 = sb; q0 < se; q0 += 32) {
                int64_t q = q0 + lane;
                bool act = q < se;
                int32_t k = act ? a.sci[q] : -1;
                rs_bump<CACHED>(a, k, act, +1, touched, nt);
                __syncwarp();
            }
        }
        {
            int64_t sb = a.srp[i], se = a.srp[i + 1];
            for (int64_t q0 = sb; q0 < se; q0 += 32) {
                int64_t q = q0 + lane;
                bool act = q < se;
                int32_t k = act ? a.sci[q] : -1;
                rs_bump<CACHED>(a, k, act, -1, touched, nt);
                __syncwarp();
            }
        }
        if (nt > a.touch_cap) {       // cannot happen with the host-side bound; fail loudly
            if (lane == 0) atomicOr(a.err, AIR_DEVERR_RS_CAP);
            break;
        }
        // re-insert every touched point under its final measure
        for (int t0 = 0; t0 < nt; t0 += 32) {
            int t = t0 + lane;
            int32_t k = t < nt ? touched[t] : -1;
            int32_t v = k >= 0 ? rs_ld<CACHED>(&a.lam[k]) : -1;
            bool ins = v > 0;
            unsigned long long key0 = ins ? (unsigned long long)v * (unsigned long long)a.w0 + (unsigned long long)(k >> 6)
                                          : ~0ull;
            unsigned m0 = __match_any_sync(FULL, key0);
            unsigned long long bit0 = ins ? (1ull << (k & 63)) : 0ull;
            unsigned lo = __reduce_or_sync(m0, (unsigned)bit0);
            unsigned hi = __reduce_or_sync(m0, (unsigned)(bit0 >> 32));
            bool lead0 = ins && (__ffs(m0) - 1) == lane;
            bool need1 = false;
            if (lead0) {
                uint64_t old = rs_ld<CACHED>((const unsigned long long *)&a.L0[key0]);
                a.L0[key0] = old | ((uint64_t)hi << 32) | lo;
                need1 = (old == 0ull);
            }
            int64_t i1 = k >> 6;
            unsigned long long key1 = need1 ? (unsigned long long)v * (unsigned long long)a.w1 + (unsigned long long)(i1 >> 6)
                                            : ~0ull;
            unsigned m1 = __match_any_sync(FULL, key1);
            unsigned long long bit1 = need1 ? (1ull << (i1 & 63)) : 0ull;
            unsigned lo1 = __reduce_or_sync(m1, (unsigned)bit1);
            unsigned hi1 = __reduce_or_sync(m1, (unsigned)(bit1 >> 32));
            bool lead1 = need1 && (__ffs(m1) - 1) == lane;
            if (lead1) {
                uint64_t old = rs_ld<CACHED>((const unsigned long long *)&a.L1[key1]);
                a.L1[key1] = old | ((uint64_t)hi1 << 32) | lo1;
                if (old == 0ull) {
                    int64_t i2 = i1 >> 6;
                    atomicOr((unsigned long long *)&L2s[(int64_t)v * a.w2 + (i2 >> 6)],
                             (unsigned long long)(1ull << (i2 & 63)));
                }
            }
            int vmax = ins ? v : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) vmax = max(vmax, __shfl_xor_sync(FULL, vmax, o));
            if (vmax > top) top = vmax;
            __syncwarp();
        }
    }
}

__global__ void rs_finish_kernel(int64_t n, const int32_t *lam, int8_t *cf) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        cf[i] = lam[i] == LAM_C ? 1 : 0;
}

// ---------------------------------------- first pass, exact-bitmap version
// The same sequential first pass, with three changes that shorten the chain
// of dependent memory accesses per pick:
//  * the bucket bitmaps are kept exact (a point is removed from its old
//    bucket whenever its measure or state changes), so the search needs no
//    validation load and never meets stale bits;
//  * for every point i the lists S^T_i, S_j (j in S^T_i, in order) and S_i
//    are gathered once into one contiguous array of (point, tag) entries, so
//    a pick reads its whole two-hop neighbourhood in one coalesced access;
//  * measures and states are int8 (measure <= 2 max|S^T| <= 124, -1 = F,
//    -2 = C), which keeps the state of ~10^7 points resident in L2.
constexpr uint32_t TAG_J = 0xffffffffu, TAG_SI = 0xfffffffeu;
constexpr int8_t L8_F = -1, L8_C = -2;

struct RS3Args {
    int64_t n;
    const int64_t *srp, *strp, *hop_ptr;
    const int32_t *sci, *stci;
    const unsigned long long *hop;
    int8_t *lam;
    int8_t *cf;
    uint64_t *L0, *L1, *L2;
    int64_t w0, w1, w2;
    int nb, top, max_st;
    int64_t cap;
    int *err;
};

__global__ void hop_count_kernel(int64_t n, const int64_t *srp, const int64_t *strp, const int32_t *stci,
                                 int32_t *cnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = (strp[i + 1] - strp[i]) + (srp[i + 1] - srp[i]);
        for (int64_t q = strp[i]; q < strp[i + 1]; ++q) {
            int32_t j = stci[q];
            c += srp[j + 1] - srp[j];
        }
        cnt[i] = (int32_t)c;
    }
}

__global__ void hop_fill_kernel(int64_t n, const int64_t *srp, const int32_t *sci, const int64_t *strp,
                                const int32_t *stci, const int64_t *hop_ptr, unsigned long long *hop) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t p = hop_ptr[i];
        for (int64_t q = strp[i]; q < strp[i + 1]; ++q)
            hop[p++] = ((unsigned long long)TAG_J << 32) | (unsigned)stci[q];
        uint32_t t = 0;
        for (int64_t q = strp[i]; q < strp[i + 1]; ++q, ++t) {
            int32_t j = stci[q];
            for (int64_t r = srp[j]; r < srp[j + 1]; ++r) hop[p++] = ((unsigned long long)t << 32) | (unsigned)sci[r];
        }
        for (int64_t r = srp[i]; r < srp[i + 1]; ++r) hop[p++] = ((unsigned long long)TAG_SI << 32) | (unsigned)sci[r];
    }
}

__global__ void rs3_init_kernel(RS3Args a) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t lam = (int32_t)(a.strp[i + 1] - a.strp[i]);
        bool isolated = (a.srp[i + 1] == a.srp[i]) && lam == 0;
        a.lam[i] = isolated ? L8_F : (int8_t)lam;
        if (!isolated && lam > 0) {
            uint64_t o0 = atomicOr((unsigned long long *)&a.L0[(int64_t)lam * a.w0 + (i >> 6)],
                                   (unsigned long long)(1ull << (i & 63)));
            if (o0 == 0) {
                int64_t i1 = i >> 6;
                uint64_t o1 = atomicOr((unsigned long long *)&a.L1[(int64_t)lam * a.w1 + (i1 >> 6)],
                                       (unsigned long long)(1ull << (i1 & 63)));
                if (o1 == 0) {
                    int64_t i2 = i1 >> 6;
                    atomicOr((unsigned long long *)&a.L2[(int64_t)lam * a.w2 + (i2 >> 6)],
                             (unsigned long long)(1ull << (i2 & 63)));
                }
            }
        }
    }
}

__device__ __forceinline__ unsigned long long warp_or_u64(unsigned m, unsigned long long v) {
    unsigned lo = __reduce_or_sync(m, (unsigned)v);
    unsigned hi = __reduce_or_sync(m, (unsigned)(v >> 32));
    return ((unsigned long long)hi << 32) | lo;
}

// Set (set = true) or clear point k in bucket b for every valid lane; the
// whole warp calls it.  Lanes hitting the same 64-bit word are combined, and
// the level-1 / level-2 summaries follow every word that becomes empty or
// non-empty.
__device__ __forceinline__ void bm_update(const RS3Args &a, uint64_t *L2s, int b, int64_t k, bool valid, bool set) {
    if (!__any_sync(FULL, valid)) return;
    int lane = threadIdx.x & 31;
    unsigned long long key0 = valid ? (unsigned long long)b * (unsigned long long)a.w0 + (unsigned long long)(k >> 6)
                                    : ~0ull;
    unsigned m0 = __match_any_sync(FULL, key0);
    unsigned long long comb = warp_or_u64(m0, valid ? (1ull << (k & 63)) : 0ull);
    bool lead = valid && (__ffs(m0) - 1) == lane;
    bool t1 = false;
    if (lead) {
        uint64_t old = a.L0[key0];
        uint64_t nw = set ? (old | comb) : (old & ~comb);
        a.L0[key0] = nw;
        t1 = (old == 0ull) != (nw == 0ull);
    }
    if (__any_sync(FULL, t1)) {
        int64_t i1 = k >> 6;
        unsigned long long key1 = t1 ? (unsigned long long)b * (unsigned long long)a.w1 + (unsigned long long)(i1 >> 6)
                                     : ~0ull;
        unsigned m1 = __match_any_sync(FULL, key1);
        unsigned long long comb1 = warp_or_u64(m1, t1 ? (1ull << (i1 & 63)) : 0ull);
        bool lead1 = t1 && (__ffs(m1) - 1) == lane;
        if (lead1) {
            uint64_t old1 = a.L1[key1];
            uint64_t nw1 = set ? (old1 | comb1) : (old1 & ~comb1);
            a.L1[key1] = nw1;
            if ((old1 == 0ull) != (nw1 == 0ull)) {
                int64_t i2 = i1 >> 6;
                unsigned long long *p2 = (unsigned long long *)&L2s[(int64_t)b * a.w2 + (i2 >> 6)];
                unsigned long long bit2 = 1ull << (i2 & 63);
                if (set) atomicOr(p2, bit2); else atomicAnd(p2, ~bit2);
            }
        }
    }
    __syncwarp();
}

// Largest measure, smallest index: -1 when the largest measure is 0, -2 on
// the iteration cap or an inconsistent bitmap.
__device__ int64_t rs3_search(const RS3Args &a, uint64_t *L2s, int *top, int64_t *iters) {
    int lane = threadIdx.x & 31;
    int b = *top;
    while (true) {
        if (b < 1) { *top = 0; return -1; }
        if (++(*iters) > a.cap) return -2;
        int64_t w = -1;
        for (int64_t base = 0; base < a.w2; base += 32) {
            uint64_t val = (base + lane < a.w2) ? L2s[(int64_t)b * a.w2 + base + lane] : 0ull;
            unsigned bal = __ballot_sync(FULL, val != 0ull);
            if (bal) { w = base + __ffs(bal) - 1; break; }
        }
        if (w < 0) { --b; continue; }
        int64_t res = -2;
        if (lane == 0) {
            uint64_t l2 = L2s[(int64_t)b * a.w2 + w];
            int64_t i1 = w * 64 + (__ffsll((long long)l2) - 1);
            uint64_t l1 = a.L1[(int64_t)b * a.w1 + i1];
            if (l1 != 0ull) {
                int64_t i0 = i1 * 64 + (__ffsll((long long)l1) - 1);
                uint64_t l0 = a.L0[(int64_t)b * a.w0 + i0];
                if (l0 != 0ull) res = i0 * 64 + (__ffsll((long long)l0) - 1);
            }
        }
        res = __shfl_sync(FULL, res, 0);
        *top = b;
        return res;
    }
}

__global__ void __launch_bounds__(32) rs3_warp_kernel(RS3Args a) {
    extern __shared__ uint64_t smem[];
    uint64_t *L2s = smem;                                              // nb * w2 words
    int8_t *jflag = (int8_t *)(smem + (int64_t)a.nb * a.w2);          // max_st + 1
    int lane = threadIdx.x & 31;
    for (int64_t t = lane; t < (int64_t)a.nb * a.w2; t += 32) L2s[t] = a.L2[t];
    int top = a.top;
    int64_t iters = 0;
    __syncwarp();
    for (int64_t pick_no = 0; pick_no <= a.n; ++pick_no) {
        int64_t i = rs3_search(a, L2s, &top, &iters);
        if (i < 0) {
            if (i == -2 && lane == 0) atomicOr(a.err, AIR_DEVERR_RS_CAP);
            break;
        }
        int b = top;
        bm_update(a, L2s, b, i, lane == 0, false);
        if (lane == 0) a.lam[i] = L8_C;
        int64_t h0 = a.hop_ptr[i], h1 = a.hop_ptr[i + 1];
        int64_t c = a.strp[i + 1] - a.strp[i];
        __syncwarp();
        // undecided strong dependants of i become F
        for (int64_t e0 = h0; e0 < h0 + c; e0 += 32) {
            int64_t e = e0 + lane;
            bool act = e < h0 + c;
            int32_t j = act ? (int32_t)(unsigned)a.hop[e] : 0;
            int old = act ? (int)a.lam[j] : -3;
            bool u = old >= 0;
            if (u) a.lam[j] = L8_F;
            if (act) jflag[e - h0] = u ? 1 : 0;
            bm_update(a, L2s, old, j, u && old >= 1, false);
        }
        // +1 on S_j of each new F point j, -1 on S_i
        int vmax = 0;
        for (int64_t e0 = h0 + c; e0 < h1; e0 += 32) {
            int64_t e = e0 + lane;
            bool act = e < h1;
            unsigned long long ent = act ? a.hop[e] : 0ull;
            int32_t k = (int32_t)(unsigned)ent;
            uint32_t tag = (uint32_t)(ent >> 32);
            int dlt = 0;
            if (act) dlt = (tag == TAG_SI) ? -1 : (jflag[tag] ? 1 : 0);
            int cur = dlt != 0 ? (int)a.lam[k] : -3;
            bool live = dlt != 0 && cur >= 0;
            unsigned m = __match_any_sync(FULL, live ? k : -1);
            int sum = __reduce_add_sync(m, live ? dlt : 0);
            bool lead = live && (__ffs(m) - 1) == lane;
            int nv = cur + sum;
            bool mv = lead && nv != cur;
            if (lead) a.lam[k] = (int8_t)nv;
            bm_update(a, L2s, cur, k, mv && cur >= 1, false);
            bm_update(a, L2s, nv, k, mv && nv >= 1, true);
            if (mv && nv > vmax) vmax = nv;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) vmax = max(vmax, __shfl_xor_sync(FULL, vmax, o));
        if (vmax > top) top = vmax;
        __syncwarp();
    }
}

__global__ void rs3_finish_kernel(int64_t n, const int8_t *lam, int8_t *cf) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        cf[i] = lam[i] == L8_C ? 1 : 0;
}

// -------------------------------------------------------------- coarse ids
__global__ void cflag_kernel(int64_t n, const int8_t *cf, int32_t *flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = cf[i] == 1 ? 1 : 0;
}

__global__ void list_flag_kernel(int64_t n, const int8_t *cf, int which, int32_t *flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = cf[i] == which ? 1 : 0;
}

__global__ void list_fill_kernel(int64_t n, const int8_t *cf, int which, const int64_t *scan, int32_t *list) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (cf[i] == which) list[scan[i]] = (int32_t)i;
}

__global__ void cid_kernel(int64_t n, const int8_t *cf, const int64_t *scan, int32_t *cid, int32_t *crows) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (cf[i] == 1) {
            cid[i] = (int32_t)scan[i];
            crows[scan[i]] = (int32_t)i;
        } else {
            cid[i] = -1;
        }
    }
}

// ------------------------------------------------------------ l-AIR solves
// N_i = S_i intersect F (distance 1), ascending.  Count m_i + 1 entries of R row i.
__global__ void lair_count_kernel(int64_t nc, const int32_t *crows, const int64_t *srp, const int32_t *sci,
                                  const int8_t *cf, int32_t *cnt) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nc; t += (int64_t)gridDim.x * blockDim.x) {
        int32_t i = crows[t];
        int c = 0;
        for (int64_t q = srp[i]; q < srp[i + 1]; ++q) c += cf[sci[q]] == CF_F;
        cnt[t] = c + 1;
    }
}

// Distance-two neighbourhood N_i = (S_i intersect F) plus (S_k intersect F)
// for every k in S_i intersect F, ascending and without repeats, built by one
// warp in buf (LAIR_CAP ints): the candidates go into an open-addressing hash
// set in buf (repeats dropped), the distinct points are compacted to the
// front and sorted by a bitonic network.  Returns m, or -1 when more than
// LAIR_CAP / 2 distinct points are found.
constexpr int LAIR_CAP = 4096;

__device__ __forceinline__ bool hash_insert(int32_t *tab, int32_t key) {
    uint32_t h = ((uint32_t)key * 2654435761u) & (LAIR_CAP - 1);
    for (int probe = 0; probe < LAIR_CAP; ++probe) {
        const int32_t old = atomicCAS(&tab[h], -1, key);
        if (old == -1) return true;         // inserted
        if (old == key) return false;       // already present
        h = (h + 1) & (LAIR_CAP - 1);
    }
    return false;
}

__device__ int lair_neighbourhood2(int32_t i, const int64_t *srp, const int32_t *sci, const int8_t *cf,
                                   int32_t *buf) {
    const int lane = threadIdx.x & 31;
    for (int t = lane; t < LAIR_CAP; t += 32) buf[t] = -1;
    __syncwarp();
    int m = 0;
    bool full = false;
    // distance one, then the F points strongly connected to each of them
    for (int64_t q0 = srp[i]; q0 < srp[i + 1]; q0 += 32) {
        const int64_t q = q0 + lane;
        const int32_t j = q < srp[i + 1] ? sci[q] : -1;
        const bool ins = j >= 0 && cf[j] == CF_F && !full && hash_insert(buf, j);
        m += __popc(__ballot_sync(FULL, ins));
        full = full || m > LAIR_CAP / 2;
    }
    __syncwarp();
    for (int64_t qa = srp[i]; qa < srp[i + 1]; ++qa) {
        const int32_t k = sci[qa];
        if (cf[k] != CF_F) continue;
        for (int64_t q0 = srp[k]; q0 < srp[k + 1]; q0 += 32) {
            const int64_t q = q0 + lane;
            const int32_t j = q < srp[k + 1] ? sci[q] : -1;
            const bool ins = j >= 0 && cf[j] == CF_F && !full && hash_insert(buf, j);
            m += __popc(__ballot_sync(FULL, ins));
            full = full || m > LAIR_CAP / 2;
        }
    }
    __syncwarp();
    if (full) return -1;
    // compact the occupied slots to the front (writes never pass the chunk being read)
    int c = 0;
    for (int t0 = 0; t0 < LAIR_CAP; t0 += 32) {
        const int32_t v = buf[t0 + lane];
        __syncwarp();
        const bool keep = v >= 0;
        const unsigned bal = __ballot_sync(FULL, keep);
        if (keep) buf[c + __popc(bal & lanemask_lt())] = v;
        c += __popc(bal);
        __syncwarp();
    }
    int P = 32;
    while (P < c) P <<= 1;
    for (int t = c + lane; t < P; t += 32) buf[t] = INT32_MAX;
    __syncwarp();
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = lane; t < P; t += 32) {
                const int u = t ^ j;
                if (u > t) {
                    const int32_t x = buf[t], y = buf[u];
                    const bool up = (t & k) == 0;
                    if ((x > y) == up) { buf[t] = y; buf[u] = x; }
                }
            }
            __syncwarp();
        }
    return c;
}

// Distance two: one warp per C point counts m_i + 1 entries of R row i.
__global__ void lair_count2_kernel(int64_t nc, const int32_t *crows, const int64_t *srp, const int32_t *sci,
                                   const int8_t *cf, int32_t *cnt, int *err) {
    extern __shared__ int32_t cbuf[];
    int32_t *buf = cbuf + (threadIdx.x >> 5) * LAIR_CAP;
    const int lane = threadIdx.x & 31;
    for (int64_t t = global_warp(); t < nc; t += warp_count()) {
        const int m = lair_neighbourhood2(crows[t], srp, sci, cf, buf);
        if (lane == 0) {
            if (m < 0) atomicOr(err, AIR_DEVERR_CAP);
            cnt[t] = (m < 0 ? 0 : m) + 1;
        }
        __syncwarp();
    }
}

__device__ __forceinline__ int find_sorted(const int32_t *arr, int m, int32_t key) {
    int lo = 0, hi = m - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int32_t v = arr[mid];
        if (v == key) return mid;
        if (v < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

// One warp per C point: gather M = A_ff(N_i, N_i)^T and rhs = -A(i, N_i)^T,
// LU with partial pivoting (ties -> smallest row), forward substitution in
// ascending and back substitution in descending column order, all with
// explicitly rounded operations.  |pivot| <= 1e-14 max|M| -> z = 0.
// One level's arrays for the local solves (one job of a batched launch).
struct LairJob {
    int64_t first;                   // index of the job's first system in the launch
    int64_t nc;
    const int32_t *crows;
    const int64_t *rp;
    const int32_t *ci;
    const double *v;
    const int64_t *srp;
    const int32_t *sci;
    const int8_t *cf;
    const int64_t *rrp;
    int32_t *rci;
    double *rv;
    unsigned long long *nsing;
};

// The local system of C point crows[t] of job J, solved by one warp in the
// warp's shared-memory slot (M: maxm x ld, z: maxm, N: the neighbourhood).
__device__ void lair_solve_one(const LairJob &J, int64_t t, int maxm, int ld, int distance, double *M, double *z,
                               int32_t *N) {
    const int lane = threadIdx.x & 31;
    const int64_t *rp = J.rp, *srp = J.srp, *rrp = J.rrp;
    const int32_t *ci = J.ci, *sci = J.sci;
    const double *v = J.v;
    const int8_t *cf = J.cf;
    int32_t *rci = J.rci;
    double *rv = J.rv;
    unsigned long long *nsing = J.nsing;
    {
        int32_t i = J.crows[t];
        // neighbourhood
        int m = 0;
        if (distance >= 2) {
            m = lair_neighbourhood2(i, srp, sci, cf, N);
            if (m < 0 || m > maxm) m = 0;      // cannot happen: the count pass saw the same sets
        } else {
            for (int64_t q0 = srp[i]; q0 < srp[i + 1]; q0 += 32) {
                int64_t q = q0 + lane;
                int32_t j = q < srp[i + 1] ? sci[q] : -1;
                bool f = j >= 0 && cf[j] == CF_F;
                unsigned bal = __ballot_sync(FULL, f);
                if (f) N[m + __popc(bal & lanemask_lt())] = j;
                m += __popc(bal);
            }
        }
        for (int64_t s = lane; s < (int64_t)m * ld; s += 32) M[s] = 0.0;
        for (int s = lane; s < m; s += 32) z[s] = 0.0;
        __syncwarp();
        double mx = 0.0;
        for (int b = 0; b < m; ++b) {
            int32_t r = N[b];
            for (int64_t q = rp[r] + lane; q < rp[r + 1]; q += 32) {
                int a = find_sorted(N, m, ci[q]);
                if (a >= 0) { M[(int64_t)a * ld + b] = v[q]; mx = fmax(mx, fabs(v[q])); }
            }
        }
        for (int64_t q = rp[i] + lane; q < rp[i + 1]; q += 32) {
            int a = find_sorted(N, m, ci[q]);
            if (a >= 0) z[a] = -v[q];
        }
        mx = warp_max_d(mx);
        double tol = __dmul_rn(1e-14, mx);
        __syncwarp();
        bool singular = false;
        for (int k = 0; k < m; ++k) {
            double best = -1.0;
            int br = m;
            for (int r = k + lane; r < m; r += 32) {
                double av = fabs(M[(int64_t)r * ld + k]);
                if (av > best) { best = av; br = r; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                double ob = __shfl_xor_sync(FULL, best, o);
                int orr = __shfl_xor_sync(FULL, br, o);
                if (ob > best || (ob == best && orr < br)) { best = ob; br = orr; }
            }
            if (best <= tol) { singular = true; break; }
            if (br != k) {
                for (int c = lane; c < m; c += 32) {
                    double t1 = M[(int64_t)k * ld + c];
                    M[(int64_t)k * ld + c] = M[(int64_t)br * ld + c];
                    M[(int64_t)br * ld + c] = t1;
                }
                if (lane == 0) { double t1 = z[k]; z[k] = z[br]; z[br] = t1; }
            }
            __syncwarp();
            double d = M[(int64_t)k * ld + k];
            for (int r = k + 1 + lane; r < m; r += 32)
                M[(int64_t)r * ld + k] = __ddiv_rn(M[(int64_t)r * ld + k], d);
            __syncwarp();
            int w = m - k - 1;
            for (int s = lane; s < w * w; s += 32) {
                int r = k + 1 + s / w, c = k + 1 + s % w;
                M[(int64_t)r * ld + c] = __dsub_rn(M[(int64_t)r * ld + c],
                                                   __dmul_rn(M[(int64_t)r * ld + k], M[(int64_t)k * ld + c]));
            }
            __syncwarp();
        }
        if (singular) {
            for (int s = lane; s < m; s += 32) z[s] = 0.0;
            if (lane == 0) atomicAdd(nsing, 1ull);
        } else {
            for (int c = 0; c < m; ++c) {
                __syncwarp();
                double yc = z[c];
                for (int r = c + 1 + lane; r < m; r += 32)
                    z[r] = __dsub_rn(z[r], __dmul_rn(M[(int64_t)r * ld + c], yc));
            }
            for (int c = m - 1; c >= 0; --c) {
                __syncwarp();
                if (lane == 0) z[c] = __ddiv_rn(z[c], M[(int64_t)c * ld + c]);
                __syncwarp();
                double xc = z[c];
                for (int r = lane; r < c; r += 32)
                    z[r] = __dsub_rn(z[r], __dmul_rn(M[(int64_t)r * ld + c], xc));
            }
        }
        __syncwarp();
        // R row: N_i with z, plus i with 1, ascending
        int64_t pos = rrp[t];
        int before = 0;
        for (int a0 = 0; a0 < m; a0 += 32) {
            int a = a0 + lane;
            bool lt = a < m && N[a] < i;
            before += __popc(__ballot_sync(FULL, lt));
            if (a < m) {
                int64_t p = pos + a + (N[a] > i ? 1 : 0);
                rci[p] = N[a];
                rv[p] = z[a];
            }
        }
        if (lane == 0) { rci[pos + before] = i; rv[pos + before] = 1.0; }
        __syncwarp();
    }
}

// Shared-memory slot of this warp: M, z, N (doubles per warp as in air_lair_solve).
__device__ __forceinline__ double *lair_slot(int maxm, int ld, int distance) {
    extern __shared__ double lsm[];
    const int nints = distance >= 2 ? LAIR_CAP : maxm;
    const int64_t per_warp = (int64_t)maxm * ld + maxm + (nints + 1) / 2 + 1;
    return lsm + (threadIdx.x >> 5) * per_warp;
}

__global__ void lair_solve_kernel(LairJob J, int maxm, int ld, int distance) {
    double *M = lair_slot(maxm, ld, distance);
    double *z = M + (int64_t)maxm * ld;
    int32_t *N = (int32_t *)(z + maxm);
    for (int64_t t = global_warp(); t < J.nc; t += warp_count()) lair_solve_one(J, t, maxm, ld, distance, M, z, N);
}

// The systems of several jobs as one index range: system t belongs to the last
// job whose first index is <= t.
__global__ void lair_solve_batch_kernel(int njobs, const LairJob *jobs, int64_t total, int maxm, int ld,
                                        int distance) {
    double *M = lair_slot(maxm, ld, distance);
    double *z = M + (int64_t)maxm * ld;
    int32_t *N = (int32_t *)(z + maxm);
    for (int64_t t = global_warp(); t < total; t += warp_count()) {
        int lo = 0, hi = njobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (jobs[mid].first <= t) lo = mid; else hi = mid - 1;
        }
        lair_solve_one(jobs[lo], t - jobs[lo].first, maxm, ld, distance, M, z, N);
    }
}

// --------------------------------------------------------- one-point P
// F point i: strong C neighbour of largest |a_ij| (ties -> smallest j), weight 1;
// none -> -1.  C point: its own coarse id.
__global__ void onepoint_kernel(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, double theta,
                                const int8_t *cf, const int32_t *cid, int32_t *pcol) {
    int lane = threadIdx.x & 31;
    for (int64_t i = global_warp(); i < n; i += warp_count()) {
        if (cf[i] == CF_C) {
            if (lane == 0) pcol[i] = cid[i];
            continue;
        }
        int64_t b = rp[i], e = rp[i + 1];
        double m = 0.0;
        for (int64_t k = b + lane; k < e; k += 32)
            if (ci[k] != i) m = fmax(m, fabs(v[k]));
        m = warp_max_d(m);
        int32_t best = INT32_MAX;
        double bv = -1.0;
        if (m > 0.0) {
            double thr = __dmul_rn(theta, m);
            for (int64_t k = b + lane; k < e; k += 32) {
                int32_t c = ci[k];
                double a = fabs(v[k]);
                if (c != i && a >= thr && cf[c] == CF_C && a > bv) { bv = a; best = c; }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double ob = __shfl_xor_sync(FULL, bv, o);
            int32_t oc = __shfl_xor_sync(FULL, best, o);
            if (ob > bv || (ob == bv && oc < best)) { bv = ob; best = oc; }
        }
        if (lane == 0) pcol[i] = (best != INT32_MAX) ? cid[best] : -1;
    }
}

// ---------------------------------------------------------------- RAP
__global__ void rap_terms_kernel(int64_t nc, const int64_t *rrp, const int32_t *rci, const int64_t *rp,
                                 int32_t *terms) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nc; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t s = 0;
        for (int64_t q = rrp[t]; q < rrp[t + 1]; ++q) s += rp[rci[q] + 1] - rp[rci[q]];
        terms[t] = (int32_t)(s < INT32_MAX ? s : INT32_MAX);
    }
}

// One warp per coarse row i.  Stage 1: (RA)_ij over R entries k ascending and
// A row k, accumulated into a per-warp hash table (within one k the columns j
// are distinct, so no two lanes touch one slot).  Stage 2: keys (P(j), j)
// sorted by a bitonic network, then every coarse column sums its terms in
// ascending j.  COUNT mode only counts the coarse columns.  The table lives in
// shared memory, or (GMEM, for rows with more terms than fit there) in a
// global scratch area of HS x 20 bytes per warp of the grid.  rows (if not
// NULL) lists the nrows coarse rows to process.
template <bool FILL, bool GMEM>
__global__ void rap_kernel(int64_t nrows, const int32_t *rows, const int64_t *rrp, const int32_t *rci,
                           const double *rv, const int64_t *rp, const int32_t *ci, const double *v,
                           const int32_t *pcol, int hs_bits, unsigned char *gscratch, int32_t *cnt,
                           const int64_t *acrp, int32_t *acci, double *acv, int *err) {
    extern __shared__ unsigned char rsm[];
    const int HS = 1 << hs_bits, HH = HS >> 1;
    int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned char *base = GMEM ? gscratch + (size_t)global_warp() * (size_t)HS * 20
                               : rsm + (size_t)wib * (size_t)HS * 20;
    double *vals = (double *)base;                          // HS
    unsigned long long *skey = (unsigned long long *)(vals + HS);   // HH
    double *sval = (double *)(skey + HH);                   // HH
    int32_t *keys = (int32_t *)(sval + HH);                 // HS
    for (int64_t u = global_warp(); u < nrows; u += warp_count()) {
        const int64_t t = rows ? (int64_t)rows[u] : u;
        for (int s = lane; s < HS; s += 32) keys[s] = -1;
        __syncwarp();
        for (int64_t q = rrp[t]; q < rrp[t + 1]; ++q) {
            int32_t k = rci[q];
            double rik = FILL ? rv[q] : 0.0;
            for (int64_t e = rp[k] + lane; e < rp[k + 1]; e += 32) {
                int32_t j = ci[e];
                unsigned h = ((unsigned)j * 2654435761u) >> (32 - hs_bits);
                bool placed = false;
                for (int probe = 0; probe < HS; ++probe) {      // the table holds twice the row's terms
                    int32_t old = atomicCAS(&keys[h], -1, j);
                    if (old == -1) { if (FILL) vals[h] = 0.0; placed = true; break; }
                    if (old == j) { placed = true; break; }
                    h = (h + 1) & (HS - 1);
                }
                if (!placed) { atomicOr(err, AIR_DEVERR_CAP); continue; }
                if (FILL) vals[h] = __dadd_rn(vals[h], __dmul_rn(rik, v[e]));
            }
            __syncwarp();
        }
        if (!FILL) {
            // COUNT: the number of distinct coarse columns P(j), from a second hash table
            int32_t *jt = (int32_t *)skey;                  // HS slots (the sort area, unused here)
            for (int s = lane; s < HS; s += 32) jt[s] = -1;
            __syncwarp();
            int heads = 0;
            for (int s0 = 0; s0 < HS; s0 += 32) {
                const int32_t j = keys[s0 + lane];
                const int32_t J = j >= 0 ? pcol[j] : -1;
                bool fresh = false;
                if (J >= 0) {
                    unsigned h = ((unsigned)J * 2654435761u) >> (32 - hs_bits);
                    bool placed = false;
                    for (int probe = 0; probe < HS; ++probe) {
                        const int32_t old = atomicCAS(&jt[h], -1, J);
                        if (old == -1) { fresh = true; placed = true; break; }
                        if (old == J) { placed = true; break; }
                        h = (h + 1) & (HS - 1);
                    }
                    if (!placed) atomicOr(err, AIR_DEVERR_CAP);
                }
                heads += __popc(__ballot_sync(FULL, fresh));
            }
            if (lane == 0) cnt[t] = heads;
            __syncwarp();
            continue;
        }
        int cntv = 0;
        for (int s0 = 0; s0 < HS; s0 += 32) {
            int s = s0 + lane;
            int32_t j = keys[s];
            int32_t J = j >= 0 ? pcol[j] : -1;
            bool ok = J >= 0;
            unsigned bal = __ballot_sync(FULL, ok);
            if (ok) {
                int p = cntv + __popc(bal & lanemask_lt());
                skey[p] = ((unsigned long long)(unsigned)J << 32) | (unsigned)j;
                if (FILL) sval[p] = vals[s];
            }
            cntv += __popc(bal);
        }
        int P = 1;
        while (P < cntv) P <<= 1;
        for (int s = cntv + lane; s < P; s += 32) skey[s] = ~0ull;
        __syncwarp();
        for (int size = 2; size <= P; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int idx = lane; idx < (P >> 1); idx += 32) {
                    int a = 2 * stride * (idx / stride) + (idx % stride);
                    int b = a + stride;
                    bool up = (a & size) == 0;
                    unsigned long long ka = skey[a], kb = skey[b];
                    if ((ka > kb) == up) {
                        skey[a] = kb; skey[b] = ka;
                        if (FILL) { double t1 = sval[a]; sval[a] = sval[b]; sval[b] = t1; }
                    }
                }
                __syncwarp();
            }
        }
        int heads = 0;
        int64_t out = FILL ? acrp[t] : 0;
        for (int s0 = 0; s0 < cntv; s0 += 32) {
            int s = s0 + lane;
            bool head = s < cntv && (s == 0 || (skey[s] >> 32) != (skey[s - 1] >> 32));
            unsigned bal = __ballot_sync(FULL, head);
            if (FILL && head) {
                unsigned long long J = skey[s] >> 32;
                double acc = 0.0;
                for (int u = s; u < cntv && (skey[u] >> 32) == J; ++u) acc = __dadd_rn(acc, sval[u]);
                int64_t p = out + heads + __popc(bal & lanemask_lt());
                acci[p] = (int32_t)J;
                acv[p] = acc;
            }
            heads += __popc(bal);
        }
        if (!FILL && lane == 0) cnt[t] = heads;
        __syncwarp();
    }
}

// ------------------------------------------------------- coarsest inverse
// Gauss-Jordan with partial pivoting (ties -> smallest row) on [A | I],
// one pivot step per pair of launches.
__global__ void dense_scatter_kernel(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                                     double *M) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) M[i * 2 * n + ci[k]] = v[k];
        M[i * 2 * n + n + i] = 1.0;
    }
}

__global__ void dense_absmax_kernel(int64_t n, const double *M, double *out) {
    __shared__ double red[32];
    double m = 0.0;
    for (int64_t s = threadIdx.x; s < n * n; s += blockDim.x) m = fmax(m, fabs(M[(s / n) * 2 * n + s % n]));
    m = warp_max_d(m);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        t = warp_max_d(t);
        if (threadIdx.x == 0) *out = t;
    }
}

// All pivot steps in one cooperative launch: block 0 picks the pivot row
// (largest |entry| of the column, ties -> smallest row), swaps it up, scales
// it and saves the column factors; then every block eliminates the column
// from the other rows.  Grid-wide barriers separate the phases; a singular
// pivot sets the error flag, which every block reads after the barrier, so
// all blocks leave together.
__global__ void __launch_bounds__(512) gj_coop_kernel(int64_t n, double *M, double *fcol, const double *amax,
                                                      int *err) {
    cg::grid_group grid = cg::this_grid();
    __shared__ double sb[16];
    __shared__ int64_t sr[16];
    __shared__ int64_t piv;
    const int tid = threadIdx.x;
    const double tol = 1e-14 * amax[0];
    for (int64_t k = 0; k < n; ++k) {
        if (blockIdx.x == 0) {
            double best = -1.0;
            int64_t br = n;
            for (int64_t r = k + tid; r < n; r += blockDim.x) {
                double av = fabs(M[r * 2 * n + k]);
                if (av > best) { best = av; br = r; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                double ob = __shfl_xor_sync(FULL, best, o);
                int64_t orr = __shfl_xor_sync(FULL, br, o);
                if (ob > best || (ob == best && orr < br)) { best = ob; br = orr; }
            }
            if ((tid & 31) == 0) { sb[tid >> 5] = best; sr[tid >> 5] = br; }
            __syncthreads();
            if (tid == 0) {
                for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
                    if (sb[w] > sb[0] || (sb[w] == sb[0] && sr[w] < sr[0])) { sb[0] = sb[w]; sr[0] = sr[w]; }
                piv = sr[0];
                if (!(sb[0] > tol)) { atomicOr(err, AIR_DEVERR_SINGULAR); piv = -1; }
            }
            __syncthreads();
            const int64_t p = piv;
            if (p >= 0) {
                if (p != k)
                    for (int64_t c = k + tid; c < 2 * n; c += blockDim.x) {
                        double t1 = M[k * 2 * n + c];
                        M[k * 2 * n + c] = M[p * 2 * n + c];
                        M[p * 2 * n + c] = t1;
                    }
                __syncthreads();
                const double d = M[k * 2 * n + k];
                __syncthreads();
                for (int64_t c = k + tid; c < 2 * n; c += blockDim.x) M[k * 2 * n + c] = M[k * 2 * n + c] / d;
                for (int64_t r = tid; r < n; r += blockDim.x) fcol[r] = (r == k) ? 0.0 : M[r * 2 * n + k];
            }
        }
        grid.sync();
        if (__ldcg(err) & AIR_DEVERR_SINGULAR) return;
        const int64_t w = 2 * n - k;
        for (int64_t q = (int64_t)blockIdx.x * blockDim.x + tid; q < n * w; q += (int64_t)gridDim.x * blockDim.x) {
            const int64_t r = q / w, c = k + q % w;
            const double f = fcol[r];
            if (r != k && f != 0.0) M[r * 2 * n + c] -= f * M[k * 2 * n + c];
        }
        grid.sync();
    }
}

__global__ void dense_extract_kernel(int64_t n, const double *M, double *inv) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n * n; s += (int64_t)gridDim.x * blockDim.x)
        inv[s] = M[(s / n) * 2 * n + n + s % n];
}

}  // namespace

// ================================================================ launchers
int air_validate_csr(int64_t n, int64_t nnz, const int64_t *rp, const int32_t *ci, const double *v, int *d_err,
                     cudaStream_t s) {
    validate_kernel<<<air_counted(grid_for(n, 256)), 256, 0, s>>>(n, nnz, rp, ci, v, d_err);
    AIR_LAUNCH();
    return AIR_OK;
}

int air_strength(const AirLevel &L, double theta, int64_t *srp, int32_t *sci, int32_t *cnt, int fill,
                 cudaStream_t s) {
    unsigned g = grid_for(L.n * 32, 256);
    if (fill)
        strength_kernel<true><<<air_counted(g), 256, 0, s>>>(L.n, L.rp, L.ci, L.v, theta, nullptr, srp, sci);
    else
        strength_kernel<false><<<air_counted(g), 256, 0, s>>>(L.n, L.rp, L.ci, L.v, theta, cnt, nullptr, nullptr);
    AIR_LAUNCH();
    return AIR_OK;
}

// work: int32 [n] scratch.  strp gets the transposed row pointer.
int air_transpose_pattern(int64_t n, int64_t nnz, const int64_t *srp, const int32_t *sci, int64_t *strp,
                          int32_t *stci, int32_t *work, cudaStream_t s) {
    AIR_CUDA(cudaMemsetAsync(work, 0, (size_t)n * sizeof(int32_t), s));
    if (nnz > 0) col_count_kernel<<<air_counted(grid_for(nnz, 256)), 256, 0, s>>>(nnz, sci, work);
    AIR_LAUNCH();
    AIR_TRY(air_exclusive_scan_i32(work, strp, n, s));
    AIR_CUDA(cudaMemsetAsync(work, 0, (size_t)n * sizeof(int32_t), s));
    transpose_scatter_kernel<<<air_counted(grid_for(n, 256)), 256, 0, s>>>(n, srp, sci, strp, work, stci);
    sort_rows_kernel<<<air_counted(grid_for(n, 256)), 256, 0, s>>>(n, strp, stci);
    AIR_LAUNCH();
    return AIR_OK;
}

static int rs_first_pass_v3(int64_t n, const int64_t *srp, const int32_t *sci, const int64_t *strp,
                            const int32_t *stci, int32_t max_st, int8_t *cf, int *d_err, cudaStream_t s) {
    RS3Args a;
    a.n = n; a.srp = srp; a.sci = sci; a.strp = strp; a.stci = stci;
    a.cf = cf;
    a.nb = 2 * max_st + 1;
    if (a.nb < 2) a.nb = 2;
    a.top = a.nb - 1;
    a.max_st = max_st;
    a.w0 = (n + 63) / 64;
    a.w1 = (a.w0 + 63) / 64;
    a.w2 = (a.w1 + 63) / 64;
    a.err = d_err;
    // each pick raises the top bucket by < nb, so the search loop runs at most
    // (n + 1) (nb + 1) times
    a.cap = (n + 1) * (int64_t)(a.nb + 1) + 4096;
    // two-hop lists
    int32_t *cnt = nullptr;
    int64_t *hop_ptr = nullptr;
    AIR_CUDA(cudaMallocAsync(&cnt, (size_t)(n > 0 ? n : 1) * sizeof(int32_t), s));
    AIR_CUDA(cudaMallocAsync(&hop_ptr, (size_t)(n + 1) * sizeof(int64_t), s));
    hop_count_kernel<<<air_counted(grid_for(n, 256)), 256, 0, s>>>(n, srp, strp, stci, cnt);
    AIR_LAUNCH();
    AIR_TRY(air_exclusive_scan_i32(cnt, hop_ptr, n, s));
    int64_t nhop = 0;
    AIR_CUDA(cudaMemcpyAsync(&nhop, hop_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    AIR_CUDA(cudaStreamSynchronize(s));
    unsigned long long *hop = nullptr;
    AIR_CUDA(cudaMallocAsync(&hop, (size_t)(nhop > 0 ? nhop : 1) * sizeof(unsigned long long), s));
    hop_fill_kernel<<<air_counted(grid_for(n, 256)), 256, 0, s>>>(n, srp, sci, strp, stci, hop_ptr, hop);
    AIR_LAUNCH();
    a.hop_ptr = hop_ptr;
    a.hop = hop;
    size_t words = (size_t)a.nb * (size_t)(a.w0 + a.w1 + a.w2);
    uint64_t *bits = nullptr;
    int8_t *lam = nullptr;
    AIR_CUDA(cudaMallocAsync(&bits, words * sizeof(uint64_t), s));
    AIR_CUDA(cudaMallocAsync(&lam, (size_t)(n > 0 ? n : 1), s));
    AIR_CUDA(cudaMemsetAsync(bits, 0, words * sizeof(uint64_t), s));
    a.L0 = bits;
    a.L1 = bits + (size_t)a.nb * a.w0;
    a.L2 = a.L1 + (size_t)a.nb * a.w1;
    a.lam = lam;
    rs3_init_kernel<<<air_counted(grid_for(n, 256)), 256, 0, s>>>(a);
    AIR_LAUNCH();
    size_t smem = (size_t)a.nb * a.w2 * sizeof(uint64_t) + (size_t)(max_st + 8);
    if (smem > AIR_SMEM_OPTIN) return AIR_ERR_UNSUPPORTED;
    AIR_CUDA(air_smem_optin(rs3_warp_kernel));
    rs3_warp_kernel<<<air_counted(1), 32, smem, s>>>(a);
    AIR_LAUNCH();
    rs3_finish_kernel<<<air_counted(grid_for(n, 256)), 256, 0, s>>>(n, lam, cf);
    AIR_LAUNCH();
    cudaFreeAsync(bits, s);
    cudaFreeAsync(lam, s);
    cudaFreeAsync(hop, s);
    cudaFreeAsync(hop_ptr, s);
    cudaFreeAsync(cnt, s);
    return AIR_OK;
}

int air_rs_first_pass(int64_t n, const int64_t *srp, const int32_t *sci, const int64_t *strp, const int32_t *stci,
                      int32_t max_st, int32_t max_s, int8_t *cf, int *d_err, int cached,
                      unsigned long long *stats, cudaStream_t s) {
    if (cached == 4) {
        const int r = air_rs_first_pass_cursor(n, srp, sci, strp, stci, max_st, cf, d_err, stats, s);
        if (r != AIR_ERR_UNSUPPORTED) return r;
        cached = 2;
    }
    if (cached >= 2 && 2 * max_st + 1 <= 125)
        return rs_first_pass_v3(n, srp, sci, strp, stci, max_st, cf, d_err, s);
    RSArgs a;
    a.n = n; a.srp = srp; a.sci = sci; a.strp = strp; a.stci = stci;
    a.cf = cf;
    a.nb = 2 * max_st + 1;
    if (a.nb < 2) a.nb = 2;
    a.top = a.nb - 1;
    a.w0 = (n + 63) / 64;
    a.w1 = (a.w0 + 63) / 64;
    a.w2 = (a.w1 + 63) / 64;
    a.err = d_err;
    a.max_st = max_st;
    // touched points per pick: S_j of every new F point j plus S_i
    a.touch_cap = (max_st + 1) * (max_s > 0 ? max_s : 1) + 64;
    int64_t nnz_s = 0;
    AIR_CUDA(cudaMemcpyAsync(&nnz_s, srp + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    AIR_CUDA(cudaStreamSynchronize(s));
    a.cap = 16 * (n + nnz_s) + 4096;
    size_t words = (size_t)a.nb * (size_t)(a.w0 + a.w1 + a.w2);
    uint64_t *bits = nullptr;
    int32_t *lam = nullptr;
    AIR_CUDA(cudaMallocAsync(&bits, words * sizeof(uint64_t), s));
    AIR_CUDA(cudaMallocAsync(&lam, (size_t)n * sizeof(int32_t), s));
    AIR_CUDA(cudaMemsetAsync(bits, 0, words * sizeof(uint64_t), s));
    a.L0 = bits;
    a.L1 = bits + (size_t)a.nb * a.w0;
    a.L2 = a.L1 + (size_t)a.nb * a.w1;
    a.lam = lam;
    rs_init_kernel<<<air_counted(grid_for(n, 256)), 256, 0, s>>>(a);
    AIR_LAUNCH();
    size_t smem = (size_t)a.nb * a.w2 * sizeof(uint64_t) + (size_t)(max_st + 1 + a.touch_cap) * sizeof(int32_t);
    if (smem > AIR_SMEM_OPTIN) return AIR_ERR_UNSUPPORTED;
    if (cached) {
        AIR_CUDA(air_smem_optin(rs_warp_kernel<true>));
        rs_warp_kernel<true><<<air_counted(1), 32, smem, s>>>(a);
    } else {
        AIR_CUDA(air_smem_optin(rs_warp_kernel<false>));
        rs_warp_kernel<false><<<air_counted(1), 32, smem, s>>>(a);
    }
    AIR_LAUNCH();
    rs_finish_kernel<<<air_counted(grid_for(n, 256)), 256, 0, s>>>(n, lam, cf);
    AIR_LAUNCH();
    cudaFreeAsync(bits, s);
    cudaFreeAsync(lam, s);
    return AIR_OK;
}

// work: int64 [n+1]
int air_coarse_ids(int64_t n, const int8_t *cf, int32_t *cid, int32_t *crows, int64_t *work, int64_t *nc,
                   cudaStream_t s) {
    int32_t *flag = nullptr;
    AIR_CUDA(cudaMallocAsync(&flag, (size_t)(n > 0 ? n : 1) * sizeof(int32_t), s));
    cflag_kernel<<<air_counted(grid_for(n, 256)), 256, 0, s>>>(n, cf, flag);
    AIR_LAUNCH();
    AIR_TRY(air_exclusive_scan_i32(flag, work, n, s));
    AIR_CUDA(cudaMemcpyAsync(nc, work + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (crows) {
        cid_kernel<<<air_counted(grid_for(n, 256)), 256, 0, s>>>(n, cf, work, cid, crows);
        AIR_LAUNCH();
    }
    cudaFreeAsync(flag, s);
    AIR_CUDA(cudaStreamSynchronize(s));
    return AIR_OK;
}

// Ascending list of the points with cf == which.  work: int64 [n+1].
int air_point_list(int64_t n, const int8_t *cf, int which, int32_t *list, int64_t *work, cudaStream_t s) {
    int32_t *flag = nullptr;
    AIR_CUDA(cudaMallocAsync(&flag, (size_t)(n > 0 ? n : 1) * sizeof(int32_t), s));
    list_flag_kernel<<<air_counted(grid_for(n, 256)), 256, 0, s>>>(n, cf, which, flag);
    AIR_LAUNCH();
    AIR_TRY(air_exclusive_scan_i32(flag, work, n, s));
    list_fill_kernel<<<air_counted(grid_for(n, 256)), 256, 0, s>>>(n, cf, which, work, list);
    AIR_LAUNCH();
    cudaFreeAsync(flag, s);
    return AIR_OK;
}

int air_lair_counts(int64_t nc, const int32_t *crows, const int64_t *srp, const int32_t *sci, const int8_t *cf,
                    int32_t *cnt, int distance, int *d_err, cudaStream_t s) {
    if (distance >= 2) {
        const size_t smem = (size_t)8 * LAIR_CAP * sizeof(int32_t);
        AIR_CUDA(air_smem_optin(lair_count2_kernel));
        lair_count2_kernel<<<air_counted(grid_for(nc * 32, 256)), 256, smem, s>>>(nc, crows, srp, sci, cf, cnt, d_err);
    } else {
        lair_count_kernel<<<air_counted(grid_for(nc, 256)), 256, 0, s>>>(nc, crows, srp, sci, cf, cnt);
    }
    AIR_LAUNCH();
    return AIR_OK;
}

namespace {

LairJob lair_job(const AirLevel &L, int64_t *d_nsing, int64_t first) {
    return LairJob{first, L.nc, L.crows, L.rp, L.ci, L.v, L.srp, L.sci, L.cf, L.rrp, L.rci, L.rv,
                   (unsigned long long *)d_nsing};
}

// Warps per block and shared memory of a local-solve launch for neighbourhoods up to max_m.
int lair_shape(int32_t max_m, int distance, int *maxm, int *ld, int *warps, size_t *smem) {
    *maxm = max_m < 1 ? 1 : max_m;
    *ld = *maxm | 1;
    const int nints = distance >= 2 ? LAIR_CAP : *maxm;
    const size_t per_warp = ((size_t)*maxm * *ld + *maxm + (nints + 1) / 2 + 1) * sizeof(double);
    *warps = (int)(((distance >= 2 ? AIR_SMEM_OPTIN : 96 * 1024)) / per_warp);
    if (*warps > 8) *warps = 8;
    if (*warps < 1) {
        if (per_warp > AIR_SMEM_OPTIN) return AIR_ERR_UNSUPPORTED;
        *warps = 1;
    }
    *smem = per_warp * *warps;
    return AIR_OK;
}

unsigned lair_blocks(int64_t systems, int warps) {
    int64_t blocks = (systems + warps - 1) / warps;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    return (unsigned)blocks;
}

}  // namespace

int air_lair_solve(const AirLevel &L, int32_t max_m, int distance, int64_t *d_nsing, cudaStream_t s) {
    int maxm = 0, ld = 0, warps = 0;
    size_t smem = 0;
    AIR_TRY(lair_shape(max_m, distance, &maxm, &ld, &warps, &smem));
    AIR_CUDA(air_smem_optin(lair_solve_kernel));
    lair_solve_kernel<<<air_counted(lair_blocks(L.nc, warps)), warps * 32, smem, s>>>(lair_job(L, d_nsing, 0), maxm,
                                                                                         ld, distance);
    AIR_LAUNCH();
    return AIR_OK;
}

int air_lair_solve_batch(int count, const AirLevel *const *levels, const int32_t *max_m, int distance,
                         int64_t *const *d_nsing, cudaStream_t s) {
    if (count <= 0) return AIR_OK;
    std::vector<LairJob> jobs((size_t)count);
    int32_t mm = 0;
    int64_t total = 0;
    for (int k = 0; k < count; ++k) {
        jobs[(size_t)k] = lair_job(*levels[k], d_nsing[k], total);
        total += levels[k]->nc;
        mm = max_m[k] > mm ? max_m[k] : mm;
    }
    int maxm = 0, ld = 0, warps = 0;
    size_t smem = 0;
    AIR_TRY(lair_shape(mm, distance, &maxm, &ld, &warps, &smem));
    LairJob *d_jobs = nullptr;
    AIR_CUDA(cudaMallocAsync(&d_jobs, (size_t)count * sizeof(LairJob), s));
    AIR_CUDA(cudaMemcpyAsync(d_jobs, jobs.data(), (size_t)count * sizeof(LairJob), cudaMemcpyHostToDevice, s));
    AIR_CUDA(air_smem_optin(lair_solve_batch_kernel));
    lair_solve_batch_kernel<<<air_counted(lair_blocks(total, warps)), warps * 32, smem, s>>>(count, d_jobs, total,
                                                                                                maxm, ld, distance);
    AIR_LAUNCH();
    AIR_CUDA(cudaStreamSynchronize(s));     // the job table is read from pageable host memory
    cudaFreeAsync(d_jobs, s);
    return AIR_OK;
}

int air_onepoint_P(const AirLevel &L, double theta, cudaStream_t s) {
    onepoint_kernel<<<air_counted(grid_for(L.n * 32, 256)), 256, 0, s>>>(L.n, L.rp, L.ci, L.v, theta, L.cf, L.cid, L.pcol);
    AIR_LAUNCH();
    return AIR_OK;
}

int air_rap_terms(const AirLevel &L, int32_t *terms, cudaStream_t s) {
    rap_terms_kernel<<<air_counted(grid_for(L.nc, 256)), 256, 0, s>>>(L.nc, L.rrp, L.rci, L.rp, terms);
    AIR_LAUNCH();
    return AIR_OK;
}

// Rows whose term count exceeds lim go to the long list, the others to the short one.
// Row classes by table size: class c holds the rows whose table of
// 2^(min_bits + c) slots is the smallest holding twice their terms (the last
// class also any longer row).  lists: ncls x nc.
__global__ void rap_class_kernel(int64_t nc, const int32_t *terms, int min_bits, int ncls, int32_t *lists,
                                 unsigned long long *counts) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nc; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t want = 2 * (int64_t)(terms[t] > 1 ? terms[t] : 1);
        int c = 0;
        while (c < ncls - 1 && ((int64_t)1 << (min_bits + c)) < want) ++c;
        lists[(int64_t)c * nc + atomicAdd(&counts[c], 1ull)] = (int32_t)t;
    }
}

template <bool FILL>
int rap_launch(const AirLevel &L, int64_t nrows, const int32_t *rows, int bits, bool gmem, int32_t *cnt,
               const int64_t *acrp, int32_t *acci, double *acv, int *err, cudaStream_t s) {
    if (nrows <= 0) return AIR_OK;
    const size_t per_warp = (size_t)(1 << bits) * 20;
    if (!gmem) {
        int warps = (int)((160 * 1024) / per_warp);
        if (warps > 8) warps = 8;
        if (warps < 1) warps = 1;
        int64_t blocks = (nrows + warps - 1) / warps;
        if (blocks > 152 * 16) blocks = 152 * 16;
        AIR_CUDA(air_smem_optin(rap_kernel<FILL, false>));
        rap_kernel<FILL, false><<<air_counted((unsigned)blocks), warps * 32, per_warp * warps, s>>>(
            nrows, rows, L.rrp, L.rci, L.rv, L.rp, L.ci, L.v, L.pcol, bits, nullptr, cnt, acrp, acci, acv, err);
        AIR_LAUNCH();
        return AIR_OK;
    }
    // one scratch table per warp of a grid of at most 152 x 4 warps (8 per block)
    int64_t blocks = (nrows + 7) / 8;
    if (blocks > 152 * 4 / 8) blocks = 152 * 4 / 8;
    unsigned char *scratch = nullptr;
    AIR_CUDA(air_dmalloc((void **)&scratch, per_warp * (size_t)blocks * 8));
    rap_kernel<FILL, true><<<air_counted((unsigned)blocks), 256, 0, s>>>(nrows, rows, L.rrp, L.rci, L.rv, L.rp, L.ci,
                                                                        L.v, L.pcol, bits, scratch, cnt, acrp, acci,
                                                                        acv, err);
    cudaError_t e = cudaGetLastError();
    air_dfree(scratch);
    if (e != cudaSuccess) return AIR_ERR_CUDA;
    return AIR_OK;
}

int air_rap(const AirLevel &L, int64_t *acrp, int32_t *acci, double *acv, int32_t *cnt, int fill,
            int32_t max_terms, const int32_t *terms, int *d_err, cudaStream_t s) {
    int bits = 5;
    while ((1 << bits) < 2 * (max_terms > 1 ? max_terms : 1)) ++bits;
    constexpr int kSmemBits = 13;                 // 8192 slots, 160 KB: the largest shared table
    constexpr int kMinBits = 9;                   // 512 slots, 10 KB: 16 warps per SM
    auto launch = [&](int64_t nrows, const int32_t *rows, int b) {
        const bool gmem = b > kSmemBits;
        return fill ? rap_launch<true>(L, nrows, rows, b, gmem, nullptr, acrp, acci, acv, d_err, s)
                    : rap_launch<false>(L, nrows, rows, b, gmem, cnt, nullptr, nullptr, nullptr, d_err, s);
    };
    if (bits <= kMinBits) return launch(L.nc, nullptr, bits);
    // rows by class: each class's table the smallest power of two that holds twice its rows'
    // terms, so short rows get small tables (more warps per SM, less table upkeep); classes
    // beyond the shared-memory tables use global scratch tables of their own size
    const int ncls = bits - kMinBits + 1;
    if (ncls > 24) return AIR_ERR_UNSUPPORTED;
    int32_t *lists = nullptr;
    unsigned long long *counts = nullptr;
    AIR_CUDA(air_dmalloc((void **)&lists, (size_t)ncls * (size_t)(L.nc > 0 ? L.nc : 1) * sizeof(int32_t)));
    AIR_CUDA(air_dmalloc((void **)&counts, (size_t)ncls * sizeof(unsigned long long)));
    AIR_CUDA(cudaMemsetAsync(counts, 0, (size_t)ncls * sizeof(unsigned long long), s));
    rap_class_kernel<<<air_counted(grid_for(L.nc, 256)), 256, 0, s>>>(L.nc, terms, kMinBits, ncls, lists, counts);
    AIR_LAUNCH();
    unsigned long long hc[24] = {};
    AIR_CUDA(cudaStreamSynchronize(s));
    AIR_CUDA(cudaMemcpyAsync(hc, counts, (size_t)ncls * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    AIR_CUDA(cudaStreamSynchronize(s));
    int st = AIR_OK;
    for (int c = 0; c < ncls && st == AIR_OK; ++c) st = launch((int64_t)hc[c], lists + (int64_t)c * L.nc, kMinBits + c);
    air_dfree(lists);
    air_dfree(counts);
    return st;
}

// inv: n*n row major.  work: 2*n*n + n + 1 doubles.
int air_coarse_inverse(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, double *inv, double *work,
                       int *d_err, cudaStream_t s) {
    double *M = work, *fcol = work + 2 * n * n, *amax = fcol + n;
    AIR_CUDA(cudaMemsetAsync(M, 0, (size_t)(2 * n * n) * sizeof(double), s));
    dense_scatter_kernel<<<air_counted(grid_for(n, 256)), 256, 0, s>>>(n, rp, ci, v, M);
    dense_absmax_kernel<<<air_counted(1), 1024, 0, s>>>(n, M, amax);
    AIR_LAUNCH();
    int dev = 0, nsm = 0, per_sm = 0;
    AIR_CUDA(cudaGetDevice(&dev));
    AIR_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    AIR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gj_coop_kernel, 512, 0));
    if (per_sm < 1) return AIR_ERR_CUDA;
    int blocks = nsm;   // one co-resident block per SM
    void *args[] = {(void *)&n, (void *)&M, (void *)&fcol, (void *)&amax, (void *)&d_err};
    AIR_CUDA(cudaLaunchCooperativeKernel((const void *)gj_coop_kernel, dim3(air_counted(blocks).x), dim3(512), args, 0, s));
    dense_extract_kernel<<<air_counted(grid_for(n * n, 256)), 256, 0, s>>>(n, M, inv);
    AIR_LAUNCH();
    return AIR_OK;
}
