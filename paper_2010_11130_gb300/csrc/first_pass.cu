// First pass of the Ruge-Stueben C/F splitting (Section 4, classical
// coarsening), cursor version.
//
// The pass is the sequential process of the classical splitting: the
// undecided point of largest measure lambda (ties -> smallest index) becomes
// C, its undecided strong dependants S^T_i become F, every undecided k in S_j
// of a new F point j gains 1 and every undecided k in S_i loses 1.  Each pick
// depends on the one before, so the whole pass runs on one warp; the kernel
// below is built to keep the dependent chain of one pick short:
//
//  * each point's two-hop neighbourhood is stored once per distinct point, in
//    a fixed-size block addressed by the point alone: the members of S^T_i
//    first (in order), then every other point of some S_j (j in S^T_i) or of
//    S_i, each with a bit mask of the S_j lists it belongs to and a flag for
//    S_i.  One load brings a pick's neighbourhood, a second the measures of
//    its points; with F_new the mask of the undecided members of S^T_i, a
//    listed undecided point then changes by popc(mask & F_new) - [k in S_i],
//    independently of every other listed point, so no combining is needed;
//  * for every bucket (measure value) the block keeps its population and a
//    cursor: a 512-point line below which the bucket has no members, with the
//    exact contents of that line.  The pick's own changes keep populations and
//    cursors exact, so the next pick (lowest member of the highest non-empty
//    bucket) is read from shared memory with no global round trip;
//  * the bucket bitmaps in global memory are updated with fire-and-forget
//    reductions: leaf words exactly (XOR of membership changes), summary
//    levels as supersets (set on insertion, cleared when a search finds them
//    stale).  They are read only when a cursor line runs empty, about one pick
//    in twenty.
#include "air_internal.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int8_t M_F = -1, M_C = -2;          // measure codes of decided points
constexpr int K_BITS = 25;
constexpr uint32_t K_MASK = (1u << K_BITS) - 1u;
constexpr uint32_t F_J = 1u << 25;             // entry is a member of S^T_i
constexpr uint32_t F_SI = 1u << 26;            // entry is a member of S_i
constexpr int NB_MAX = 128;                    // buckets; measures <= 124 fit int8
constexpr int BLK_E = 64;                      // positions per block: header + 63 entries
constexpr int BLK_W = BLK_E + 2 * BLK_E;       // 32-bit words per block: entries, then 64-bit masks
constexpr int EMAX = 1024;                     // positions per list (header + 1023 entries)
constexpr int F_BIAS = 4096;                   // contribution of a point that becomes F (> 2 EMAX)
constexpr int32_t CL_INF = 0x7fffffff;         // cursor of an empty bucket
static_assert(F_BIAS > 2 * EMAX, "an F mark must dominate any sum of +-1 contributions");

struct RS5Args {
    int32_t n;
    int nb;                    // buckets 0 .. nb-1 (bucket 0 is never stored)
    const uint32_t *blocks;    // n * BLK_W words: [0] header, [1 + e] entry e (e < 63), masks at word 64 + 2 (1 + e)
    const int64_t *optr;       // start of each point's overflow entries (e >= 63)
    const uint32_t *ovf;       // overflow entries
    const uint64_t *ovfm;      // overflow masks
    int8_t *lam;
    uint64_t *L0, *L1;         // nb * w0 leaf words, nb * w1 summary words
    const uint64_t *L2;        // nb * w2 second summary (initial copy)
    int32_t w0, w1, w2;        // w0 is a multiple of 8 (one cursor line = 8 words)
    const int32_t *pop0;       // initial bucket populations
    int64_t cap;               // bound on search steps
    int *err;
    unsigned long long *stats; // [0] picks, [1] cursor refills, [2] lines visited, [3] long lists
};

unsigned blocks_for(int64_t items, int threads) {
    int64_t b = (items + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)b;
}

__device__ __forceinline__ void red_xor(uint64_t *p, uint64_t v) {
    atomicXor((unsigned long long *)p, (unsigned long long)v);
}
__device__ __forceinline__ void red_or(uint64_t *p, uint64_t v) {
    atomicOr((unsigned long long *)p, (unsigned long long)v);
}
__device__ __forceinline__ void red_and(uint64_t *p, uint64_t v) {
    atomicAnd((unsigned long long *)p, (unsigned long long)v);
}

// Upper bound on the distinct points of a neighbourhood: |S^T_i| + sum |S_j| + |S_i|.
__global__ void list_count_kernel(int64_t n, const int64_t *srp, const int64_t *strp, const int32_t *stci,
                                  int32_t *cnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = (strp[i + 1] - strp[i]) + (srp[i + 1] - srp[i]);
        for (int64_t q = strp[i]; q < strp[i + 1]; ++q) {
            const int32_t j = stci[q];
            c += srp[j + 1] - srp[j];
        }
        cnt[i] = (int32_t)(c < 0x7fffffff ? c : 0x7fffffff);
    }
}

__global__ void overflow_count_kernel(int64_t n, const int32_t *cnt, int32_t *ocnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        ocnt[i] = cnt[i] + 1 > BLK_E ? cnt[i] + 1 - BLK_E : 0;
}

// Neighbourhood block of point i, one entry per distinct point other than i:
// the members j_0, j_1, ... of S^T_i first (flag F_J), then the points of the
// lists S_{j_t} (mask bit t) and of S_i (flag F_SI) in first-seen order.
// Header: entries | |S^T_i| << 11.
__global__ void list_fill_kernel(int64_t n, const int64_t *srp, const int32_t *sci, const int64_t *strp,
                                 const int32_t *stci, const int64_t *optr, uint32_t *blocks, uint32_t *ovf,
                                 uint64_t *ovfm) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t *blk = blocks + (size_t)i * BLK_W;
        uint64_t *msk = (uint64_t *)(blk + BLK_E);
        const int64_t o = optr[i];
        auto ent = [&](int e) -> uint32_t & { return e < BLK_E - 1 ? blk[1 + e] : ovf[o + (e - (BLK_E - 1))]; };
        auto mask = [&](int e) -> uint64_t & { return e < BLK_E - 1 ? msk[1 + e] : ovfm[o + (e - (BLK_E - 1))]; };
        auto find = [&](int u, int32_t k) {
            for (int e = 0; e < u; ++e)
                if ((int32_t)(ent(e) & K_MASK) == k) return e;
            return -1;
        };
        int u = 0;
        for (int64_t q = strp[i]; q < strp[i + 1]; ++q) {
            ent(u) = F_J | (uint32_t)stci[q];
            mask(u) = 0ull;
            ++u;
        }
        int t = 0;
        for (int64_t q = strp[i]; q < strp[i + 1]; ++q, ++t) {
            const int32_t j = stci[q];
            for (int64_t r = srp[j]; r < srp[j + 1]; ++r) {
                const int32_t k = sci[r];
                if (k == (int32_t)i) continue;          // i itself becomes C
                const int e = find(u, k);
                if (e >= 0) {
                    mask(e) |= 1ull << t;
                } else {
                    ent(u) = (uint32_t)k;
                    mask(u) = 1ull << t;
                    ++u;
                }
            }
        }
        for (int64_t r = srp[i]; r < srp[i + 1]; ++r) {
            const int32_t k = sci[r];
            const int e = find(u, k);
            if (e >= 0) {
                ent(e) |= F_SI;
            } else {
                ent(u) = F_SI | (uint32_t)k;
                mask(u) = 0ull;
                ++u;
            }
        }
        blk[0] = (uint32_t)u | ((uint32_t)(strp[i + 1] - strp[i]) << 11);
    }
}

// Measures, exact bitmaps at all three levels and bucket populations.
__global__ void rs5_init_kernel(RS5Args a, const int64_t *srp, const int64_t *strp, uint64_t *L2, int32_t *pop) {
    __shared__ int32_t hist[NB_MAX];
    for (int b = threadIdx.x; b < NB_MAX; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t lam = (int32_t)(strp[i + 1] - strp[i]);
        const bool isolated = (srp[i + 1] == srp[i]) && lam == 0;
        a.lam[i] = isolated ? M_F : (int8_t)lam;
        if (!isolated && lam > 0) {
            atomicAdd(&hist[lam], 1);
            const int64_t i0 = i >> 6, i1 = i0 >> 6, i2 = i1 >> 6;
            const uint64_t o0 = atomicOr((unsigned long long *)&a.L0[(int64_t)lam * a.w0 + i0],
                                         (unsigned long long)(1ull << (i & 63)));
            if (o0 == 0ull) {
                const uint64_t o1 = atomicOr((unsigned long long *)&a.L1[(int64_t)lam * a.w1 + i1],
                                             (unsigned long long)(1ull << (i0 & 63)));
                if (o1 == 0ull)
                    atomicOr((unsigned long long *)&L2[(int64_t)lam * a.w2 + i2], (unsigned long long)(1ull << (i1 & 63)));
            }
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < NB_MAX; b += blockDim.x)
        if (hist[b]) atomicAdd(&pop[b], hist[b]);
}

__global__ void rs5_finish_kernel(int64_t n, const int8_t *lam, int8_t *cf) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        cf[i] = lam[i] == M_C ? 1 : 0;
}

struct Shared {
    uint32_t *cv;     // NB_MAX * 16: contents of each bucket's cursor line (512 points)
    uint32_t *L2s;    // nb * s2 second-level summary bits (bit q: summary word q may be non-zero)
    int32_t *pop;     // NB_MAX bucket populations
    int32_t *cl;      // NB_MAX cursor line (-1: not yet searched, CL_INF: never had a cursor)
    int32_t *pl;      // NB_MAX lowest line of insertions below the cursor (CL_INF: none)
    int32_t *rk;      // EMAX records of long lists: point, bucket left, bucket entered
    int8_t *rob, *rnb;
    int s2;           // 32-bit words of L2s per bucket
};

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Measures are read through L1: only this warp writes them, with plain
// stores that the same SM's L1 sees, and a __syncwarp orders every pick's
// stores before the next pick's loads.
__device__ __forceinline__ int lam_load(const int8_t *p) {
    return (int)__ldca((const signed char *)p);
}

__device__ __forceinline__ void prefetch_block(const uint32_t *p) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "r"(BLK_W * 4u)
                 : "memory");
}

// Bucket b has members but its cursor line is empty: find the first non-empty
// leaf line after it, using the summary levels as supersets and clearing the
// stale bits met on the way.  Returns false on an inconsistency or the cap.
__device__ bool rs5_refill(const RS5Args &a, const Shared &s, int b, int64_t *steps, unsigned long long *visits) {
    const int lane = threadIdx.x & 31;
    int32_t w = (s.cl[b] + 1) * 8;                  // first candidate leaf word (a line start)
    uint32_t *l2b = s.L2s + (int64_t)b * s.s2;
    while (true) {
        if (++(*steps) > a.cap || w >= a.w0) return false;
        const int32_t q = w >> 6;                   // summary word holding w
        const int32_t qq = q + lane;
        const bool in = qq < a.w1;
        const bool l2 = in && ((l2b[qq >> 5] >> (qq & 31)) & 1u);
        const uint64_t l1full = l2 ? __ldcg((const unsigned long long *)&a.L1[(int64_t)b * a.w1 + qq]) : 0ull;
        if (l2 && l1full == 0ull) atomicAnd(&l2b[qq >> 5], ~(1u << (qq & 31)));   // stale second-level bit
        const uint64_t l1 = lane == 0 ? (l1full & (~0ull << (w & 63))) : l1full;
        const unsigned bal = __ballot_sync(FULL, l1 != 0ull);
        if (bal == 0u) {
            // nothing in the next 32 summary words: jump to the next set second-level bit
            const int32_t from = q + 32;
            int32_t nq = a.w1;
            for (int32_t base = from >> 5; base < s.s2; base += 32) {
                const int32_t x = base + lane;
                uint32_t v = x < s.s2 ? l2b[x] : 0u;
                if (x == (from >> 5)) v &= ~0u << (from & 31);
                const unsigned vb = __ballot_sync(FULL, v != 0u);
                if (vb) {
                    const int src = __ffs(vb) - 1;
                    const uint32_t vv = __shfl_sync(FULL, v, src);
                    nq = (base + src) * 32 + (__ffs(vv) - 1);
                    break;
                }
            }
            __syncwarp();
            if (nq >= a.w1) return false;
            w = nq * 64;
            continue;
        }
        const int src = __ffs(bal) - 1;
        const uint64_t l1w = __shfl_sync(FULL, l1, src);
        const int32_t wf = (q + src) * 64 + (__ffsll((long long)l1w) - 1);
        const int32_t line = wf >> 3;
        const uint64_t lw = lane < 8 ? __ldcg((const unsigned long long *)&a.L0[(int64_t)b * a.w0 + line * 8 + lane]) : 0ull;
        ++(*visits);
        if (__ballot_sync(FULL, lw != 0ull)) {
            if (lane < 8) {
                s.cv[b * 16 + 2 * lane] = (uint32_t)lw;
                s.cv[b * 16 + 2 * lane + 1] = (uint32_t)(lw >> 32);
            }
            if (lane == 0) { s.cl[b] = line; s.pl[b] = CL_INF; }
            __syncwarp();
            return true;
        }
        if (lane == 0)                              // the whole line is empty: its summary bits are stale
            red_and(&a.L1[(int64_t)b * a.w1 + ((line * 8) >> 6)], ~(0xffull << ((line * 8) & 63)));
        __syncwarp();
        w = (line + 1) * 8;
    }
}

__global__ void __launch_bounds__(32) rs5_warp_kernel(RS5Args a) {
    extern __shared__ uint32_t smem[];
    Shared s;
    s.s2 = 2 * a.w2;
    s.cv = smem;
    s.L2s = s.cv + NB_MAX * 16;
    s.pop = (int32_t *)(s.L2s + (int64_t)a.nb * s.s2);
    s.cl = s.pop + NB_MAX;
    s.pl = s.cl + NB_MAX;
    s.rk = s.pl + NB_MAX;
    s.rob = (int8_t *)(s.rk + EMAX);
    s.rnb = s.rob + EMAX;
    const int lane = threadIdx.x & 31;
    const uint32_t *L2g = (const uint32_t *)a.L2;
    for (int64_t t = lane; t < (int64_t)a.nb * s.s2; t += 32) s.L2s[t] = L2g[t];
    for (int t = lane; t < NB_MAX * 16; t += 32) s.cv[t] = 0u;
    int top = 0;
    for (int b = lane; b < NB_MAX; b += 32) {
        const int32_t p = (b >= 1 && b < a.nb) ? a.pop0[b] : 0;
        s.pop[b] = p;
        s.cl[b] = p > 0 ? -1 : CL_INF;
        s.pl[b] = CL_INF;
        if (p > 0) top = b;
    }
    top = (int)__reduce_max_sync(FULL, (unsigned)top);
    __syncwarp();
    int64_t steps = 0;
    unsigned long long picks = 0, refills = 0, visits = 0, longs = 0, moves = 0;
    bool failed = false;
    // the block of the predicted next pick (the next member of the current
    // cursor line), loaded while the current pick settles
    int32_t pi = -1;
    uint32_t pe0 = 0u, pe1 = 0u;
    uint64_t pm0 = 0ull, pm1 = 0ull;
    while (true) {
        // ---- the pick: lowest member of the highest non-empty bucket (the state
        // of the previous top bucket is read at once: it usually still has members)
        int B = top;
        int32_t popB = s.pop[B], plB = s.pl[B], clB = s.cl[B];
        uint32_t wv = lane < 16 ? s.cv[B * 16 + lane] : 0u;
        if (popB == 0) {
            while (top >= 1 && s.pop[top] == 0) --top;
            if (top < 1) break;
            B = top;
            plB = s.pl[B];
            clB = s.cl[B];
            wv = lane < 16 ? s.cv[B * 16 + lane] : 0u;
        }
        if (plB < clB) {
            // insertions below the cursor: move it down to the lowest of them and
            // read that line (the bucket has no members below it)
            const int32_t line = plB;
            const uint64_t lw = lane < 8 ? __ldcg((const unsigned long long *)&a.L0[(int64_t)B * a.w0 + line * 8 + lane]) : 0ull;
            if (lane < 8) {
                s.cv[B * 16 + 2 * lane] = (uint32_t)lw;
                s.cv[B * 16 + 2 * lane + 1] = (uint32_t)(lw >> 32);
            }
            __syncwarp();
            if (lane == 0) { s.cl[B] = line; s.pl[B] = CL_INF; }
            ++moves;
            __syncwarp();
            clB = line;
            wv = lane < 16 ? s.cv[B * 16 + lane] : 0u;
        }
        unsigned bal = __ballot_sync(FULL, wv != 0u);
        if (bal == 0u) {
            ++refills;
            if (!rs5_refill(a, s, B, &steps, &visits)) { failed = true; break; }
            wv = lane < 16 ? s.cv[B * 16 + lane] : 0u;
            clB = s.cl[B];
            bal = __ballot_sync(FULL, wv != 0u);
            if (bal == 0u) { failed = true; break; }
        }
        const int sw = __ffs(bal) - 1;
        const uint32_t word = __shfl_sync(FULL, wv, sw);
        const int32_t lbase = clB * 512;
        const int32_t i = lbase + sw * 32 + (__ffs(word) - 1);
        if (++picks > (unsigned long long)a.n || i >= a.n) { failed = true; break; }
        // the next member of the same line is the likely next pick
        int32_t nxt = -1;
        {
            const uint32_t rest = lane == sw ? (word & (word - 1u)) : wv;
            const unsigned nz = __ballot_sync(FULL, rest != 0u);
            if (nz) {
                const int fl = __ffs(nz) - 1;
                const uint32_t rw = __shfl_sync(FULL, rest, fl);
                nxt = lbase + fl * 32 + (__ffs(rw) - 1);
                if (nxt >= a.n) nxt = -1;                // a stray bit past the last point: no speculative load
            }
        }

        // ---- round trip 1: the neighbourhood of i (positions lane and lane + 32),
        // already in registers when i was the predicted pick
        uint32_t e0, e1;
        uint64_t m0, m1;
        if (i == pi) {
            e0 = pe0; e1 = pe1; m0 = pm0; m1 = pm1;
        } else {
            const uint32_t *blk = a.blocks + (size_t)i * BLK_W;
            const uint64_t *bmk = (const uint64_t *)(blk + BLK_E);
            e0 = __ldcg(blk + lane);
            e1 = __ldcg(blk + 32 + lane);
            m0 = __ldcg((const unsigned long long *)bmk + lane);
            m1 = __ldcg((const unsigned long long *)bmk + 32 + lane);
        }
        pi = nxt;                                        // start loading the predicted next block
        if (nxt >= 0) {
            const uint32_t *nb = a.blocks + (size_t)nxt * BLK_W;
            const uint64_t *nm = (const uint64_t *)(nb + BLK_E);
            pe0 = __ldcg(nb + lane);
            pe1 = __ldcg(nb + 32 + lane);
            pm0 = __ldcg((const unsigned long long *)nm + lane);
            pm1 = __ldcg((const unsigned long long *)nm + 32 + lane);
        }
        const uint32_t hdr = __shfl_sync(FULL, e0, 0);
        const int np = (int)(hdr & 2047u) + 1;           // positions: header + entries
        const int nj = (int)((hdr >> 11) & 63u);         // entries 0 .. nj-1 are S^T_i (positions 1 .. nj)
        const bool two = np > 32;

        // ---- round trip 2: measures of the listed points
        const int32_t k0 = (int32_t)(e0 & K_MASK), k1 = (int32_t)(e1 & K_MASK);
        const int l0 = (lane >= 1 && lane < np) ? lam_load(a.lam + k0) : -3;
        const int l1 = (two && lane + 32 < np) ? lam_load(a.lam + k1) : -3;
        // F_new: the undecided members of S^T_i, bit t for entry t
        const unsigned f0 = __ballot_sync(FULL, lane >= 1 && lane <= nj && l0 >= 0);
        const unsigned f1 = __ballot_sync(FULL, lane + 32 <= nj && l1 >= 0);
        const uint64_t fnew = (uint64_t)(f0 >> 1) | ((uint64_t)f1 << 31);
        int vmax = 0;
        bool bad = false;
        // new state of a listed point from its measure l and its change c (F_BIAS: becomes F)
        auto settle = [&](int32_t k, int l, int c, int &ob, int &nbk) {
            ob = 0;
            nbk = 0;
            if (c >= F_BIAS / 2) {
                a.lam[k] = M_F;
                ob = l >= 1 ? l : 0;
            } else if (c != 0) {
                int nv = l + c;
                if (nv < 0 || nv >= a.nb) { bad = true; nv = 0; }   // cannot happen: 0 <= measure <= 2 max|S^T|
                a.lam[k] = (int8_t)nv;
                ob = l >= 1 ? l : 0;
                nbk = nv >= 1 ? nv : 0;
            }
            if (ob) red_xor(&a.L0[(int64_t)ob * a.w0 + (k >> 6)], 1ull << (k & 63));
            if (nbk) {
                red_xor(&a.L0[(int64_t)nbk * a.w0 + (k >> 6)], 1ull << (k & 63));
                red_or(&a.L1[(int64_t)nbk * a.w1 + (k >> 12)], 1ull << ((k >> 6) & 63));
                atomicOr(&s.L2s[(int64_t)nbk * s.s2 + (k >> 17)], 1u << ((k >> 12) & 31));
                if (nbk > B) prefetch_block(a.blocks + (size_t)k * BLK_W);   // a candidate for the next pick
            }
            vmax = max(vmax, nbk);
        };
        auto change = [&](uint32_t e, uint64_t m, int l, bool is_j) {
            if (l < 0) return 0;
            if (is_j) return F_BIAS;
            return __popcll(m & fnew) - ((e & F_SI) ? 1 : 0);
        };
        // one record per changed point: two in registers per lane, the rest of a long list in shared memory
        int32_t rk0 = k0, rk1 = k1;
        int ob0, nb0, ob1 = 0, nb1 = 0;
        settle(k0, l0, change(e0, m0, l0, lane <= nj), ob0, nb0);
        if (two) settle(k1, l1, change(e1, m1, l1, lane + 32 <= nj), ob1, nb1);
        if (lane == 0) {                                   // the header slot carries the pick's own record
            rk0 = i;
            ob0 = B;
            nb0 = 0;
            a.lam[i] = M_C;
            red_xor(&a.L0[(int64_t)B * a.w0 + (i >> 6)], 1ull << (i & 63));
        }
        int nx = 0;
        if (np > BLK_E) {                                  // long list: entries 63.. from the overflow area
            ++longs;
            const int64_t op = a.optr[i];
            for (int base = BLK_E; base < np; base += 32) {
                const int p = base + lane;
                int ob = 0, nbk = 0;
                int32_t k = 0;
                if (p < np) {
                    const uint32_t e = __ldcg(a.ovf + op + (p - BLK_E));
                    const uint64_t m = __ldcg((const unsigned long long *)a.ovfm + op + (p - BLK_E));
                    k = (int32_t)(e & K_MASK);
                    const int l = lam_load(a.lam + k);
                    settle(k, l, change(e, m, l, false), ob, nbk);   // S^T_i has at most 62 members
                }
                const bool has = ob != 0 || nbk != 0;
                const unsigned hb = __ballot_sync(FULL, has);
                if (has) {
                    const int q = nx + __popc(hb & lanemask_lt());
                    s.rk[q] = k;
                    s.rob[q] = (int8_t)ob;
                    s.rnb[q] = (int8_t)nbk;
                }
                nx += __popc(hb);
            }
        }
        if (__any_sync(FULL, bad)) { failed = true; break; }
        __syncwarp();
        // visit every record of the pick
        auto each = [&](auto fn) {
            fn(rk0, ob0, nb0);
            if (two) fn(rk1, ob1, nb1);
            for (int q = lane; q < nx; q += 32) fn(s.rk[q], (int)s.rob[q], (int)s.rnb[q]);
        };
        // populations and cursors.  A change inside a bucket's cursor line
        // toggles its bit (a removal clears a set bit, an insertion sets a clear
        // one); an insertion below the cursor only lowers the pending line, which
        // the next pick from that bucket reads from the leaf bitmap.  A bucket
        // left empty forgets its cursor, so that its next members all count as
        // insertions below it.  A: removals
        {
            auto forget = [&](int b) { s.cl[b] = CL_INF; s.pl[b] = CL_INF; };
            if (ob0 && atomicSub(&s.pop[ob0], 1) == 1) forget(ob0);
            if (two && ob1 && atomicSub(&s.pop[ob1], 1) == 1) forget(ob1);
            for (int q = lane; q < nx; q += 32) {
                const int ob = s.rob[q];
                if (ob && atomicSub(&s.pop[ob], 1) == 1) forget(ob);
            }
        }
        each([&](int32_t k, int ob, int) {
            if (ob && (k >> 9) == s.cl[ob]) atomicXor(&s.cv[ob * 16 + ((k >> 5) & 15)], 1u << (k & 31));
        });
        __syncwarp();
        // B: insertions
        if (nb0) atomicAdd(&s.pop[nb0], 1);
        if (two && nb1) atomicAdd(&s.pop[nb1], 1);
        for (int q = lane; q < nx; q += 32)
            if (s.rnb[q]) atomicAdd(&s.pop[s.rnb[q]], 1);
        each([&](int32_t k, int, int nbk) {
            if (nbk) {
                const int32_t L = k >> 9, c = s.cl[nbk];
                if (L == c) atomicXor(&s.cv[nbk * 16 + ((k >> 5) & 15)], 1u << (k & 31));
                else if (L < c) atomicMin(&s.pl[nbk], L);
            }
        });
        __syncwarp();
        vmax = (int)__reduce_max_sync(FULL, (unsigned)vmax);
        if (vmax > top) top = vmax;
    }
    if (lane == 0) {
        if (failed) atomicOr(a.err, AIR_DEVERR_RS_CAP);
        a.stats[0] += picks;
        a.stats[1] += refills;
        a.stats[2] += visits;
        a.stats[3] += longs;
        a.stats[4] += moves;
    }
}

}  // namespace

// Returns AIR_ERR_UNSUPPORTED (nothing launched) when the level is outside
// this kernel's limits: n >= 2^25, measures above 124, or a two-hop list of
// EMAX entries or more.  The caller then takes another variant.
int air_rs_first_pass_cursor(int64_t n, const int64_t *srp, const int32_t *sci, const int64_t *strp,
                             const int32_t *stci, int32_t max_st, int8_t *cf, int *d_err,
                             unsigned long long *stats, cudaStream_t s) {
    const int nb = 2 * max_st + 1 < 2 ? 2 : 2 * max_st + 1;
    if (n <= 0 || n >= (int64_t)1 << K_BITS || nb > 125 || max_st > 62) return AIR_ERR_UNSUPPORTED;
    int32_t *cnt = nullptr, *dmax = nullptr;
    AIR_CUDA(cudaMallocAsync(&cnt, (size_t)n * sizeof(int32_t), s));
    AIR_CUDA(cudaMallocAsync(&dmax, sizeof(int32_t), s));
    AIR_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int32_t), s));
    list_count_kernel<<<air_counted(blocks_for(n, 256)), 256, 0, s>>>(n, srp, strp, stci, cnt);
    AIR_LAUNCH();
    AIR_TRY(air_reduce_max_i32(cnt, n, dmax, s));
    int32_t maxcnt = 0;
    AIR_CUDA(cudaMemcpyAsync(&maxcnt, dmax, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AIR_CUDA(cudaStreamSynchronize(s));
    cudaFreeAsync(dmax, s);
    if (maxcnt + 1 > EMAX) {
        cudaFreeAsync(cnt, s);
        return AIR_ERR_UNSUPPORTED;
    }
    // overflow area for neighbourhoods longer than a block (sized by the upper bound)
    int32_t *ocnt = nullptr;
    int64_t *optr = nullptr;
    AIR_CUDA(cudaMallocAsync(&ocnt, (size_t)n * sizeof(int32_t), s));
    AIR_CUDA(cudaMallocAsync(&optr, (size_t)(n + 1) * sizeof(int64_t), s));
    overflow_count_kernel<<<air_counted(blocks_for(n, 256)), 256, 0, s>>>(n, cnt, ocnt);
    AIR_LAUNCH();
    AIR_TRY(air_exclusive_scan_i32(ocnt, optr, n, s));
    int64_t novf = 0;
    AIR_CUDA(cudaMemcpyAsync(&novf, optr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    AIR_CUDA(cudaStreamSynchronize(s));
    cudaFreeAsync(ocnt, s);
    cudaFreeAsync(cnt, s);
    RS5Args a{};
    a.n = (int32_t)n;
    a.nb = nb;
    a.w0 = (int32_t)((((n + 63) / 64) + 7) / 8 * 8);
    a.w1 = (a.w0 + 63) / 64;
    a.w2 = (a.w1 + 63) / 64;
    a.err = d_err;
    a.stats = stats;
    // every search step returns, clears a stale summary bit or moves past an
    // empty line; stale bits come only from insertions (at most one per list
    // entry per pick)
    a.cap = 4 * (int64_t)n * (int64_t)EMAX + 4096;
    uint32_t *blocks = nullptr, *ovf = nullptr;
    uint64_t *ovfm = nullptr;
    AIR_CUDA(cudaMallocAsync(&blocks, (size_t)n * BLK_W * sizeof(uint32_t), s));
    AIR_CUDA(cudaMallocAsync(&ovf, (size_t)(novf > 0 ? novf : 1) * sizeof(uint32_t), s));
    AIR_CUDA(cudaMallocAsync(&ovfm, (size_t)(novf > 0 ? novf : 1) * sizeof(uint64_t), s));
    list_fill_kernel<<<air_counted(blocks_for(n, 256)), 256, 0, s>>>(n, srp, sci, strp, stci, optr, blocks, ovf,
                                                                      ovfm);
    AIR_LAUNCH();
    const size_t words = (size_t)nb * (size_t)(a.w0 + a.w1 + a.w2);
    uint64_t *bits = nullptr;
    int32_t *pop = nullptr;
    int8_t *lam = nullptr;
    AIR_CUDA(cudaMallocAsync(&bits, words * sizeof(uint64_t), s));
    AIR_CUDA(cudaMallocAsync(&pop, NB_MAX * sizeof(int32_t), s));
    AIR_CUDA(cudaMallocAsync(&lam, (size_t)n, s));
    AIR_CUDA(cudaMemsetAsync(bits, 0, words * sizeof(uint64_t), s));
    AIR_CUDA(cudaMemsetAsync(pop, 0, NB_MAX * sizeof(int32_t), s));
    a.L0 = bits;
    a.L1 = bits + (size_t)nb * a.w0;
    uint64_t *L2 = a.L1 + (size_t)nb * a.w1;
    a.L2 = L2;
    a.lam = lam;
    a.blocks = blocks;
    a.optr = optr;
    a.ovf = ovf;
    a.ovfm = ovfm;
    a.pop0 = pop;
    rs5_init_kernel<<<air_counted(blocks_for(n, 256)), 256, 0, s>>>(a, srp, strp, L2, pop);
    AIR_LAUNCH();
    const size_t smem = (size_t)NB_MAX * 16 * 4 + (size_t)nb * 2 * a.w2 * 4 + 3 * NB_MAX * 4 + (size_t)EMAX * 4 +
                        2 * (size_t)EMAX + 64;
    int st = AIR_OK;
    if (smem > AIR_SMEM_OPTIN) {
        st = AIR_ERR_UNSUPPORTED;
    } else {
        AIR_CUDA(air_smem_optin(rs5_warp_kernel));
        rs5_warp_kernel<<<air_counted(1), 32, smem, s>>>(a);
        AIR_LAUNCH();
        rs5_finish_kernel<<<air_counted(blocks_for(n, 256)), 256, 0, s>>>(n, lam, cf);
        AIR_LAUNCH();
    }
    cudaFreeAsync(bits, s);
    cudaFreeAsync(pop, s);
    cudaFreeAsync(lam, s);
    cudaFreeAsync(blocks, s);
    cudaFreeAsync(ovf, s);
    cudaFreeAsync(ovfm, s);
    cudaFreeAsync(optr, s);
    return st;
}
