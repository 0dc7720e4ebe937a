// First pass of the Ruge-Stueben C/F splitting (Section 4, classical
// coarsening), cursor version.
//
// The pass is the sequential process of the classical splitting: the
// undecided point of largest measure lambda (ties -> smallest index) becomes
// C, its undecided strong dependants S^T_i become F, every undecided k in S_j
// of a new F point j gains 1 and every undecided k in S_i loses 1.  Each pick
// depends on the one before, so the whole pass runs on one warp; the kernel
// below is built to keep the dependent chain of one pick to two memory round
// trips:
//
//  * each point's two-hop list (S^T_i, then S_j for each j in S^T_i, then S_i)
//    sits in a fixed-size line of 32-bit entries (point index in the low 25
//    bits, the role in the high 7), so a pick's whole list arrives in one
//    coalesced load addressed by the point alone;
//  * the measures of the listed points arrive in the second load; every
//    consequence of the pick (new F points, summed measure changes) is then
//    combined in registers and a shared-memory hash table;
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
constexpr uint32_t ROLE_SI = 126u, ROLE_J = 127u;
constexpr int K_BITS = 25;
constexpr uint32_t K_MASK = (1u << K_BITS) - 1u;
constexpr int NB_MAX = 128;                    // buckets; measures <= 124 fit int8
constexpr int LINE = 128;                      // words per list line: header + 127 entries
constexpr int EMAX = 1024;                     // positions per list (header + 1023 entries)
constexpr int TS_BITS = 11;
constexpr int TS = 1 << TS_BITS;               // hash slots, >= 2x the entries of one list
constexpr int F_BIAS = 4096;                   // hash value of a point that becomes F (> 2 EMAX)
constexpr int32_t CL_INF = 0x7fffffff;         // cursor of an empty bucket
constexpr int OWNER = 4096;                    // slot code of the position that claimed the slot
static_assert(OWNER >= TS && OWNER + TS <= 32767, "slot codes must fit int16");
static_assert(F_BIAS > 2 * EMAX, "an F mark must dominate any sum of +-1 contributions");

struct RS5Args {
    int32_t n;
    int nb;                    // buckets 0 .. nb-1 (bucket 0 is never stored)
    const uint32_t *lines;     // n * LINE words
    const int64_t *optr;       // start of each point's overflow entries (positions >= LINE)
    const uint32_t *ovf;
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

// Line of point i: word 0 = entries | |S^T_i| << 11, word p = entry p - 1 for
// p < LINE, the rest at ovf[optr[i] + p - LINE].  Roles: ROLE_J for S^T_i, t
// (the position of j in S^T_i) for S_j, ROLE_SI for S_i.
__global__ void list_fill_kernel(int64_t n, const int64_t *srp, const int32_t *sci, const int64_t *strp,
                                 const int32_t *stci, const int64_t *optr, uint32_t *lines, uint32_t *ovf) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t *line = lines + (size_t)i * LINE;
        const int64_t o = optr[i];
        int p = 1;
        auto put = [&](uint32_t v) {
            if (p < LINE) line[p] = v; else ovf[o + (p - LINE)] = v;
            ++p;
        };
        for (int64_t q = strp[i]; q < strp[i + 1]; ++q) put((ROLE_J << K_BITS) | (uint32_t)stci[q]);
        uint32_t t = 0;
        for (int64_t q = strp[i]; q < strp[i + 1]; ++q, ++t) {
            const int32_t j = stci[q];
            for (int64_t r = srp[j]; r < srp[j + 1]; ++r) put((t << K_BITS) | (uint32_t)sci[r]);
        }
        for (int64_t r = srp[i]; r < srp[i + 1]; ++r) put((ROLE_SI << K_BITS) | (uint32_t)sci[r]);
        line[0] = (uint32_t)(p - 1) | ((uint32_t)(strp[i + 1] - strp[i]) << 11);
    }
}

__global__ void overflow_count_kernel(int64_t n, const int32_t *cnt, int32_t *ocnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        ocnt[i] = cnt[i] + 1 > LINE ? cnt[i] + 1 - LINE : 0;
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
    int32_t *cl;      // NB_MAX cursor line (-1: not yet searched, CL_INF: empty bucket)
    int32_t *cl2;     // NB_MAX shadow of cl collecting the lowest new line
    int32_t *tk;      // TS hash keys (-1 empty)
    int32_t *tv;      // TS hash values
    uint32_t *sent;   // EMAX list entries of the current pick (position p = entry p - 1)
    int32_t *rk;      // EMAX records: point, bucket left, bucket entered
    int8_t *rob, *rnb;
    int8_t *slv;      // EMAX measures of the listed points at the start of the pick (-3: not live)
    int16_t *sslot;   // EMAX hash slot of the position (+ OWNER when it owns the slot), -1 none
    int8_t *jf;       // 64 new-F flags of the S^T_i entries
    int s2;           // 32-bit words of L2s per bucket
};

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ void prefetch_line(const uint32_t *p) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "r"(LINE * 4u)
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
            if (lane == 0) { s.cl[b] = line; s.cl2[b] = line; }
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
    s.cl2 = s.cl + NB_MAX;
    s.tk = s.cl2 + NB_MAX;
    s.tv = s.tk + TS;
    s.sent = (uint32_t *)(s.tv + TS);
    s.rk = (int32_t *)(s.sent + EMAX);
    s.sslot = (int16_t *)(s.rk + EMAX + 32);
    s.rob = (int8_t *)(s.sslot + EMAX);
    s.rnb = s.rob + EMAX + 32;
    s.slv = s.rnb + EMAX + 32;
    s.jf = s.slv + EMAX;
    const int lane = threadIdx.x & 31;
    const uint32_t *L2g = (const uint32_t *)a.L2;
    for (int64_t t = lane; t < (int64_t)a.nb * s.s2; t += 32) s.L2s[t] = L2g[t];
    for (int t = lane; t < NB_MAX * 16; t += 32) s.cv[t] = 0u;
    int top = 0;
    for (int b = lane; b < NB_MAX; b += 32) {
        const int32_t p = (b >= 1 && b < a.nb) ? a.pop0[b] : 0;
        s.pop[b] = p;
        s.cl[b] = p > 0 ? -1 : CL_INF;
        s.cl2[b] = s.cl[b];
        if (p > 0) top = b;
    }
    for (int t = lane; t < TS; t += 32) { s.tk[t] = -1; s.tv[t] = 0; }
    top = (int)__reduce_max_sync(FULL, (unsigned)top);
    __syncwarp();
    int64_t steps = 0;
    unsigned long long picks = 0, refills = 0, visits = 0, longs = 0;
    bool failed = false;
    while (true) {
        // ---- the pick: lowest member of the highest non-empty bucket
        while (top >= 1 && s.pop[top] == 0) --top;
        if (top < 1) break;
        const int B = top;
        uint32_t wv = lane < 16 ? s.cv[B * 16 + lane] : 0u;
        unsigned bal = __ballot_sync(FULL, wv != 0u);
        if (bal == 0u) {
            ++refills;
            if (!rs5_refill(a, s, B, &steps, &visits)) { failed = true; break; }
            wv = lane < 16 ? s.cv[B * 16 + lane] : 0u;
            bal = __ballot_sync(FULL, wv != 0u);
            if (bal == 0u) { failed = true; break; }
        }
        const int sw = __ffs(bal) - 1;
        const uint32_t word = __shfl_sync(FULL, wv, sw);
        const int32_t lbase = s.cl[B] * 512;
        const int32_t i = lbase + sw * 32 + (__ffs(word) - 1);
        if (++picks > (unsigned long long)a.n || i >= a.n) { failed = true; break; }
        // the next members of the same line are the likely next picks: warm their lists in L2
        {
            const uint32_t rest = lane == sw ? (word & (word - 1u)) : wv;
            const unsigned nz = __ballot_sync(FULL, rest != 0u);
            if (rest != 0u && __popc(nz & lanemask_lt()) < 3)
                prefetch_line(a.lines + (size_t)(lbase + lane * 32 + (__ffs(rest) - 1)) * LINE);
        }

        // ---- round trip 1: the two-hop list of i
        const uint32_t *line = a.lines + (size_t)i * LINE;
        uint32_t ent[LINE / 32];
#pragma unroll
        for (int r = 0; r < LINE / 32; ++r) ent[r] = __ldcg(line + lane + 32 * r);
        const uint32_t hdr = __shfl_sync(FULL, ent[0], 0);
        const int np = (int)(hdr & 2047u) + 1;          // positions: header + entries
        const int nj = (int)((hdr >> 11) & 63u);

        // ---- round trip 2: measures of the listed points
        int lv[LINE / 32];
#pragma unroll
        for (int r = 0; r < LINE / 32; ++r) {
            const int p = lane + 32 * r;
            const int32_t k = (int32_t)(ent[r] & K_MASK);
            lv[r] = (p >= 1 && p < np && k != i) ? (int)__ldcg(a.lam + k) : -3;
        }
        // Each changed point gets one record (point, bucket left, bucket entered;
        // 0 = none): in a register of the owning lane when the list fits one
        // position per lane, else in shared memory.
        const bool fast = np <= 32;
        int32_t fk = 0;
        int fob = 0, fnb = 0;
        int nrec = 0, vmax = 0;
        bool bad = false;
        // new state of a changed point from its measure l and summed contribution v
        auto settle = [&](int32_t k, int l, int v, int &ob, int &nbk) {
            ob = 0;
            nbk = 0;
            if (v >= F_BIAS / 2) {
                a.lam[k] = M_F;
                ob = l >= 1 ? l : 0;
            } else if (v != 0) {
                int nv = l + v;
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
                if (nbk > B) prefetch_line(a.lines + (size_t)k * LINE);   // a candidate for the next pick
            }
            vmax = max(vmax, nbk);
        };
        if (fast) {
            // one position per lane: combine duplicates with warp matching
            const int32_t k = (int32_t)(ent[0] & K_MASK);
            const uint32_t role = ent[0] >> K_BITS;
            const int l = lv[0];
            const bool newF = lane >= 1 && lane - 1 < nj && l >= 0;     // undecided members of S^T_i
            const bool jnew = __shfl_sync(FULL, newF, role < ROLE_SI ? (int)(role + 1) & 31 : 0);
            int contrib = 0;
            if (l >= 0) contrib = (lane - 1 < nj) ? F_BIAS : (role == ROLE_SI ? -1 : (jnew ? 1 : 0));
            // per-group sums from three full-warp ballots (a reduction over each
            // match group would serialise over the distinct groups)
            const unsigned m = __match_any_sync(FULL, contrib != 0 ? (uint32_t)k : (0x80000000u | (uint32_t)lane));
            const unsigned bF = __ballot_sync(FULL, contrib == F_BIAS);
            const unsigned bP = __ballot_sync(FULL, contrib == 1);
            const unsigned bM = __ballot_sync(FULL, contrib == -1);
            const int v = F_BIAS * __popc(bF & m) + __popc(bP & m) - __popc(bM & m);
            if (contrib != 0 && lane == __ffs(m) - 1) {
                fk = k;
                settle(k, l, v, fob, fnb);
            }
            if (lane == 0) {                              // the header lane carries the pick's record
                fk = i;
                fob = B;
                fnb = 0;
            }
        } else {
#pragma unroll
            for (int r = 0; r < LINE / 32; ++r) {
                const int p = lane + 32 * r;
                if (p < np) { s.sent[p] = ent[r]; s.slv[p] = (int8_t)lv[r]; }
                if (p >= 1 && p - 1 < nj) s.jf[p - 1] = lv[r] >= 0 ? 1 : 0;   // new F points: undecided S^T_i
            }
            if (np > LINE) {                             // long list: the rest from the overflow area
                ++longs;
                const int64_t op = a.optr[i];
                for (int p = LINE + lane; p < np; p += 32) {
                    const uint32_t e = __ldcg(a.ovf + op + (p - LINE));
                    const int32_t k = (int32_t)(e & K_MASK);
                    s.sent[p] = e;
                    s.slv[p] = (int8_t)(k != i ? (int)__ldcg(a.lam + k) : -3);
                }
            }
            __syncwarp();
            // contributions of every live entry, summed per point in the hash table
            for (int p = lane; p < np; p += 32) {
                int16_t sl = -1;
                const int l = p >= 1 ? (int)s.slv[p] : -3;
                if (l >= 0) {
                    const uint32_t ev = s.sent[p];
                    const uint32_t role = ev >> K_BITS;
                    const int32_t k = (int32_t)(ev & K_MASK);
                    const int contrib = (p - 1 < nj) ? F_BIAS : (role == ROLE_SI ? -1 : (s.jf[role] ? 1 : 0));
                    if (contrib != 0) {
                        int h = (int)(((uint32_t)k * 2654435761u) >> (32 - TS_BITS));
                        bool own = false;
                        for (int t = 0; t < TS; ++t) {
                            const int old = atomicCAS(&s.tk[h], -1, k);
                            if (old == -1) { own = true; break; }
                            if (old == k) break;
                            h = (h + 1) & (TS - 1);
                        }
                        atomicAdd(&s.tv[h], contrib);
                        sl = (int16_t)(h + (own ? OWNER : 0));
                    }
                }
                s.sslot[p] = sl;
            }
            __syncwarp();
            // owners settle their point and append its record
            for (int base = 0; base < np; base += 32) {
                const int p = base + lane;
                int ob = 0, nbk = 0;
                int32_t k = 0;
                const int sl = p < np ? (int)s.sslot[p] : -1;
                if (sl >= OWNER) {
                    const int h = sl - OWNER;
                    const int v = s.tv[h];
                    s.tk[h] = -1;
                    s.tv[h] = 0;
                    k = (int32_t)(s.sent[p] & K_MASK);
                    settle(k, (int)s.slv[p], v, ob, nbk);
                }
                const bool has = ob != 0 || nbk != 0;
                const unsigned hb = __ballot_sync(FULL, has);
                if (has) {
                    const int q = nrec + __popc(hb & lanemask_lt());
                    s.rk[q] = k;
                    s.rob[q] = (int8_t)ob;
                    s.rnb[q] = (int8_t)nbk;
                }
                nrec += __popc(hb);
            }
            if (lane == 0) {                              // the pick's record
                s.rk[nrec] = i;
                s.rob[nrec] = (int8_t)B;
                s.rnb[nrec] = 0;
            }
            ++nrec;
        }
        if (__any_sync(FULL, bad)) { failed = true; break; }
        if (lane == 0) {                                  // the pick itself leaves bucket B
            a.lam[i] = M_C;
            red_xor(&a.L0[(int64_t)B * a.w0 + (i >> 6)], 1ull << (i & 63));
        }
        __syncwarp();
        // visit every record of the pick
        auto each = [&](auto fn) {
            if (fast) {
                fn(fk, fob, fnb);
            } else {
                for (int q = lane; q < nrec; q += 32) fn(s.rk[q], (int)s.rob[q], (int)s.rnb[q]);
            }
        };
        // cursors and populations.  A: removals (the fast path adds one
        // population change per bucket, from warp matching)
        if (fast) {
            const unsigned m = __match_any_sync(FULL, fob ? (uint32_t)fob : (0x100u | (uint32_t)lane));
            if (fob && lane == __ffs(m) - 1) atomicSub(&s.pop[fob], __popc(m));
        }
        each([&](int32_t k, int ob, int) {
            if (ob) {
                if (!fast) atomicSub(&s.pop[ob], 1);
                if ((k >> 9) == s.cl[ob]) atomicXor(&s.cv[ob * 16 + ((k >> 5) & 15)], 1u << (k & 31));
            }
        });
        __syncwarp();
        // B: a bucket left empty forgets its cursor
        each([&](int32_t, int ob, int) {
            if (ob && s.pop[ob] == 0) { s.cl[ob] = CL_INF; s.cl2[ob] = CL_INF; }
        });
        __syncwarp();
        // C: insertions; a point below a bucket's cursor pulls the cursor down
        if (fast) {
            const unsigned m = __match_any_sync(FULL, fnb ? (uint32_t)fnb : (0x100u | (uint32_t)lane));
            if (fnb && lane == __ffs(m) - 1) atomicAdd(&s.pop[fnb], __popc(m));
        }
        each([&](int32_t k, int, int nbk) {
            if (nbk) {
                if (!fast) atomicAdd(&s.pop[nbk], 1);
                if ((k >> 9) < s.cl[nbk]) atomicMin(&s.cl2[nbk], k >> 9);
            }
        });
        __syncwarp();
        // D: a moved cursor starts from an empty line (the bucket had no members
        // there); several records may move the same cursor, all to the same line
        each([&](int32_t, int, int nbk) {
            if (nbk && s.cl2[nbk] < s.cl[nbk]) {
                for (int t = 0; t < 16; ++t) s.cv[nbk * 16 + t] = 0u;
                s.cl[nbk] = s.cl2[nbk];
            }
        });
        __syncwarp();
        // E: insertions into the cursor line
        each([&](int32_t k, int, int nbk) {
            if (nbk && (k >> 9) == s.cl[nbk]) atomicOr(&s.cv[nbk * 16 + ((k >> 5) & 15)], 1u << (k & 31));
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
    if (n <= 0 || n >= (int64_t)1 << K_BITS || nb > 125) return AIR_ERR_UNSUPPORTED;
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
    // overflow area for lists longer than a line
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
    uint32_t *lines = nullptr, *ovf = nullptr;
    AIR_CUDA(cudaMallocAsync(&lines, (size_t)n * LINE * sizeof(uint32_t), s));
    AIR_CUDA(cudaMallocAsync(&ovf, (size_t)(novf > 0 ? novf : 1) * sizeof(uint32_t), s));
    list_fill_kernel<<<air_counted(blocks_for(n, 256)), 256, 0, s>>>(n, srp, sci, strp, stci, optr, lines, ovf);
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
    a.lines = lines;
    a.optr = optr;
    a.ovf = ovf;
    a.pop0 = pop;
    rs5_init_kernel<<<air_counted(blocks_for(n, 256)), 256, 0, s>>>(a, srp, strp, L2, pop);
    AIR_LAUNCH();
    const size_t smem = (size_t)NB_MAX * 16 * 4 + (size_t)nb * 2 * a.w2 * 4 + 3 * NB_MAX * 4 + 2 * TS * 4 +
                        (size_t)EMAX * 4 + (size_t)(EMAX + 32) * 4 + (size_t)EMAX * 2 + 2 * (size_t)(EMAX + 32) +
                        (size_t)EMAX + 64;
    int st = AIR_OK;
    if (smem > 200 * 1024) {
        st = AIR_ERR_UNSUPPORTED;
    } else {
        AIR_CUDA(cudaFuncSetAttribute(rs5_warp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        rs5_warp_kernel<<<air_counted(1), 32, smem, s>>>(a);
        AIR_LAUNCH();
        rs5_finish_kernel<<<air_counted(blocks_for(n, 256)), 256, 0, s>>>(n, lam, cf);
        AIR_LAUNCH();
    }
    cudaFreeAsync(bits, s);
    cudaFreeAsync(pop, s);
    cudaFreeAsync(lam, s);
    cudaFreeAsync(lines, s);
    cudaFreeAsync(ovf, s);
    cudaFreeAsync(optr, s);
    return st;
}
