/*
 * Plain CPU oracle of the AIR-preconditioned GMRES path -- TEST INFRASTRUCTURE.
 *
 * Only the test suite, the package smoke check and the benchmark's CPU
 * baseline call into this file.  It shares no code with the CUDA library.
 * Single-threaded, FP64, compiled with -O2 -ffp-contract=off so that every
 * a*b+c is one rounded multiply followed by one rounded add.
 *
 * Method (arXiv:2010.11130, Section 3 and the solver settings of Section 4):
 *   x <- x + P (R A P)^{-1} R r        two-level correction      (Section 3)
 *   R ~ R_ideal = [-A_cf A_ff^{-1}, I] by local l-AIR solves       (Section 3)
 *   P = [W; I], one-point interpolation                            (Section 4)
 *   classical strength, C/F splitting, relaxation, Krylov acceleration.
 *
 * Readings of what the paper leaves open (all stated once here):
 *  - strength: j in S_i iff j != i and |a_ij| >= theta * max_{k != i} |a_ik|
 *    over the stored entries of row i (theta * max is one IEEE multiply);
 *    S_i is empty when that maximum is 0.
 *  - C/F splitting: first pass of Ruge-Stueben with measure lambda_i = |S^T_i|;
 *    the undecided point of largest lambda is made C (ties -> smallest
 *    index); its undecided strong dependants S^T_i become F and every
 *    undecided k in S_j of a new F point j gains 1; every undecided k in
 *    S_i loses 1.  Points with S_i and S^T_i both empty start as F; points
 *    still undecided when the largest lambda is 0 become F.
 *  - Falgout-style splitting (optional, the coarsening of the paper's Section 4
 *    settings, whose details the paper leaves to its library): the points
 *    are cut into consecutive index blocks of a fixed size; the first pass
 *    above runs in each block on the strength graph restricted to the block
 *    (measures count only dependants inside the block; a point with no strong
 *    connection inside its block starts F).  Interface points (a strong
 *    connection, either way, to another block) that end F with S_i non-empty
 *    but no C point in S_i are then fixed by rounds of a parallel independent
 *    set: weight w_i = |S^T_i| + frac(i), frac(i) in [0, 1) from the
 *    SplitMix64 hash of i; a remaining point becomes C when its weight beats
 *    every remaining point of S_i and S^T_i (ties -> smaller index), and
 *    points that now have a C point in S_i leave.  One block = the first pass.
 *  - the strength threshold may differ between the C/F splitting (with
 *    one-point P) and the l-AIR neighbourhoods (Section 4 uses 0.2 for the
 *    coarsening and 0.3 for R); R then uses its own strength graph.
 *  - l-AIR neighbourhood N_i: distance 1 = S_i intersect F; distance d adds
 *    S_k intersect F for every k found at distance d-1.  N_i ascending.
 *    Local system A_ff(N_i,N_i)^T z = -A(i,N_i)^T by LU with partial
 *    pivoting (ties -> smallest row), forward substitution in ascending and
 *    back substitution in descending column order.  A pivot with
 *    |pivot| <= 1e-14 * max|M| marks the system singular: z = 0.
 *    R row i = [z on N_i, 1 at i], columns ascending.
 *  - one-point P: F point i takes its value from the strong C neighbour of
 *    largest |a_ij| (ties -> smallest j) with weight 1; no strong C
 *    neighbour -> empty row.  C point i -> identity onto its coarse id
 *    (rank among the C points in ascending order).
 *  - A_c = (R A) P with structural patterns (no dropping): (RA)_ij sums over
 *    the entries k of R row i in ascending k, and for each k over A row k;
 *    then column j goes to coarse column P(j) and the terms meet in
 *    ascending j.
 *  - coarsening stops when n <= max_coarse, when the next level would keep
 *    more than 0.9 n points (or none), or at max_levels; the coarsest level
 *    is solved by dense LU with partial pivoting.
 *  - V-cycle: zero initial guess on every level, restrict, recurse,
 *    interpolate, then the sweeps of the relaxation string, one per
 *    character: 'F', 'C', 'A' = a Jacobi sweep (weight omega) over the F, C
 *    or all points ("FCF" = F, C, F); 'f', 'c', 'a' = a forward Gauss-Seidel
 *    sweep (weight omega, ascending index, each point using the values
 *    already updated) over the F, C or all points.  "fa" is the paper's
 *    post-relaxation: forward Gauss-Seidel on the F points, then on all
 *    points (Section 4 settings).
 *  - GMRES(m): right preconditioned, modified Gram-Schmidt, Givens
 *    rotations, x0 = 0, flexible (stores Z = M^{-1} V), stops when the
 *    true relative residual ||b - A x|| / ||b|| <= rtol (checked at the
 *    end of every cycle; inside a cycle the Givens estimate decides).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_MAX_LEVELS 32

enum { ORA_OK = 0, ORA_ERR_ARG = -1, ORA_ERR_OOM = -2, ORA_ERR_COARSE = -3 };

typedef struct {
    int64_t n, nnz;
    int64_t *rp;
    int32_t *ci;
    double *v;
} ora_csr;

typedef struct {
    ora_csr A;          /* level operator */
    ora_csr S;          /* strength pattern (v unused) */
    ora_csr ST;         /* its transpose */
    ora_csr SR;         /* strength pattern for R when its threshold differs (else empty) */
    int8_t *cf;         /* 1 = C, 0 = F */
    int32_t *cid;       /* coarse id of C points, -1 for F */
    int64_t nc;
    ora_csr R;          /* nc x n */
    int32_t *pcol;      /* coarse column of each fine row, -1 if empty */
    double *pw;         /* its weight */
    int64_t n_singular; /* l-AIR systems treated as singular */
    int32_t max_m;      /* largest l-AIR system */
} ora_level;

typedef struct {
    int nlev;                       /* levels 0 .. nlev-1, last one is coarsest */
    ora_level lev[ORA_MAX_LEVELS];
    double *lu;                     /* dense LU of the coarsest operator (row major) */
    int32_t *piv;
    double omega;
    char relax[64];
} ora_hier;

static void csr_free(ora_csr *M) {
    free(M->rp); free(M->ci); free(M->v);
    memset(M, 0, sizeof(*M));
}

static int csr_alloc(ora_csr *M, int64_t n, int64_t nnz, int with_val) {
    M->n = n; M->nnz = nnz;
    M->rp = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    M->ci = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    M->v = with_val ? (double *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double)) : NULL;
    if (!M->rp || !M->ci || (with_val && !M->v)) return ORA_ERR_OOM;
    return ORA_OK;
}

/* value of A(r, c), 0 if not stored (binary search, columns ascending) */
static double csr_get(const ora_csr *A, int64_t r, int32_t c) {
    int64_t lo = A->rp[r], hi = A->rp[r + 1] - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (A->ci[mid] == c) return A->v[mid];
        if (A->ci[mid] < c) lo = mid + 1; else hi = mid - 1;
    }
    return 0.0;
}

/* ---------------------------------------------------------------- SpMV */
void ora_spmv(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
              const double *x, double *y) {
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s += v[k] * x[ci[k]];
        y[i] = s;
    }
}

/* ------------------------------------------------ classical strength (a1) */
static int strength(const ora_csr *A, double theta, ora_csr *S) {
    int64_t n = A->n, cnt = 0;
    double *thr = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (!thr) return ORA_ERR_OOM;
    for (int64_t i = 0; i < n; ++i) {
        double m = 0.0;
        for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k)
            if (A->ci[k] != i && fabs(A->v[k]) > m) m = fabs(A->v[k]);
        thr[i] = (m > 0.0) ? theta * m : -1.0;   /* -1: row has no strong entries */
        if (m > 0.0)
            for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k)
                if (A->ci[k] != i && fabs(A->v[k]) >= thr[i]) ++cnt;
    }
    if (csr_alloc(S, n, cnt, 0)) { free(thr); return ORA_ERR_OOM; }
    int64_t pos = 0;
    for (int64_t i = 0; i < n; ++i) {
        S->rp[i] = pos;
        if (thr[i] >= 0.0)
            for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k)
                if (A->ci[k] != i && fabs(A->v[k]) >= thr[i]) S->ci[pos++] = A->ci[k];
    }
    S->rp[n] = pos;
    free(thr);
    return ORA_OK;
}

/* ---------------------------------------------------------- transpose (a2) */
static int transpose_pattern(const ora_csr *S, ora_csr *T) {
    int64_t n = S->n;
    if (csr_alloc(T, n, S->nnz, 0)) return ORA_ERR_OOM;
    for (int64_t k = 0; k < S->nnz; ++k) T->rp[S->ci[k] + 1]++;
    for (int64_t i = 0; i < n; ++i) T->rp[i + 1] += T->rp[i];
    int64_t *fill = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!fill) return ORA_ERR_OOM;
    memcpy(fill, T->rp, (size_t)n * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i)              /* rows ascending -> columns of T ascending */
        for (int64_t k = S->rp[i]; k < S->rp[i + 1]; ++k) T->ci[fill[S->ci[k]]++] = (int32_t)i;
    free(fill);
    return ORA_OK;
}

/* ------------------------------------- RS first pass (a3), lazy max-heap */
typedef struct { int64_t lam; int64_t idx; } heap_item;

static int heap_less(heap_item a, heap_item b) {     /* a has lower priority than b */
    if (a.lam != b.lam) return a.lam < b.lam;
    return a.idx > b.idx;                              /* smaller index wins ties */
}

typedef struct { heap_item *h; int64_t size, cap; } heap_t;

static int heap_push(heap_t *H, heap_item it) {
    if (H->size == H->cap) {
        int64_t nc = H->cap ? 2 * H->cap : 1024;
        heap_item *p = (heap_item *)realloc(H->h, (size_t)nc * sizeof(heap_item));
        if (!p) return ORA_ERR_OOM;
        H->h = p; H->cap = nc;
    }
    int64_t i = H->size++;
    H->h[i] = it;
    while (i > 0) {
        int64_t par = (i - 1) / 2;
        if (!heap_less(H->h[par], H->h[i])) break;
        heap_item t = H->h[par]; H->h[par] = H->h[i]; H->h[i] = t;
        i = par;
    }
    return ORA_OK;
}

static heap_item heap_pop(heap_t *H) {
    heap_item top = H->h[0];
    H->h[0] = H->h[--H->size];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < H->size && heap_less(H->h[m], H->h[l])) m = l;
        if (r < H->size && heap_less(H->h[m], H->h[r])) m = r;
        if (m == i) break;
        heap_item t = H->h[m]; H->h[m] = H->h[i]; H->h[i] = t;
        i = m;
    }
    return top;
}

#define U_PT 2   /* undecided */

/* First pass on the points [lo, hi) with the strength graph restricted to
 * them (the whole graph for lo = 0, hi = n). */
static int rs_first_pass_range(const ora_csr *S, const ora_csr *ST, int8_t *cf, int64_t lo, int64_t hi) {
    int64_t n = S->n;
    int64_t *lam = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    heap_t H = {0};
    if (!lam) return ORA_ERR_OOM;
#define IN_RANGE(x) ((x) >= lo && (x) < hi)
    for (int64_t i = lo; i < hi; ++i) {
        int64_t m = 0, ns = 0;
        for (int64_t a = ST->rp[i]; a < ST->rp[i + 1]; ++a) m += IN_RANGE(ST->ci[a]);
        for (int64_t a = S->rp[i]; a < S->rp[i + 1]; ++a) ns += IN_RANGE(S->ci[a]);
        lam[i] = m;
        int isolated = ns == 0 && m == 0;
        cf[i] = isolated ? 0 : U_PT;
        if (!isolated && heap_push(&H, (heap_item){lam[i], i})) { free(lam); return ORA_ERR_OOM; }
    }
    while (H.size > 0) {
        heap_item it = heap_pop(&H);
        int64_t i = it.idx;
        if (cf[i] != U_PT || it.lam != lam[i]) continue;       /* stale entry */
        if (lam[i] == 0) break;                                 /* largest measure is 0 */
        cf[i] = 1;
        for (int64_t a = ST->rp[i]; a < ST->rp[i + 1]; ++a) {
            int64_t j = ST->ci[a];
            if (!IN_RANGE(j) || cf[j] != U_PT) continue;
            cf[j] = 0;
            for (int64_t b = S->rp[j]; b < S->rp[j + 1]; ++b) {
                int64_t k = S->ci[b];
                if (!IN_RANGE(k) || cf[k] != U_PT) continue;
                lam[k] += 1;
                if (heap_push(&H, (heap_item){lam[k], k})) { free(lam); free(H.h); return ORA_ERR_OOM; }
            }
        }
        for (int64_t a = S->rp[i]; a < S->rp[i + 1]; ++a) {
            int64_t k = S->ci[a];
            if (!IN_RANGE(k) || cf[k] != U_PT) continue;
            lam[k] -= 1;
            if (heap_push(&H, (heap_item){lam[k], k})) { free(lam); free(H.h); return ORA_ERR_OOM; }
        }
    }
#undef IN_RANGE
    for (int64_t i = lo; i < hi; ++i)
        if (cf[i] == U_PT) cf[i] = 0;
    free(lam);
    free(H.h);
    return ORA_OK;
}

static int rs_first_pass(const ora_csr *S, const ora_csr *ST, int8_t *cf) {
    return rs_first_pass_range(S, ST, cf, 0, S->n);
}

/* SplitMix64 (Steele, Lea and Flood, 2014) of x, its top 53 bits as a
 * fraction in [0, 1). */
double ora_hash_frac(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

static int has_strong_c(const ora_csr *S, const int8_t *cf, int64_t i) {
    for (int64_t a = S->rp[i]; a < S->rp[i + 1]; ++a)
        if (cf[S->ci[a]] == 1) return 1;
    return 0;
}

/* Falgout-style splitting with blocks of `block` points (see the header). */
static int falgout_split(const ora_csr *S, const ora_csr *ST, int8_t *cf, int64_t block) {
    int64_t n = S->n;
    for (int64_t lo = 0; lo < n; lo += block) {
        int st = rs_first_pass_range(S, ST, cf, lo, lo + block < n ? lo + block : n);
        if (st) return st;
    }
    int8_t *inU = (int8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    int8_t *sel = (int8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!inU || !sel) { free(inU); free(sel); return ORA_ERR_OOM; }
    int64_t nu = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (cf[i] != 0 || S->rp[i + 1] == S->rp[i] || has_strong_c(S, cf, i)) continue;
        int64_t bi = i / block, cross = 0;
        for (int64_t a = S->rp[i]; a < S->rp[i + 1] && !cross; ++a) cross = S->ci[a] / block != bi;
        for (int64_t a = ST->rp[i]; a < ST->rp[i + 1] && !cross; ++a) cross = ST->ci[a] / block != bi;
        if (cross) { inU[i] = 1; ++nu; }
    }
    while (nu > 0) {
        /* select: weight beats every remaining strong neighbour (either direction) */
        for (int64_t i = 0; i < n; ++i) {
            sel[i] = 0;
            if (!inU[i]) continue;
            double wi = (double)(ST->rp[i + 1] - ST->rp[i]) + ora_hash_frac((uint64_t)i);
            int best = 1;
            for (int pass = 0; pass < 2 && best; ++pass) {
                const ora_csr *G = pass == 0 ? S : ST;
                for (int64_t a = G->rp[i]; a < G->rp[i + 1] && best; ++a) {
                    int64_t j = G->ci[a];
                    if (!inU[j]) continue;
                    double wj = (double)(ST->rp[j + 1] - ST->rp[j]) + ora_hash_frac((uint64_t)j);
                    if (wj > wi || (wj == wi && j < i)) best = 0;
                }
            }
            sel[i] = (int8_t)best;
        }
        for (int64_t i = 0; i < n; ++i)
            if (sel[i]) { cf[i] = 1; inU[i] = 0; --nu; }
        for (int64_t i = 0; i < n; ++i)
            if (inU[i] && has_strong_c(S, cf, i)) { inU[i] = 0; --nu; }
    }
    free(inU);
    free(sel);
    return ORA_OK;
}

/* ----------------------------------------- dense LU used by l-AIR and coarsest */
/* In-place LU of the m x m row-major matrix M with partial pivoting (ties ->
 * smallest row); the row swaps are applied to rhs as they happen.  Returns 1
 * if a pivot falls to <= tol, 0 otherwise. */
static int lu_factor_rhs(double *M, int m, double *rhs, int32_t *perm, double tol) {
    for (int k = 0; k < m; ++k) {
        int p = k;
        double pv = fabs(M[(size_t)k * m + k]);
        for (int r = k + 1; r < m; ++r)
            if (fabs(M[(size_t)r * m + k]) > pv) { pv = fabs(M[(size_t)r * m + k]); p = r; }
        if (pv <= tol) return 1;
        if (perm) perm[k] = p;
        if (p != k) {
            for (int c = 0; c < m; ++c) {
                double t = M[(size_t)k * m + c]; M[(size_t)k * m + c] = M[(size_t)p * m + c]; M[(size_t)p * m + c] = t;
            }
            if (rhs) { double t = rhs[k]; rhs[k] = rhs[p]; rhs[p] = t; }
        }
        double d = M[(size_t)k * m + k];
        for (int r = k + 1; r < m; ++r) {
            double l = M[(size_t)r * m + k] / d;
            M[(size_t)r * m + k] = l;
            for (int c = k + 1; c < m; ++c) {
                double prod = l * M[(size_t)k * m + c];
                M[(size_t)r * m + c] = M[(size_t)r * m + c] - prod;
            }
        }
    }
    return 0;
}

/* Solve L U x = y (y already row-permuted) in place: forward substitution in
 * ascending, back substitution in descending column order. */
static void lu_solve_inplace(const double *M, int m, double *y) {
    for (int r = 0; r < m; ++r) {
        double s = y[r];
        for (int c = 0; c < r; ++c) { double prod = M[(size_t)r * m + c] * y[c]; s = s - prod; }
        y[r] = s;
    }
    for (int r = m - 1; r >= 0; --r) {
        double s = y[r];
        for (int c = m - 1; c > r; --c) { double prod = M[(size_t)r * m + c] * y[c]; s = s - prod; }
        y[r] = s / M[(size_t)r * m + r];
    }
}

/* ------------------------------------------------ l-AIR restriction (a4) */
static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static int64_t find_i32(const int32_t *arr, int64_t m, int32_t key) {
    int64_t lo = 0, hi = m - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (arr[mid] == key) return mid;
        if (arr[mid] < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* Neighbourhood N_i of C point i (sorted, unique) into nb; returns its size. */
static int64_t lair_neighbourhood(const ora_csr *S, const int8_t *cf, int64_t i, int distance,
                                  int32_t *nb, int32_t *mark, int64_t stamp) {
    int64_t m = 0, lo = 0;
    for (int64_t a = S->rp[i]; a < S->rp[i + 1]; ++a) {
        int32_t j = S->ci[a];
        if (cf[j] == 0 && mark[j] != (int32_t)stamp) { mark[j] = (int32_t)stamp; nb[m++] = j; }
    }
    for (int d = 2; d <= distance; ++d) {
        int64_t hi = m;
        for (int64_t t = lo; t < hi; ++t) {
            int32_t k = nb[t];
            for (int64_t a = S->rp[k]; a < S->rp[k + 1]; ++a) {
                int32_t j = S->ci[a];
                if (cf[j] == 0 && mark[j] != (int32_t)stamp) { mark[j] = (int32_t)stamp; nb[m++] = j; }
            }
        }
        if (hi == m) break;
        lo = hi;
    }
    qsort(nb, (size_t)m, sizeof(int32_t), cmp_i32);
    return m;
}

static int build_R(ora_level *L, int distance) {
    const ora_csr *A = &L->A, *S = L->SR.rp ? &L->SR : &L->S;
    int64_t n = A->n;
    int32_t *mark = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t *nb = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!mark || !nb) return ORA_ERR_OOM;
    for (int64_t i = 0; i < n; ++i) mark[i] = -1;
    /* pass 1: sizes */
    int64_t nnz = 0, max_m = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (L->cf[i] != 1) continue;
        int64_t m = lair_neighbourhood(S, L->cf, i, distance, nb, mark, i);
        nnz += m + 1;
        if (m > max_m) max_m = m;
    }
    if (csr_alloc(&L->R, L->nc, nnz, 1)) return ORA_ERR_OOM;
    double *M = (double *)malloc((size_t)(max_m > 0 ? max_m * max_m : 1) * sizeof(double));
    double *z = (double *)malloc((size_t)(max_m > 0 ? max_m : 1) * sizeof(double));
    if (!M || !z) return ORA_ERR_OOM;
    for (int64_t i = 0; i < n; ++i) mark[i] = -1;
    int64_t pos = 0, row = 0;
    L->n_singular = 0;
    L->max_m = (int32_t)max_m;
    for (int64_t i = 0; i < n; ++i) {
        if (L->cf[i] != 1) continue;
        int64_t m = lair_neighbourhood(S, L->cf, i, distance, nb, mark, n + i);
        /* M[a][b] = A(N[b], N[a])  i.e. M = A_ff(N, N)^T ; rhs = -A(i, N)^T */
        memset(M, 0, (size_t)(m * m) * sizeof(double));
        double mx = 0.0;
        for (int64_t bcol = 0; bcol < m; ++bcol) {
            int64_t r = nb[bcol];
            for (int64_t k = A->rp[r]; k < A->rp[r + 1]; ++k) {
                int64_t a = find_i32(nb, m, A->ci[k]);
                if (a < 0) continue;
                M[a * m + bcol] = A->v[k];
                if (fabs(A->v[k]) > mx) mx = fabs(A->v[k]);
            }
        }
        for (int64_t a = 0; a < m; ++a) z[a] = -csr_get(A, i, nb[a]);
        if (m > 0) {
            int sing = lu_factor_rhs(M, (int)m, z, NULL, 1e-14 * mx);
            if (sing) {
                for (int64_t a = 0; a < m; ++a) z[a] = 0.0;
                L->n_singular++;
            } else {
                lu_solve_inplace(M, (int)m, z);
            }
        }
        /* R row: sorted N_i union {i} */
        L->R.rp[row] = pos;
        int placed = 0;
        for (int64_t a = 0; a < m; ++a) {
            if (!placed && nb[a] > i) { L->R.ci[pos] = (int32_t)i; L->R.v[pos++] = 1.0; placed = 1; }
            L->R.ci[pos] = nb[a]; L->R.v[pos++] = z[a];
        }
        if (!placed) { L->R.ci[pos] = (int32_t)i; L->R.v[pos++] = 1.0; }
        ++row;
    }
    L->R.rp[row] = pos;
    free(M); free(z); free(mark); free(nb);
    return ORA_OK;
}

/* ------------------------------------------------- one-point P (a5) */
static void build_P(ora_level *L) {
    const ora_csr *A = &L->A, *S = &L->S;
    for (int64_t i = 0; i < A->n; ++i) {
        if (L->cf[i] == 1) { L->pcol[i] = L->cid[i]; L->pw[i] = 1.0; continue; }
        int64_t best = -1;
        double bv = -1.0;
        for (int64_t a = S->rp[i]; a < S->rp[i + 1]; ++a) {
            int32_t j = S->ci[a];
            if (L->cf[j] != 1) continue;
            double v = fabs(csr_get(A, i, j));
            if (v > bv) { bv = v; best = j; }
        }
        L->pcol[i] = best >= 0 ? L->cid[best] : -1;
        L->pw[i] = best >= 0 ? 1.0 : 0.0;
    }
}

/* --------------------------------------------------------- RAP (a6) */
static int galerkin(const ora_level *L, ora_csr *Ac) {
    const ora_csr *A = &L->A, *R = &L->R;
    int64_t n = A->n, nc = L->nc;
    double *acc = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    int32_t *seen = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t *list = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    double *acc2 = (double *)calloc((size_t)(nc > 0 ? nc : 1), sizeof(double));
    int32_t *seen2 = (int32_t *)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(int32_t));
    int32_t *list2 = (int32_t *)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(int32_t));
    if (!acc || !seen || !list || !acc2 || !seen2 || !list2) return ORA_ERR_OOM;
    for (int64_t j = 0; j < n; ++j) seen[j] = -1;
    for (int64_t j = 0; j < nc; ++j) seen2[j] = -1;
    int64_t cap = 1024, nnz = 0;
    int32_t *ci = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    double *v = (double *)malloc((size_t)cap * sizeof(double));
    int64_t *rp = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
    if (!ci || !v || !rp) return ORA_ERR_OOM;
    for (int64_t i = 0; i < nc; ++i) {
        int64_t m = 0, m2 = 0;
        for (int64_t a = R->rp[i]; a < R->rp[i + 1]; ++a) {     /* k ascending */
            int64_t k = R->ci[a];
            double rik = R->v[a];
            for (int64_t b = A->rp[k]; b < A->rp[k + 1]; ++b) {
                int32_t j = A->ci[b];
                if (seen[j] != (int32_t)i) { seen[j] = (int32_t)i; acc[j] = 0.0; list[m++] = j; }
                double prod = rik * A->v[b];
                acc[j] = acc[j] + prod;
            }
        }
        qsort(list, (size_t)m, sizeof(int32_t), cmp_i32);
        for (int64_t t = 0; t < m; ++t) {                         /* j ascending */
            int32_t j = list[t];
            int32_t J = L->pcol[j];
            if (J < 0) continue;
            if (seen2[J] != (int32_t)i) { seen2[J] = (int32_t)i; acc2[J] = 0.0; list2[m2++] = J; }
            double prod = acc[j] * L->pw[j];
            acc2[J] = acc2[J] + prod;
        }
        qsort(list2, (size_t)m2, sizeof(int32_t), cmp_i32);
        if (nnz + m2 > cap) {
            while (nnz + m2 > cap) cap *= 2;
            ci = (int32_t *)realloc(ci, (size_t)cap * sizeof(int32_t));
            v = (double *)realloc(v, (size_t)cap * sizeof(double));
            if (!ci || !v) return ORA_ERR_OOM;
        }
        for (int64_t t = 0; t < m2; ++t) { ci[nnz] = list2[t]; v[nnz] = acc2[list2[t]]; ++nnz; }
        rp[i + 1] = nnz;
    }
    Ac->n = nc; Ac->nnz = nnz; Ac->rp = rp; Ac->ci = ci; Ac->v = v;
    free(acc); free(seen); free(list); free(acc2); free(seen2); free(list2);
    return ORA_OK;
}

/* ------------------------------------------------------- setup (a1-a7) */
void ora_free(ora_hier *H);

ora_hier *ora_setup(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                    double theta, double theta_r, int distance, int max_coarse, int max_levels,
                    int max_dense, const char *relax, double omega, int64_t falgout_block, int *status) {
    *status = ORA_OK;
    if (n <= 0 || max_levels < 1 || max_levels > ORA_MAX_LEVELS || distance < 1) { *status = ORA_ERR_ARG; return NULL; }
    ora_hier *H = (ora_hier *)calloc(1, sizeof(ora_hier));
    if (!H) { *status = ORA_ERR_OOM; return NULL; }
    H->omega = omega;
    strncpy(H->relax, relax ? relax : "FCF", sizeof(H->relax) - 1);
    ora_level *L0 = &H->lev[0];
    int64_t nnz = rp[n];
    if (csr_alloc(&L0->A, n, nnz, 1)) { *status = ORA_ERR_OOM; return H; }
    memcpy(L0->A.rp, rp, (size_t)(n + 1) * sizeof(int64_t));
    memcpy(L0->A.ci, ci, (size_t)nnz * sizeof(int32_t));
    memcpy(L0->A.v, v, (size_t)nnz * sizeof(double));
    int l = 0;
    for (;;) {
        ora_level *L = &H->lev[l];
        int64_t nl = L->A.n;
        H->nlev = l + 1;
        if (nl <= max_coarse || l == max_levels - 1) break;
        if ((*status = strength(&L->A, theta, &L->S))) return H;
        if ((*status = transpose_pattern(&L->S, &L->ST))) return H;
        L->cf = (int8_t *)malloc((size_t)nl);
        L->cid = (int32_t *)malloc((size_t)nl * sizeof(int32_t));
        if (!L->cf || !L->cid) { *status = ORA_ERR_OOM; return H; }
        if (falgout_block > 0) {
            if ((*status = falgout_split(&L->S, &L->ST, L->cf, falgout_block))) return H;
        } else if ((*status = rs_first_pass(&L->S, &L->ST, L->cf))) {
            return H;
        }
        int64_t nc = 0;
        for (int64_t i = 0; i < nl; ++i) L->cid[i] = L->cf[i] == 1 ? (int32_t)nc++ : -1;
        L->nc = nc;
        if (nc == 0 || (double)nc > 0.9 * (double)nl) {
            /* coarsening stalled: this level is the coarsest */
            csr_free(&L->S); csr_free(&L->ST);
            free(L->cf); free(L->cid); L->cf = NULL; L->cid = NULL; L->nc = 0;
            break;
        }
        if (theta_r >= 0.0 && theta_r != theta && (*status = strength(&L->A, theta_r, &L->SR))) return H;
        if ((*status = build_R(L, distance))) return H;
        L->pcol = (int32_t *)malloc((size_t)nl * sizeof(int32_t));
        L->pw = (double *)malloc((size_t)nl * sizeof(double));
        if (!L->pcol || !L->pw) { *status = ORA_ERR_OOM; return H; }
        build_P(L);
        if ((*status = galerkin(L, &H->lev[l + 1].A))) return H;
        ++l;
    }
    /* coarsest: dense LU */
    ora_level *Lc = &H->lev[H->nlev - 1];
    int64_t m = Lc->A.n;
    if (m > max_dense) { *status = ORA_ERR_COARSE; return H; }
    H->lu = (double *)calloc((size_t)(m * m), sizeof(double));
    H->piv = (int32_t *)malloc((size_t)m * sizeof(int32_t));
    if (!H->lu || !H->piv) { *status = ORA_ERR_OOM; return H; }
    double mx = 0.0;
    for (int64_t i = 0; i < m; ++i)
        for (int64_t k = Lc->A.rp[i]; k < Lc->A.rp[i + 1]; ++k) {
            H->lu[i * m + Lc->A.ci[k]] = Lc->A.v[k];
            if (fabs(Lc->A.v[k]) > mx) mx = fabs(Lc->A.v[k]);
        }
    if (lu_factor_rhs(H->lu, (int)m, NULL, H->piv, 1e-14 * mx)) *status = ORA_ERR_COARSE;
    return H;
}

void ora_free(ora_hier *H) {
    if (!H) return;
    for (int l = 0; l < ORA_MAX_LEVELS; ++l) {
        ora_level *L = &H->lev[l];
        csr_free(&L->A); csr_free(&L->S); csr_free(&L->ST); csr_free(&L->SR); csr_free(&L->R);
        free(L->cf); free(L->cid); free(L->pcol); free(L->pw);
    }
    free(H->lu); free(H->piv);
    free(H);
}

/* ---------------------------------------------------------- V-cycle (a9) */
static void coarse_solve(const ora_hier *H, const double *b, double *x) {
    int64_t m = H->lev[H->nlev - 1].A.n;
    memcpy(x, b, (size_t)m * sizeof(double));
    for (int64_t k = 0; k < m; ++k) {                 /* replay the row swaps */
        int32_t p = H->piv[k];
        if (p != k) { double t = x[k]; x[k] = x[p]; x[p] = t; }
    }
    lu_solve_inplace(H->lu, (int)m, x);
}

/* which: 0 = F points, 1 = C points, 2 = all points; every update from the old x */
static void jacobi_sweep(const ora_csr *A, const int8_t *cf, int which, double omega,
                         const double *b, double *x, double *tmp) {
    for (int64_t i = 0; i < A->n; ++i) {
        tmp[i] = x[i];
        if (which != 2 && cf[i] != which) continue;
        double r = b[i], d = 0.0;
        for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
            if (A->ci[k] == i) d = A->v[k];
            r -= A->v[k] * x[A->ci[k]];
        }
        tmp[i] = x[i] + omega * r / d;
    }
    memcpy(x, tmp, (size_t)A->n * sizeof(double));
}

/* which: 0 = F points, 1 = C points, 2 = all points; in place, ascending index */
static void gauss_seidel_sweep(const ora_csr *A, const int8_t *cf, int which, double omega,
                               const double *b, double *x) {
    for (int64_t i = 0; i < A->n; ++i) {
        if (which != 2 && cf[i] != which) continue;
        double r = b[i], d = 0.0;
        for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
            if (A->ci[k] == i) d = A->v[k];
            r -= A->v[k] * x[A->ci[k]];
        }
        x[i] = x[i] + omega * r / d;
    }
}

static void vcycle_level(const ora_hier *H, int l, const double *b, double *x) {
    if (l == H->nlev - 1) { coarse_solve(H, b, x); return; }
    const ora_level *L = &H->lev[l];
    int64_t n = L->A.n, nc = L->nc;
    double *bc = (double *)malloc((size_t)nc * sizeof(double));
    double *xc = (double *)calloc((size_t)nc, sizeof(double));
    double *tmp = (double *)malloc((size_t)n * sizeof(double));
    for (int64_t i = 0; i < nc; ++i) {                /* b_c = R b */
        double s = 0.0;
        for (int64_t k = L->R.rp[i]; k < L->R.rp[i + 1]; ++k) s += L->R.v[k] * b[L->R.ci[k]];
        bc[i] = s;
    }
    vcycle_level(H, l + 1, bc, xc);
    for (int64_t i = 0; i < n; ++i)                   /* x = P x_c */
        x[i] = L->pcol[i] >= 0 ? L->pw[i] * xc[L->pcol[i]] : 0.0;
    for (const char *c = H->relax; *c; ++c) {
        int which = (*c == 'C' || *c == 'c') ? 1 : (*c == 'A' || *c == 'a') ? 2 : 0;
        if (*c >= 'a') gauss_seidel_sweep(&L->A, L->cf, which, H->omega, b, x);
        else jacobi_sweep(&L->A, L->cf, which, H->omega, b, x, tmp);
    }
    free(bc); free(xc); free(tmp);
}

void ora_vcycle(const ora_hier *H, const double *b, double *x) { vcycle_level(H, 0, b, x); }

/* ------------------------------------------------------------ GMRES (a10) */
static double dot(int64_t n, const double *a, const double *b) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Returns 0 if converged, 1 if not; iters = total inner steps; resid history
 * (Givens estimates, relative) written to hist[0..iters] if hist != NULL. */
int ora_gmres(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
              const ora_hier *H, const double *b, double *x, double rtol, int restart,
              int max_iter, int *iters, double *relres, double *hist) {
    int m = restart;
    double *V = (double *)malloc((size_t)(m + 1) * n * sizeof(double));
    double *Z = (double *)malloc((size_t)m * n * sizeof(double));
    double *w = (double *)malloc((size_t)n * sizeof(double));
    double *Hh = (double *)calloc((size_t)(m + 1) * m, sizeof(double));
    double *cs = (double *)malloc((size_t)m * sizeof(double));
    double *sn = (double *)malloc((size_t)m * sizeof(double));
    double *g = (double *)malloc((size_t)(m + 1) * sizeof(double));
    double *y = (double *)malloc((size_t)m * sizeof(double));
    int it = 0, conv = 0;
    double bn = sqrt(dot(n, b, b));
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    if (bn == 0.0) { *iters = 0; *relres = 0.0; conv = 1; goto done; }
    if (hist) hist[0] = 1.0;
    for (;;) {
        ora_spmv(n, rp, ci, v, x, w);
        for (int64_t i = 0; i < n; ++i) w[i] = b[i] - w[i];
        double beta = sqrt(dot(n, w, w));
        *relres = beta / bn;
        if (*relres <= rtol) { conv = 1; break; }
        if (it >= max_iter) break;
        for (int64_t i = 0; i < n; ++i) V[i] = w[i] / beta;
        memset(g, 0, (size_t)(m + 1) * sizeof(double));
        g[0] = beta;
        int j, k = 0;
        for (j = 0; j < m && it < max_iter; ++j) {
            double *vj = V + (size_t)j * n, *zj = Z + (size_t)j * n;
            if (H) ora_vcycle(H, vj, zj); else memcpy(zj, vj, (size_t)n * sizeof(double));
            ora_spmv(n, rp, ci, v, zj, w);
            for (int i = 0; i <= j; ++i) {                        /* modified Gram-Schmidt */
                double h = dot(n, w, V + (size_t)i * n);
                Hh[i * m + j] = h;
                for (int64_t t = 0; t < n; ++t) w[t] -= h * V[(size_t)i * n + t];
            }
            double hn = sqrt(dot(n, w, w));
            Hh[(j + 1) * m + j] = hn;
            if (hn > 0.0)
                for (int64_t t = 0; t < n; ++t) V[(size_t)(j + 1) * n + t] = w[t] / hn;
            for (int i = 0; i < j; ++i) {                         /* previous rotations */
                double a = Hh[i * m + j], c = Hh[(i + 1) * m + j];
                Hh[i * m + j] = cs[i] * a + sn[i] * c;
                Hh[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
            }
            double a = Hh[j * m + j], c = Hh[(j + 1) * m + j];
            double r = hypot(a, c);
            cs[j] = r > 0.0 ? a / r : 1.0;
            sn[j] = r > 0.0 ? c / r : 0.0;
            Hh[j * m + j] = r;
            Hh[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++it;
            k = j + 1;
            if (hist) hist[it] = fabs(g[j + 1]) / bn;
            if (fabs(g[j + 1]) / bn <= rtol || hn == 0.0) break;
        }
        for (int i = k - 1; i >= 0; --i) {                        /* H y = g */
            double s = g[i];
            for (int c2 = i + 1; c2 < k; ++c2) s -= Hh[i * m + c2] * y[c2];
            y[i] = s / Hh[i * m + i];
        }
        for (int i = 0; i < k; ++i)
            for (int64_t t = 0; t < n; ++t) x[t] += y[i] * Z[(size_t)i * n + t];
    }
done:
    *iters = it;
    free(V); free(Z); free(w); free(Hh); free(cs); free(sn); free(g); free(y);
    return conv ? 0 : 1;
}

/* ------------------------------------------------------------ BiCGSTAB */
/* Right-preconditioned BiCGSTAB (van der Vorst, 1992), the Krylov method the
 * paper pairs with AIR (Section 5.1, Table 2): M^{-1} = one V-cycle (identity
 * when H is NULL), x0 = 0, shadow residual r^ = r0.  Per iteration:
 *   rho = (r^, r); beta = (rho / rho_prev)(alpha / omega);
 *   p = r + beta (p - omega v); p^ = M^{-1} p; v = A p^; alpha = rho / (r^, v);
 *   s = r - alpha v; s^ = M^{-1} s; t = A s^; omega = (t, s) / (t, t);
 *   x += alpha p^ + omega s^; r = s - omega t.
 * Stop when ||r|| / ||b|| <= rtol and the true residual b - A x agrees; if the
 * true residual is still above rtol the iteration restarts from it (r^ = r,
 * p = v = 0, rho_prev = alpha = omega = 1).  rho = 0, (r^, v) = 0 or omega = 0
 * end the solve unconverged.  iters counts iterations (two V-cycles each);
 * relres is the true relative residual at exit.  Returns 0 if converged. */
int ora_bicgstab(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                 const ora_hier *H, const double *b, double *x, double rtol, int max_iter,
                 int *iters, double *relres) {
    double *r = (double *)malloc((size_t)n * sizeof(double));
    double *rh = (double *)malloc((size_t)n * sizeof(double));
    double *p = (double *)calloc((size_t)n, sizeof(double));
    double *vv = (double *)calloc((size_t)n, sizeof(double));
    double *ph = (double *)malloc((size_t)n * sizeof(double));
    double *s = (double *)malloc((size_t)n * sizeof(double));
    double *sh = (double *)malloc((size_t)n * sizeof(double));
    double *t = (double *)malloc((size_t)n * sizeof(double));
    int it = 0, conv = 0;
    double bn = sqrt(dot(n, b, b));
    for (int64_t i = 0; i < n; ++i) { x[i] = 0.0; r[i] = b[i]; rh[i] = b[i]; }
    *relres = 0.0;
    if (bn == 0.0) { conv = 1; goto done; }
    *relres = 1.0;
    double rho_prev = 1.0, alpha = 1.0, omega = 1.0;
    while (it < max_iter) {
        double rho = dot(n, rh, r);
        if (rho == 0.0) break;
        double beta = (rho / rho_prev) * (alpha / omega);
        for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * vv[i]);
        if (H) ora_vcycle(H, p, ph); else memcpy(ph, p, (size_t)n * sizeof(double));
        ora_spmv(n, rp, ci, v, ph, vv);
        double den = dot(n, rh, vv);
        if (den == 0.0) break;
        alpha = rho / den;
        for (int64_t i = 0; i < n; ++i) s[i] = r[i] - alpha * vv[i];
        if (H) ora_vcycle(H, s, sh); else memcpy(sh, s, (size_t)n * sizeof(double));
        ora_spmv(n, rp, ci, v, sh, t);
        double tt = dot(n, t, t), ts = dot(n, t, s);
        omega = tt > 0.0 ? ts / tt : 0.0;
        for (int64_t i = 0; i < n; ++i) x[i] += alpha * ph[i] + omega * sh[i];
        for (int64_t i = 0; i < n; ++i) r[i] = s[i] - omega * t[i];
        rho_prev = rho;
        ++it;
        if (sqrt(dot(n, r, r)) / bn <= rtol) {
            ora_spmv(n, rp, ci, v, x, t);                       /* true residual */
            for (int64_t i = 0; i < n; ++i) r[i] = b[i] - t[i];
            *relres = sqrt(dot(n, r, r)) / bn;
            if (*relres <= rtol) { conv = 1; break; }
            for (int64_t i = 0; i < n; ++i) { rh[i] = r[i]; p[i] = 0.0; vv[i] = 0.0; }
            rho_prev = alpha = omega = 1.0;
            continue;
        }
        if (omega == 0.0) break;
    }
    if (!conv) {
        ora_spmv(n, rp, ci, v, x, t);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - t[i];
        *relres = sqrt(dot(n, r, r)) / bn;
    }
done:
    *iters = it;
    free(r); free(rh); free(p); free(vv); free(ph); free(s); free(sh); free(t);
    return conv ? 0 : 1;
}

/* ------------------------------------------------------------ accessors */
int ora_nlevels(const ora_hier *H) { return H ? H->nlev : 0; }

/* info: n, nnz(A), nnz(S), nc, nnz(R), n_singular, max_m */
void ora_level_info(const ora_hier *H, int l, int64_t *info) {
    const ora_level *L = &H->lev[l];
    info[0] = L->A.n; info[1] = L->A.nnz; info[2] = L->S.nnz; info[3] = L->nc;
    info[4] = L->R.nnz; info[5] = L->n_singular; info[6] = L->max_m;
}

/* what: 0 A.rp 1 A.ci 2 A.v 3 S.rp 4 S.ci 5 cf 6 cid 7 R.rp 8 R.ci 9 R.v 10 pcol 11 pw */
int ora_level_copy(const ora_hier *H, int l, int what, void *dst) {
    const ora_level *L = &H->lev[l];
    int64_t n = L->A.n;
    switch (what) {
    case 0: memcpy(dst, L->A.rp, (size_t)(n + 1) * 8); break;
    case 1: memcpy(dst, L->A.ci, (size_t)L->A.nnz * 4); break;
    case 2: memcpy(dst, L->A.v, (size_t)L->A.nnz * 8); break;
    case 3: if (!L->S.rp) return -1; memcpy(dst, L->S.rp, (size_t)(n + 1) * 8); break;
    case 4: if (!L->S.rp) return -1; memcpy(dst, L->S.ci, (size_t)L->S.nnz * 4); break;
    case 5: if (!L->cf) return -1; memcpy(dst, L->cf, (size_t)n); break;
    case 6: if (!L->cid) return -1; memcpy(dst, L->cid, (size_t)n * 4); break;
    case 7: if (!L->R.rp) return -1; memcpy(dst, L->R.rp, (size_t)(L->nc + 1) * 8); break;
    case 8: if (!L->R.rp) return -1; memcpy(dst, L->R.ci, (size_t)L->R.nnz * 4); break;
    case 9: if (!L->R.rp) return -1; memcpy(dst, L->R.v, (size_t)L->R.nnz * 8); break;
    case 10: if (!L->pcol) return -1; memcpy(dst, L->pcol, (size_t)n * 4); break;
    case 11: if (!L->pw) return -1; memcpy(dst, L->pw, (size_t)n * 8); break;
    default: return -1;
    }
    return 0;
}
