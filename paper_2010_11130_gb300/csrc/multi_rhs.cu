// Many right-hand sides through one hierarchy at once.
//
// The V-cycle (Section 3: restriction of b, coarsest solve, one-point
// interpolation, FCF-Jacobi sweeps) is bandwidth-bound: one right-hand side
// reads every stored entry of every level for a few flops.  With k right-hand
// sides stored row-major (row i holds x_i of all k systems, k <= 32) one warp
// handles one matrix row: lane j carries system j, the row's entries are read
// once (coalesced, then broadcast by shuffles) and serve all k systems, and
// the gathered x rows are k contiguous values.  The matrix traffic of one
// V-cycle is shared by k systems.
//
// Every kernel sums a row in the CSR entry order with fused multiply-adds,
// like the single-right-hand-side SELL kernels, so column j of the result is
// the FP64 V-cycle of column j.
#include <string.h>

#include "air_internal.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int MK = 32;                // largest k
constexpr int MR_SPMV = 0, MR_RESID = 1, MR_JACOBI = 2;

unsigned grid_for(int64_t items, int threads, int64_t cap = 152 * 32) {
    int64_t b = (items + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

// One warp per listed row (rows == NULL: row p itself).
//  MR_SPMV:   Y[row] = A_row X
//  MR_RESID:  Y[row] = B[row] - A_row X
//  MR_JACOBI: Y[p]   = X[row] + omega (B[row] - A_row X) / a_row,row   (compact; scattered afterwards)
template <int MODE, typename T>
__global__ void __launch_bounds__(256) csr_multi_kernel(int64_t m, const int32_t *__restrict__ rows,
                                                        const int64_t *__restrict__ rp,
                                                        const int32_t *__restrict__ ci,
                                                        const T *__restrict__ v, int k,
                                                        const T *__restrict__ X, T *__restrict__ Y,
                                                        const T *__restrict__ B,
                                                        const T *__restrict__ dinv, T omega) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < m; p += nw) {
        const int64_t row = rows ? (int64_t)rows[p] : p;
        const int64_t e0 = rp[row], e1 = rp[row + 1];
        T acc = 0;
        for (int64_t base = e0; base < e1; base += 32) {
            const int64_t e = base + lane;
            const int32_t ce = e < e1 ? ci[e] : 0;
            const T ve = e < e1 ? v[e] : (T)0;
            const int cnt = (int)(e1 - base < 32 ? e1 - base : 32);
            for (int t = 0; t < cnt; ++t) {
                const int32_t c = __shfl_sync(FULL, ce, t);
                const T w = __shfl_sync(FULL, ve, t);
                if (lane < k) acc += w * X[(int64_t)c * k + lane];
            }
        }
        if (lane < k) {
            if (MODE == MR_SPMV) {
                Y[row * k + lane] = acc;
            } else if (MODE == MR_RESID) {
                Y[row * k + lane] = B[row * k + lane] - acc;
            } else {
                Y[p * k + lane] = X[row * k + lane] + omega * (B[row * k + lane] - acc) * dinv[row];
            }
        }
    }
}

template <typename T>
__global__ void scatter_multi_kernel(int64_t m, const int32_t *rows, int k, const T *Tc, T *X) {
    const int64_t tot = m * k;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = q / k;
        X[(int64_t)rows[p] * k + (q - p * k)] = Tc[q];
    }
}

template <typename T>
__global__ void interp_multi_kernel(int64_t n, const int32_t *pcol, int k, const T *XC, T *X) {
    const int64_t tot = n * k;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q / k;
        const int32_t pc = pcol[i];
        X[q] = pc >= 0 ? XC[(int64_t)pc * k + (q - i * k)] : (T)0;
    }
}

// X = Cinv B on the coarsest level (Cinv row-major m x m), one warp per row
template <typename T>
__global__ void dense_multi_kernel(int64_t m, const T *__restrict__ Ci, int k, const T *__restrict__ B,
                                   T *__restrict__ X) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < m; r += nw) {
        T acc = 0;
        for (int64_t c0 = 0; c0 < m; c0 += 32) {
            const T cv = c0 + lane < m ? Ci[r * m + c0 + lane] : (T)0;
            const int cnt = (int)(m - c0 < 32 ? m - c0 : 32);
            for (int t = 0; t < cnt; ++t) {
                const T w = __shfl_sync(FULL, cv, t);
                if (lane < k) acc += w * B[(c0 + t) * k + lane];
            }
        }
        if (lane < k) X[r * k + lane] = acc;
    }
}

// partial column dots: part[blk * 2k + d * k + j] = sum over this block's rows of U_ij W_ij
// (d = 0) and, with U2, U2_ij W_ij (d = 1)
constexpr int DT = 256;
__global__ void __launch_bounds__(DT) coldot_kernel(int64_t n, int k, const double *__restrict__ U,
                                                    const double *__restrict__ U2, const double *__restrict__ W,
                                                    double *__restrict__ part) {
    __shared__ double red[2][DT / 32][MK];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double a0 = 0.0, a1 = 0.0;
    if (lane < k) {
        for (int64_t i = (int64_t)blockIdx.x * (DT / 32) + wid; i < n; i += (int64_t)gridDim.x * (DT / 32)) {
            const double w = W[i * k + lane];
            a0 += U[i * k + lane] * w;
            if (U2) a1 += U2[i * k + lane] * w;
        }
    }
    red[0][wid][lane] = a0;
    red[1][wid][lane] = a1;
    __syncthreads();
    if (threadIdx.x < 2 * MK) {
        const int d = threadIdx.x / MK, j = threadIdx.x % MK;
        double s = 0.0;
        for (int q = 0; q < DT / 32; ++q) s += red[d][q][j];
        if (j < k) part[(int64_t)blockIdx.x * 2 * k + d * k + j] = s;
    }
}

__global__ void coldot_reduce_kernel(int nblk, int k, const double *part, double *out) {
    const int t = threadIdx.x;   // 2k threads
    if (t >= 2 * k) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * 2 * k + t];
    out[t] = s;
}

// out = ca_j a + cb_j b (+ cc_j c), coefficients per column j
__global__ void lincomb_multi_kernel(int64_t n, int k, double *out, const double *a, const double *ca,
                                     const double *b, const double *cb, const double *c, const double *cc) {
    const int64_t tot = n * k;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(q % k);
        double v = ca[j] * a[q] + cb[j] * b[q];
        if (c) v += cc[j] * c[q];
        out[q] = v;
    }
}

__global__ void d2f_multi_kernel(int64_t tot, const double *in, float *out) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x)
        out[q] = (float)in[q];
}

__global__ void f2d_multi_kernel(int64_t tot, const float *in, double *out) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x)
        out[q] = (double)in[q];
}

// columns j with mask[j] != 0: dst_j = src_j
__global__ void copy_cols_kernel(int64_t n, int k, const int *mask, const double *src, double *dst) {
    const int64_t tot = n * k;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x)
        if (mask[q % k]) dst[q] = src[q];
}

template <int MODE, typename T>
void csr_multi(int64_t m, const int32_t *rows, const int64_t *rp, const int32_t *ci, const T *v, int k, const T *X,
               T *Y, const T *B, const T *dinv, T omega, cudaStream_t s) {
    if (m <= 0) return;
    csr_multi_kernel<MODE, T><<<air_counted(grid_for(m * 32, 256)), 256, 0, s>>>(m, rows, rp, ci, v, k, X, Y, B,
                                                                                dinv, omega);
}

// the V-cycle buffers only: the Krylov vectors of a solve in progress stay
void free_vcycle_multi(air_hierarchy *H) {
    for (int l = 0; l < AIR_MAX_LEVELS; ++l) {
        air_dfree(H->mb[l]);
        air_dfree(H->mx[l]);
        air_dfree(H->mt[l]);
        H->mb[l] = H->mx[l] = H->mt[l] = nullptr;
    }
    H->mk = 0;
}

int ensure_multi(air_hierarchy *H, int k) {
    if (H->mk == k) return AIR_OK;
    free_vcycle_multi(H);
    for (int l = 0; l < H->nlev; ++l) {
        const AirLevel &L = H->lev[l];
        const int64_t n = L.n > 0 ? L.n : 1;
        const int64_t mt = (L.nf > L.nc ? L.nf : L.nc) > 0 ? (L.nf > L.nc ? L.nf : L.nc) : 1;
        AIR_CUDA(air_dmalloc((void **)&H->mb[l], (size_t)n * k * sizeof(double)));
        AIR_CUDA(air_dmalloc((void **)&H->mx[l], (size_t)n * k * sizeof(double)));
        AIR_CUDA(air_dmalloc((void **)&H->mt[l], (size_t)mt * k * sizeof(double)));
    }
    H->mk = k;
    return AIR_OK;
}

// FP32 copies of the level operators, R, 1 / a_ii and the coarsest inverse
// (round to nearest from the FP64 hierarchy) for the FP32 multi V-cycle
int ensure_multi32(air_hierarchy *H, cudaStream_t s) {
    if (H->m32) return AIR_OK;
    for (int l = 0; l < H->nlev; ++l) {
        AirLevel &L = H->lev[l];
        AIR_CUDA(air_dmalloc((void **)&H->mv32[l], (size_t)(L.nnz > 0 ? L.nnz : 1) * sizeof(float)));
        AIR_TRY(air_cast_d2f(L.v, H->mv32[l], L.nnz, s));
        AIR_CUDA(air_dmalloc((void **)&H->md32[l], (size_t)(L.n > 0 ? L.n : 1) * sizeof(float)));
        if (L.dinv) AIR_TRY(air_cast_d2f(L.dinv, H->md32[l], L.n, s));
        if (l + 1 < H->nlev) {
            AIR_CUDA(air_dmalloc((void **)&H->mr32[l], (size_t)(L.nnz_r > 0 ? L.nnz_r : 1) * sizeof(float)));
            AIR_TRY(air_cast_d2f(L.rv, H->mr32[l], L.nnz_r, s));
        }
    }
    AIR_CUDA(air_dmalloc((void **)&H->mc32, (size_t)(H->nco > 0 ? H->nco * H->nco : 1) * sizeof(float)));
    AIR_TRY(air_cast_d2f(H->cinv, H->mc32, H->nco * H->nco, s));
    H->m32 = 1;
    return AIR_OK;
}

}  // namespace

void air_free_multi(air_hierarchy *H) {
    free_vcycle_multi(H);
    for (int l = 0; l < AIR_MAX_LEVELS; ++l) {
        air_dfree(H->mv32[l]);
        air_dfree(H->md32[l]);
        air_dfree(H->mr32[l]);
        H->mv32[l] = H->md32[l] = H->mr32[l] = nullptr;
    }
    air_dfree(H->mc32);
    H->mc32 = nullptr;
    H->m32 = 0;
    air_dfree(H->mkry);
    H->mkry = nullptr;
    H->mkry_n = 0;
}

// x = M^{-1} b for k columns, the V-cycle of vcycle_t column by column: in
// FP64 on the FP64 hierarchy data, or in FP32 on its round-to-nearest copies
// (the level vectors reuse the FP64 buffers)
template <typename T>
int vcycle_multi_t(air_hierarchy *H, int k, const T *b0, T *x0, cudaStream_t s) {
    constexpr bool F = sizeof(T) == 4;
    AIR_TRY(ensure_multi(H, k));
    if (F) AIR_TRY(ensure_multi32(H, s));
    const int L = H->nlev;
    const char *relax = H->opt.relax;
    const int ns = (int)strnlen(relax, sizeof(H->opt.relax));
    const T omega = (T)H->opt.omega;
    auto vals = [&](int l) { return F ? (const T *)H->mv32[l] : (const T *)H->lev[l].v; };
    auto rvals = [&](int l) { return F ? (const T *)H->mr32[l] : (const T *)H->lev[l].rv; };
    auto dinv = [&](int l) { return F ? (const T *)H->md32[l] : (const T *)H->lev[l].dinv; };
    auto mb = [&](int l) { return (T *)H->mb[l]; };
    auto mx = [&](int l) { return (T *)H->mx[l]; };
    for (int l = 0; l + 1 < L; ++l) {                      // restriction of b
        const AirLevel &A = H->lev[l];
        const T *bl = l == 0 ? b0 : mb(l);
        csr_multi<MR_SPMV, T>(A.nc, nullptr, A.rrp, A.rci, rvals(l), k, bl, mb(l + 1), nullptr, nullptr, (T)0, s);
    }
    {                                                      // coarsest
        const AirLevel &C = H->lev[L - 1];
        const T *bl = L == 1 ? b0 : mb(L - 1);
        T *xl = L == 1 ? x0 : mx(L - 1);
        const T *Ci = F ? (const T *)H->mc32 : (const T *)H->cinv;
        dense_multi_kernel<T><<<air_counted(grid_for(C.n * 32, 256, 152 * 8)), 256, 0, s>>>(C.n, Ci, k, bl, xl);
    }
    for (int l = L - 2; l >= 0; --l) {                     // interpolation and sweeps
        const AirLevel &A = H->lev[l];
        const T *bl = l == 0 ? b0 : mb(l);
        T *out = l == 0 ? x0 : mx(l);
        interp_multi_kernel<T><<<air_counted(grid_for(A.n * k, 256)), 256, 0, s>>>(A.n, A.pcol, k, mx(l + 1), out);
        for (int q = 0; q < ns; ++q) {
            const bool c = relax[q] == 'C';
            const int64_t m = c ? A.nc : A.nf;
            const int32_t *rows = c ? A.crows : A.frows;
            if (m <= 0) continue;
            T *tl = (T *)H->mt[l];
            csr_multi<MR_JACOBI, T>(m, rows, A.rp, A.ci, vals(l), k, out, tl, bl, dinv(l), omega, s);
            scatter_multi_kernel<T><<<air_counted(grid_for(m * k, 256)), 256, 0, s>>>(m, rows, k, tl, out);
        }
    }
    AIR_LAUNCH();
    return AIR_OK;
}

int air_vcycle_multi_run(const air_hierarchy *H, int k, const double *b0, double *x0, cudaStream_t s) {
    return vcycle_multi_t<double>(const_cast<air_hierarchy *>(H), k, b0, x0, s);
}

int air_vcycle_multi_run_f32(const air_hierarchy *H, int k, const float *b0, float *x0, cudaStream_t s) {
    return vcycle_multi_t<float>(const_cast<air_hierarchy *>(H), k, b0, x0, s);
}

// Lockstep BiCGSTAB on k systems sharing A and H: the iteration of the
// single-system solve with per-column scalars.  A converged column is frozen
// (its coefficients leave it unchanged); a column whose recursive residual
// meets rtol but whose true residual does not restarts from the true one.
int air_bicgstab_multi_impl(const air_hierarchy *Hc, int k, const double *b, double *x, double rtol,
                            cudaStream_t s, air_solve_info *info) {
    air_hierarchy *H = const_cast<air_hierarchy *>(Hc);
    const AirLevel &A0 = H->lev[0];
    const int64_t n = A0.n;
    const int nblk = (int)grid_for(n, DT / 32, 152 * 8);
    const size_t vec = (size_t)n * k;
    // Krylov vectors r, r^, p, v, s, t, p^, s^, an FP32 pair for the FP32
    // V-cycle; then partial sums, device scalars and flags
    const size_t need = 9 * vec + (size_t)nblk * 2 * k + 16 * MK + MK;
    if (H->mkry_n < need) {
        air_dfree(H->mkry);
        H->mkry = nullptr;
        AIR_CUDA(air_dmalloc((void **)&H->mkry, need * sizeof(double)));
        H->mkry_n = need;
    }
    double *r = H->mkry, *rh = r + vec, *p = rh + vec, *v = p + vec, *sv = v + vec, *t = sv + vec, *ph = t + vec,
           *sh = ph + vec;
    float *f_in = (float *)(sh + vec), *f_out = f_in + vec;
    double *part = sh + 2 * vec, *dsc = part + (size_t)nblk * 2 * k;   // dsc: 2k dots, then coefficient rows
    // the preconditioner in the hierarchy's precision (FP32 for FP32 and BF16 storage)
    const bool f32 = H->opt.precision != AIR_PREC_F64;
    auto precond = [&](const double *in, double *out) -> int {
        if (!f32) return air_vcycle_multi_run(H, k, in, out, s);
        d2f_multi_kernel<<<air_counted(grid_for((int64_t)vec, 256)), 256, 0, s>>>((int64_t)vec, in, f_in);
        AIR_TRY(air_vcycle_multi_run_f32(H, k, f_in, f_out, s));
        f2d_multi_kernel<<<air_counted(grid_for((int64_t)vec, 256)), 256, 0, s>>>((int64_t)vec, f_out, out);
        AIR_LAUNCH();
        return AIR_OK;
    };
    double *c1 = dsc + 2 * MK, *c2 = c1 + MK, *c3 = c2 + MK, *ones = c3 + MK, *zeros = ones + MK;
    int *dmask = (int *)(zeros + MK);
    double hd[2 * MK], hc1[MK], hc2[MK], hc3[MK], hone[MK], hzero[MK];
    int hmask[MK];
    auto dots = [&](const double *U, const double *U2, const double *W) -> int {
        coldot_kernel<<<air_counted(nblk), DT, 0, s>>>(n, k, U, U2, W, part);
        coldot_reduce_kernel<<<air_counted(1), 64, 0, s>>>(nblk, k, part, dsc);
        AIR_LAUNCH();
        AIR_CUDA(cudaMemcpyAsync(hd, dsc, 2 * (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, s));
        AIR_CUDA(cudaStreamSynchronize(s));
        return AIR_OK;
    };
    auto coef = [&](const double *h, double *d) -> int {
        AIR_CUDA(cudaMemcpyAsync(d, h, (size_t)k * sizeof(double), cudaMemcpyHostToDevice, s));
        return AIR_OK;
    };
    auto lincomb = [&](double *out, const double *a, const double *ca, const double *bb, const double *cb,
                       const double *c, const double *cc) -> int {
        lincomb_multi_kernel<<<air_counted(grid_for((int64_t)vec, 256)), 256, 0, s>>>(n, k, out, a, ca, bb, cb, c, cc);
        AIR_LAUNCH();
        return AIR_OK;
    };
    for (int j = 0; j < k; ++j) {
        hone[j] = 1.0;
        hzero[j] = 0.0;
        info[j].iters = 0;
        info[j].restarts = 0;
        info[j].vcycles = 0;
        info[j].relres = 0.0;
        info[j].status = AIR_NOT_CONVERGED;
    }
    AIR_TRY(coef(hone, ones));
    AIR_TRY(coef(hzero, zeros));
    AIR_CUDA(cudaMemsetAsync(x, 0, vec * sizeof(double), s));
    AIR_TRY(dots(b, nullptr, b));
    double bn[MK], rho_prev[MK], alpha[MK], omega[MK];
    bool done[MK];
    int active = 0;
    for (int j = 0; j < k; ++j) {
        bn[j] = sqrt(hd[j]);
        rho_prev[j] = alpha[j] = omega[j] = 1.0;
        done[j] = bn[j] == 0.0;
        if (done[j]) info[j].status = AIR_OK;
        else ++active;
    }
    AIR_CUDA(cudaMemcpyAsync(r, b, vec * sizeof(double), cudaMemcpyDeviceToDevice, s));
    AIR_CUDA(cudaMemcpyAsync(rh, b, vec * sizeof(double), cudaMemcpyDeviceToDevice, s));
    AIR_CUDA(cudaMemsetAsync(p, 0, vec * sizeof(double), s));
    AIR_CUDA(cudaMemsetAsync(v, 0, vec * sizeof(double), s));
    for (int it = 0; it < H->opt.max_iter && active > 0; ++it) {
        AIR_TRY(dots(rh, nullptr, r));
        double rho[MK];
        for (int j = 0; j < k; ++j) {
            rho[j] = hd[j];
            if (!done[j] && rho[j] == 0.0) { done[j] = true; --active; }     // breakdown
            const double beta = done[j] ? 0.0 : (rho[j] / rho_prev[j]) * (alpha[j] / omega[j]);
            hc1[j] = beta;
            hc2[j] = -beta * (done[j] ? 0.0 : omega[j]);
        }
        AIR_TRY(coef(hc1, c1));
        AIR_TRY(coef(hc2, c2));
        AIR_TRY(lincomb(p, r, ones, p, c1, v, c2));                       // p = r + beta (p - omega v)
        AIR_TRY(precond(p, ph));
        csr_multi<MR_SPMV, double>(n, nullptr, A0.rp, A0.ci, A0.v, k, ph, v, nullptr, nullptr, 0.0, s);
        AIR_TRY(dots(rh, nullptr, v));
        for (int j = 0; j < k; ++j) {
            if (!done[j] && hd[j] == 0.0) { done[j] = true; --active; }
            alpha[j] = done[j] ? 0.0 : rho[j] / hd[j];
            hc1[j] = -alpha[j];
        }
        AIR_TRY(coef(hc1, c1));
        AIR_TRY(lincomb(sv, r, ones, v, c1, nullptr, nullptr));           // s = r - alpha v
        AIR_TRY(precond(sv, sh));
        csr_multi<MR_SPMV, double>(n, nullptr, A0.rp, A0.ci, A0.v, k, sh, t, nullptr, nullptr, 0.0, s);
        AIR_TRY(dots(sv, t, t));                                           // (s, t), (t, t)
        for (int j = 0; j < k; ++j) {
            const double ts = hd[j], tt = hd[k + j];
            omega[j] = done[j] ? 0.0 : (tt > 0.0 ? ts / tt : 0.0);
            hc1[j] = alpha[j];
            hc2[j] = omega[j];
            hc3[j] = -omega[j];
        }
        AIR_TRY(coef(hc1, c1));
        AIR_TRY(coef(hc2, c2));
        AIR_TRY(coef(hc3, c3));
        AIR_TRY(lincomb(x, x, ones, ph, c1, sh, c2));                     // x += alpha p^ + omega s^
        AIR_TRY(lincomb(r, sv, ones, t, c3, nullptr, nullptr));           // r = s - omega t
        for (int j = 0; j < k; ++j) {
            if (done[j]) continue;
            rho_prev[j] = rho[j];
            info[j].iters++;
            info[j].vcycles += 2;
        }
        AIR_TRY(dots(r, nullptr, r));
        double rr[MK];
        bool check = false;
        for (int j = 0; j < k; ++j) {
            rr[j] = sqrt(hd[j]) / bn[j];
            check |= !done[j] && rr[j] <= rtol;
        }
        if (check) {
            // the true residual decides the columns whose recursive residual met rtol;
            // those above rtol restart from it
            csr_multi<MR_RESID, double>(n, nullptr, A0.rp, A0.ci, A0.v, k, x, t, b, nullptr, 0.0, s);
            AIR_TRY(dots(t, nullptr, t));
            bool restart = false;
            for (int j = 0; j < k; ++j) {
                hmask[j] = 0;
                if (done[j] || rr[j] > rtol) continue;
                const double tr = sqrt(hd[j]) / bn[j];
                if (tr <= rtol) {
                    done[j] = true;
                    --active;
                    info[j].relres = tr;
                    info[j].status = AIR_OK;
                } else {
                    hmask[j] = 1;
                    restart = true;
                }
            }
            if (restart) {
                AIR_CUDA(cudaMemcpyAsync(dmask, hmask, (size_t)k * sizeof(int), cudaMemcpyHostToDevice, s));
                copy_cols_kernel<<<air_counted(grid_for((int64_t)vec, 256)), 256, 0, s>>>(n, k, dmask, t, r);
                copy_cols_kernel<<<air_counted(grid_for((int64_t)vec, 256)), 256, 0, s>>>(n, k, dmask, t, rh);
                AIR_LAUNCH();
                for (int j = 0; j < k; ++j) hc1[j] = hmask[j] ? 0.0 : 1.0;
                AIR_TRY(coef(hc1, c1));
                AIR_TRY(lincomb(p, p, c1, p, zeros, nullptr, nullptr));   // p = v = 0 on restarted columns
                AIR_TRY(lincomb(v, v, c1, v, zeros, nullptr, nullptr));
                for (int j = 0; j < k; ++j)
                    if (hmask[j]) {
                        rho_prev[j] = alpha[j] = omega[j] = 1.0;
                        info[j].restarts++;
                    }
            }
        }
        for (int j = 0; j < k; ++j)
            if (!done[j] && omega[j] == 0.0) { done[j] = true; --active; }   // stagnation
    }
    // true residual of the columns that did not converge
    csr_multi<MR_RESID, double>(n, nullptr, A0.rp, A0.ci, A0.v, k, x, t, b, nullptr, 0.0, s);
    AIR_TRY(dots(t, nullptr, t));
    for (int j = 0; j < k; ++j)
        if (info[j].status != AIR_OK) info[j].relres = bn[j] > 0.0 ? sqrt(hd[j]) / bn[j] : 0.0;
    AIR_CUDA(cudaStreamSynchronize(s));
    int st = AIR_OK;
    for (int j = 0; j < k; ++j)
        if (info[j].status != AIR_OK) st = AIR_NOT_CONVERGED;
    return st;
}
