// Space-time HDG assembly on the GPU: element matrices of the bilinear form
// (arXiv:2010.11130, Section 2.3, eqs. st-hdg and bilin, upwind flux sigma_a
// and interior-penalty flux sigma_d of eq. IPpenalty), static condensation
// S_K = D_K - C_K A_K^{-1} B_K, H_K = G_K - C_K A_K^{-1} F_K (Section 2.5,
// eqs. linsys and systemLambda), scatter into the facet CSR pattern and the
// left scaling by the facet block-diagonal inverse (Section 4 settings).
//
// For an element K with test (v, mu) and trial (u, lambda), unit space-time
// normal n_hat = (n_t, n), a_hat = (1, a), a_hat_n = a_hat . n_hat,
// c+ = (a_hat_n + |a_hat_n|)/2, c- = (a_hat_n - |a_hat_n|)/2, pen = nu alpha / h_K
// (h_K the longest edge), the local blocks are
//   A(v, u)   = int_K -u a_hat.grad_hat v + nu grad u . grad v
//             + int_dK (c+ + pen) u v - nu (grad u . n) v - nu u (grad v . n)
//   B(v, lam) = int_dK (c- - pen) lam v + nu lam (grad v . n)
//   C(mu, u)  = int_dK -(c+ + pen) u mu + nu (grad u . n) mu
//   D(mu, lam)= int_dK -(c- - pen) lam mu  (+ c+ lam mu on Neumann facets)
//   F(v)      = int_K f v,   G(mu) = int_{dK on Neumann} g mu, g = -a_hat_n u0 where a_hat_n < 0
// (grad and grad . n spatial).  The Dirichlet trace is the L2 projection of
// the data onto the facet basis and moves to the right-hand side.
//
// One warp per element: the local matrices live in shared memory, lanes run
// over matrix entries (each summing over the quadrature points) and over the
// rows / columns of the elimination.  One warp per free facet then sums the
// two diagonal contributions in element order, inverts the diagonal block by
// Gauss-Jordan and scales its row.  FP64 throughout.
#include <math.h>

#include "air_internal.cuh"
#include "warp_dense.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int WPB = 4;         // elements (warps) per block
constexpr int FWPB = 4;        // facets (warps) per block
constexpr int8_t K_DIR = 1, K_NEU = 2;

__host__ __device__ constexpr int binom(int n, int k) { return k == 0 ? 1 : binom(n - 1, k - 1) * n / k; }
__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }
__host__ __device__ constexpr int fact(int n) { return n <= 1 ? 1 : n * fact(n - 1); }

template <int D, int P>
struct Dims {
    static constexpr int NB = binom(P + D, D);       // element basis
    static constexpr int B = binom(P + D - 1, D - 1); // trace basis per facet
    static constexpr int NF = D + 1;
    static constexpr int NT = NF * B;
    static constexpr int NX = NT + 1;                // columns of [B | F]
    static constexpr int Q = P + 2;
    static constexpr int NQ = ipow(Q, D);
    static constexpr int NQF = ipow(Q, D - 1);
    static constexpr int NPERM = fact(D);
    static constexpr int SQ = NQ * (D + 1) > NQF * 4 ? NQ * (D + 1) : NQF * 4;
    static constexpr int WARP_DOUBLES = NB * NB + NB * NX + NT * NB + NF * B * B + NT + NT * NT + SQ;
    static constexpr int MAXN = 2 * D;               // off-diagonal facet blocks per row
};

template <int D>
struct Geo {
    double X0[D];
    double J[D][D];      // J[r][c] = X_{c+1}[r] - X_0[r]
    double Jinv[D][D];
    double det;          // |det J|
    double h;            // longest edge
};

template <int D>
__device__ void geometry(const double *verts, const int32_t *ev, Geo<D> &g) {
    double X[D + 1][D];
#pragma unroll
    for (int v = 0; v <= D; ++v)
#pragma unroll
        for (int d = 0; d < D; ++d) X[v][d] = verts[(int64_t)ev[v] * D + d];
#pragma unroll
    for (int d = 0; d < D; ++d) g.X0[d] = X[0][d];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) g.J[r][c] = X[c + 1][r] - X[0][r];
    double det;
    if constexpr (D == 2) {
        det = g.J[0][0] * g.J[1][1] - g.J[0][1] * g.J[1][0];
        g.Jinv[0][0] = g.J[1][1] / det;
        g.Jinv[0][1] = -g.J[0][1] / det;
        g.Jinv[1][0] = -g.J[1][0] / det;
        g.Jinv[1][1] = g.J[0][0] / det;
    } else {
        const double(*J)[D] = g.J;
        double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
        g.Jinv[0][0] = c00 / det;
        g.Jinv[1][0] = c01 / det;
        g.Jinv[2][0] = c02 / det;
        g.Jinv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
        g.Jinv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
        g.Jinv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
        g.Jinv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
        g.Jinv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
        g.Jinv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    }
    g.det = fabs(det);
    double h = 0.0;
#pragma unroll
    for (int i = 0; i <= D; ++i)
#pragma unroll
        for (int j = i + 1; j <= D; ++j) {
            double s = 0.0;
#pragma unroll
            for (int d = 0; d < D; ++d) s += (X[i][d] - X[j][d]) * (X[i][d] - X[j][d]);
            h = fmax(h, sqrt(s));
        }
    g.h = h;
}

// Index s of the canonical frame of local facet k: the facet's local vertices
// (ascending local index) sorted by global id; perms[s] lists, for canonical
// vertex m, the position within the local list.
template <int D>
__device__ int facet_perm(const int32_t *ev, int k, const int32_t *perms) {
    int loc[D], ord[D];
    int32_t gid[D];
    int c = 0;
#pragma unroll
    for (int v = 0; v <= D; ++v)
        if (v != k) loc[c++] = v;
#pragma unroll
    for (int m = 0; m < D; ++m) {
        gid[m] = ev[loc[m]];
        ord[m] = m;
    }
    for (int i = 1; i < D; ++i)          // stable insertion sort of positions by global id
        for (int j = i; j > 0 && gid[ord[j - 1]] > gid[ord[j]]; --j) {
            int t = ord[j];
            ord[j] = ord[j - 1];
            ord[j - 1] = t;
        }
    for (int s = 0; s < fact(D); ++s) {
        bool eq = true;
#pragma unroll
        for (int m = 0; m < D; ++m) eq = eq && perms[s * D + m] == ord[m];
        if (eq) return s;
    }
    return 0;
}

struct ElemArgs {
    int64_t E;
    double nu, alpha;
    int dlen;                    // stored entries of a diagonal row block: 1 (scaled) or b
    const double *verts;
    const int32_t *elems, *elem_facets, *facet_elems;
    const int8_t *kind;
    const int32_t *rnum, *nbr, *nbr_cnt;
    const int64_t *row_ptr;
    const double *wq, *phi, *gphi, *wf, *psi, *phi_f, *gphi_f;
    const int32_t *perms;
    const double *vel_vol, *src, *vel_face, *u0_face, *lam_dir;
    double *val, *dpart, *hpart;
    // velocity gradient (adjoint) mode
    const double *lam_full, *mu_full;   // n_facets x b trace and unscaled adjoint (0 on Dirichlet)
    double *grad;                       // E x (D-1)
    int *err;
};

// Builds A, [B | F], C, the diagonal blocks of D and G of one element in the
// warp's shared memory.  With dvel >= 0 it builds instead the derivatives of
// A, B, C, D with respect to velocity component dvel (constant on the
// element); F and G are then left as they are.
template <int D, int P>
__device__ void local_matrices(const ElemArgs &a, int64_t e, const Geo<D> &g, double *sA, double *sX, double *sC,
                               double *sD, double *sG, double *sQ, int dvel) {
    using Dm = Dims<D, P>;
    constexpr int NB = Dm::NB, B = Dm::B, NF = Dm::NF, NX = Dm::NX, NQ = Dm::NQ, NQF = Dm::NQF,
                  NPERM = Dm::NPERM;
    const int lane = threadIdx.x & 31;
    const int32_t *ev = a.elems + e * (D + 1);
    const double nu = dvel >= 0 ? 0.0 : a.nu;          // the diffusion terms do not depend on a
    // ---- volume: per point W_q and (Jinv a_hat)_k (its velocity derivative: Jinv e_{dvel+1})
    for (int q = lane; q < NQ; q += 32) {
        double ah[D];
        ah[0] = dvel >= 0 ? 0.0 : 1.0;
#pragma unroll
        for (int m = 0; m < D - 1; ++m)
            ah[m + 1] = dvel >= 0 ? (m == dvel ? 1.0 : 0.0) : a.vel_vol[(e * NQ + q) * (D - 1) + m];
        sQ[q * (D + 1)] = g.det * a.wq[q];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            double at = 0.0;
#pragma unroll
            for (int d = 0; d < D; ++d) at += g.Jinv[k][d] * ah[d];
            sQ[q * (D + 1) + 1 + k] = at;
        }
    }
    double Mm[D][D];   // spatial metric: sum over spatial s of Jinv[k][s] Jinv[l][s]
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
        for (int l = 0; l < D; ++l) {
            double s = 0.0;
#pragma unroll
            for (int d = 1; d < D; ++d) s += g.Jinv[k][d] * g.Jinv[l][d];
            Mm[k][l] = s;
        }
    __syncwarp();
    for (int t = lane; t < NB * NB; t += 32) {
        const int i = t / NB, j = t % NB;
        double acc = 0.0;
        for (int q = 0; q < NQ; ++q) {
            const double *gi = a.gphi + (q * NB + i) * D, *gj = a.gphi + (q * NB + j) * D;
            double adv = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) adv += sQ[q * (D + 1) + 1 + k] * gi[k];
            double term = -a.phi[q * NB + j] * adv;
            if (nu != 0.0) {
                double dif = 0.0;
#pragma unroll
                for (int k = 0; k < D; ++k)
#pragma unroll
                    for (int l = 0; l < D; ++l) dif += Mm[k][l] * gi[k] * gj[l];
                term += nu * dif;
            }
            acc += sQ[q * (D + 1)] * term;
        }
        sA[t] = acc;
    }
    if (dvel < 0)
        for (int i = lane; i < NB; i += 32) {
            double acc = 0.0;
            if (a.src)
                for (int q = 0; q < NQ; ++q) acc += sQ[q * (D + 1)] * a.src[e * NQ + q] * a.phi[q * NB + i];
            sX[i * NX + Dm::NT] = acc;
        }
    const double pen = nu * a.alpha / g.h;
    for (int k = 0; k < NF; ++k) {
        const int s = facet_perm<D>(ev, k, a.perms);
        double gl[D];   // Jinv^T grad_ref(lambda_k): lambda_0 = 1 - sum xi, lambda_k = xi_{k-1}
#pragma unroll
        for (int d = 0; d < D; ++d) {
            if (k == 0) {
                double sum = 0.0;
#pragma unroll
                for (int kk = 0; kk < D; ++kk) sum -= g.Jinv[kk][d];
                gl[d] = sum;
            } else {
                gl[d] = g.Jinv[k - 1][d];
            }
        }
        double gn = 0.0;
#pragma unroll
        for (int d = 0; d < D; ++d) gn += gl[d] * gl[d];
        gn = sqrt(gn);
        double nh[D];
#pragma unroll
        for (int d = 0; d < D; ++d) nh[d] = -gl[d] / gn;      // outward unit space-time normal
        const double wscale = (double)D * (g.det / (double)fact(D)) * gn * (double)fact(D - 1);
        double jv[D];    // (grad phi . n) = grad_ref phi . (Jinv (0, n))
#pragma unroll
        for (int kk = 0; kk < D; ++kk) {
            double sum = 0.0;
#pragma unroll
            for (int d = 1; d < D; ++d) sum += g.Jinv[kk][d] * nh[d];
            jv[kk] = sum;
        }
        const int32_t f = a.elem_facets[e * NF + k];
        const bool neu = a.kind[f] == K_NEU;
        const double *phf = a.phi_f + (size_t)(k * NPERM + s) * NQF * NB;
        const double *gphf = a.gphi_f + (size_t)(k * NPERM + s) * NQF * NB * D;
        __syncwarp();
        for (int q = lane; q < NQF; q += 32) {
            double an = dvel >= 0 ? 0.0 : nh[0];
            double dan = 0.0;
            if (dvel >= 0) {
                // a_hat_n at the point (for the side of the kink) and its derivative n_{dvel+1}
                an = nh[0];
#pragma unroll
                for (int m = 0; m < D - 1; ++m) an += a.vel_face[((e * NF + k) * NQF + q) * (D - 1) + m] * nh[m + 1];
                dan = nh[dvel + 1];
            } else {
#pragma unroll
                for (int m = 0; m < D - 1; ++m) an += a.vel_face[((e * NF + k) * NQF + q) * (D - 1) + m] * nh[m + 1];
            }
            double cup, cdn, gN = 0.0;
            if (dvel >= 0) {
                // d/da of (an +- |an|)/2; the kink an = 0 takes the mean slope
                const double sg = an > 0.0 ? 1.0 : (an < 0.0 ? -1.0 : 0.0);
                cup = 0.5 * (1.0 + sg) * dan;
                cdn = 0.5 * (1.0 - sg) * dan;
            } else {
                cup = 0.5 * (an + fabs(an));
                cdn = 0.5 * (an - fabs(an));
                if (neu && an < 0.0 && a.u0_face) gN = -an * a.u0_face[(e * NF + k) * NQF + q];
            }
            sQ[q * 4 + 0] = wscale * a.wf[q];
            sQ[q * 4 + 1] = cup;
            sQ[q * 4 + 2] = cdn;
            sQ[q * 4 + 3] = gN;
        }
        __syncwarp();
        for (int t = lane; t < NB * NB; t += 32) {
            const int i = t / NB, j = t % NB;
            double acc = 0.0;
            for (int q = 0; q < NQF; ++q) {
                const double W = sQ[q * 4], cup = sQ[q * 4 + 1];
                const double fi = phf[q * NB + i], fj = phf[q * NB + j];
                double term = (cup + pen) * fi * fj;
                if (nu != 0.0) {
                    double dni = 0.0, dnj = 0.0;
#pragma unroll
                    for (int d = 0; d < D; ++d) {
                        dni += gphf[(q * NB + i) * D + d] * jv[d];
                        dnj += gphf[(q * NB + j) * D + d] * jv[d];
                    }
                    term -= nu * (fi * dnj + dni * fj);
                }
                acc += W * term;
            }
            sA[t] += acc;
        }
        for (int t = lane; t < NB * B; t += 32) {
            const int i = t / B, l = t % B;
            double acc = 0.0;
            for (int q = 0; q < NQF; ++q) {
                const double W = sQ[q * 4], cdn = sQ[q * 4 + 2];
                const double fi = phf[q * NB + i], pl = a.psi[q * B + l];
                double term = (cdn - pen) * fi * pl;
                if (nu != 0.0) {
                    double dni = 0.0;
#pragma unroll
                    for (int d = 0; d < D; ++d) dni += gphf[(q * NB + i) * D + d] * jv[d];
                    term += nu * dni * pl;
                }
                acc += W * term;
            }
            sX[i * NX + k * B + l] = acc;
        }
        for (int t = lane; t < B * NB; t += 32) {
            const int l = t / NB, j = t % NB;
            double acc = 0.0;
            for (int q = 0; q < NQF; ++q) {
                const double W = sQ[q * 4], cup = sQ[q * 4 + 1];
                const double fj = phf[q * NB + j], pl = a.psi[q * B + l];
                double term = -(cup + pen) * fj * pl;
                if (nu != 0.0) {
                    double dnj = 0.0;
#pragma unroll
                    for (int d = 0; d < D; ++d) dnj += gphf[(q * NB + j) * D + d] * jv[d];
                    term += nu * dnj * pl;
                }
                acc += W * term;
            }
            sC[(k * B + l) * NB + j] = acc;
        }
        for (int t = lane; t < B * B; t += 32) {
            const int m = t / B, l = t % B;
            double acc = 0.0;
            for (int q = 0; q < NQF; ++q) {
                const double W = sQ[q * 4], cup = sQ[q * 4 + 1], cdn = sQ[q * 4 + 2];
                acc += W * (-(cdn - pen) + (neu ? cup : 0.0)) * a.psi[q * B + l] * a.psi[q * B + m];
            }
            sD[(k * B + m) * B + l] = acc;
        }
        if (dvel < 0)
            for (int m = lane; m < B; m += 32) {
                double acc = 0.0;
                for (int q = 0; q < NQF; ++q) acc += sQ[q * 4] * sQ[q * 4 + 3] * a.psi[q * B + m];
                sG[k * B + m] = acc;
            }
    }
    __syncwarp();
}

// Gaussian elimination with partial pivoting (ties -> smallest row) of the
// warp's A (n x n, row-major) applied to the ncol columns of X (row stride
// ldx), then back substitution: X <- A^{-1} X.  A is overwritten by its LU
// factors.  Returns false if a pivot is zero.
__device__ bool warp_solve(double *A, int n, double *X, int ldx, int ncol) {
    const int lane = threadIdx.x & 31;
    bool ok = true;
    for (int c = 0; c < n; ++c) {
        double v = -1.0;
        int r = n;
        for (int rr = c + lane; rr < n; rr += 32) {
            const double av = fabs(A[rr * n + c]);
            if (av > v) { v = av; r = rr; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_down_sync(FULL, v, o);
            const int orow = __shfl_down_sync(FULL, r, o);
            if (ov > v || (ov == v && orow < r)) { v = ov; r = orow; }
        }
        r = __shfl_sync(FULL, r, 0);
        v = __shfl_sync(FULL, v, 0);
        if (!(v > 0.0)) { ok = false; break; }
        if (r != c) {
            for (int t = lane; t < n; t += 32) {
                const double x = A[c * n + t];
                A[c * n + t] = A[r * n + t];
                A[r * n + t] = x;
            }
            for (int t = lane; t < ncol; t += 32) {
                const double x = X[c * ldx + t];
                X[c * ldx + t] = X[r * ldx + t];
                X[r * ldx + t] = x;
            }
        }
        __syncwarp();
        const double piv = A[c * n + c];
        for (int rr = c + 1 + lane; rr < n; rr += 32) A[rr * n + c] = A[rr * n + c] / piv;
        __syncwarp();
        const int rows = n - c - 1, wa = n - c - 1, w = wa + ncol;
        for (int t = lane; t < rows * w; t += 32) {
            const int rr = c + 1 + t / w, cc = t % w;
            const double l = A[rr * n + c];
            if (cc < wa) A[rr * n + c + 1 + cc] -= l * A[c * n + c + 1 + cc];
            else X[rr * ldx + (cc - wa)] -= l * X[c * ldx + (cc - wa)];
        }
        __syncwarp();
    }
    if (!ok) return false;
    for (int t = lane; t < ncol; t += 32)
        for (int r = n - 1; r >= 0; --r) {
            double s = X[r * ldx + t];
            for (int cc = r + 1; cc < n; ++cc) s -= A[r * n + cc] * X[cc * ldx + t];
            X[r * ldx + t] = s / A[r * n + r];
        }
    __syncwarp();
    return true;
}

template <int D, int P>
__global__ void __launch_bounds__(WPB * 32) hdg_element_kernel(ElemArgs a) {
    using Dm = Dims<D, P>;
    constexpr int NB = Dm::NB, B = Dm::B, NF = Dm::NF, NT = Dm::NT, NX = Dm::NX, MAXN = Dm::MAXN;
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t e = (int64_t)blockIdx.x * WPB + w;
    if (e >= a.E) return;                                 // the whole warp leaves together
    double *sA = smem + (size_t)w * Dm::WARP_DOUBLES;
    double *sX = sA + NB * NB, *sC = sX + NB * NX, *sD = sC + NT * NB, *sG = sD + NF * B * B, *sS = sG + NT,
           *sQ = sS + NT * NT;
    Geo<D> g;
    geometry<D>(a.verts, a.elems + e * (D + 1), g);
    local_matrices<D, P>(a, e, g, sA, sX, sC, sD, sG, sQ, -1);
    if (!warp_solve(sA, NB, sX, NX, NX)) {
        if (lane == 0) atomicOr(a.err, AIR_DEVERR_SINGULAR);
        return;
    }
    // S = D - C X_B (D block diagonal), H = G - C X_F
    for (int t = lane; t < NT * NT; t += 32) {
        const int r = t / NT, c = t % NT;
        double acc = 0.0;
        for (int i = 0; i < NB; ++i) acc += sC[r * NB + i] * sX[i * NX + c];
        const double dv = (r / B == c / B) ? sD[r * B + c % B] : 0.0;
        sS[t] = dv - acc;
    }
    for (int r = lane; r < NT; r += 32) {
        double acc = 0.0;
        for (int i = 0; i < NB; ++i) acc += sC[r * NB + i] * sX[i * NX + NT];
        sG[r] = sG[r] - acc;
    }
    __syncwarp();
    const int32_t *ef = a.elem_facets + e * NF;
    for (int k = 0; k < NF; ++k) {
        const int32_t f = ef[k];
        if (a.kind[f] == K_DIR) continue;
        const int slot = a.facet_elems[2 * (int64_t)f] == (int32_t)e ? 0 : 1;
        for (int t = lane; t < B * B; t += 32) {
            const int m = t / B, l = t % B;
            a.dpart[((int64_t)(2 * (int64_t)f + slot) * B + m) * B + l] = sS[(k * B + m) * NT + k * B + l];
        }
        for (int m = lane; m < B; m += 32) {
            double h = sG[k * B + m];
            for (int l = 0; l < NF; ++l) {
                if (l == k || a.kind[ef[l]] != K_DIR) continue;
                const double *ld = a.lam_dir + (int64_t)ef[l] * B;
                for (int l2 = 0; l2 < B; ++l2) h -= sS[(k * B + m) * NT + l * B + l2] * ld[l2];
            }
            a.hpart[(2 * (int64_t)f + slot) * B + m] = h;
        }
        const int32_t rf = a.rnum[f];
        const int cnt = a.nbr_cnt[rf];
        const int32_t *nb = a.nbr + (int64_t)rf * MAXN;
        for (int l = 0; l < NF; ++l) {
            const int32_t gf = ef[l];
            if (l == k || a.kind[gf] == K_DIR) continue;
            const int32_t rg = a.rnum[gf];
            int rank = 0;
            while (rank < cnt && nb[rank] != rg) ++rank;
            if (rank == cnt) {
                if (lane == 0) atomicOr(a.err, AIR_DEVERR_CSR);
                continue;
            }
            const int64_t off = (int64_t)rank * B + (rg > rf ? a.dlen : 0);
            for (int t = lane; t < B * B; t += 32) {
                const int m = t / B, l2 = t % B;
                a.val[a.row_ptr[(int64_t)rf * B + m] + off + l2] = sS[(k * B + m) * NT + l * B + l2];
            }
        }
    }
}

// ---------------------------------------------------------------- pattern
__global__ void free_flag_kernel(int64_t F, const int8_t *kind, int32_t *flag) {
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < F; f += (int64_t)gridDim.x * blockDim.x)
        flag[f] = kind[f] != K_DIR ? 1 : 0;
}

__global__ void renumber_kernel(int64_t F, const int8_t *kind, const int64_t *scan, int32_t *rnum,
                                int32_t *free_ids) {
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < F; f += (int64_t)gridDim.x * blockDim.x) {
        if (kind[f] != K_DIR) {
            rnum[f] = (int32_t)scan[f];
            free_ids[scan[f]] = (int32_t)f;
        } else {
            rnum[f] = -1;
        }
    }
}

// Sorted free neighbour facets (by free number) of every free facet: the
// other facets of its one or two elements.
template <int D>
__global__ void neighbour_kernel(int64_t nfree, int B, int dlen, const int32_t *free_ids, const int32_t *facet_elems,
                                 const int32_t *elem_facets, const int8_t *kind, const int32_t *rnum, int32_t *nbr,
                                 int32_t *cnt, int32_t *rowlen) {
    constexpr int MAXN = 2 * D;
    for (int64_t rf = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; rf < nfree;
         rf += (int64_t)gridDim.x * blockDim.x) {
        const int32_t f = free_ids[rf];
        int32_t list[MAXN];
        int c = 0;
        for (int s = 0; s < 2; ++s) {
            const int32_t e = facet_elems[2 * (int64_t)f + s];
            if (e < 0) continue;
            for (int l = 0; l <= D; ++l) {
                const int32_t g = elem_facets[(int64_t)e * (D + 1) + l];
                if (g == f || kind[g] == K_DIR || c >= MAXN) continue;
                int32_t v = rnum[g];
                int j = c++;
                while (j > 0 && list[j - 1] > v) { list[j] = list[j - 1]; --j; }
                list[j] = v;
            }
        }
        for (int t = 0; t < MAXN; ++t) nbr[rf * MAXN + t] = t < c ? list[t] : -1;
        cnt[rf] = c;
        for (int i = 0; i < B; ++i) rowlen[rf * B + i] = c * B + dlen;
    }
}

template <int MAXN>
__global__ void columns_kernel(int64_t nfree, int B, int dlen, const int32_t *nbr, const int32_t *cnt,
                               const int64_t *row_ptr, int32_t *col) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nfree * B;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t rf = r / B;
        const int i = (int)(r % B);
        const int c = cnt[rf];
        int64_t p = row_ptr[r];
        bool diag = false;
        for (int t = 0; t <= c; ++t) {
            const int32_t g = t < c ? nbr[rf * MAXN + t] : INT32_MAX;
            if (!diag && g > rf) {
                diag = true;
                if (dlen == 1) col[p++] = (int32_t)(rf * B + i);
                else for (int j = 0; j < B; ++j) col[p++] = (int32_t)(rf * B + j);
            }
            if (t < c)
                for (int j = 0; j < B; ++j) col[p++] = g * B + j;
        }
    }
}

__global__ void dirichlet_kernel(int64_t F, int B, int NQF, const int8_t *kind, const double *proj, const double *gd,
                                 double *lam) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < F * B; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = t / B;
        const int m = (int)(t % B);
        double s = 0.0;
        if (kind[f] == K_DIR && gd)
            for (int q = 0; q < NQF; ++q) s += proj[m * NQF + q] * gd[f * NQF + q];
        lam[t] = s;
    }
}

struct FacetArgs {
    int64_t nfree;
    int B, dlen, maxn, scale;
    const int32_t *free_ids, *facet_elems, *nbr, *cnt;
    const int64_t *row_ptr;
    const double *dpart, *hpart;
    double *val, *rhs, *diag;
    int *err;
};

// One warp per free facet: Sd = sum of the element contributions (element
// order), H likewise; scaled: Dinv = Sd^{-1}, rhs = Dinv H and every
// off-diagonal block of the row block becomes Dinv blk; the diagonal block is
// stored as its b ones.  Unscaled: Sd goes into the row, rhs = H.
__global__ void __launch_bounds__(FWPB * 32) facet_kernel(FacetArgs a) {
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t rf = (int64_t)blockIdx.x * FWPB + w;
    if (rf >= a.nfree) return;
    const int B = a.B, BB = B * B;
    double *sS = smem + (size_t)w * 6 * BB, *sI = sS + BB, *sW = sI + BB, *sT = sW + 2 * BB, *sH = sT + BB;
    const int32_t f = a.free_ids[rf];
    const bool two = a.facet_elems[2 * (int64_t)f + 1] >= 0;
    for (int t = lane; t < BB; t += 32) {
        double v = a.dpart[(2 * (int64_t)f) * BB + t];
        if (two) v = v + a.dpart[(2 * (int64_t)f + 1) * BB + t];
        sS[t] = v;
        if (a.diag) a.diag[rf * BB + t] = v;
    }
    for (int m = lane; m < B; m += 32) {
        double v = a.hpart[(2 * (int64_t)f) * B + m];
        if (two) v = v + a.hpart[(2 * (int64_t)f + 1) * B + m];
        sH[m] = v;
    }
    __syncwarp();
    const int c = a.cnt[rf];
    const int32_t *nb = a.nbr + rf * a.maxn;
    int nbefore = 0;
    for (int t = 0; t < c; ++t) nbefore += nb[t] < rf ? 1 : 0;
    if (!a.scale) {
        for (int t = lane; t < BB; t += 32) {
            const int m = t / B, l = t % B;
            a.val[a.row_ptr[rf * B + m] + (int64_t)nbefore * B + l] = sS[t];
        }
        for (int m = lane; m < B; m += 32) a.rhs[rf * B + m] = sH[m];
        return;
    }
    if (!warp_inverse(sS, B, sW, sI)) {
        if (lane == 0) atomicOr(a.err, AIR_DEVERR_SINGULAR);
        return;
    }
    for (int m = lane; m < B; m += 32) {
        double s = 0.0;
        for (int l = 0; l < B; ++l) s += sI[m * B + l] * sH[l];
        a.rhs[rf * B + m] = s;
        a.val[a.row_ptr[rf * B + m] + (int64_t)nbefore * B] = 1.0;
    }
    for (int t = 0; t < c; ++t) {
        const int64_t off = (int64_t)t * B + (nb[t] > rf ? a.dlen : 0);
        for (int u = lane; u < BB; u += 32) {
            const int m = u / B, l = u % B;
            sT[u] = a.val[a.row_ptr[rf * B + m] + off + l];
        }
        __syncwarp();
        for (int u = lane; u < BB; u += 32) {
            const int m = u / B, l = u % B;
            double s = 0.0;
            for (int j = 0; j < B; ++j) s += sI[m * B + j] * sT[j * B + l];
            a.val[a.row_ptr[rf * B + m] + off + l] = s;
        }
        __syncwarp();
    }
}

// --------------------------------------------------------------- points
template <int D>
__global__ void points_kernel(int64_t E, int nq, int nqf, int nperm, const double *verts, const int32_t *elems,
                              const double *xq, const double *xi_f, const int32_t *perms, double *x_vol,
                              double *x_face) {
    const int64_t per = (int64_t)nq + (int64_t)(D + 1) * nqf;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < E * per;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = t / per;
        const int r = (int)(t % per);
        const int32_t *ev = elems + e * (D + 1);
        double X0[D], J[D][D];
#pragma unroll
        for (int d = 0; d < D; ++d) X0[d] = verts[(int64_t)ev[0] * D + d];
#pragma unroll
        for (int d = 0; d < D; ++d)
#pragma unroll
            for (int c = 0; c < D; ++c) J[d][c] = verts[(int64_t)ev[c + 1] * D + d] - X0[d];
        const double *xi;
        double *out;
        if (r < nq) {
            if (!x_vol) continue;
            xi = xq + r * D;
            out = x_vol + (e * nq + r) * D;
        } else {
            if (!x_face) continue;
            const int k = (r - nq) / nqf, q = (r - nq) % nqf;
            const int s = facet_perm<D>(ev, k, perms);
            xi = xi_f + ((int64_t)(k * nperm + s) * nqf + q) * D;
            out = x_face + ((e * (D + 1) + k) * nqf + q) * D;
        }
#pragma unroll
        for (int d = 0; d < D; ++d) {
            double v = X0[d];
#pragma unroll
            for (int c = 0; c < D; ++c) v += J[d][c] * xi[c];
            out[d] = v;
        }
    }
}

__global__ void facet_points_kernel(int64_t F, int D, int nqf, const double *verts, const int32_t *facets,
                                    const double *sq, double *x_facet) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < F * nqf;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = t / nqf;
        const int q = (int)(t % nqf);
        const int32_t *fv = facets + f * D;
        for (int d = 0; d < D; ++d) {
            const double w0 = verts[(int64_t)fv[0] * D + d];
            double v = w0;
            for (int m = 0; m + 1 < D; ++m) v += (verts[(int64_t)fv[m + 1] * D + d] - w0) * sq[q * (D - 1) + m];
            x_facet[t * D + d] = v;
        }
    }
}

// ------------------------------------------------------ velocity gradient
// mu_f = Sd_f^{-T} adj_f per free facet (the unscaled adjoint), spread to all
// facets with zeros on Dirichlet ones; Lambda likewise with the Dirichlet
// values.  One warp per free facet.
__global__ void __launch_bounds__(FWPB * 32) adjoint_unscale_kernel(int64_t F, int64_t nfree, int B,
                                                                    const int32_t *free_ids, const double *diag,
                                                                    const double *lam, const double *adj,
                                                                    double *mu_full, double *lam_full, int *err) {
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t rf = (int64_t)blockIdx.x * FWPB + w;
    if (rf >= nfree) return;
    const int BB = B * B;
    double *sS = smem + (size_t)w * 4 * BB, *sI = sS + BB, *sW = sI + BB;
    for (int t = lane; t < BB; t += 32) sS[t] = diag[rf * BB + (t % B) * B + t / B];   // transpose
    __syncwarp();
    if (!warp_inverse(sS, B, sW, sI)) {
        if (lane == 0) atomicOr(err, AIR_DEVERR_SINGULAR);
        return;
    }
    const int32_t f = free_ids[rf];
    for (int m = lane; m < B; m += 32) {
        double s = 0.0;
        for (int l = 0; l < B; ++l) s += sI[m * B + l] * adj[rf * B + l];
        mu_full[(int64_t)f * B + m] = s;
        lam_full[(int64_t)f * B + m] = lam[rf * B + m];
    }
}

__global__ void spread_dirichlet_kernel(int64_t F, int B, const int8_t *kind, const double *lam_dir, double *mu_full,
                                        double *lam_full) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < F * B; t += (int64_t)gridDim.x * blockDim.x)
        if (kind[t / B] == K_DIR) {
            mu_full[t] = 0.0;
            lam_full[t] = lam_dir[t];
        }
}

// dL/da_e,m = mu^T (dH/da - dS/da Lambda) = -mu^T dC U + y^T dA U - mu^T dD Lambda + y^T dB Lambda
// with U = A^{-1}(F - B Lambda), y = A^{-T} C^T mu (the source and the
// Neumann data do not depend on the element velocity here: on the t faces the
// spatial normal vanishes).
template <int D, int P>
__global__ void __launch_bounds__(WPB * 32) velocity_gradient_kernel(ElemArgs a) {
    using Dm = Dims<D, P>;
    constexpr int NB = Dm::NB, B = Dm::B, NF = Dm::NF, NT = Dm::NT, NX = Dm::NX;
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t e = (int64_t)blockIdx.x * WPB + w;
    if (e >= a.E) return;
    double *sA = smem + (size_t)w * Dm::WARP_DOUBLES;
    double *sX = sA + NB * NB, *sC = sX + NB * NX, *sD = sC + NT * NB, *sG = sD + NF * B * B, *sS = sG + NT,
           *sQ = sS + NT * NT;
    // sS holds: Lam (NT), mu (NT), U (NB), y (NB), AT (NB x NB) for the transposed solve
    double *sLam = sS, *sMu = sLam + NT, *sU = sMu + NT, *sY = sU + NB, *sAT = sY + NB;
    Geo<D> g;
    geometry<D>(a.verts, a.elems + e * (D + 1), g);
    const int32_t *ef = a.elem_facets + e * NF;
    for (int t = lane; t < NT; t += 32) {
        const int k = t / B, m = t % B;
        sLam[t] = a.lam_full[(int64_t)ef[k] * B + m];
        sMu[t] = a.mu_full[(int64_t)ef[k] * B + m];
    }
    local_matrices<D, P>(a, e, g, sA, sX, sC, sD, sG, sQ, -1);
    // right-hand sides: F - B Lam (column NT of sX), C^T mu (into sY); A^T copy
    for (int i = lane; i < NB; i += 32) {
        double s = sX[i * NX + NT];
        for (int c = 0; c < NT; ++c) s -= sX[i * NX + c] * sLam[c];
        sU[i] = s;
        double y = 0.0;
        for (int r = 0; r < NT; ++r) y += sC[r * NB + i] * sMu[r];
        sY[i] = y;
    }
    for (int t = lane; t < NB * NB; t += 32) sAT[t] = sA[(t % NB) * NB + t / NB];
    __syncwarp();
    bool ok = warp_solve(sA, NB, sU, 1, 1);
    ok = ok && warp_solve(sAT, NB, sY, 1, 1);
    if (!ok) {
        if (lane == 0) atomicOr(a.err, AIR_DEVERR_SINGULAR);
        return;
    }
    // sU, sY must survive the derivative builds: they sit in sS, which
    // local_matrices does not touch
    for (int m = 0; m < D - 1; ++m) {
        local_matrices<D, P>(a, e, g, sA, sX, sC, sD, sG, sQ, m);
        double part = 0.0;
        for (int t = lane; t < NB * NB; t += 32) part += sY[t / NB] * sA[t] * sU[t % NB];
        for (int t = lane; t < NB * NT; t += 32) part += sY[t / NT] * sX[(t / NT) * NX + t % NT] * sLam[t % NT];
        for (int t = lane; t < NT * NB; t += 32) part -= sMu[t / NB] * sC[t] * sU[t % NB];
        for (int t = lane; t < NT * B; t += 32) {
            const int r = t / B, l = t % B;
            part -= sMu[r] * sD[t] * sLam[(r / B) * B + l];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(FULL, part, o);
        if (lane == 0) a.grad[e * (D - 1) + m] = part;
        __syncwarp();
    }
}

// ---------------------------------------------------------------- host side
unsigned grid_for(int64_t items, int threads) {
    int64_t b = (items + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)b;
}

int check_ref(const air_hdg_mesh *M, const air_hdg_ref *R) {
    if (!M || !R || (M->D != 2 && M->D != 3) || R->p < 1 || R->p > 3) return AIR_ERR_INVALID_ARG;
    const int D = M->D, p = R->p, q = p + 2;
    if (R->nb != binom(p + D, D) || R->b != binom(p + D - 1, D - 1) || R->nq != ipow(q, D) ||
        R->nqf != ipow(q, D - 1) || R->nperm != fact(D))
        return AIR_ERR_INVALID_ARG;
    if (M->n_elems <= 0 || M->n_facets <= 0 || M->n_verts <= 0 || !M->verts || !M->elems || !M->elem_facets ||
        !M->facets || !M->facet_elems || !M->facet_kind)
        return AIR_ERR_INVALID_ARG;
    if (M->n_elems > INT32_MAX || M->n_facets > INT32_MAX) return AIR_ERR_INVALID_ARG;
    return AIR_OK;
}

template <typename T>
int dalloc(T **p, int64_t count) {
    *p = nullptr;
    if (count <= 0) count = 1;
    AIR_CUDA(air_dmalloc((void **)p, (size_t)count * sizeof(T)));
    return AIR_OK;
}

// Facet renumbering and the neighbour lists (the pattern of every row).
struct Pattern {
    int64_t nfree = 0, nnz = 0;
    int32_t *rnum = nullptr, *free_ids = nullptr, *nbr = nullptr, *cnt = nullptr, *rowlen = nullptr;
    int64_t *scan = nullptr;
    ~Pattern() {
        air_dfree(rnum); air_dfree(free_ids); air_dfree(nbr); air_dfree(cnt); air_dfree(rowlen); air_dfree(scan);
    }
};

int build_pattern(const air_hdg_mesh *M, const air_hdg_ref *R, int dlen, int64_t *row_ptr, Pattern &P,
                  cudaStream_t s) {
    const int64_t F = M->n_facets;
    const int D = M->D, B = R->b, MAXN = 2 * D;
    int32_t *flag = nullptr;
    AIR_TRY(dalloc(&flag, F));
    AIR_TRY(dalloc(&P.scan, F + 1));
    free_flag_kernel<<<air_counted(grid_for(F, 256)), 256, 0, s>>>(F, M->facet_kind, flag);
    AIR_LAUNCH();
    int st = air_exclusive_scan_i32(flag, P.scan, F, s);
    air_dfree(flag);
    AIR_TRY(st);
    AIR_CUDA(cudaMemcpyAsync(&P.nfree, P.scan + F, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    AIR_CUDA(cudaStreamSynchronize(s));
    AIR_TRY(dalloc(&P.rnum, F));
    AIR_TRY(dalloc(&P.free_ids, P.nfree));
    renumber_kernel<<<air_counted(grid_for(F, 256)), 256, 0, s>>>(F, M->facet_kind, P.scan, P.rnum, P.free_ids);
    AIR_LAUNCH();
    AIR_TRY(dalloc(&P.nbr, P.nfree * MAXN));
    AIR_TRY(dalloc(&P.cnt, P.nfree));
    AIR_TRY(dalloc(&P.rowlen, P.nfree * B));
    if (D == 2)
        neighbour_kernel<2><<<air_counted(grid_for(P.nfree, 256)), 256, 0, s>>>(
            P.nfree, B, dlen, P.free_ids, M->facet_elems, M->elem_facets, M->facet_kind, P.rnum, P.nbr, P.cnt,
            P.rowlen);
    else
        neighbour_kernel<3><<<air_counted(grid_for(P.nfree, 256)), 256, 0, s>>>(
            P.nfree, B, dlen, P.free_ids, M->facet_elems, M->elem_facets, M->facet_kind, P.rnum, P.nbr, P.cnt,
            P.rowlen);
    AIR_LAUNCH();
    int64_t *rp = row_ptr;
    if (!rp) AIR_TRY(dalloc(&rp, P.nfree * B + 1));
    st = air_exclusive_scan_i32(P.rowlen, rp, P.nfree * B, s);
    if (st == AIR_OK) {
        cudaError_t e = cudaMemcpyAsync(&P.nnz, rp + P.nfree * B, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = AIR_ERR_CUDA;
    }
    if (!row_ptr) air_dfree(rp);
    return st;
}

template <int D, int P>
int launch_element(const ElemArgs &a, bool gradient, cudaStream_t s) {
    using Dm = Dims<D, P>;
    const size_t smem = (size_t)WPB * Dm::WARP_DOUBLES * sizeof(double);
    if (smem > AIR_SMEM_OPTIN) return AIR_ERR_UNSUPPORTED;
    const unsigned grid = (unsigned)((a.E + WPB - 1) / WPB);
    if (gradient) {
        AIR_CUDA(air_smem_optin(velocity_gradient_kernel<D, P>));
        velocity_gradient_kernel<D, P><<<air_counted(grid), WPB * 32, smem, s>>>(a);
    } else {
        AIR_CUDA(air_smem_optin(hdg_element_kernel<D, P>));
        hdg_element_kernel<D, P><<<air_counted(grid), WPB * 32, smem, s>>>(a);
    }
    AIR_LAUNCH();
    return AIR_OK;
}

int dispatch_element(int D, int p, const ElemArgs &a, bool gradient, cudaStream_t s) {
    switch (D * 10 + p) {
    case 21: return launch_element<2, 1>(a, gradient, s);
    case 22: return launch_element<2, 2>(a, gradient, s);
    case 23: return launch_element<2, 3>(a, gradient, s);
    case 31: return launch_element<3, 1>(a, gradient, s);
    case 32: return launch_element<3, 2>(a, gradient, s);
    case 33: return launch_element<3, 3>(a, gradient, s);
    default: return AIR_ERR_INVALID_ARG;
    }
}

ElemArgs element_args(const air_hdg_mesh *M, const air_hdg_ref *R, const air_hdg_data *d) {
    ElemArgs a{};
    a.E = M->n_elems;
    a.nu = d->nu;
    a.alpha = d->alpha;
    a.verts = M->verts;
    a.elems = M->elems;
    a.elem_facets = M->elem_facets;
    a.facet_elems = M->facet_elems;
    a.kind = M->facet_kind;
    a.wq = R->wq; a.phi = R->phi; a.gphi = R->gphi; a.wf = R->wf; a.psi = R->psi;
    a.phi_f = R->phi_f; a.gphi_f = R->gphi_f; a.perms = R->perms;
    a.vel_vol = d->vel_vol; a.src = d->src; a.vel_face = d->vel_face; a.u0_face = d->u0_face;
    return a;
}

int read_err(int *d_err, cudaStream_t s) {
    int h = 0;
    AIR_CUDA(cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    AIR_CUDA(cudaStreamSynchronize(s));
    if (h & AIR_DEVERR_SINGULAR) return AIR_ERR_SINGULAR_COARSE;
    if (h & AIR_DEVERR_CSR) return AIR_ERR_CSR_MALFORMED;
    return AIR_OK;
}

int assemble_impl(const air_hdg_mesh *M, const air_hdg_ref *R, const air_hdg_data *d, int scale, int64_t *row_ptr,
                  int32_t *col, double *val, double *rhs, double *diag, double *lam_dir, cudaStream_t s) {
    const int D = M->D, B = R->b, dlen = scale ? 1 : B;
    const int64_t F = M->n_facets;
    Pattern P;
    AIR_TRY(build_pattern(M, R, dlen, row_ptr, P, s));
    if (D == 2)
        columns_kernel<4><<<air_counted(grid_for(P.nfree * B, 256)), 256, 0, s>>>(P.nfree, B, dlen, P.nbr, P.cnt,
                                                                                   row_ptr, col);
    else
        columns_kernel<6><<<air_counted(grid_for(P.nfree * B, 256)), 256, 0, s>>>(P.nfree, B, dlen, P.nbr, P.cnt,
                                                                                   row_ptr, col);
    AIR_LAUNCH();
    double *ld = lam_dir, *dpart = nullptr, *hpart = nullptr;
    int *d_err = nullptr;
    int st = AIR_OK;
    if (!ld) st = dalloc(&ld, F * B);
    if (st == AIR_OK) st = dalloc(&dpart, 2 * F * B * B);
    if (st == AIR_OK) st = dalloc(&hpart, 2 * F * B);
    if (st == AIR_OK) st = dalloc(&d_err, 1);
    if (st == AIR_OK) {
        cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(int), s);
        if (e != cudaSuccess) st = AIR_ERR_CUDA;
    }
    if (st == AIR_OK) {
        dirichlet_kernel<<<air_counted(grid_for(F * B, 256)), 256, 0, s>>>(F, B, R->nqf, M->facet_kind, R->dir_proj,
                                                                          d->g_dir, ld);
        if (cudaGetLastError() != cudaSuccess) st = AIR_ERR_CUDA;
    }
    if (st == AIR_OK) {
        ElemArgs a = element_args(M, R, d);
        a.dlen = dlen;
        a.rnum = P.rnum; a.nbr = P.nbr; a.nbr_cnt = P.cnt; a.row_ptr = row_ptr;
        a.lam_dir = ld; a.val = val; a.dpart = dpart; a.hpart = hpart; a.err = d_err;
        st = dispatch_element(D, R->p, a, false, s);
    }
    if (st == AIR_OK) {
        FacetArgs fa{};
        fa.nfree = P.nfree; fa.B = B; fa.dlen = dlen; fa.maxn = 2 * D; fa.scale = scale;
        fa.free_ids = P.free_ids; fa.facet_elems = M->facet_elems; fa.nbr = P.nbr; fa.cnt = P.cnt;
        fa.row_ptr = row_ptr; fa.dpart = dpart; fa.hpart = hpart; fa.val = val; fa.rhs = rhs; fa.diag = diag;
        fa.err = d_err;
        const size_t smem = (size_t)FWPB * 6 * B * B * sizeof(double);
        facet_kernel<<<air_counted((unsigned)((P.nfree + FWPB - 1) / FWPB)), FWPB * 32, smem, s>>>(fa);
        if (cudaGetLastError() != cudaSuccess) st = AIR_ERR_CUDA;
    }
    if (st == AIR_OK) st = read_err(d_err, s);
    if (!lam_dir) air_dfree(ld);
    air_dfree(dpart);
    air_dfree(hpart);
    air_dfree(d_err);
    return st;
}

}  // namespace

extern "C" {

int air_hdg_points(const air_hdg_mesh *M, const air_hdg_ref *R, double *x_vol, double *x_face, double *x_facet,
                   void *stream) {
    AIR_TRY(check_ref(M, R));
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t E = M->n_elems, F = M->n_facets;
    const int D = M->D;
    if (x_vol || x_face) {
        const int64_t items = E * (R->nq + (int64_t)(D + 1) * R->nqf);
        if (D == 2)
            points_kernel<2><<<air_counted(grid_for(items, 256)), 256, 0, s>>>(E, R->nq, R->nqf, R->nperm, M->verts,
                                                                               M->elems, R->xq, R->xi_f, R->perms,
                                                                               x_vol, x_face);
        else
            points_kernel<3><<<air_counted(grid_for(items, 256)), 256, 0, s>>>(E, R->nq, R->nqf, R->nperm, M->verts,
                                                                               M->elems, R->xq, R->xi_f, R->perms,
                                                                               x_vol, x_face);
        AIR_LAUNCH();
    }
    if (x_facet) {
        facet_points_kernel<<<air_counted(grid_for(F * R->nqf, 256)), 256, 0, s>>>(F, D, R->nqf, M->verts, M->facets,
                                                                                   R->sq, x_facet);
        AIR_LAUNCH();
    }
    return AIR_OK;
}

int air_hdg_size(const air_hdg_mesh *M, const air_hdg_ref *R, int scale, int64_t *n_rows, int64_t *nnz,
                 void *stream) {
    AIR_TRY(check_ref(M, R));
    if (!n_rows || !nnz) return AIR_ERR_INVALID_ARG;
    AirCallStream call((cudaStream_t)stream);
    Pattern P;
    AIR_TRY(build_pattern(M, R, scale ? 1 : R->b, nullptr, P, (cudaStream_t)stream));
    *n_rows = P.nfree * R->b;
    *nnz = P.nnz;
    return AIR_OK;
}

int air_hdg_assemble(const air_hdg_mesh *M, const air_hdg_ref *R, const air_hdg_data *data, int scale,
                     int64_t *row_ptr, int32_t *col, double *val, double *rhs, double *diag, double *lam_dir,
                     void *stream) {
    AIR_TRY(check_ref(M, R));
    if (!data || !row_ptr || !col || !val || !rhs || !data->vel_vol || !data->vel_face || !(data->nu >= 0.0))
        return AIR_ERR_INVALID_ARG;
    AirCallStream call((cudaStream_t)stream);
    return assemble_impl(M, R, data, scale ? 1 : 0, row_ptr, col, val, rhs, diag, lam_dir, (cudaStream_t)stream);
}

int air_hdg_velocity_gradient(const air_hdg_mesh *M, const air_hdg_ref *R, const air_hdg_data *data,
                              const double *diag, const double *lam_dir, const double *lam, const double *adj,
                              double *grad, void *stream) {
    AIR_TRY(check_ref(M, R));
    if (!data || !diag || !lam_dir || !lam || !adj || !grad || !data->vel_vol || !data->vel_face)
        return AIR_ERR_INVALID_ARG;
    AirCallStream call((cudaStream_t)stream);
    cudaStream_t s = (cudaStream_t)stream;
    const int D = M->D, B = R->b;
    const int64_t F = M->n_facets;
    Pattern P;
    AIR_TRY(build_pattern(M, R, 1, nullptr, P, s));
    double *mu_full = nullptr, *lam_full = nullptr;
    int *d_err = nullptr;
    int st = dalloc(&mu_full, F * B);
    if (st == AIR_OK) st = dalloc(&lam_full, F * B);
    if (st == AIR_OK) st = dalloc(&d_err, 1);
    if (st == AIR_OK && cudaMemsetAsync(d_err, 0, sizeof(int), s) != cudaSuccess) st = AIR_ERR_CUDA;
    if (st == AIR_OK) {
        const size_t smem = (size_t)FWPB * 4 * B * B * sizeof(double);
        adjoint_unscale_kernel<<<air_counted((unsigned)((P.nfree + FWPB - 1) / FWPB)), FWPB * 32, smem, s>>>(
            F, P.nfree, B, P.free_ids, diag, lam, adj, mu_full, lam_full, d_err);
        spread_dirichlet_kernel<<<air_counted(grid_for(F * B, 256)), 256, 0, s>>>(F, B, M->facet_kind, lam_dir,
                                                                                   mu_full, lam_full);
        if (cudaGetLastError() != cudaSuccess) st = AIR_ERR_CUDA;
    }
    if (st == AIR_OK) {
        ElemArgs a = element_args(M, R, data);
        a.lam_full = lam_full;
        a.mu_full = mu_full;
        a.grad = grad;
        a.err = d_err;
        st = dispatch_element(D, R->p, a, true, s);
    }
    if (st == AIR_OK) st = read_err(d_err, s);
    air_dfree(mu_full);
    air_dfree(lam_full);
    air_dfree(d_err);
    return st;
}

}  // extern "C"
