// Small dense kernels shared by the warp-per-block routines: one warp
// inverts a b x b matrix held in shared memory.
#pragma once

#include <math.h>

// Gauss-Jordan inversion of the warp's n x n matrix M (row-major) into Minv,
// with partial pivoting (ties -> smallest row).  W is 2 n^2 scratch; every
// pointer is shared memory of the calling warp and all 32 lanes call it.
// Returns false if a pivot is zero.
__device__ inline bool warp_inverse(const double *M, int n, double *W, double *Minv) {
    const unsigned FULLM = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int w2 = 2 * n;
    for (int t = lane; t < n * w2; t += 32) {
        const int r = t / w2, c = t % w2;
        W[t] = c < n ? M[r * n + c] : (c - n == r ? 1.0 : 0.0);
    }
    __syncwarp();
    for (int c = 0; c < n; ++c) {
        double v = -1.0;
        int r = n;
        for (int rr = c + lane; rr < n; rr += 32) {
            const double av = fabs(W[rr * w2 + c]);
            if (av > v) { v = av; r = rr; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_down_sync(FULLM, v, o);
            const int orow = __shfl_down_sync(FULLM, r, o);
            if (ov > v || (ov == v && orow < r)) { v = ov; r = orow; }
        }
        r = __shfl_sync(FULLM, r, 0);
        v = __shfl_sync(FULLM, v, 0);
        if (!(v > 0.0)) return false;
        if (r != c)
            for (int t = lane; t < w2; t += 32) {
                const double x = W[c * w2 + t];
                W[c * w2 + t] = W[r * w2 + t];
                W[r * w2 + t] = x;
            }
        __syncwarp();
        const double piv = W[c * w2 + c];
        for (int t = lane; t < w2; t += 32) W[c * w2 + t] = W[c * w2 + t] / piv;
        __syncwarp();
        for (int t = lane; t < n * w2; t += 32) {
            const int rr = t / w2, cc = t % w2;
            if (rr == c || cc == c) continue;
            W[t] -= W[rr * w2 + c] * W[c * w2 + cc];
        }
        __syncwarp();
        for (int rr = lane; rr < n; rr += 32)
            if (rr != c) W[rr * w2 + c] = 0.0;
        __syncwarp();
    }
    for (int t = lane; t < n * n; t += 32) Minv[t] = W[(t / n) * w2 + n + t % n];
    __syncwarp();
    return true;
}
