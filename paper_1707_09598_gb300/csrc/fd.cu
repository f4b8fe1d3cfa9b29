// Fast-diagonalisation preconditioner: batched mode products with the 1D
// generalised eigenvectors (not in the paper; it cites fast-diagonalisation
// solvers among the fast-IGA methods and lists their combination with sparse
// grids as future work, Sec. 5).
//
//   z = (U_d x .. x U_1) diag(sum_k lambda_{k,i_k})^{-1} (U_d x .. x U_1)^T r
//
// One pass applies U_k^T (forward) or U_k (backward) along direction k of every
// component: out[a][i][b] = sum_j Mat[i][j] in[a][j][b], a GEMM with
// M = K = n_k and N = (ndof / n_k) columns. A block computes a 32 x 64 output
// tile with a 16-deep K loop staged in shared memory; each thread owns 2 x 4
// outputs in registers. The last forward pass divides by the eigenvalue sums.
#include "kernels.h"

namespace sgiga {

__global__ void __launch_bounds__(256)
k_fd_pass(DevPlan P, const FDItem* __restrict__ items, int dir, int forward, int scale,
          const double* __restrict__ in, double* __restrict__ out, const int* __restrict__ active) {
    __shared__ double As[16][33];
    __shared__ double Bs[16][65];
    const FDItem it = items[blockIdx.x];
    if (active && !active[it.grid]) return;
    const GridDesc& g = P.grids[it.grid];
    const int d = P.d;
    const int n = g.n[dir];
    long long B = 1, A = 1;
    for (int k = 0; k < dir; ++k) B *= g.n[k];
    for (int k = dir + 1; k < d; ++k) A *= g.n[k];
    const long long Ncol = A * B;
    const Eig1D e = P.eigs[g.eig[dir]];
    const double* __restrict__ U = P.U + e.uoff;
    const double* vin = in + g.dof_off;
    double* vout = out + g.dof_off;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[2][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = 0.0;
    for (int j0 = 0; j0 < n; j0 += 16) {
        for (int l = threadIdx.x; l < 512; l += 256) {
            int kk, ii;
            if (forward) { ii = l & 31; kk = l >> 5; } else { kk = l & 15; ii = l >> 4; }
            int i = it.i0 + ii, j = j0 + kk;
            double v = 0.0;
            if (i < n && j < n) v = forward ? U[(long long)j * n + i] : U[(long long)i * n + j];
            As[kk][ii] = v;
        }
        for (int l = threadIdx.x; l < 1024; l += 256) {
            int kk, cc;
            if (B == 1) { kk = l & 15; cc = l >> 4; } else { cc = l & 63; kk = l >> 6; }
            long long c = it.c0 + cc;
            int j = j0 + kk;
            double v = 0.0;
            if (c < Ncol && j < n) {
                long long a = c / B, b = c - a * B;
                v = vin[a * n * B + (long long)j * B + b];
            }
            Bs[kk][cc] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double a0 = As[kk][ty], a1 = As[kk][ty + 16];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                double b = Bs[kk][tx + 16 * c];
                acc[0][c] += a0 * b;
                acc[1][c] += a1 * b;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        int i = it.i0 + ty + 16 * r;
        if (i >= n) continue;
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4) {
            long long c = it.c0 + tx + 16 * c4;
            if (c >= Ncol) continue;
            long long a = c / B, b = c - a * B;
            long long idx = a * n * B + (long long)i * B + b;
            double v = acc[r][c4];
            if (scale) {
                long long rem = idx;
                double s = 0.0;
                for (int k = 0; k < d; ++k) {
                    int ik = (int)(rem % g.n[k]);
                    rem /= g.n[k];
                    s += P.lam[P.eigs[g.eig[k]].loff + ik];
                }
                v /= s;
            }
            vout[idx] = v;
        }
    }
}

cudaError_t launch_fd_pass(const DevPlan& P, const FDItem* items, int nitems, int dir, int forward, int scale,
                           const double* in, double* out, const int* active, cudaStream_t s) {
    if (nitems == 0) return cudaSuccess;
    SGIGA_COUNT_LAUNCH();
    k_fd_pass<<<nitems, 256, 0, s>>>(P, items, dir, forward, scale, in, out, active);
    return cudaGetLastError();
}

}  // namespace sgiga
