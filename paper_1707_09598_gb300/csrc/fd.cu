// Fast-diagonalisation preconditioner: batched mode products with the 1D
// generalised eigenvectors (not in the paper; it cites fast-diagonalisation
// solvers among the fast-IGA methods and lists their combination with sparse
// grids as future work, Sec. 5).
//
//   z = (U_d x .. x U_1) diag(sum_k lambda_{k,i_k})^{-1} (U_d x .. x U_1)^T r
//
// One pass applies Mat = U_k^T (forward) or U_k (backward) along direction k of
// every component: out[a][i][b] = sum_j Mat[i][j] in[a][j][b], a GEMM with
// M = K = n_k and ncol = ndof / n_k columns. Work items pick one of three
// shapes so that FP64 work is not wasted on padding:
//   SMALL (n_k <= 64): one thread per output, Mat staged in shared memory;
//   ROWS  (long direction, < 64 columns): one lane per row, a group of at most
//         8 columns in registers; Mat is read through its transpose so that a
//         warp's loads are coalesced, the input entries are warp broadcasts;
//   TILE  (otherwise): 32 x 64 output tile, 16-deep K loop through shared
//         memory, 2 x 4 outputs per thread.
// Long contractions (n_k > 128) are split into 128-deep ranges of j so that no
// block carries more than ~10^5 FMAs; such items add their partial sums
// atomically into an output that was cleared before the pass. The division by
// the eigenvalue sums is a separate elementwise pass between the forward and
// the backward passes, with the reciprocals precomputed per DoF.
#include "kernels.h"

namespace sgiga {

template <typename Real, int NC>
__device__ __forceinline__ void fd_rows(const Real* __restrict__ MT, const Real* __restrict__ vin,
                                        Real* __restrict__ vout, int n, long long B, int i, bool act,
                                        long long c0, int j0, int j1, bool split) {
    long long base[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        long long col = c0 + c, a = col / B;
        base[c] = a * n * B + (col - a * B);
    }
    Real acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0;
    const Real* mp = MT + (act ? i : 0);
    for (int j = j0; j < j1; ++j) {
        const Real m = act ? mp[(long long)j * n] : Real(0);
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] += m * __ldg(vin + base[c] + (long long)j * B);
    }
    if (!act) return;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        Real* o = vout + base[c] + (long long)i * B;
        if (split) atomicAdd(o, acc[c]); else *o = acc[c];
    }
}

template <typename Real> struct FDData;
template <> struct FDData<double> {
    static __device__ __forceinline__ const double* U(const DevPlan& P) { return P.U; }
    static __device__ __forceinline__ const double* Ut(const DevPlan& P) { return P.Ut; }
    static __device__ __forceinline__ const double* dinv(const DevPlan& P) { return P.dinv; }
};
template <> struct FDData<float> {
    static __device__ __forceinline__ const float* U(const DevPlan& P) { return P.Uf; }
    static __device__ __forceinline__ const float* Ut(const DevPlan& P) { return P.Utf; }
    static __device__ __forceinline__ const float* dinv(const DevPlan& P) { return P.dinvf; }
};

template <typename Real>
__global__ void __launch_bounds__(256, 2)
k_fd_pass(DevPlan P, const FDItem* __restrict__ items, int dir, int forward,
          const Real* __restrict__ in, Real* __restrict__ out, const int* __restrict__ active) {
    __shared__ double sm_raw[64 * 65];
    Real* sm = reinterpret_cast<Real*>(sm_raw);
    const FDItem it = items[blockIdx.x];
    const GridDesc& g = P.grids[it.grid];
    if (active && !active[g.comp]) return;
    const int d = P.d;
    const int n = g.fn[dir];
    long long B = 1, A = 1;
    for (int k = 0; k < dir; ++k) B *= g.fn[k];
    for (int k = dir + 1; k < d; ++k) A *= g.fn[k];
    const long long Ncol = A * B;
    const Eig1D e = P.eigs[g.eig[dir]];
    // Mat[i][j] = U[j][i] (forward) or U[i][j] (backward); MT[j][i] = Mat[i][j]
    const Real* __restrict__ U = FDData<Real>::U(P) + e.uoff;
    const Real* __restrict__ MT = forward ? FDData<Real>::U(P) + e.uoff : FDData<Real>::Ut(P) + e.uoff;
    const Real* vin = in + g.fd_off;
    Real* vout = out + g.fd_off;
    const bool split = it.j0 > 0 || it.j1 < n;

    if (it.mode == FD_SMALL) {
        for (int l = threadIdx.x; l < n * n; l += blockDim.x) {
            int i = l / n, j = l - i * n;
            sm[i * 65 + j] = forward ? U[(long long)j * n + i] : U[(long long)i * n + j];
        }
        __syncthreads();
        long long lin = it.c0 + threadIdx.x;
        if (lin >= g.fd_n) return;
        long long b = lin % B, r = lin / B;
        int i = (int)(r % n);
        long long a = r / n;
        const Real* vp = vin + a * n * B + b;
        Real acc = 0;
        for (int j = 0; j < n; ++j) acc += sm[i * 65 + j] * vp[(long long)j * B];
        vout[lin] = acc;
        return;
    }
    if (it.mode == FD_ROWS) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int i_w = it.i0 + 32 * warp;
        if (i_w >= n) return;
        const int i = i_w + lane;
        const bool act = i < n;
        switch (it.nc) {
#define CASE(NCV) case NCV: fd_rows<Real, NCV>(MT, vin, vout, n, B, i, act, it.c0, it.j0, it.j1, split); break;
            CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
        }
        return;
    }
    // FD_TILE
    Real (*As)[33] = reinterpret_cast<Real (*)[33]>(sm);
    Real (*Bs)[65] = reinterpret_cast<Real (*)[65]>(sm + 16 * 33);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    Real acc[2][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = 0;
    for (int j0 = it.j0; j0 < it.j1; j0 += 16) {
        for (int l = threadIdx.x; l < 512; l += 256) {
            int ii = l & 31, kk = l >> 5;
            int i = it.i0 + ii, j = j0 + kk;
            As[kk][ii] = (i < n && j < it.j1) ? MT[(long long)j * n + i] : Real(0);
        }
        for (int l = threadIdx.x; l < 1024; l += 256) {
            int kk, cc;
            if (B == 1) { kk = l & 15; cc = l >> 4; } else { cc = l & 63; kk = l >> 6; }
            long long c = it.c0 + cc;
            int j = j0 + kk;
            Real v = 0;
            if (c < Ncol && j < it.j1) {
                long long a = c / B, b = c - a * B;
                v = vin[a * n * B + (long long)j * B + b];
            }
            Bs[kk][cc] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            Real a0 = As[kk][ty], a1 = As[kk][ty + 16];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                Real b = Bs[kk][tx + 16 * c];
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
            if (split) atomicAdd(vout + idx, acc[r][c4]); else vout[idx] = acc[r][c4];
        }
    }
}

template <typename Real>
cudaError_t launch_fd_pass(const DevPlan& P, const FDItem* items, int nitems, int dir, int forward,
                           const Real* in, Real* out, const int* active, cudaStream_t s) {
    if (nitems == 0) return cudaSuccess;
    SGIGA_COUNT_LAUNCH();
    k_fd_pass<Real><<<nitems, 256, 0, s>>>(P, items, dir, forward, in, out, active);
    return cudaGetLastError();
}
template cudaError_t launch_fd_pass<double>(const DevPlan&, const FDItem*, int, int, int, const double*, double*,
                                            const int*, cudaStream_t);
template cudaError_t launch_fd_pass<float>(const DevPlan&, const FDItem*, int, int, int, const float*, float*,
                                           const int*, cudaStream_t);

// z[i] *= dinv[i] = 1 / sum_k lambda_{k, i_k} over every entry of the local layout.
template <typename Real>
__global__ void k_fd_scale(const Chunk* __restrict__ chunks, DevPlan P, Real* __restrict__ z,
                           const int* __restrict__ active) {
    const Chunk c = chunks[blockIdx.x];
    if (active && !active[c.grid]) return;
    const Real* dinv = FDData<Real>::dinv(P);
    for (int i = threadIdx.x; i < c.len; i += blockDim.x) z[c.start + i] *= dinv[c.start + i];
}

template <typename Real>
cudaError_t launch_fd_scale(const DevPlan& P, Real* z, const int* active, cudaStream_t s) {
    if (P.nfdchunks == 0) return cudaSuccess;
    SGIGA_COUNT_LAUNCH();
    k_fd_scale<Real><<<P.nfdchunks, 256, 0, s>>>(P.fdchunks, P, z, active);
    return cudaGetLastError();
}
template cudaError_t launch_fd_scale<double>(const DevPlan&, double*, const int*, cudaStream_t);
template cudaError_t launch_fd_scale<float>(const DevPlan&, float*, const int*, cudaStream_t);

// Multi-patch preconditioner (weighted additive Schwarz over the patches):
//   z = sum_pieces R_p^T D_p A_p^{-1} D_p R_p r,
// with A_p the piece's stiffness on its kept functions and natural conditions
// at patch interfaces, inverted exactly by fast diagonalisation. R_p gathers
// the piece's kept functions (interface functions appear in both pieces that
// share them) into the local layout; R_p^T adds them back. D_p = 1 / (number
// of pieces sharing the function), the Neumann-Neumann weighting: 1/2 on an
// interface. The excluded (0,0) corner of a piece is a zero entry of its
// tensor on the way in and dropped on the way out (the principal part of the
// local inverse stays SPD).
__device__ __forceinline__ double share_weight(const GridDesc& g, int f0, int f1) {
    const int m = 1 + (f0 == 0 && g.klo[0] == 0) + (f1 == 0 && g.klo[1] == 0);
    return m == 1 ? 1.0 : 1.0 / m;
}

template <typename Real>
__global__ void k_fd_gather(DevPlan P, const Real* __restrict__ r, Real* __restrict__ loc,
                            const int* __restrict__ active) {
    const Chunk c = P.fdchunks[blockIdx.x];
    if (active && !active[c.grid]) return;
    const GridDesc& g = P.grids[c.piece];
    for (int i = threadIdx.x; i < c.len; i += blockDim.x) {
        const long long l = c.start - g.fd_off + i;
        const int f0 = (int)(l % g.fn[0]) + g.klo[0], f1 = (int)(l / g.fn[0]) + g.klo[1];
        Real v = Real(0);
        if (!(g.xcorner && f0 == 0 && f1 == 0)) v = r[piece_addr2(P.grids, g, f0, f1)] * (Real)share_weight(g, f0, f1);
        loc[c.start + i] = v;
    }
}

template <typename Real>
__global__ void k_fd_scatter(DevPlan P, const Real* __restrict__ loc, Real* __restrict__ z,
                             const int* __restrict__ active) {
    const Chunk c = P.fdchunks[blockIdx.x];
    if (active && !active[c.grid]) return;
    const GridDesc& g = P.grids[c.piece];
    for (int i = threadIdx.x; i < c.len; i += blockDim.x) {
        const long long l = c.start - g.fd_off + i;
        const int f0 = (int)(l % g.fn[0]) + g.klo[0], f1 = (int)(l / g.fn[0]) + g.klo[1];
        if (g.xcorner && f0 == 0 && f1 == 0) continue;
        atomicAdd(z + piece_addr2(P.grids, g, f0, f1), loc[c.start + i] * (Real)share_weight(g, f0, f1));
    }
}

template <typename Real>
cudaError_t launch_fd_gather(const DevPlan& P, const Real* r, Real* loc, const int* active, cudaStream_t s) {
    if (P.nfdchunks == 0) return cudaSuccess;
    SGIGA_COUNT_LAUNCH();
    k_fd_gather<Real><<<P.nfdchunks, 256, 0, s>>>(P, r, loc, active);
    return cudaGetLastError();
}
template <typename Real>
cudaError_t launch_fd_scatter(const DevPlan& P, const Real* loc, Real* z, const int* active, cudaStream_t s) {
    if (P.nfdchunks == 0) return cudaSuccess;
    SGIGA_COUNT_LAUNCH();
    k_fd_scatter<Real><<<P.nfdchunks, 256, 0, s>>>(P, loc, z, active);
    return cudaGetLastError();
}
template cudaError_t launch_fd_gather<double>(const DevPlan&, const double*, double*, const int*, cudaStream_t);
template cudaError_t launch_fd_gather<float>(const DevPlan&, const float*, float*, const int*, cudaStream_t);
template cudaError_t launch_fd_scatter<double>(const DevPlan&, const double*, double*, const int*, cudaStream_t);
template cudaError_t launch_fd_scatter<float>(const DevPlan&, const float*, float*, const int*, cudaStream_t);

}  // namespace sgiga
