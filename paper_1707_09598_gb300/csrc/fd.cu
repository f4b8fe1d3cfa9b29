// Fast-diagonalisation preconditioner: batched mode products with the 1D
// generalised eigenvectors (not in the paper; it cites fast-diagonalisation
// solvers among the fast-IGA methods and lists their combination with sparse
// grids as future work, Sec. 5).
//
//   z = (U_d x .. x U_1) diag(sum_k lambda_{k,i_k})^{-1} (U_d x .. x U_1)^T r
//
// One pass applies Mat = U_k^T (forward) or U_k (backward) along direction k of
// every component: out[a][i][b] = sum_j Mat[i][j] in[a][j][b], a GEMM with
// M = K = n_k and ncol = ndof / n_k columns. Two work layouts; the autotuner
// measures both and keeps the faster for the plan's precision:
//   per piece: SMALL (n_k <= 64), ROWS (long direction, < 64 columns) and
//         TILE (otherwise) items of one piece each, shaped so that FP64 work
//         is not wasted on padding (FP64 is bound by its FMA pipe);
//   grouped: SMALL items, and for longer directions all pieces whose
//         direction k uses the same eigenvector matrix form one GEMM over all
//         their fibres (a "segment"), cut into output tiles of 64x64, 128x32
//         or 256x16 (by column count) with 4 x 4 outputs per thread. Each
//         element of U read from memory then serves many pieces' columns,
//         which is what the latency-bound FP32 instances need.
// Contractions longer than the autotuned depth are split into items whose
// partial sums add atomically into an output cleared before the pass.
// The division by the eigenvalue sums is a separate elementwise pass between
// the forward and the backward passes, with the reciprocals precomputed per
// entry.
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

// Per-piece items: SMALL (one output per thread, Mat in shared memory), ROWS
// (one lane per row, a group of at most 8 columns in registers; Mat read through
// its transpose so that a warp's loads are coalesced) and TILE (32 x 64 output
// tile, 16-deep K loop through shared memory, 2 x 4 outputs per thread).
template <typename Real>
__global__ void __launch_bounds__(256, 2)
k_fd_pass(DevPlan P, const FDItem* __restrict__ items, int dir, int forward,
          const Real* __restrict__ in, Real* __restrict__ out, const int* __restrict__ active) {
    __shared__ double sm_raw[6144];
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
        // a tile of nc fibres: Mat (n x n) and the fibres (n x nc) staged in
        // shared memory, each read from memory once, then Y = Mat X. With
        // B = 1 a fibre is contiguous, so threads run along the fibre;
        // otherwise neighbouring fibres are neighbours in memory, so threads
        // run across fibres.
        const long long rest = Ncol - it.c0;
        const int nc = rest < fd_small_cols(n) ? (int)rest : fd_small_cols(n);
        const int ms = n + 1, xs = nc + 1;
        Real* Ms = sm;
        Real* Xs = sm + n * ms;
        for (int l = threadIdx.x; l < n * n; l += blockDim.x) {
            const int i = l / n, j = l - i * n;
            Ms[i * ms + j] = forward ? U[(long long)j * n + i] : U[(long long)i * n + j];
        }
        const bool unit = B == 1;
        for (int l = threadIdx.x; l < n * nc; l += blockDim.x) {
            const int j = unit ? l % n : l / nc, cl = unit ? l / n : l % nc;
            const long long col = it.c0 + cl, a = col / B, b = col - a * B;
            Xs[j * xs + cl] = vin[a * n * B + (long long)j * B + b];
        }
        __syncthreads();
        for (int l = threadIdx.x; l < n * nc; l += blockDim.x) {
            const int i = unit ? l % n : l / nc, cl = unit ? l / n : l % nc;
            Real acc = 0;
            for (int j = 0; j < n; ++j) acc += Ms[i * ms + j] * Xs[j * xs + cl];
            const long long col = it.c0 + cl, a = col / B, b = col - a * B;
            const long long oi = a * n * B + (long long)i * B + b;
            if (SGIGA_GUARD(P, oi >= 0 && oi < g.fd_n, CHK_FD_SMALL)) vout[oi] = acc;
        }
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

// Four consecutive values from shared memory (16-byte aligned): one 128-bit
// load for FP32, two for FP64.
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
    const double2 q0 = *reinterpret_cast<const double2*>(p);
    const double2 q1 = *reinterpret_cast<const double2*>(p + 2);
    v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}

// Asynchronous element copy global -> shared (cp.async, L1-allocating), or
// zero fill when src is null (src-size 0: nothing is read; the instruction
// still gets a valid global address, `any`).
template <typename Real>
__device__ __forceinline__ void cp_async_elem(Real* dst, const Real* src, const Real* any) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int n = src ? (int)sizeof(Real) : 0;
    const Real* g = src ? src : any;
    if constexpr (sizeof(Real) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(g), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(g), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Dynamic shared memory of k_fd_level<Real, TN>: two stages of the MT tile
// [16][TM + 4] and the X tile [16][TN + 4].
template <typename Real, int TN>
constexpr size_t fd_level_smem() {
    return 2 * 16 * ((4096 / TN + 4) + (TN + 4)) * sizeof(Real);
}

// LEVEL items: Y[i][c] = sum_j MT[j][i] X[j][c] over one TM x TN tile
// (TM = 4096 / TN); thread (tx, ty) owns rows 4 ty .. 4 ty + 3 and columns
// 4 tx .. 4 tx + 3. Segments with few columns (the long directions of the most
// anisotropic components) take tall tiles so that the lanes stay busy. Rows and
// columns past the segment's end are neither computed nor written: the last
// row tile of an n = 2^l + p - 2 direction holds only p - 2 rows.
// The K loop is double-buffered: the copies of the next 16 rows of MT and X
// (cp.async, zero-filled past the item's range) are in flight while the
// current 16 are multiplied out of shared memory.
template <typename Real, int TN>
__global__ void __launch_bounds__(256)
k_fd_level(DevPlan P, const FDItem* __restrict__ items, int forward, const Real* __restrict__ in,
           Real* __restrict__ out, const int* __restrict__ active) {
    constexpr int TM = 4096 / TN, NTX = TN / 4;
    constexpr int LA = 16 * TM / 256, LB = 16 * TN / 256;   // tile copies per thread per K step
    constexpr int SA = 16 * (TM + 4), SB = 16 * (TN + 4);  // elements per stage
    extern __shared__ __align__(16) unsigned char fd_smem[];
    Real* const Abuf = reinterpret_cast<Real*>(fd_smem);   // [2][16][TM + 4]
    Real* const Bbuf = Abuf + 2 * SA;                       // [2][16][TN + 4]
    const FDItem it = items[blockIdx.x];
    const FDSeg sg = P.fdsegs[it.grid];
    const Eig1D e = P.eigs[sg.eig];
    const Real* __restrict__ MT = forward ? FDData<Real>::U(P) + e.uoff : FDData<Real>::Ut(P) + e.uoff;
    const int n = sg.n, tid = threadIdx.x;
    const long long* cb = P.fdcb + sg.col0;
    const int* cs = P.fdcs + sg.col0;
    const int* cc = P.fdcc + sg.col0;
    const int i0 = it.i0;
    const int c0 = (int)it.c0;
    const int nrows = min(TM, n - i0), ncols = min(TN, sg.ncols - c0);
    const bool split = it.j0 > 0 || it.j1 < n;
    // this thread's copies of the X tile per K step: (kk, column) fixed over the loop
    int ldk[LB], ldc[LB];
    const Real* ldp[LB];
    long long lds[LB];
#pragma unroll
    for (int u = 0; u < LB; ++u) {
        const int l = tid + 256 * u;
        int kk, col;
        if (sg.unit) { kk = l & 15; col = l >> 4; }   // stride-1 fibres: runs of 16 along j
        else { col = l % TN; kk = l / TN; }            // strided fibres: neighbouring columns
        ldk[u] = kk;
        ldc[u] = col;
        const bool ok = col < ncols && (!active || active[cc[c0 + col]]);
        ldp[u] = ok ? in + cb[c0 + col] : nullptr;
        lds[u] = ok ? cs[c0 + col] : 0;
    }
    // stage `buf` <- rows j0 .. j0 + 15 of MT (this item's rows) and of X
    auto issue = [&](int buf, int j0) {
        const int kn = min(16, it.j1 - j0);
        Real* As = Abuf + buf * SA;
        Real* Bs = Bbuf + buf * SB;
#pragma unroll
        for (int u = 0; u < LA; ++u) {
            const int l = tid + 256 * u;
            const int kk = l / TM, ii = l % TM;
            cp_async_elem(As + kk * (TM + 4) + ii,
                          (ii < nrows && kk < kn) ? MT + (long long)(j0 + kk) * n + i0 + ii : nullptr, MT);
        }
#pragma unroll
        for (int u = 0; u < LB; ++u)
            cp_async_elem(Bs + ldk[u] * (TN + 4) + ldc[u],
                          (ldp[u] && ldk[u] < kn) ? ldp[u] + (long long)(j0 + ldk[u]) * lds[u] : nullptr, MT);
        cp_async_commit();
    };
    const int tx = tid % NTX, ty = tid / NTX;
    const bool work = 4 * ty < nrows && 4 * tx < ncols;
    Real acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = Real(0);
    const int nsteps = (it.j1 - it.j0 + 15) / 16;
    if (nsteps > 0) issue(0, it.j0);
    for (int st = 0; st < nsteps; ++st) {
        const int buf = st & 1;
        if (st + 1 < nsteps) {
            issue(buf ^ 1, it.j0 + 16 * (st + 1));
            cp_async_wait<1>();   // this step's stage has landed (the next may be in flight)
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        if (work) {
            const Real* As = Abuf + buf * SA;
            const Real* Bs = Bbuf + buf * SB;
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {   // rows past the item's range are zero
                Real a[4], b[4];
                ld4(As + kk * (TM + 4) + 4 * ty, a);
                ld4(Bs + kk * (TN + 4) + 4 * tx, b);
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] += a[r] * b[c];
            }
        }
        __syncthreads();   // the stage is read before the next issue overwrites it
    }
    if (!work) return;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int col = 4 * tx + c;
        if (col >= ncols) continue;
        if (active && !active[cc[c0 + col]]) continue;
        Real* o = out + cb[c0 + col];
        const long long st = cs[c0 + col];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = 4 * ty + r;
            if (i >= nrows) continue;
            const long long oi = cb[c0 + col] + (long long)(i0 + i) * st;
            if (!SGIGA_GUARD(P, oi >= 0 && oi < P.nfd, CHK_FD_LEVEL)) continue;
            if (split) atomicAdd(o + (long long)(i0 + i) * st, acc[r][c]);
            else o[(long long)(i0 + i) * st] = acc[r][c];
        }
    }
}

// The level kernels' dynamic shared memory above the 48 KB default (FP64, TN =
// 16 needs 70 KB); set once per process and device before the first launch.
cudaError_t fd_prepare() {
    cudaError_t e = cudaSuccess;
#define FDSET(R, TN)                                                                                    \
    if (e == cudaSuccess)                                                                               \
        e = cudaFuncSetAttribute(k_fd_level<R, TN>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                                 (int)fd_level_smem<R, TN>());
    FDSET(double, 16) FDSET(double, 32) FDSET(double, 64) FDSET(float, 16) FDSET(float, 32) FDSET(float, 64)
#undef FDSET
    return e;
}

template <typename Real>
cudaError_t launch_fd_pass(const DevPlan& P, const FDLists& L, int dir, int forward, const Real* in, Real* out,
                           const int* active, cudaStream_t s, const FDStreams* fs) {
    cudaError_t e = cudaSuccess;
    const int nk = (L.nlvl[0] > 0) + (L.nlvl[1] > 0) + (L.nlvl[2] > 0) + (L.nsmall > 0);
    const bool fork = fs && nk > 1;
    if (fork && (e = cudaEventRecord(fs->fork, s)) != cudaSuccess) return e;
    int branch = 0;
    // the first kernel runs on s, each further one on its own branch
    auto begin = [&](cudaStream_t& ks) -> cudaError_t {
        ks = s;
        if (!fork || branch == 0) return cudaSuccess;
        ks = fs->aux[branch - 1];
        return cudaStreamWaitEvent(ks, fs->fork, 0);
    };
    auto end = [&](cudaStream_t ks) -> cudaError_t {
        cudaError_t r = cudaGetLastError();
        if (r == cudaSuccess && fork && branch > 0) r = cudaEventRecord(fs->join[branch - 1], ks);
        ++branch;
        return r;
    };
    cudaStream_t ks;
    if (L.nlvl[0] > 0) {
        if ((e = begin(ks)) != cudaSuccess) return e;
        SGIGA_COUNT_LAUNCH();
        k_fd_level<Real, 16><<<L.nlvl[0], 256, fd_level_smem<Real, 16>(), ks>>>(P, L.lvl[0], forward, in, out, active);
        if ((e = end(ks)) != cudaSuccess) return e;
    }
    if (L.nlvl[1] > 0) {
        if ((e = begin(ks)) != cudaSuccess) return e;
        SGIGA_COUNT_LAUNCH();
        k_fd_level<Real, 32><<<L.nlvl[1], 256, fd_level_smem<Real, 32>(), ks>>>(P, L.lvl[1], forward, in, out, active);
        if ((e = end(ks)) != cudaSuccess) return e;
    }
    if (L.nlvl[2] > 0) {
        if ((e = begin(ks)) != cudaSuccess) return e;
        SGIGA_COUNT_LAUNCH();
        k_fd_level<Real, 64><<<L.nlvl[2], 256, fd_level_smem<Real, 64>(), ks>>>(P, L.lvl[2], forward, in, out, active);
        if ((e = end(ks)) != cudaSuccess) return e;
    }
    if (L.nsmall > 0) {
        if ((e = begin(ks)) != cudaSuccess) return e;
        SGIGA_COUNT_LAUNCH();
        k_fd_pass<Real><<<L.nsmall, 256, 0, ks>>>(P, L.small, dir, forward, in, out, active);
        if ((e = end(ks)) != cudaSuccess) return e;
    }
    for (int b = 1; fork && b < branch; ++b)
        if ((e = cudaStreamWaitEvent(s, fs->join[b - 1], 0)) != cudaSuccess) return e;
    return cudaSuccess;
}
template cudaError_t launch_fd_pass<double>(const DevPlan&, const FDLists&, int, int, const double*, double*,
                                            const int*, cudaStream_t, const FDStreams*);
template cudaError_t launch_fd_pass<float>(const DevPlan&, const FDLists&, int, int, const float*, float*,
                                           const int*, cudaStream_t, const FDStreams*);

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
