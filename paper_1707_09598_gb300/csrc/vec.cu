// Batched preconditioned-CG vector kernels: every component keeps its own
// scalars (alpha, beta, residual norms) and convergence flag. Packed vectors
// are cut into chunks of at most 4096 entries that never straddle two
// components; a block reduces its chunk, and a second kernel sums each
// component's chunk partials in a fixed order (deterministic dot products). Vectors may be FP64
// or FP32; scalars and reductions are FP64.
#include "kernels.h"

namespace sgiga {

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double ws[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) ws[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = threadIdx.x < nw ? ws[threadIdx.x] : 0.0;
    if (wid == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    return v;
}

__global__ void k_reduce(const CompDesc* __restrict__ comps, int ncomps, const double* __restrict__ partial,
                         double* __restrict__ out) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ncomps) return;
    double s = 0.0;
    const int c0 = comps[g].chunk0, nc = comps[g].nchunk;
    for (int c = 0; c < nc; ++c) s += partial[c0 + c];
    out[g] = s;
}

static cudaError_t reduce(const DevPlan& P, const double* partial, double* out, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_reduce<<<(P.ncomps + 127) / 128, 128, 0, s>>>(P.comps, P.ncomps, partial, out);
    return cudaGetLastError();
}

template <typename Real>
__global__ void k_dot(const Chunk* __restrict__ chunks, const Real* __restrict__ a, const Real* __restrict__ b,
                      double* __restrict__ partial) {
    const Chunk c = chunks[blockIdx.x];
    double s = 0.0;
    for (int i = threadIdx.x; i < c.len; i += blockDim.x) s += (double)a[c.start + i] * (double)b[c.start + i];
    s = block_sum(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

template <typename Real>
cudaError_t launch_dot(const DevPlan& P, const Real* a, const Real* b, double* partial, double* out,
                       cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_dot<Real><<<P.nchunks, 256, 0, s>>>(P.chunks, a, b, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return reduce(P, partial, out, s);
}

// x = 0, r = b, partial sums of ||b||^2
template <typename Real>
__global__ void k_pcg_init(const Chunk* __restrict__ chunks, const Real* __restrict__ b, Real* __restrict__ x,
                           Real* __restrict__ r, double* __restrict__ partial) {
    const Chunk c = chunks[blockIdx.x];
    double s = 0.0;
    for (int i = threadIdx.x; i < c.len; i += blockDim.x) {
        Real v = b[c.start + i];
        x[c.start + i] = Real(0);
        r[c.start + i] = v;
        s += (double)v * (double)v;
    }
    s = block_sum(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

template <typename Real>
cudaError_t launch_pcg_init(const DevPlan& P, const Real* b, Real* x, Real* r, double* partial, double* bb,
                            cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_pcg_init<Real><<<P.nchunks, 256, 0, s>>>(P.chunks, b, x, r, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return reduce(P, partial, bb, s);
}

template <typename Real>
__global__ void k_update_xr(const Chunk* __restrict__ chunks, Real* __restrict__ x, Real* __restrict__ r,
                            const Real* __restrict__ p, const Real* __restrict__ q,
                            const double* __restrict__ alpha, const int* __restrict__ active,
                            double* __restrict__ partial) {
    const Chunk c = chunks[blockIdx.x];
    double s = 0.0;
    if (active[c.grid]) {
        const Real al = (Real)alpha[c.grid];
        for (int i = threadIdx.x; i < c.len; i += blockDim.x) {
            long long k = c.start + i;
            x[k] += al * p[k];
            Real rv = r[k] - al * q[k];
            r[k] = rv;
            s += (double)rv * (double)rv;
        }
    } else {
        for (int i = threadIdx.x; i < c.len; i += blockDim.x) {
            double rv = r[c.start + i];
            s += rv * rv;
        }
    }
    s = block_sum(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

template <typename Real>
cudaError_t launch_pcg_update_xr(const DevPlan& P, Real* x, Real* r, const Real* p, const Real* q,
                                 const double* alpha, const int* active, double* partial, double* rr,
                                 cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_update_xr<Real><<<P.nchunks, 256, 0, s>>>(P.chunks, x, r, p, q, alpha, active, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return reduce(P, partial, rr, s);
}

template <typename Real>
__global__ void k_update_p(const Chunk* __restrict__ chunks, Real* __restrict__ p, const Real* __restrict__ z,
                           const double* __restrict__ beta, const int* __restrict__ active) {
    const Chunk c = chunks[blockIdx.x];
    if (!active[c.grid]) return;
    const Real be = (Real)beta[c.grid];
    for (int i = threadIdx.x; i < c.len; i += blockDim.x) {
        long long k = c.start + i;
        p[k] = z[k] + be * p[k];
    }
}

template <typename Real>
cudaError_t launch_pcg_update_p(const DevPlan& P, Real* p, const Real* z, const double* beta, const int* active,
                                cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_update_p<Real><<<P.nchunks, 256, 0, s>>>(P.chunks, p, z, beta, active);
    return cudaGetLastError();
}

template <typename Real>
__global__ void k_copy(Real* __restrict__ dst, const Real* __restrict__ src, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride) dst[i] = src[i];
}

template <typename Real>
cudaError_t launch_copy(Real* dst, const Real* src, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    SGIGA_COUNT_LAUNCH();
    k_copy<Real><<<(int)blocks, 256, 0, s>>>(dst, src, n);
    return cudaGetLastError();
}

#define INST(R)                                                                                                  \
    template cudaError_t launch_dot<R>(const DevPlan&, const R*, const R*, double*, double*, cudaStream_t);    \
    template cudaError_t launch_pcg_init<R>(const DevPlan&, const R*, R*, R*, double*, double*, cudaStream_t);  \
    template cudaError_t launch_pcg_update_xr<R>(const DevPlan&, R*, R*, const R*, const R*, const double*,     \
                                                 const int*, double*, double*, cudaStream_t);                  \
    template cudaError_t launch_pcg_update_p<R>(const DevPlan&, R*, const R*, const double*, const int*,        \
                                                cudaStream_t);                                                 \
    template cudaError_t launch_copy<R>(R*, const R*, long long, cudaStream_t);
INST(double)
INST(float)
#undef INST

__global__ void k_alpha(int ng, const double* __restrict__ rz, const double* __restrict__ pq,
                        double* __restrict__ alpha, const int* __restrict__ active) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    double den = pq[g];
    alpha[g] = (active[g] && den != 0.0) ? rz[g] / den : 0.0;
}

cudaError_t launch_pcg_alpha(const DevPlan& P, const double* rz, const double* pq, double* alpha,
                             const int* active, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_alpha<<<(P.ncomps + 127) / 128, 128, 0, s>>>(P.ncomps, rz, pq, alpha, active);
    return cudaGetLastError();
}

// beta = (rz_new - rz_mid) / rz; rz_mid = r_new . z_old for the flexible
// (Polak-Ribiere) variant, absent for plain PCG
__global__ void k_beta(int ng, double* __restrict__ rz, const double* __restrict__ rznew,
                       const double* __restrict__ rzmid, double* __restrict__ beta) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    double old = rz[g];
    double num = rznew[g] - (rzmid ? rzmid[g] : 0.0);
    beta[g] = old != 0.0 ? num / old : 0.0;
    rz[g] = rznew[g];
}

cudaError_t launch_pcg_beta(const DevPlan& P, double* rz, const double* rznew, const double* rzmid, double* beta,
                            cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_beta<<<(P.ncomps + 127) / 128, 128, 0, s>>>(P.ncomps, rz, rznew, rzmid, beta);
    return cudaGetLastError();
}

// active[g] stays 1 while ||r_g||^2 > tol^2 ||b_g||^2; counts the active grids.
__global__ void k_check(int ng, const double* __restrict__ rr, const double* __restrict__ bb, double tol2,
                        int* __restrict__ active, int* __restrict__ iters, int* __restrict__ nactive) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    if (!active[g]) return;
    iters[g] += 1;
    if (rr[g] <= tol2 * bb[g]) active[g] = 0;
    else atomicAdd(nactive, 1);
}

cudaError_t launch_pcg_check(const DevPlan& P, const double* rr, const double* bb, double tol2, int* active,
                             int* iters, int* nactive, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(nactive, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    SGIGA_COUNT_LAUNCH();
    k_check<<<(P.ncomps + 127) / 128, 128, 0, s>>>(P.ncomps, rr, bb, tol2, active, iters, nactive);
    return cudaGetLastError();
}

// Start mask: active[g] = (bb[g] > 0) && (outer == null || outer[g]); iters[g] = 0.
__global__ void k_start(int ng, const double* __restrict__ bb, const int* __restrict__ outer,
                        int* __restrict__ active, int* __restrict__ iters) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    active[g] = (bb[g] > 0.0 && (!outer || outer[g])) ? 1 : 0;
    iters[g] = 0;
}

cudaError_t launch_pcg_start(const DevPlan& P, const double* bb, const int* outer, int* active, int* iters,
                             cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_start<<<(P.ncomps + 127) / 128, 128, 0, s>>>(P.ncomps, bb, outer, active, iters);
    return cudaGetLastError();
}

// End of one iteration of a graph-captured CG loop: counts the iteration and
// keeps the loop's while-condition set while some grid is active and the
// iteration limit is not reached.
__global__ void k_loop_cond(int* __restrict__ counter, const int* __restrict__ nactive, int max_iter,
                            cudaGraphConditionalHandle h) {
    int it = *counter + 1;
    *counter = it;
    cudaGraphSetConditional(h, (*nactive > 0 && it < max_iter) ? 1u : 0u);
}

cudaError_t launch_loop_cond(int* counter, const int* nactive, int max_iter, cudaGraphConditionalHandle h,
                             cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_loop_cond<<<1, 1, 0, s>>>(counter, nactive, max_iter, h);
    return cudaGetLastError();
}

// Iterative refinement helpers (FP64 outer loop around an FP32 inner solve).
// r32 = (float) r64 on active grids, 0 elsewhere
__global__ void k_ir_down(const Chunk* __restrict__ chunks, const double* __restrict__ r64, float* __restrict__ r32,
                          const int* __restrict__ active) {
    const Chunk c = chunks[blockIdx.x];
    const bool a = active[c.grid] != 0;
    for (int i = threadIdx.x; i < c.len; i += blockDim.x) r32[c.start + i] = a ? (float)r64[c.start + i] : 0.0f;
}

cudaError_t launch_ir_down(const DevPlan& P, const double* r64, float* r32, const int* active, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_ir_down<<<P.nchunks, 256, 0, s>>>(P.chunks, r64, r32, active);
    return cudaGetLastError();
}

// x64 += d on active grids (d FP32 from the inner solve, or FP64 from the fallback)
template <typename Real>
__global__ void k_ir_up(const Chunk* __restrict__ chunks, double* __restrict__ x64, const Real* __restrict__ d,
                        const int* __restrict__ active) {
    const Chunk c = chunks[blockIdx.x];
    if (!active[c.grid]) return;
    for (int i = threadIdx.x; i < c.len; i += blockDim.x) x64[c.start + i] += (double)d[c.start + i];
}

cudaError_t launch_ir_up(const DevPlan& P, double* x64, const float* d32, const int* active, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_ir_up<float><<<P.nchunks, 256, 0, s>>>(P.chunks, x64, d32, active);
    return cudaGetLastError();
}

// x = 0 on active grids (restart of a refinement whose iterate went non-finite)
__global__ void k_zero_active(const Chunk* __restrict__ chunks, double* __restrict__ x, const int* __restrict__ active) {
    const Chunk c = chunks[blockIdx.x];
    if (!active[c.grid]) return;
    for (int i = threadIdx.x; i < c.len; i += blockDim.x) x[c.start + i] = 0.0;
}

cudaError_t launch_zero_active(const DevPlan& P, double* x, const int* active, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_zero_active<<<P.nchunks, 256, 0, s>>>(P.chunks, x, active);
    return cudaGetLastError();
}

cudaError_t launch_ir_up64(const DevPlan& P, double* x64, const double* d64, const int* active, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_ir_up<double><<<P.nchunks, 256, 0, s>>>(P.chunks, x64, d64, active);
    return cudaGetLastError();
}

// r64 = b - q on active grids (q = K x64 in FP64); partial ||r64||^2 for every grid
__global__ void k_ir_residual(const Chunk* __restrict__ chunks, const double* __restrict__ b,
                              const double* __restrict__ q, double* __restrict__ r, const int* __restrict__ active,
                              double* __restrict__ partial) {
    const Chunk c = chunks[blockIdx.x];
    double s = 0.0;
    const bool a = active[c.grid] != 0;
    for (int i = threadIdx.x; i < c.len; i += blockDim.x) {
        long long k = c.start + i;
        double v = a ? b[k] - q[k] : r[k];
        r[k] = v;
        s += v * v;
    }
    s = block_sum(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

cudaError_t launch_ir_residual(const DevPlan& P, const double* b, const double* q, double* r, const int* active,
                               double* partial, double* rr, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_ir_residual<<<P.nchunks, 256, 0, s>>>(P.chunks, b, q, r, active, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return reduce(P, partial, rr, s);
}

// z64 = (double) z32 on the active components (the FP32 preconditioner's
// output handed back to FP64 CG).
__global__ void k_widen_active(const Chunk* __restrict__ chunks, double* __restrict__ dst,
                               const float* __restrict__ src, const int* __restrict__ active) {
    const Chunk c = chunks[blockIdx.x];
    if (active && !active[c.grid]) return;
    for (int i = threadIdx.x; i < c.len; i += blockDim.x) dst[c.start + i] = (double)src[c.start + i];
}

cudaError_t launch_widen_active(const DevPlan& P, double* dst, const float* src, const int* active, cudaStream_t s) {
    if (P.nchunks == 0) return cudaSuccess;
    SGIGA_COUNT_LAUNCH();
    k_widen_active<<<P.nchunks, 256, 0, s>>>(P.chunks, dst, src, active);
    return cudaGetLastError();
}

// Narrow an FP64 array to FP32 (plan set-up of the mixed-precision copies).
__global__ void k_narrow(float* __restrict__ dst, const double* __restrict__ src, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride) dst[i] = (float)src[i];
}

cudaError_t launch_narrow(float* dst, const double* src, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    SGIGA_COUNT_LAUNCH();
    k_narrow<<<(int)blocks, 256, 0, s>>>(dst, src, n);
    return cudaGetLastError();
}

}  // namespace sgiga
