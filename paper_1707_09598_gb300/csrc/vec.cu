// Batched preconditioned-CG vector kernels: every component grid keeps its own
// scalars (alpha, beta, residual norms) and convergence flag. Packed vectors
// are cut into chunks of at most 4096 entries that never straddle two grids;
// a block reduces its chunk, and a second kernel sums each grid's chunk
// partials in a fixed order (deterministic dot products).
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

__global__ void k_dot(const Chunk* __restrict__ chunks, const double* __restrict__ a, const double* __restrict__ b,
                      double* __restrict__ partial) {
    const Chunk c = chunks[blockIdx.x];
    double s = 0.0;
    for (int i = threadIdx.x; i < c.len; i += blockDim.x) s += a[c.start + i] * b[c.start + i];
    s = block_sum(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_reduce(const GridDesc* __restrict__ grids, int ngrids, const double* __restrict__ partial,
                         double* __restrict__ out) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ngrids) return;
    double s = 0.0;
    const int c0 = grids[g].chunk0, nc = grids[g].nchunk;
    for (int c = 0; c < nc; ++c) s += partial[c0 + c];
    out[g] = s;
}

static cudaError_t reduce(const DevPlan& P, const double* partial, double* out, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_reduce<<<(P.ngrids + 127) / 128, 128, 0, s>>>(P.grids, P.ngrids, partial, out);
    return cudaGetLastError();
}

cudaError_t launch_dot(const DevPlan& P, const double* a, const double* b, double* partial, double* out,
                       cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_dot<<<P.nchunks, 256, 0, s>>>(P.chunks, a, b, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return reduce(P, partial, out, s);
}

__global__ void k_pcg_init(const Chunk* __restrict__ chunks, const double* __restrict__ b, double* __restrict__ x,
                           double* __restrict__ r, double* __restrict__ partial) {
    const Chunk c = chunks[blockIdx.x];
    double s = 0.0;
    for (int i = threadIdx.x; i < c.len; i += blockDim.x) {
        double v = b[c.start + i];
        x[c.start + i] = 0.0;
        r[c.start + i] = v;
        s += v * v;
    }
    s = block_sum(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

cudaError_t launch_pcg_init(const DevPlan& P, const double* b, double* x, double* r, double* partial, double* bb,
                            cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_pcg_init<<<P.nchunks, 256, 0, s>>>(P.chunks, b, x, r, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return reduce(P, partial, bb, s);
}

__global__ void k_update_xr(const Chunk* __restrict__ chunks, double* __restrict__ x, double* __restrict__ r,
                            const double* __restrict__ p, const double* __restrict__ q,
                            const double* __restrict__ alpha, const int* __restrict__ active,
                            double* __restrict__ partial) {
    const Chunk c = chunks[blockIdx.x];
    double s = 0.0;
    if (active[c.grid]) {
        const double al = alpha[c.grid];
        for (int i = threadIdx.x; i < c.len; i += blockDim.x) {
            long long k = c.start + i;
            x[k] += al * p[k];
            double rv = r[k] - al * q[k];
            r[k] = rv;
            s += rv * rv;
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

cudaError_t launch_pcg_update_xr(const DevPlan& P, double* x, double* r, const double* p, const double* q,
                                 const double* alpha, const int* active, double* partial, double* rr,
                                 cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_update_xr<<<P.nchunks, 256, 0, s>>>(P.chunks, x, r, p, q, alpha, active, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return reduce(P, partial, rr, s);
}

__global__ void k_update_p(const Chunk* __restrict__ chunks, double* __restrict__ p, const double* __restrict__ z,
                           const double* __restrict__ beta, const int* __restrict__ active) {
    const Chunk c = chunks[blockIdx.x];
    if (!active[c.grid]) return;
    const double be = beta[c.grid];
    for (int i = threadIdx.x; i < c.len; i += blockDim.x) {
        long long k = c.start + i;
        p[k] = z[k] + be * p[k];
    }
}

cudaError_t launch_pcg_update_p(const DevPlan& P, double* p, const double* z, const double* beta,
                                const int* active, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_update_p<<<P.nchunks, 256, 0, s>>>(P.chunks, p, z, beta, active);
    return cudaGetLastError();
}

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
    k_alpha<<<(P.ngrids + 127) / 128, 128, 0, s>>>(P.ngrids, rz, pq, alpha, active);
    return cudaGetLastError();
}

__global__ void k_beta(int ng, double* __restrict__ rz, const double* __restrict__ rznew, double* __restrict__ beta) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    double old = rz[g];
    beta[g] = old != 0.0 ? rznew[g] / old : 0.0;
    rz[g] = rznew[g];
}

cudaError_t launch_pcg_beta(const DevPlan& P, double* rz, const double* rznew, double* beta, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_beta<<<(P.ngrids + 127) / 128, 128, 0, s>>>(P.ngrids, rz, rznew, beta);
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
                             int* iters, int* nactive, double* maxrel, cudaStream_t s) {
    (void)maxrel;
    cudaError_t e = cudaMemsetAsync(nactive, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    SGIGA_COUNT_LAUNCH();
    k_check<<<(P.ngrids + 127) / 128, 128, 0, s>>>(P.ngrids, rr, bb, tol2, active, iters, nactive);
    return cudaGetLastError();
}

// Every component with a nonzero load vector starts active, with 0 iterations.
__global__ void k_start(int ng, const double* __restrict__ bb, int* __restrict__ active, int* __restrict__ iters) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    active[g] = bb[g] > 0.0 ? 1 : 0;
    iters[g] = 0;
}

cudaError_t launch_pcg_start(const DevPlan& P, const double* bb, int* active, int* iters, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_start<<<(P.ngrids + 127) / 128, 128, 0, s>>>(P.ngrids, bb, active, iters);
    return cudaGetLastError();
}

__global__ void k_copy(double* __restrict__ dst, const double* __restrict__ src, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride) dst[i] = src[i];
}

cudaError_t launch_copy(double* dst, const double* src, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    SGIGA_COUNT_LAUNCH();
    k_copy<<<(int)blocks, 256, 0, s>>>(dst, src, n);
    return cudaGetLastError();
}

}  // namespace sgiga
