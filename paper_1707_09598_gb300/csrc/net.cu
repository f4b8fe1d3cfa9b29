// Network of the learned scaling of the fast-diagonalisation preconditioner
// (not in the paper; its conclusions name fast solvers used as
// preconditioners as future work, Sec. 5), and the elementwise kernels of the
// scaled preconditioner and of its training loss:
//
//   M(r) = S * FD(S * r),  S = exp(-phi / 2 + 4 tanh(N(phi) / 4)),  phi = log
//   of the local effective coefficient of each DoF,
//
// N = three 3x3(x3) convolutions over each component's DoF tensor with zero
// padding, 1 -> 32 -> 32 -> 1 channels, ReLU after the first two (conv.cu).
// Weights are kept as an FP32 master copy (Adam) and a BF16 copy used by
// every forward and backward kernel; all accumulation is FP32.
//
// Kernels here: features, scaling, pair loss and gradient, Adam.
#include <cuda_bf16.h>

#include "kernels.h"

namespace sgiga {

__global__ void k_fill(float* __restrict__ x, float v, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride) x[i] = v;
}

// phi = log(num / den) (FP64 ratio, FP32 result)
__global__ void k_log_ratio(const double* __restrict__ num, const double* __restrict__ den, float* __restrict__ out,
                            long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride) out[i] = (float)log(num[i] / den[i]);
}

// per component: ok[g] = all entries of y finite (partial flags by chunk)
__global__ void k_finite(DevPlan P, const float* __restrict__ y, int* __restrict__ ok) {
    const Chunk c = P.chunks[blockIdx.x];
    bool bad = false;
    for (int i = threadIdx.x; i < c.len; i += blockDim.x) bad |= !isfinite(y[c.start + i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicAnd(&ok[c.grid], 0);
}

// log S = A phi + L tanh(y / L) with A = SGIGA_LOGS_SKIP and L =
// SGIGA_LOGS_MAX: the network output y corrects the network-free scaling
// S = c^(-1/2) (phi = log c), which the untrained network (y = 0) gives
// exactly; the tanh is a smooth bound on the correction (a factor within
// [e^-L, e^L]) that keeps a training step from driving one component's
// preconditioner far from it.
#define SGIGA_LOGS_MAX 4.0f
#define SGIGA_LOGS_SKIP (-0.5f)

// S = exp(A phi + L tanh(y / L)) where the component's y is finite, else 1
// (plain FD there)
__global__ void k_exp_scaling(DevPlan P, const float* __restrict__ y, const float* __restrict__ phi,
                              const int* __restrict__ ok, float* __restrict__ S) {
    const Chunk c = P.chunks[blockIdx.x];
    const bool use = ok[c.grid] != 0;
    for (int i = threadIdx.x; i < c.len; i += blockDim.x) {
        const long long k = c.start + i;
        S[k] = use ? expf(SGIGA_LOGS_SKIP * phi[k] + SGIGA_LOGS_MAX * tanhf(y[k] * (1.0f / SGIGA_LOGS_MAX))) : 1.0f;
    }
}

// out = S * in on the active components (out may alias in)
__global__ void k_mul_active(DevPlan P, const float* __restrict__ S, const float* in, float* out,
                             const int* __restrict__ active) {
    const Chunk c = P.chunks[blockIdx.x];
    if (active && !active[c.grid]) return;
    for (int i = threadIdx.x; i < c.len; i += blockDim.x) {
        const long long k = c.start + i;
        out[k] = S[k] * in[k];
    }
}

// res = S * z1 - e
__global__ void k_pair_residual(long long n, const float* __restrict__ S, const float* __restrict__ z1,
                                const float* __restrict__ e, float* __restrict__ res) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride) res[i] = S[i] * z1[i] - e[i];
}

// The components a sample counts: mask[g] != 0 (all when mask is null) and
// e_g != 0; their number goes to cnt[0] (one block).
__global__ void k_pair_count(int ng, const int* __restrict__ mask, const double* __restrict__ ee,
                             double* __restrict__ cnt) {
    __shared__ int red[32];
    int v = 0;
    for (int g = threadIdx.x; g < ng; g += blockDim.x) v += ((!mask || mask[g]) && ee[g] > 0.0) ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        cnt[0] = (double)t;
    }
}

// delta = 2 res / (||e_g||^2 count) on the counted components, 0 elsewhere;
// t2 = S delta
__global__ void k_pair_delta(DevPlan P, const float* __restrict__ S, const float* __restrict__ res,
                             const double* __restrict__ ee, const int* __restrict__ mask,
                             const double* __restrict__ cnt, float* __restrict__ delta, float* __restrict__ t2) {
    const Chunk c = P.chunks[blockIdx.x];
    const double e2 = ee[c.grid];
    const bool use = (!mask || mask[c.grid]) && e2 > 0.0 && cnt[0] > 0.0;
    const float f = use ? (float)(2.0 / (e2 * cnt[0])) : 0.0f;
    for (int i = threadIdx.x; i < c.len; i += blockDim.x) {
        const long long k = c.start + i;
        const float dl = f * res[k];
        delta[k] = dl;
        t2[k] = S[k] * dl;
    }
}

// acc[0] += mean over the counted components of rr_g / ee_g (one block)
__global__ void k_pair_loss(int ng, const double* __restrict__ rr, const double* __restrict__ ee,
                            const int* __restrict__ mask, const double* __restrict__ cnt, double* __restrict__ acc) {
    __shared__ double red[32];
    double v = 0.0;
    for (int g = threadIdx.x; g < ng; g += blockDim.x)
        v += ((!mask || mask[g]) && ee[g] > 0.0) ? rr[g] / ee[g] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        if (cnt[0] > 0.0) acc[0] += t / cnt[0];
    }
}

// mask[g] = ||r_g||^2 > thr2 ||b_g||^2: the component had not converged when
// the pair was recorded (a converged component's error is the noise of two
// solves, not the error of its residual)
__global__ void k_pair_mask(int ng, const double* __restrict__ rr, const double* __restrict__ bb, double thr2,
                            int* __restrict__ mask) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < ng) mask[g] = rr[g] > thr2 * bb[g] ? 1 : 0;
}

// dls += weight * S (delta z1 + r z2): the gradient with respect to log S
__global__ void k_pair_grad(long long n, const float* __restrict__ S, const float* __restrict__ delta,
                            const float* __restrict__ z1, const float* __restrict__ r, const float* __restrict__ z2,
                            float weight, float* __restrict__ dls) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride) dls[i] += weight * S[i] * (delta[i] * z1[i] + r[i] * z2[i]);
}

// chain rule from d/dlog S to d/dy through log S = L tanh(y / L); no gradient
// through a component that fell back to S = 1
__global__ void k_mask_scaled(DevPlan P, float* __restrict__ dy, const int* __restrict__ ok,
                              const float* __restrict__ y) {
    const Chunk c = P.chunks[blockIdx.x];
    const bool use = ok[c.grid] != 0;
    for (int i = threadIdx.x; i < c.len; i += blockDim.x) {
        const long long k = c.start + i;
        const float t = tanhf(y[k] * (1.0f / SGIGA_LOGS_MAX));   // dlog S / dy = 1 - t^2
        dy[k] = use ? dy[k] * (1.0f - t * t) : 0.0f;
    }
}

// Adam update of the FP32 master parameters and their BF16 copy
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       __nv_bfloat16* __restrict__ wb, const int* __restrict__ wmap, int n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (wmap[i] >= 0) wb[wmap[i]] = __float2bfloat16(pi);
}

__global__ void k_f2bf(const float* __restrict__ p, const int* __restrict__ wmap, __nv_bfloat16* __restrict__ wb,
                       int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && wmap[i] >= 0) wb[wmap[i]] = __float2bfloat16(p[i]);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static unsigned eblocks(long long n) {
    long long b = (n + 255) / 256;
    return (unsigned)(b > 152 * 32 ? 152 * 32 : (b < 1 ? 1 : b));
}

cudaError_t launch_fill(float* x, float v, long long n, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_fill<<<eblocks(n), 256, 0, s>>>(x, v, n);
    return cudaGetLastError();
}

cudaError_t launch_log_ratio(const double* num, const double* den, float* out, long long n, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_log_ratio<<<eblocks(n), 256, 0, s>>>(num, den, out, n);
    return cudaGetLastError();
}

cudaError_t launch_exp_scaling(const DevPlan& P, const float* y, const float* phi, int* ok, float* S,
                               cudaStream_t s) {
    if (P.nchunks == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(ok, 0xff, sizeof(int) * P.ncomps, s);   // all ones = finite
    if (e != cudaSuccess) return e;
    SGIGA_COUNT_LAUNCH();
    k_finite<<<P.nchunks, 256, 0, s>>>(P, y, ok);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    SGIGA_COUNT_LAUNCH();
    k_exp_scaling<<<P.nchunks, 256, 0, s>>>(P, y, phi, ok, S);
    return cudaGetLastError();
}

cudaError_t launch_mul_active(const DevPlan& P, const float* S, const float* in, float* out, const int* active,
                              cudaStream_t s) {
    if (P.nchunks == 0) return cudaSuccess;
    SGIGA_COUNT_LAUNCH();
    k_mul_active<<<P.nchunks, 256, 0, s>>>(P, S, in, out, active);
    return cudaGetLastError();
}

cudaError_t launch_pair_residual(const DevPlan& P, const float* S, const float* z1, const float* e, float* res,
                                 cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_pair_residual<<<eblocks(P.ndof), 256, 0, s>>>(P.ndof, S, z1, e, res);
    return cudaGetLastError();
}

cudaError_t launch_pair_delta(const DevPlan& P, const float* S, const float* res, const double* rr, const double* ee,
                              const int* mask, double* cnt, float* delta, float* t2, double* lossacc, cudaStream_t s) {
    if (P.nchunks == 0) return cudaSuccess;
    SGIGA_COUNT_LAUNCH();
    k_pair_count<<<1, 256, 0, s>>>(P.ncomps, mask, ee, cnt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    SGIGA_COUNT_LAUNCH();
    k_pair_delta<<<P.nchunks, 256, 0, s>>>(P, S, res, ee, mask, cnt, delta, t2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    SGIGA_COUNT_LAUNCH();
    k_pair_loss<<<1, 256, 0, s>>>(P.ncomps, rr, ee, mask, cnt, lossacc);
    return cudaGetLastError();
}

cudaError_t launch_pair_mask(int ng, const double* rr, const double* bb, double thr2, int* mask, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_pair_mask<<<(ng + 127) / 128, 128, 0, s>>>(ng, rr, bb, thr2, mask);
    return cudaGetLastError();
}

cudaError_t launch_pair_grad(const DevPlan& P, const float* S, const float* delta, const float* z1, const float* r,
                             const float* z2, float weight, float* dls, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_pair_grad<<<eblocks(P.ndof), 256, 0, s>>>(P.ndof, S, delta, z1, r, z2, weight, dls);
    return cudaGetLastError();
}

cudaError_t launch_mask_scaled(const DevPlan& P, float* dy, const int* ok, const float* y, cudaStream_t s) {
    if (P.nchunks == 0) return cudaSuccess;
    SGIGA_COUNT_LAUNCH();
    k_mask_scaled<<<P.nchunks, 256, 0, s>>>(P, dy, ok, y);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, void* wb, const int* wmap, int n, float lr,
                        float b1, float b2, float eps, int step, cudaStream_t s) {
    float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    SGIGA_COUNT_LAUNCH();
    k_adam<<<(n + 255) / 256, 256, 0, s>>>(p, g, m, v, (__nv_bfloat16*)wb, wmap, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_f2bf(const float* p, const int* wmap, void* wb, int n, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_f2bf<<<(n + 255) / 256, 256, 0, s>>>(p, wmap, (__nv_bfloat16*)wb, n);
    return cudaGetLastError();
}

// one training pair from an FP64 CG iterate: rd = (float) r, ed = (float)(x* - x)
__global__ void k_pair_store(long long n, const double* __restrict__ r, const double* __restrict__ xs,
                             const double* __restrict__ x, float* __restrict__ rd, float* __restrict__ ed) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride) {
        rd[i] = (float)r[i];
        ed[i] = (float)(xs[i] - x[i]);
    }
}

cudaError_t launch_pair_store(const DevPlan& P, const double* r, const double* xstar, const double* x, float* rd,
                              float* ed, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_pair_store<<<eblocks(P.ndof), 256, 0, s>>>(P.ndof, r, xstar, x, rd, ed);
    return cudaGetLastError();
}

}  // namespace sgiga
