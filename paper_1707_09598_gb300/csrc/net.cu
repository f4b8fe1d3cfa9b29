// Network of the learned scaling of the fast-diagonalisation preconditioner
// (not in the paper; its conclusions name fast solvers used as
// preconditioners as future work, Sec. 5), and the elementwise kernels of the
// scaled preconditioner and of its training loss:
//
//   M(r) = S * FD(S * r),  S = exp(N(phi)),  phi = log of the local effective
//   coefficient of each DoF,
//
// N = three 3x3(x3) convolutions over each component's DoF tensor with zero
// padding, 1 -> 32 -> 32 -> 1 channels, ReLU after the first two. Weights are
// kept as an FP32 master copy (Adam) and a BF16 copy used by every forward and
// backward kernel; all accumulation is FP32. Activations are channel planes
// over the packed vector of all components: X[c][v].
//
// Kernels (one thread per DoF for the convolutions, weights staged in shared
// memory as FP32 [tap][c_in][c_out]):
//   conv      Y[co][v] = b[co] + sum_{tap,ci} W[co][ci][tap] X[ci][nb(v,tap)]
//   convT     data gradient: the same with W transposed and taps mirrored
//   wgrad     dW[co][ci][tap] += sum_v dZ[co][v] X[ci][nb(v,tap)] (tiles of 32
//             DoFs gathered im2col-style in shared memory, 8x32 thread grid,
//             partial sums in registers, one atomic add per block and weight)
//   relu/mask, features, scaling, pair loss and gradient, Adam.
#include <cuda_bf16.h>

#include "kernels.h"

namespace sgiga {

// neighbour of packed DoF (grid-local index loc) at tap offset (ox, oy, oz)
struct NbInfo {
    int n0, n1, n2;
    long long off;
};

__device__ __forceinline__ long long nb_index(const NbInfo& g, int i0, int i1, int i2, int tap, int d) {
    int o0, o1, o2;
    if (d == 3) { o0 = tap % 3 - 1; o1 = (tap / 3) % 3 - 1; o2 = tap / 9 - 1; }
    else { o0 = tap % 3 - 1; o1 = tap / 3 - 1; o2 = 0; }
    int j0 = i0 + o0, j1 = i1 + o1, j2 = i2 + o2;
    if (j0 < 0 || j0 >= g.n0 || j1 < 0 || j1 >= g.n1 || j2 < 0 || j2 >= g.n2) return -1;
    return g.off + j0 + (long long)g.n0 * (j1 + (long long)g.n1 * j2);
}

// ---------------------------------------------------------------------------
// convolution (forward, or data gradient with mirrored taps and swapped channels)
// ---------------------------------------------------------------------------
template <int CIN, int COUT>
__global__ void __launch_bounds__(256, 2)
k_conv(DevPlan P, const __nv_bfloat16* __restrict__ W, const float* __restrict__ bias, const float* __restrict__ X,
       float* __restrict__ Y, long long N, int transpose, int relu) {
    extern __shared__ float ws[];   // [taps][CIN][COUT]
    const int d = P.d, T = d == 3 ? 27 : 9;
    // stage weights: forward ws[(t*CIN+ci)*COUT+co] = W[co][ci][t];
    // transposed (layer with cout=CIN, cin=COUT): W[ci'][co'][T-1-t] with ci' = co, co' = ci
    const int nw = T * CIN * COUT;
    for (int i = threadIdx.x; i < nw; i += blockDim.x) {
        int co = i % COUT, r = i / COUT, ci = r % CIN, t = r / CIN;
        float v;
        if (!transpose) v = __bfloat162float(W[((long long)co * CIN + ci) * T + t]);
        else v = __bfloat162float(W[((long long)ci * COUT + co) * T + (T - 1 - t)]);
        ws[i] = v;
    }
    __syncthreads();
    const Chunk c = P.chunks[blockIdx.x];
    const GridDesc& g = P.grids[c.grid];
    NbInfo nb{g.n[0], d > 1 ? g.n[1] : 1, d > 2 ? g.n[2] : 1, g.dof_off};
    for (int k = threadIdx.x; k < c.len; k += blockDim.x) {
        const long long v = c.start + k;
        long long loc = v - g.dof_off;
        int i0 = (int)(loc % nb.n0);
        loc /= nb.n0;
        int i1 = (int)(loc % nb.n1);
        int i2 = (int)(loc / nb.n1);
        float acc[COUT];
#pragma unroll
        for (int co = 0; co < COUT; ++co) acc[co] = bias ? bias[co] : 0.0f;
        for (int t = 0; t < T; ++t) {
            long long u = nb_index(nb, i0, i1, i2, t, d);
            if (u < 0) continue;
            const float* wt = ws + t * CIN * COUT;
#pragma unroll 2
            for (int ci = 0; ci < CIN; ++ci) {
                const float x = X[(long long)ci * N + u];
#pragma unroll
                for (int co = 0; co < COUT; ++co) acc[co] += wt[ci * COUT + co] * x;
            }
        }
#pragma unroll
        for (int co = 0; co < COUT; ++co) {
            float y = acc[co];
            if (relu) y = y > 0.0f ? y : 0.0f;
            Y[(long long)co * N + v] = y;
        }
    }
}

// ---------------------------------------------------------------------------
// weight gradient: dW[co][ci][t] += sum_v dZ[co][v] X[ci][nb(v, t)],
// db[co] += sum_v dZ[co][v]
// ---------------------------------------------------------------------------
template <int CIN, int COUT, int RPT>
__global__ void __launch_bounds__(256, 1)
k_wgrad(DevPlan P, const float* __restrict__ X, const float* __restrict__ dZ, float* __restrict__ dW,
        float* __restrict__ db, long long N) {
    extern __shared__ float sh[];
    const int d = P.d, T = d == 3 ? 27 : 9;
    const int ROWS = CIN * T;
    constexpr int VT = 32;                          // DoFs per tile
    float* xcol = sh;                               // [VT][ROWS]
    float* dzt = sh + VT * ROWS;                    // [VT][COUT]
    const int RG = 256 / COUT;                      // row groups
    const int col = threadIdx.x % COUT, rg = threadIdx.x / COUT;
    float acc[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) acc[i] = 0.0f;
    float bacc = 0.0f;
    for (int ch = blockIdx.x; ch < P.nchunks; ch += gridDim.x) {
        const Chunk c = P.chunks[ch];
        const GridDesc& g = P.grids[c.grid];
        NbInfo nb{g.n[0], d > 1 ? g.n[1] : 1, d > 2 ? g.n[2] : 1, g.dof_off};
        for (int t0 = 0; t0 < c.len; t0 += VT) {
            const int nv = min(VT, c.len - t0);
            __syncthreads();
            for (int i = threadIdx.x; i < VT * ROWS; i += blockDim.x) {
                int vv = i / ROWS, row = i % ROWS;
                float val = 0.0f;
                if (vv < nv) {
                    long long v = c.start + t0 + vv, loc = v - g.dof_off;
                    int i0 = (int)(loc % nb.n0);
                    loc /= nb.n0;
                    int i1 = (int)(loc % nb.n1), i2 = (int)(loc / nb.n1);
                    int ci = row / T, t = row % T;
                    long long u = nb_index(nb, i0, i1, i2, t, d);
                    if (u >= 0) val = X[(long long)ci * N + u];
                }
                xcol[i] = val;
            }
            for (int i = threadIdx.x; i < VT * COUT; i += blockDim.x) {
                int vv = i / COUT, co = i % COUT;
                dzt[i] = vv < nv ? dZ[(long long)co * N + c.start + t0 + vv] : 0.0f;
            }
            __syncthreads();
            for (int vv = 0; vv < nv; ++vv) {
                const float z = dzt[vv * COUT + col];
                if (rg == 0) bacc += z;
                const float* xr = xcol + vv * ROWS;
#pragma unroll
                for (int i = 0; i < RPT; ++i) {
                    int row = rg + i * RG;
                    if (row < ROWS) acc[i] += xr[row] * z;
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        int row = rg + i * RG;
        if (row < ROWS) {
            int ci = row / T, t = row % T;
            atomicAdd(&dW[((long long)col * CIN + ci) * T + t], acc[i]);
        }
    }
    if (rg == 0) atomicAdd(&db[col], bacc);
}

// dA *= (A > 0): ReLU backward through the post-activation values
__global__ void k_relu_mask(float* __restrict__ dA, const float* __restrict__ A, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride)
        if (!(A[i] > 0.0f)) dA[i] = 0.0f;
}

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

// log S = L tanh(y / L) with L = SGIGA_LOGS_MAX: a smooth bound on the
// scaling (S in [e^-L, e^L]) that keeps a training step from driving one
// component's preconditioner far from FD; the scalings that matter here have
// |log S| below 2.
#define SGIGA_LOGS_MAX 4.0f

// S = exp(L tanh(y / L)) where the component's y is finite, else 1 (plain FD there)
__global__ void k_exp_scaling(DevPlan P, const float* __restrict__ y, const int* __restrict__ ok,
                              float* __restrict__ S) {
    const Chunk c = P.chunks[blockIdx.x];
    const bool use = ok[c.grid] != 0;
    for (int i = threadIdx.x; i < c.len; i += blockDim.x) {
        const long long k = c.start + i;
        S[k] = use ? expf(SGIGA_LOGS_MAX * tanhf(y[k] * (1.0f / SGIGA_LOGS_MAX))) : 1.0f;
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
        const float t = tanhf(y[k] * (1.0f / SGIGA_LOGS_MAX));
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

cudaError_t launch_conv(const DevPlan& P, int cin, int cout, const void* W, const float* bias, const float* X,
                        float* Y, int transpose, int relu, cudaStream_t s) {
    const int T = P.d == 3 ? 27 : 9;
    const long long N = P.ndof;
    if (P.nchunks == 0) return cudaSuccess;
    const size_t sm = (size_t)T * cin * cout * sizeof(float);
    const __nv_bfloat16* w = (const __nv_bfloat16*)W;
    SGIGA_COUNT_LAUNCH();
#define CONV(CI, CO)                                                                                       \
    if (cin == CI && cout == CO) {                                                                         \
        cudaFuncSetAttribute(k_conv<CI, CO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);      \
        k_conv<CI, CO><<<P.nchunks, 256, sm, s>>>(P, w, bias, X, Y, N, transpose, relu);                 \
        return cudaGetLastError();                                                                         \
    }
    CONV(32, 32) CONV(32, 1) CONV(1, 32)
#undef CONV
    return cudaErrorInvalidValue;
}

cudaError_t launch_wgrad(const DevPlan& P, int cin, int cout, const float* X, const float* dZ, float* dW, float* db,
                         cudaStream_t s) {
    const int T = P.d == 3 ? 27 : 9;
    const long long N = P.ndof;
    if (P.nchunks == 0) return cudaSuccess;
    const size_t sm = (size_t)32 * (cin * T + cout) * sizeof(float);
    const int blocks = P.nchunks < 2 * 152 ? P.nchunks : 2 * 152;
    SGIGA_COUNT_LAUNCH();
#define WG(CI, CO, R)                                                                                      \
    if (cin == CI && cout == CO) {                                                                         \
        cudaFuncSetAttribute(k_wgrad<CI, CO, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);  \
        k_wgrad<CI, CO, R><<<blocks, 256, sm, s>>>(P, X, dZ, dW, db, N);                                  \
        return cudaGetLastError();                                                                         \
    }
    WG(1, 32, 4) WG(32, 32, 108) WG(32, 1, 4)
#undef WG
    return cudaErrorInvalidValue;
}

cudaError_t launch_relu_mask(float* dA, const float* A, long long n, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_relu_mask<<<eblocks(n), 256, 0, s>>>(dA, A, n);
    return cudaGetLastError();
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

cudaError_t launch_exp_scaling(const DevPlan& P, const float* y, int* ok, float* S, cudaStream_t s) {
    if (P.nchunks == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(ok, 0xff, sizeof(int) * P.ncomps, s);   // all ones = finite
    if (e != cudaSuccess) return e;
    SGIGA_COUNT_LAUNCH();
    k_finite<<<P.nchunks, 256, 0, s>>>(P, y, ok);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    SGIGA_COUNT_LAUNCH();
    k_exp_scaling<<<P.nchunks, 256, 0, s>>>(P, y, ok, S);
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
