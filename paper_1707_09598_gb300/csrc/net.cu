// Learned correction of the fast-diagonalisation preconditioner (not in the
// paper; its conclusions suggest the combination technique itself as a
// preconditioner, Sec. 5 — this is a different, data-driven companion):
//
//   M(r) = z + s_z N([r / s_r, z / s_z]),  z = FD(r),  s_* = RMS per component,
//
// N = three 3x3(x3) convolutions over each component's DoF tensor with zero
// padding, 2 -> 32 -> 32 -> 1 channels, ReLU after the first two. Weights are
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
//   relu/mask, per-component RMS scaling, loss, Adam.
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

// x[c][v] *= scale[grid(v)] over every channel c (per-component scaling)
__global__ void k_scale_grid(DevPlan P, float* __restrict__ x, const double* __restrict__ scale, int nch,
                             long long N, int invert) {
    const Chunk c = P.chunks[blockIdx.x];
    double s = scale[c.grid];
    float f = (float)(invert ? (s > 0.0 ? 1.0 / s : 0.0) : s);
    for (int ch = 0; ch < nch; ++ch)
        for (int i = threadIdx.x; i < c.len; i += blockDim.x) x[(long long)ch * N + c.start + i] *= f;
}

// cand = z + s_z * y (all grids)
__global__ void k_net_candidate(DevPlan P, const float* __restrict__ z, const float* __restrict__ y,
                                const double* __restrict__ sz, float* __restrict__ cand) {
    const Chunk c = P.chunks[blockIdx.x];
    const float s = (float)sz[c.grid];
    for (int i = threadIdx.x; i < c.len; i += blockDim.x) {
        long long k = c.start + i;
        cand[k] = z[k] + s * y[k];
    }
}

// out = cand where the component's network output is finite and
// r.cand >= r.z / 2 (the learned direction keeps the descent property of FD),
// else z; active grids only
__global__ void k_net_select(DevPlan P, const float* __restrict__ z, const float* __restrict__ cand,
                             const int* __restrict__ ok, const double* __restrict__ rz, const double* __restrict__ rc,
                             float* __restrict__ out, const int* __restrict__ active) {
    const Chunk c = P.chunks[blockIdx.x];
    if (active && !active[c.grid]) return;
    const bool use = ok[c.grid] != 0 && rc[c.grid] >= 0.5 * rz[c.grid];
    for (int i = threadIdx.x; i < c.len; i += blockDim.x) {
        long long k = c.start + i;
        out[k] = use ? cand[k] : z[k];
    }
}

// per-component: ok[g] = all entries of y finite (partial flags by chunk)
__global__ void k_finite(DevPlan P, const float* __restrict__ y, int* __restrict__ ok) {
    const Chunk c = P.chunks[blockIdx.x];
    bool bad = false;
    for (int i = threadIdx.x; i < c.len; i += blockDim.x) bad |= !isfinite(y[c.start + i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicAnd(&ok[c.grid], 0);
}

// loss = sum_v (y - t)^2 / sum_v t^2 (partials: [0] numerator, [1] denominator);
// dy = 2 (y - t) / sum t^2 is written in a second pass
__global__ void k_loss_partial(const float* __restrict__ y, const float* __restrict__ t, long long n,
                               double* __restrict__ acc) {
    double a = 0.0, b = 0.0;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride) {
        double e = (double)y[i] - (double)t[i];
        a += e * e;
        b += (double)t[i] * (double)t[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&acc[0], a);
        atomicAdd(&acc[1], b);
    }
}

__global__ void k_loss_grad(const float* __restrict__ y, const float* __restrict__ t, long long n,
                            const double* __restrict__ acc, float* __restrict__ dy) {
    const float f = (float)(2.0 / acc[1]);
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride) dy[i] = f * (y[i] - t[i]);
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
    CONV(2, 32) CONV(32, 32) CONV(32, 1) CONV(1, 32)
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
    WG(2, 32, 7) WG(32, 32, 108) WG(32, 1, 4)
#undef WG
    return cudaErrorInvalidValue;
}

cudaError_t launch_relu_mask(float* dA, const float* A, long long n, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_relu_mask<<<eblocks(n), 256, 0, s>>>(dA, A, n);
    return cudaGetLastError();
}

cudaError_t launch_scale_grid(const DevPlan& P, float* x, const double* scale, int nch, int invert, cudaStream_t s) {
    if (P.nchunks == 0) return cudaSuccess;
    SGIGA_COUNT_LAUNCH();
    k_scale_grid<<<P.nchunks, 256, 0, s>>>(P, x, scale, nch, P.ndof, invert);
    return cudaGetLastError();
}

cudaError_t launch_net_candidate(const DevPlan& P, const float* z, const float* y, const double* sz, int* ok,
                                 float* cand, cudaStream_t s) {
    if (P.nchunks == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(ok, 0xff, sizeof(int) * P.ngrids, s);   // all ones = finite
    if (e != cudaSuccess) return e;
    SGIGA_COUNT_LAUNCH();
    k_finite<<<P.nchunks, 256, 0, s>>>(P, y, ok);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    SGIGA_COUNT_LAUNCH();
    k_net_candidate<<<P.nchunks, 256, 0, s>>>(P, z, y, sz, cand);
    return cudaGetLastError();
}

cudaError_t launch_net_select(const DevPlan& P, const float* z, const float* cand, const int* ok, const double* rz,
                              const double* rc, float* out, const int* active, cudaStream_t s) {
    if (P.nchunks == 0) return cudaSuccess;
    SGIGA_COUNT_LAUNCH();
    k_net_select<<<P.nchunks, 256, 0, s>>>(P, z, cand, ok, rz, rc, out, active);
    return cudaGetLastError();
}

cudaError_t launch_loss(const float* y, const float* t, long long n, double* acc, float* dy, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(acc, 0, 2 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    SGIGA_COUNT_LAUNCH();
    k_loss_partial<<<eblocks(n), 256, 0, s>>>(y, t, n, acc);
    e = cudaGetLastError();
    if (e != cudaSuccess || !dy) return e;
    SGIGA_COUNT_LAUNCH();
    k_loss_grad<<<eblocks(n), 256, 0, s>>>(y, t, n, acc, dy);
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

// rms[g] = sqrt(dots[g] / ndof_g)
__global__ void k_rms(DevPlan P, const double* __restrict__ dots, double* __restrict__ rms) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= P.ngrids) return;
    long long n = P.grids[g].ndof;
    rms[g] = n > 0 ? sqrt(dots[g] / (double)n) : 0.0;
}

cudaError_t launch_rms(const DevPlan& P, const double* dots, double* rms, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_rms<<<(P.ngrids + 127) / 128, 128, 0, s>>>(P, dots, rms);
    return cudaGetLastError();
}

// training target t = (e - z) / s_z per component
__global__ void k_target(DevPlan P, const float* __restrict__ e, const float* __restrict__ z,
                         const double* __restrict__ sz, float* __restrict__ t) {
    const Chunk c = P.chunks[blockIdx.x];
    const double s = sz[c.grid];
    const float f = (float)(s > 0.0 ? 1.0 / s : 0.0);
    for (int i = threadIdx.x; i < c.len; i += blockDim.x) {
        long long k = c.start + i;
        t[k] = (e[k] - z[k]) * f;
    }
}

cudaError_t launch_target(const DevPlan& P, const float* e, const float* z, const double* sz, float* t, cudaStream_t s) {
    if (P.nchunks == 0) return cudaSuccess;
    SGIGA_COUNT_LAUNCH();
    k_target<<<P.nchunks, 256, 0, s>>>(P, e, z, sz, t);
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
