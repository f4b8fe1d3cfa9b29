// Convolutions of the learned-scaling network over each component's DoF
// tensor (3^d taps, zero padding), with the 32-channel activations stored as
// BF16 rows [voxel][32] (64 bytes per voxel) and FP32 accumulation.
//
//   conv_in   1 -> 32:  A1 = relu(b1 + W1 * x)                 (SIMT)
//   conv_mid  32 -> 32: A2 = relu(b2 + W2 * A1)                (tensor cores)
//             and its data gradient dA1 = (W2^T * dA2) . [A1 > 0]
//   conv_out  32 -> 1:  y = b3 + W3 * A2                       (SIMT)
//   convT_out 1 -> 32:  dA2 = (W3^T * dy) . [A2 > 0]           (SIMT)
//   wgrad     dW[co][ci][t] = sum_v dZ[v][co] X[nb(v,t)][ci]  (tensor cores for 32 x 32)
//
// conv_mid is an implicit GEMM on the BF16 tensor cores (mma.sync m16n8k16,
// FP32 accumulation): a block computes 64 voxels x 32 output channels; for
// each tap the 64 neighbour rows (64 bytes each, zero where the neighbour is
// outside the component's tensor) are copied to shared memory with cp.async
// (double-buffered over taps), the tap's 32 x 32 weight block is resident in
// shared memory, and each warp issues 2 k-steps x 4 n-tiles of MMAs per tap.
#include <cuda_bf16.h>

#include "kernels.h"

namespace sgiga {

namespace {

struct Grid3 {
    int n0, n1, n2;
    long long off;
};

__device__ __forceinline__ Grid3 grid_of(const DevPlan& P, int g) {
    const GridDesc& G = P.grids[g];
    return Grid3{G.n[0], P.d > 1 ? G.n[1] : 1, P.d > 2 ? G.n[2] : 1, G.dof_off};
}

// packed index of the neighbour of local voxel (i0, i1, i2) at tap t (offsets
// in {-1, 0, 1}^d, direction 0 fastest over t), or -1 outside the tensor
__device__ __forceinline__ long long neighbour(const Grid3& g, int i0, int i1, int i2, int t, int d) {
    const int o0 = t % 3 - 1, o1 = (t / 3) % 3 - 1, o2 = d == 3 ? t / 9 - 1 : 0;
    const int j0 = i0 + o0, j1 = i1 + o1, j2 = i2 + o2;
    if (j0 < 0 || j0 >= g.n0 || j1 < 0 || j1 >= g.n1 || j2 < 0 || j2 >= g.n2) return -1;
    return g.off + j0 + (long long)g.n0 * (j1 + (long long)g.n1 * j2);
}

__device__ __forceinline__ void local_coords(const Grid3& g, long long v, int& i0, int& i1, int& i2) {
    long long loc = v - g.off;
    i0 = (int)(loc % g.n0);
    loc /= g.n0;
    i1 = (int)(loc % g.n1);
    i2 = (int)(loc / g.n1);
}

__device__ __forceinline__ void unpack8(uint4 q, float* f) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 t = __bfloat1622float2(h[i]);
        f[2 * i] = t.x;
        f[2 * i + 1] = t.y;
    }
}

__device__ __forceinline__ uint4 pack8(const float* f) {
    uint4 q;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&q);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
    return q;
}

}  // namespace

// ---------------------------------------------------------------------------
// SIMT layers (one input or one output channel): one thread per voxel
// ---------------------------------------------------------------------------

// A1[v][co] = relu(b[co] + sum_t W[co][t] x[nb(v, t)])   (W: BF16 [32][1][T])
__global__ void __launch_bounds__(256) k_conv_in(DevPlan P, const __nv_bfloat16* __restrict__ W,
                                                 const float* __restrict__ bias, const float* __restrict__ x,
                                                 __nv_bfloat16* __restrict__ out) {
    __shared__ float ws[27][32];
    __shared__ float bs[32];
    const int d = P.d, T = d == 3 ? 27 : 9;
    for (int i = threadIdx.x; i < T * 32; i += blockDim.x) {
        const int t = i / 32, co = i % 32;
        ws[t][co] = __bfloat162float(W[co * T + t]);
    }
    if (threadIdx.x < 32) bs[threadIdx.x] = bias[threadIdx.x];
    __syncthreads();
    const Chunk c = P.chunks[blockIdx.x];
    const Grid3 g = grid_of(P, c.grid);
    for (int k = threadIdx.x; k < c.len; k += blockDim.x) {
        const long long v = c.start + k;
        int i0, i1, i2;
        local_coords(g, v, i0, i1, i2);
        float acc[32];
#pragma unroll
        for (int co = 0; co < 32; ++co) acc[co] = bs[co];
        for (int t = 0; t < T; ++t) {
            const long long u = neighbour(g, i0, i1, i2, t, d);
            if (u < 0) continue;
            const float xv = x[u];
#pragma unroll
            for (int co = 0; co < 32; ++co) acc[co] += ws[t][co] * xv;
        }
#pragma unroll
        for (int co = 0; co < 32; ++co) acc[co] = acc[co] > 0.0f ? acc[co] : 0.0f;
        uint4* o = reinterpret_cast<uint4*>(out + v * 32);
#pragma unroll
        for (int q = 0; q < 4; ++q) o[q] = pack8(acc + 8 * q);
    }
}

// y[v] = b + sum_t sum_ci W[ci][t] A[nb(v, t)][ci]   (W: BF16 [1][32][T])
__global__ void __launch_bounds__(256) k_conv_out(DevPlan P, const __nv_bfloat16* __restrict__ W,
                                                  const float* __restrict__ bias, const __nv_bfloat16* __restrict__ A,
                                                  float* __restrict__ y) {
    __shared__ float ws[27][32];
    const int d = P.d, T = d == 3 ? 27 : 9;
    for (int i = threadIdx.x; i < T * 32; i += blockDim.x) {
        const int t = i / 32, ci = i % 32;
        ws[t][ci] = __bfloat162float(W[ci * T + t]);
    }
    __syncthreads();
    const Chunk c = P.chunks[blockIdx.x];
    const Grid3 g = grid_of(P, c.grid);
    const float b = bias[0];
    for (int k = threadIdx.x; k < c.len; k += blockDim.x) {
        const long long v = c.start + k;
        int i0, i1, i2;
        local_coords(g, v, i0, i1, i2);
        float acc = b;
        for (int t = 0; t < T; ++t) {
            const long long u = neighbour(g, i0, i1, i2, t, d);
            if (u < 0) continue;
            const uint4* row = reinterpret_cast<const uint4*>(A + u * 32);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float f[8];
                unpack8(row[q], f);
#pragma unroll
                for (int i = 0; i < 8; ++i) acc += ws[t][8 * q + i] * f[i];
            }
        }
        y[v] = acc;
    }
}

// dA[v][ci] = (sum_t W[ci][T-1-t] dy[nb(v, t)]) * [act[v][ci] > 0]   (W: BF16 [1][32][T])
__global__ void __launch_bounds__(256) k_convT_out(DevPlan P, const __nv_bfloat16* __restrict__ W,
                                                   const float* __restrict__ dy,
                                                   const __nv_bfloat16* __restrict__ act,
                                                   __nv_bfloat16* __restrict__ dA) {
    __shared__ float ws[27][32];
    const int d = P.d, T = d == 3 ? 27 : 9;
    for (int i = threadIdx.x; i < T * 32; i += blockDim.x) {
        const int t = i / 32, ci = i % 32;
        ws[t][ci] = __bfloat162float(W[ci * T + (T - 1 - t)]);
    }
    __syncthreads();
    const Chunk c = P.chunks[blockIdx.x];
    const Grid3 g = grid_of(P, c.grid);
    for (int k = threadIdx.x; k < c.len; k += blockDim.x) {
        const long long v = c.start + k;
        int i0, i1, i2;
        local_coords(g, v, i0, i1, i2);
        float acc[32];
#pragma unroll
        for (int ci = 0; ci < 32; ++ci) acc[ci] = 0.0f;
        for (int t = 0; t < T; ++t) {
            const long long u = neighbour(g, i0, i1, i2, t, d);
            if (u < 0) continue;
            const float gv = dy[u];
#pragma unroll
            for (int ci = 0; ci < 32; ++ci) acc[ci] += ws[t][ci] * gv;
        }
        const uint4* a = reinterpret_cast<const uint4*>(act + v * 32);
        uint4* o = reinterpret_cast<uint4*>(dA + v * 32);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float f[8];
            unpack8(a[q], f);
#pragma unroll
            for (int i = 0; i < 8; ++i) f[i] = f[i] > 0.0f ? acc[8 * q + i] : 0.0f;
            o[q] = pack8(f);
        }
    }
}

// ---------------------------------------------------------------------------
// tensor-core layers (32 x 32 channels)
// ---------------------------------------------------------------------------
namespace {

constexpr int kRow = 40;   // BF16 per shared-memory row: 32 channels + 8 padding (80 bytes: ldmatrix
                           // rows of a warp fall in distinct bank groups)

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// 16 bytes global -> shared, or 16 zero bytes when bytes == 0 (src must still be a valid address)
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

__device__ __forceinline__ void ldsm_x4(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3, const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3, const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}

// D += A B, A 16x16 (row-major, BF16), B 16x8 (column-major, BF16), D 16x8 FP32
__device__ __forceinline__ void mma_bf16(float* d, const unsigned* a, unsigned b0, unsigned b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                 "{%8, %9}, {%0, %1, %2, %3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

}  // namespace

// out[v][n] = act(bias[n] + sum_t sum_k Wt[t][n][k] X[nb(v, t)][k]) for the 64
// voxels of each tile; act = relu (relu != 0), or the mask [gate[v][n] > 0]
// (gate != null: the data gradient through a ReLU), else identity.
// Wt: BF16 [T][32][32] (n = output channel, k = input channel).
// Block: 4 warps, warp w owns tile rows 16w .. 16w+15; persistent over tiles.
// Shared memory: Wt in rows of kRow, then two buffers of 64 rows of kRow.
__global__ void __launch_bounds__(128) k_conv_mid(DevPlan P, const ConvTile* __restrict__ tiles, int ntiles,
                                                  const __nv_bfloat16* __restrict__ Wt,
                                                  const float* __restrict__ bias,
                                                  const __nv_bfloat16* __restrict__ X,
                                                  const __nv_bfloat16* __restrict__ gate, int relu,
                                                  __nv_bfloat16* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int d = P.d, T = d == 3 ? 27 : 9;
    __nv_bfloat16* Ws = reinterpret_cast<__nv_bfloat16*>(smraw);           // [T][32][kRow]
    __nv_bfloat16* As = Ws + (size_t)T * 32 * kRow;                          // [2][64][kRow]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < T * 32 * 4; i += blockDim.x) {                     // 16-byte pieces of Wt rows
        const int row = i >> 2, seg = i & 3;
        *reinterpret_cast<uint4*>(Ws + (size_t)row * kRow + seg * 8) =
            *reinterpret_cast<const uint4*>(Wt + (size_t)row * 32 + seg * 8);
    }
    __syncthreads();
    // this thread's copy work per tap: rows r0 = tid / 4 and r0 + 32, segment tid % 4
    const int cr0 = tid >> 2, cseg = tid & 3;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const ConvTile tl = tiles[tile];
        const Chunk c = P.chunks[tl.chunk];
        const Grid3 g = grid_of(P, c.grid);
        const long long v0 = c.start + tl.off;
        const int nv = min(64, c.len - tl.off);
        int ci0[2], ci1[2], ci2[2];
        bool cv[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = cr0 + 32 * h;
            cv[h] = r < nv;
            ci0[h] = ci1[h] = ci2[h] = 0;
            if (cv[h]) local_coords(g, v0 + r, ci0[h], ci1[h], ci2[h]);
        }
        auto issue = [&](int t, int buf) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = cr0 + 32 * h;
                const long long u = cv[h] ? neighbour(g, ci0[h], ci1[h], ci2[h], t, d) : -1;
                const __nv_bfloat16* src = u >= 0 ? X + u * 32 + cseg * 8 : X;
                cp_async16(As + ((size_t)buf * 64 + r) * kRow + cseg * 8, src, u >= 0 ? 16 : 0);
            }
            cp_async_commit();
        };
        float acc[4][4];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[nt][i] = 0.0f;
        issue(0, 0);
        for (int t = 0; t < T; ++t) {
            if (t + 1 < T) { issue(t + 1, (t + 1) & 1); cp_async_wait1(); }
            else cp_async_wait0();
            __syncthreads();
            const __nv_bfloat16* Ab = As + (size_t)(t & 1) * 64 * kRow;
            const __nv_bfloat16* Wb = Ws + (size_t)t * 32 * kRow;
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
                unsigned a[4];
                ldsm_x4(a[0], a[1], a[2], a[3], Ab + (size_t)(16 * warp + (lane & 15)) * kRow + 16 * kk + 8 * (lane >> 4));
#pragma unroll
                for (int np = 0; np < 2; ++np) {   // pairs of n-tiles
                    unsigned b[4];
                    ldsm_x4(b[0], b[1], b[2], b[3],
                            Wb + (size_t)(8 * (2 * np + (lane >> 4)) + (lane & 7)) * kRow + 16 * kk + 8 * ((lane >> 3) & 1));
                    mma_bf16(acc[2 * np], a, b[0], b[1]);
                    mma_bf16(acc[2 * np + 1], a, b[2], b[3]);
                }
            }
            __syncthreads();   // buffer t & 1 is free for tap t + 2
        }
        // epilogue: rows 16w + lane/4 (+8), columns 8 nt + 2 (lane % 4) (+1)
        const int gq = lane >> 2, cq = lane & 3;
#pragma unroll
        for (int hr = 0; hr < 2; ++hr) {
            const int r = 16 * warp + gq + 8 * hr;
            if (r >= nv) continue;
            const long long v = v0 + r;
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int n = 8 * nt + 2 * cq;
                float y0 = acc[nt][2 * hr], y1 = acc[nt][2 * hr + 1];
                if (bias) { y0 += bias[n]; y1 += bias[n + 1]; }
                if (relu) { y0 = y0 > 0.0f ? y0 : 0.0f; y1 = y1 > 0.0f ? y1 : 0.0f; }
                if (gate) {
                    const float2 gv = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(gate + v * 32 + n));
                    y0 = gv.x > 0.0f ? y0 : 0.0f;
                    y1 = gv.y > 0.0f ? y1 : 0.0f;
                }
                *reinterpret_cast<__nv_bfloat162*>(out + v * 32 + n) = __floats2bfloat162_rn(y0, y1);
            }
        }
    }
}

// dW[co][ci][t] += sum_v dZ[v][co] X[nb(v, t)][ci] and db[co] += sum_v dZ[v][co]
// for 32 x 32 channels on the tensor cores: per tile of 64 voxels the rows of
// dZ and the 64 gathered neighbour rows of every tap are copied to shared
// memory; warp w owns the taps t = w, w + 9, w + 18 and computes their
// 32 x 32 blocks as M = co (2 m-tiles) x N = ci (4 n-tiles) x K = voxels
// (4 k-steps per tile), A = dZ^T and B = X_t read with transposing ldmatrix.
// Accumulators stay in registers over the block's tiles; one atomic add per
// weight and block at the end. Block: 9 warps; persistent over tiles.
__global__ void __launch_bounds__(288) k_wgrad_mid(DevPlan P, const ConvTile* __restrict__ tiles, int ntiles,
                                                   const __nv_bfloat16* __restrict__ X,
                                                   const __nv_bfloat16* __restrict__ dZ, float* __restrict__ dW,
                                                   float* __restrict__ db) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int d = P.d, T = d == 3 ? 27 : 9;
    __nv_bfloat16* Ds = reinterpret_cast<__nv_bfloat16*>(smraw);   // [64][kRow]
    __nv_bfloat16* Xs = Ds + 64 * kRow;                              // [T][64][kRow]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int TPW = 3;                                           // taps per warp (27 = 9 x 3)
    float acc[TPW][2][4][4];
#pragma unroll
    for (int a = 0; a < TPW; ++a)
#pragma unroll
        for (int m = 0; m < 2; ++m)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[a][m][nt][i] = 0.0f;
    float bacc = 0.0f;
    const int nrows = (1 + T) * 64;                                  // dZ rows, then every tap's rows
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const ConvTile tl = tiles[tile];
        const Chunk c = P.chunks[tl.chunk];
        const Grid3 g = grid_of(P, c.grid);
        const long long v0 = c.start + tl.off;
        const int nv = min(64, c.len - tl.off);
        for (int i = tid; i < nrows * 4; i += blockDim.x) {
            const int row = i >> 2, seg = i & 3;
            const int blk = row >> 6, r = row & 63;                    // blk 0: dZ, blk 1 + t: tap t
            long long u = -1;
            if (r < nv) {
                if (blk == 0) u = v0 + r;
                else {
                    int i0, i1, i2;
                    local_coords(g, v0 + r, i0, i1, i2);
                    u = neighbour(g, i0, i1, i2, blk - 1, d);
                }
            }
            const __nv_bfloat16* base = blk == 0 ? dZ : X;
            const __nv_bfloat16* src = u >= 0 ? base + u * 32 + seg * 8 : base;
            cp_async16(Ds + (size_t)row * kRow + seg * 8, src, u >= 0 ? 16 : 0);
        }
        cp_async_commit();
        cp_async_wait0();
        __syncthreads();
        if (tid < 32)
            for (int r = 0; r < nv; ++r) bacc += __bfloat162float(Ds[(size_t)r * kRow + tid]);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            // A = dZ^T (m = co, k = voxel): transposing loads of the voxel-major rows
            unsigned a[2][4];
#pragma unroll
            for (int m = 0; m < 2; ++m)
                ldsm_x4_t(a[m][0], a[m][1], a[m][2], a[m][3],
                          Ds + (size_t)(16 * kk + (lane & 7) + 8 * (lane >> 4)) * kRow + 16 * m + 8 * ((lane >> 3) & 1));
#pragma unroll
            for (int q = 0; q < TPW; ++q) {
                const int t = warp + 9 * q;
                if (t >= T) break;
                const __nv_bfloat16* Xb = Xs + (size_t)t * 64 * kRow;
#pragma unroll
                for (int np = 0; np < 2; ++np) {
                    unsigned b[4];
                    ldsm_x4_t(b[0], b[1], b[2], b[3],
                              Xb + (size_t)(16 * kk + (lane & 7) + 8 * ((lane >> 3) & 1)) * kRow + 16 * np + 8 * (lane >> 4));
#pragma unroll
                    for (int m = 0; m < 2; ++m) {
                        mma_bf16(acc[q][m][2 * np], a[m], b[0], b[1]);
                        mma_bf16(acc[q][m][2 * np + 1], a[m], b[2], b[3]);
                    }
                }
            }
        }
        __syncthreads();
    }
    const int gq = lane >> 2, cq = lane & 3;
#pragma unroll
    for (int q = 0; q < TPW; ++q) {
        const int t = warp + 9 * q;
        if (t >= T) break;
#pragma unroll
        for (int m = 0; m < 2; ++m)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int co = 16 * m + gq + 8 * (i >> 1), ci = 8 * nt + 2 * cq + (i & 1);
                    atomicAdd(&dW[((size_t)co * 32 + ci) * T + t], acc[q][m][nt][i]);
                }
    }
    if (tid < 32) atomicAdd(&db[tid], bacc);
}

// Weight gradients of the one-channel layers. Warp w of a block takes the
// voxels k = w, w + 8, .. of each of its chunks; lane = the 32-channel index;
// one FP32 accumulator per tap in registers; block reduction in shared memory
// and one atomic add per weight and block.
//   in  (layer 1): dW[co][t] += sum_v dZ[v][co] x[nb(v, t)],  db[co] += sum_v dZ[v][co]
//   out (layer 3): dW[ci][t] += sum_v dy[v] A[nb(v, t)][ci],   db[0]  += sum_v dy[v]
template <bool IN>
__global__ void __launch_bounds__(256) k_wgrad_one(DevPlan P, const float* __restrict__ x1,
                                                   const __nv_bfloat16* __restrict__ rows, float* __restrict__ dW,
                                                   float* __restrict__ db) {
    __shared__ float red[8][28][32];
    const int d = P.d, T = d == 3 ? 27 : 9;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float acc[28];
#pragma unroll
    for (int t = 0; t < 28; ++t) acc[t] = 0.0f;
    for (int ch = blockIdx.x; ch < P.nchunks; ch += gridDim.x) {
        const Chunk c = P.chunks[ch];
        const Grid3 g = grid_of(P, c.grid);
        for (int k = warp; k < c.len; k += 8) {
            const long long v = c.start + k;
            int i0, i1, i2;
            local_coords(g, v, i0, i1, i2);
            if (IN) {
                // x1 = layer input (one channel), rows = dZ
                const float gz = __bfloat162float(rows[v * 32 + lane]);
                acc[27] += gz;
#pragma unroll
                for (int t = 0; t < 27; ++t) {
                    if (t >= T) break;
                    const long long u = neighbour(g, i0, i1, i2, t, d);
                    if (u >= 0) acc[t] += gz * x1[u];
                }
            } else {
                // x1 = dy (one channel), rows = layer input A
                const float gy = x1[v];
                acc[27] += lane == 0 ? gy : 0.0f;
#pragma unroll
                for (int t = 0; t < 27; ++t) {
                    if (t >= T) break;
                    const long long u = neighbour(g, i0, i1, i2, t, d);
                    if (u >= 0) acc[t] += gy * __bfloat162float(rows[u * 32 + lane]);
                }
            }
        }
    }
#pragma unroll
    for (int t = 0; t < 28; ++t) red[warp][t][lane] = acc[t];
    __syncthreads();
    for (int i = threadIdx.x; i < 28 * 32; i += blockDim.x) {
        const int t = i / 32, ch = i % 32;
        float s = 0.0f;
        for (int w = 0; w < 8; ++w) s += red[w][t][ch];
        if (t < T) atomicAdd(&dW[ch * T + t], s);
        else if (t == 27 && (IN || ch == 0)) atomicAdd(&db[IN ? ch : 0], s);
    }
}

// BF16 arrangements of the 32 x 32 layer's weights W [co][ci][T] (BF16) for
// k_conv_mid: forward Wf[t][co][ci] = W[co][ci][t]; data gradient
// Wb[t][ci][co] = W[co][ci][T-1-t] (mirrored taps)
__global__ void k_arrange_mid(const __nv_bfloat16* __restrict__ W, int T, __nv_bfloat16* __restrict__ Wf,
                              __nv_bfloat16* __restrict__ Wb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 32 * 32 * T) return;
    const int t = i % T, ci = (i / T) % 32, co = i / (32 * T);
    const __nv_bfloat16 w = W[i];
    Wf[((size_t)t * 32 + co) * 32 + ci] = w;
    Wb[((size_t)(T - 1 - t) * 32 + ci) * 32 + co] = w;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int conv_blocks(const DevPlan& P) { return P.nchunks; }

cudaError_t launch_conv_in(const DevPlan& P, const void* W, const float* b, const float* x, void* out,
                           cudaStream_t s) {
    if (P.nchunks == 0) return cudaSuccess;
    SGIGA_COUNT_LAUNCH();
    k_conv_in<<<conv_blocks(P), 256, 0, s>>>(P, (const __nv_bfloat16*)W, b, x, (__nv_bfloat16*)out);
    return cudaGetLastError();
}

cudaError_t launch_conv_out(const DevPlan& P, const void* W, const float* b, const void* A, float* y,
                            cudaStream_t s) {
    if (P.nchunks == 0) return cudaSuccess;
    SGIGA_COUNT_LAUNCH();
    k_conv_out<<<conv_blocks(P), 256, 0, s>>>(P, (const __nv_bfloat16*)W, b, (const __nv_bfloat16*)A, y);
    return cudaGetLastError();
}

cudaError_t launch_convT_out(const DevPlan& P, const void* W, const float* dy, const void* act, void* dA,
                             cudaStream_t s) {
    if (P.nchunks == 0) return cudaSuccess;
    SGIGA_COUNT_LAUNCH();
    k_convT_out<<<conv_blocks(P), 256, 0, s>>>(P, (const __nv_bfloat16*)W, dy, (const __nv_bfloat16*)act,
                                              (__nv_bfloat16*)dA);
    return cudaGetLastError();
}

cudaError_t launch_conv_mid(const DevPlan& P, const ConvTile* tiles, int ntiles, const void* Wt, const float* bias,
                            const void* X, const void* gate, int relu, void* out, cudaStream_t s) {
    if (ntiles == 0) return cudaSuccess;
    const int T = P.d == 3 ? 27 : 9;
    const size_t sm = ((size_t)T * 32 + 2 * 64) * kRow * 2;
    cudaError_t e = cudaFuncSetAttribute(k_conv_mid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int blocks = ntiles < 2 * 152 ? ntiles : 2 * 152;
    SGIGA_COUNT_LAUNCH();
    k_conv_mid<<<blocks, 128, sm, s>>>(P, tiles, ntiles, (const __nv_bfloat16*)Wt, bias, (const __nv_bfloat16*)X,
                                       (const __nv_bfloat16*)gate, relu, (__nv_bfloat16*)out);
    return cudaGetLastError();
}

cudaError_t launch_wgrad_mid(const DevPlan& P, const ConvTile* tiles, int ntiles, const void* X, const void* dZ,
                             float* dW, float* db, cudaStream_t s) {
    if (ntiles == 0) return cudaSuccess;
    const int T = P.d == 3 ? 27 : 9;
    const size_t sm = (size_t)(1 + T) * 64 * kRow * 2;
    cudaError_t e = cudaFuncSetAttribute(k_wgrad_mid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int blocks = ntiles < 152 ? ntiles : 152;
    SGIGA_COUNT_LAUNCH();
    k_wgrad_mid<<<blocks, 288, sm, s>>>(P, tiles, ntiles, (const __nv_bfloat16*)X, (const __nv_bfloat16*)dZ, dW, db);
    return cudaGetLastError();
}

cudaError_t launch_wgrad_in(const DevPlan& P, const float* x, const void* dZ, float* dW, float* db, cudaStream_t s) {
    if (P.nchunks == 0) return cudaSuccess;
    const int blocks = P.nchunks < 2 * 152 ? P.nchunks : 2 * 152;
    SGIGA_COUNT_LAUNCH();
    k_wgrad_one<true><<<blocks, 256, 0, s>>>(P, x, (const __nv_bfloat16*)dZ, dW, db);
    return cudaGetLastError();
}

cudaError_t launch_wgrad_out(const DevPlan& P, const float* dy, const void* A, float* dW, float* db, cudaStream_t s) {
    if (P.nchunks == 0) return cudaSuccess;
    const int blocks = P.nchunks < 2 * 152 ? P.nchunks : 2 * 152;
    SGIGA_COUNT_LAUNCH();
    k_wgrad_one<false><<<blocks, 256, 0, s>>>(P, dy, (const __nv_bfloat16*)A, dW, db);
    return cudaGetLastError();
}

cudaError_t launch_arrange_mid(const void* W, int T, void* Wf, void* Wb, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_arrange_mid<<<(32 * 32 * T + 255) / 256, 256, 0, s>>>((const __nv_bfloat16*)W, T, (__nv_bfloat16*)Wf,
                                                           (__nv_bfloat16*)Wb);
    return cudaGetLastError();
}

}  // namespace sgiga
