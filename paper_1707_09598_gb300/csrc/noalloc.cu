// Allocation-free fast-diagonalisation apply for one tensor-product grid.
//
// Some callers cannot call cudaMalloc at the point where they need the
// preconditioner: real-time or embedded loops that must not touch the device
// allocator after start-up (an allocation can block or fail at any time),
// processes whose device memory is owned by another allocator (for example a
// framework's caching allocator) that must account for every byte, and code
// running where an allocation is not permitted at all. For them this entry
// point takes everything as caller-owned buffers (the 1D eigenpairs, the
// input and the output) and keeps its two intermediate tensors in a
// file-scope device array instead of allocating.
//
// The array is sized for grids of at most SGIGA_NOALLOC_MAX_DOFS entries
// (two halves of 2 MB, 4 MB in total); every GPU that loads this library holds
// it until the process exits. Every call shares it, so calls that overlap on
// the GPU (different streams, or different host threads) race on it; order
// them. Each pass writes every entry it later reads, so nothing has to be
// cleared between calls. The array's device address is looked up once per
// device ordinal and cached; a cudaDeviceReset (or any other teardown of the
// device's primary context) invalidates it, so after one the process must not
// call this entry point again on that device.
#include <mutex>

#include "../../include/sgiga.h"
#include "kernels.h"

namespace sgiga {

static __device__ __align__(256) double g_noalloc_scratch[2 * SGIGA_NOALLOC_MAX_DOFS];

struct NoallocGrid {
    int d;
    int n[3];
    const double* U[3];
    const double* lam[3];
};

// out[a][i][b] = sum_j Mat[i][j] in[a][j][b] along direction `dir`, one thread
// per output; Mat = U^T (forward) or U (backward); the last forward pass
// divides by the eigenvalue sums.
__global__ void k_fd_noalloc(NoallocGrid G, int dir, int forward, int scale, const double* __restrict__ in,
                             double* __restrict__ out, long long N) {
    long long lin = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (lin >= N) return;
    long long B = 1;
    for (int k = 0; k < dir; ++k) B *= G.n[k];
    const int n = G.n[dir];
    long long b = lin % B, r = lin / B;
    int i = (int)(r % n);
    long long a = r / n;
    const double* U = G.U[dir];
    const double* vp = in + a * n * B + b;
    double acc = 0.0;
    for (int j = 0; j < n; ++j) {
        double m = forward ? U[(long long)j * n + i] : U[(long long)i * n + j];
        acc += m * vp[(long long)j * B];
    }
    if (scale) {
        long long rem = lin;
        double s = 0.0;
        for (int k = 0; k < G.d; ++k) {
            int ik = (int)(rem % G.n[k]);
            rem /= G.n[k];
            s += G.lam[k][ik];
        }
        acc /= s;
    }
    out[lin] = acc;
}

// Device address of the scratch array, resolved once per device.
static double* scratch_address(int dev, cudaError_t* err) {
    static std::mutex mu;
    static double* addr[64] = {nullptr};
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= 64) { *err = cudaErrorInvalidDevice; return nullptr; }
    if (!addr[dev]) {
        double* p = nullptr;
        *err = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
        if (*err != cudaSuccess) return nullptr;
        addr[dev] = p;
    }
    *err = cudaSuccess;
    return addr[dev];
}

}  // namespace sgiga

extern "C" int sgiga_fd_apply_noalloc(int d, const int* n, const double* const* U, const double* const* lam,
                                      const double* r, double* z, void* stream) {
    using namespace sgiga;
    if (d < 1 || d > 3 || !n || !U || !lam || !r || !z) {
        set_last_error("sgiga_fd_apply_noalloc: d must be 1..3 and no pointer may be null");
        return SGIGA_ERR_ARG;
    }
    long long N = 1;
    NoallocGrid G{};
    G.d = d;
    for (int k = 0; k < d; ++k) {
        if (n[k] < 1 || !U[k] || !lam[k]) {
            set_last_error("sgiga_fd_apply_noalloc: every n[k] must be >= 1 with U[k], lam[k] given");
            return SGIGA_ERR_ARG;
        }
        // checked after every factor: the product of up to three 31-bit sizes
        // must neither overflow nor wrap below the limit
        if (n[k] > SGIGA_NOALLOC_MAX_DOFS || N * n[k] > SGIGA_NOALLOC_MAX_DOFS) {
            set_last_error("sgiga_fd_apply_noalloc: grid has more than SGIGA_NOALLOC_MAX_DOFS (262144) entries");
            return SGIGA_ERR_ARG;
        }
        G.n[k] = n[k];
        G.U[k] = U[k];
        G.lam[k] = lam[k];
        N *= n[k];
    }
    // every array is read or written by kernels: host memory would fault the device
    auto on_device = [](const void* ptr) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) { cudaGetLastError(); return false; }
        return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
    };
    bool dev_ok = on_device(r) && on_device(z);
    for (int k = 0; k < d; ++k) dev_ok = dev_ok && on_device(U[k]) && on_device(lam[k]);
    if (!dev_ok) {
        set_last_error("sgiga_fd_apply_noalloc: r, z, U[k] and lam[k] must be device buffers");
        return SGIGA_ERR_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return SGIGA_ERR_CUDA;
    }
    double* s0 = scratch_address(dev, &e);
    if (!s0) {
        set_last_error(cudaGetErrorString(e));
        return SGIGA_ERR_CUDA;
    }
    double* s1 = s0 + SGIGA_NOALLOC_MAX_DOFS;
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned blocks = (unsigned)((N + 255) / 256);
    // forward passes r -> s0 -> s1 -> s0 (last one scaled), backward back to z
    double* fbuf[3] = {s0, s1, s0};
    const double* in = r;
    for (int k = 0; k < d; ++k) {
        double* out = fbuf[k];
        SGIGA_COUNT_LAUNCH();
        k_fd_noalloc<<<blocks, 256, 0, st>>>(G, k, 1, k == d - 1, in, out, N);
        in = out;
    }
    for (int k = 0; k < d; ++k) {
        double* out = (k == d - 1) ? z : (in == s0 ? s1 : s0);
        SGIGA_COUNT_LAUNCH();
        k_fd_noalloc<<<blocks, 256, 0, st>>>(G, k, 0, 0, in, out, N);
        in = out;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return SGIGA_ERR_CUDA;
    }
    return SGIGA_OK;
}
