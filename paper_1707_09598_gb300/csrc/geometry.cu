// Geometry coefficients and load density at every quadrature point.
//
// For the Galerkin stiffness of Problem 1 pulled back to the parametric
// domain (Sec. 2.2, eqs. F-B-splines, spline_space_phys):
//   K_ij = sum_q grad R_i^T G_q grad R_j,  G_q = w_q |det J_q| (J_q^T J_q)^{-1},
//   b_i  = sum_q R_i rho_q,               rho_q = f(F(xi_q)) w_q |det J_q|.
// G is stored as d(d+1)/2 planes in the LOGICAL axis order of the operator
// kernel's tiles (a, b, c = perm of the physical directions), tile-major.
#include <math.h>

#include "kernels.h"
#include "op_common.cuh"
#include "spline_dev.cuh"

namespace sgiga {

// Tile-major qp index -> per-physical-direction global qp coordinate.
struct QpLoc {
    int qg[3];   // global qp index along each physical direction
};

__device__ __forceinline__ QpLoc tile_qp(const GridDesc& g, const TileDesc& t, int d, int Q, int idx) {
    const int pa = g.perm[0], pb = g.perm[1], pc = g.perm[2];
    int QTb = Q * g.T[pb];
    int npen = d == 3 ? QTb * Q * g.T[pc] : QTb;
    int qa = idx / npen, pid = idx - qa * npen;
    int qb = pid % QTb, qc = pid / QTb;
    QpLoc L;
    L.qg[0] = L.qg[1] = L.qg[2] = 0;
    L.qg[pa] = Q * t.e0[pa] + qa;
    L.qg[pb] = Q * t.e0[pb] + qb;
    if (d == 3) L.qg[pc] = Q * t.e0[pc] + qc;
    return L;
}

__device__ __forceinline__ long long natural_index(const GridDesc& g, int d, int Q, const QpLoc& L) {
    long long i = L.qg[0];
    if (d >= 2) i += (long long)Q * g.E[0] * L.qg[1];
    if (d == 3) i += (long long)Q * g.E[0] * Q * g.E[1] * L.qg[2];
    return g.qp_off + i;
}

__device__ __forceinline__ void qp_param(const DevPlan& P, const GridDesc& g, const QpLoc& L, double* xi,
                                         double& wq) {
    wq = 1.0;
    for (int k = 0; k < P.d; ++k) {
        const Table1D& tb = P.tabs[g.tab[k]];
        xi[k] = P.xi[tb.off + L.qg[k]];
        wq *= P.w[tb.off + L.qg[k]];
    }
    for (int k = P.d; k < 3; ++k) xi[k] = 0.0;
}

// Symmetric inverse of J^T J (d x d) times s; returns det J.
__device__ __forceinline__ double metric(int d, const double J[3][3], double s, double Gp[3][3]) {
    double A[3][3];
    for (int k = 0; k < d; ++k)
        for (int l = 0; l < d; ++l) {
            double v = 0.0;
            for (int i = 0; i < d; ++i) v += J[i][k] * J[i][l];
            A[k][l] = v;
        }
    double det;
    if (d == 2) {
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        double da = A[0][0] * A[1][1] - A[0][1] * A[1][0];
        double f = s * fabs(det) / da;
        Gp[0][0] = A[1][1] * f;
        Gp[1][1] = A[0][0] * f;
        Gp[0][1] = Gp[1][0] = -A[0][1] * f;
    } else {
        det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
              J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
              J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
        double c01 = A[0][2] * A[2][1] - A[0][1] * A[2][2];
        double c02 = A[0][1] * A[1][2] - A[0][2] * A[1][1];
        double c11 = A[0][0] * A[2][2] - A[0][2] * A[2][0];
        double c12 = A[0][2] * A[1][0] - A[0][0] * A[1][2];
        double c22 = A[0][0] * A[1][1] - A[0][1] * A[1][0];
        double da = A[0][0] * c00 + A[0][1] * (A[1][2] * A[2][0] - A[1][0] * A[2][2]) + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
        double f = s * fabs(det) / da;
        Gp[0][0] = c00 * f; Gp[0][1] = Gp[1][0] = c01 * f; Gp[0][2] = Gp[2][0] = c02 * f;
        Gp[1][1] = c11 * f; Gp[1][2] = Gp[2][1] = c12 * f; Gp[2][2] = c22 * f;
    }
    return det;
}

__global__ void k_geometry(DevPlan P) {
    const TileDesc t = P.tiles[blockIdx.x];
    const GridDesc g = P.grids[t.grid];
    const int d = P.d, Q = P.Q;
    long long nq = 1;
    for (int k = 0; k < d; ++k) nq *= (long long)Q * g.T[k];
    const int ncomp = d * (d + 1) / 2;
    const Patch& pt = P.patch[g.patch];
    for (int idx = threadIdx.x; idx < nq; idx += blockDim.x) {
        QpLoc L = tile_qp(g, t, d, Q, idx);
        double xi[3], wq;
        qp_param(P, g, L, xi, wq);
        double x[3], J[3][3];
        patch_eval(pt, xi, x, J);
        double Gp[3][3];
        double s = wq;
        if (P.acoef) {                                        // diffusion coefficient a(x_q)
            const double a = P.acoef[natural_index(g, d, Q, L)];
            if (!(a > 0.0 && a < INFINITY)) atomicOr(&P.flags[0], 2);
            s *= a;
        }
        double det = metric(d, J, s, Gp);
        if (!(det * (pt.orient < 0 ? -1.0 : 1.0) > 0.0)) atomicOr(&P.flags[0], 1);
        long long o = t.g_off + idx;
        int c = 0;
        for (int a = 0; a < d; ++a)
            for (int b = a; b < d; ++b) P.G[(long long)(c++) * P.nqp + o] = Gp[g.perm[a]][g.perm[b]];
        (void)ncomp;
        P.mw[o] = wq * fabs(det);   // mass weight: no coefficient (load vector)
    }
}

// flag = 1 if some off-diagonal geometry coefficient is nonzero
__global__ void k_offdiag(const double* __restrict__ G, long long nqp, int d, int* __restrict__ flag) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    const int planes3[3] = {1, 2, 4};
    const int np = d == 3 ? 3 : 1;
    bool nz = false;
    for (; i < nqp; i += stride)
        for (int k = 0; k < np; ++k) nz |= G[(long long)(d == 3 ? planes3[k] : 1) * nqp + i] != 0.0;
    if (__syncthreads_or(nz) && threadIdx.x == 0) atomicOr(flag, 1);
}

cudaError_t launch_offdiag_check(const DevPlan& P, int* flag, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    long long blocks = (P.nqp + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    SGIGA_COUNT_LAUNCH();
    k_offdiag<<<(unsigned)blocks, 256, 0, s>>>(P.G, P.nqp, P.d, flag);
    return cudaGetLastError();
}

// a(x_q) = exp(amp * sum_f cos(omega_f . x_q + phase_f)) at every quadrature
// point, natural order (random Fourier features of a log-normal field).
__global__ void k_coef_features(DevPlan P, const double* __restrict__ feat, int nfeat, double amp,
                                double* __restrict__ a) {
    const TileDesc t = P.tiles[blockIdx.x];
    const GridDesc g = P.grids[t.grid];
    const int d = P.d, Q = P.Q;
    long long nq = 1;
    for (int k = 0; k < d; ++k) nq *= (long long)Q * g.T[k];
    for (int idx = threadIdx.x; idx < nq; idx += blockDim.x) {
        QpLoc L = tile_qp(g, t, d, Q, idx);
        double xi[3], wq, x[3];
        qp_param(P, g, L, xi, wq);
        patch_point(P.patch[g.patch], xi, x);
        double f = 0.0;
        for (int i = 0; i < nfeat; ++i) {
            const double* ft = feat + 4 * i;
            double arg = ft[3];
            for (int k = 0; k < d; ++k) arg += ft[k] * x[k];
            f += cos(arg);
        }
        a[natural_index(g, d, Q, L)] = exp(amp * f);
    }
}

cudaError_t launch_coef_features(const DevPlan& P, const double* feat, int nfeat, double amp, double* a,
                                 cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_coef_features<<<P.ntiles, 256, 0, s>>>(P, feat, nfeat, amp, a);
    return cudaGetLastError();
}

cudaError_t launch_geometry(const DevPlan& P, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_geometry<<<P.ntiles, 256, 0, s>>>(P);
    return cudaGetLastError();
}

__global__ void k_qp_coords(DevPlan P, double* xq) {
    const TileDesc t = P.tiles[blockIdx.x];
    const GridDesc g = P.grids[t.grid];
    const int d = P.d, Q = P.Q;
    long long nq = 1;
    for (int k = 0; k < d; ++k) nq *= (long long)Q * g.T[k];
    for (int idx = threadIdx.x; idx < nq; idx += blockDim.x) {
        QpLoc L = tile_qp(g, t, d, Q, idx);
        double xi[3], wq, x[3];
        qp_param(P, g, L, xi, wq);
        patch_point(P.patch[g.patch], xi, x);
        long long nat = natural_index(g, d, Q, L);
        for (int k = 0; k < d; ++k) xq[(long long)k * P.nqp + nat] = x[k];
    }
}

cudaError_t launch_qp_coords(const DevPlan& P, double* xq, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_qp_coords<<<P.ntiles, 256, 0, s>>>(P, xq);
    return cudaGetLastError();
}

// f = -Laplace(u) of the built-in manufactured solutions (derived by hand).
__device__ double builtin_source(int src, int d, const double* x) {
    const double pi = 3.14159265358979323846;
    switch (src) {
    case 0: {  // u = prod sin(pi x_k)
        double v = d * pi * pi;
        for (int k = 0; k < d; ++k) v *= sin(pi * x[k]);
        return v;
    }
    case 1: {  // u = prod x_k (1 - x_k): -Laplace u = sum_k 2 prod_{j != k} x_j (1 - x_j)
        double v = 0.0;
        for (int k = 0; k < d; ++k) {
            double t = 2.0;
            for (int j = 0; j < d; ++j) if (j != k) t *= x[j] * (1.0 - x[j]);
            v += t;
        }
        return v;
    }
    case 2: {  // u = x y phi sin x, phi = (r^2-1)(r^2-4)
        double X = x[0], Y = x[1], r2 = X * X + Y * Y;
        double phi = (r2 - 1.0) * (r2 - 4.0);
        double sx = sin(X), cx = cos(X);
        double lap = phi * (2.0 * Y * cx - X * Y * sx) + 2.0 * (4.0 * r2 - 10.0) * (2.0 * X * Y * sx + X * X * Y * cx) +
                     X * Y * sx * (16.0 * r2 - 20.0);
        return -lap;
    }
    case 3: {  // u = -phi x y^2 [sin(pi z)]
        double X = x[0], Y = x[1], r2 = X * X + Y * Y;
        double phi = (r2 - 1.0) * (r2 - 4.0);
        double u2 = -phi * X * Y * Y;
        double lap2 = phi * (-2.0 * X) + 2.0 * (4.0 * r2 - 10.0) * (-3.0 * X * Y * Y) + (-X * Y * Y) * (16.0 * r2 - 20.0);
        if (d == 2) return -lap2;
        return (-lap2 + pi * pi * u2) * sin(pi * x[2]);
    }
    case SRC_LSHAPE_CORNER:
    case SRC_HARMONIC_QUADRATIC:   // harmonic: f = 0, the data is on the boundary
        return 0.0;
    default:
        return 1.0;
    }
}

__global__ void k_rhs_density(DevPlan P, int src, const double* __restrict__ fnat) {
    const TileDesc t = P.tiles[blockIdx.x];
    const GridDesc g = P.grids[t.grid];
    const int d = P.d, Q = P.Q;
    long long nq = 1;
    for (int k = 0; k < d; ++k) nq *= (long long)Q * g.T[k];
    for (int idx = threadIdx.x; idx < nq; idx += blockDim.x) {
        QpLoc L = tile_qp(g, t, d, Q, idx);
        double f;
        if (fnat) {
            f = fnat[natural_index(g, d, Q, L)];
        } else {
            double xi[3], wq, x[3];
            qp_param(P, g, L, xi, wq);
            patch_point(P.patch[g.patch], xi, x);
            f = builtin_source(src, d, x);
        }
        long long o = t.g_off + idx;
        P.rho[o] = f * P.mw[o];
    }
}

// f(x_q) of a built-in source at every quadrature point, natural order.
__global__ void k_source_qp(DevPlan P, int src, double* __restrict__ fout) {
    const TileDesc t = P.tiles[blockIdx.x];
    const GridDesc g = P.grids[t.grid];
    const int d = P.d, Q = P.Q;
    long long nq = 1;
    for (int k = 0; k < d; ++k) nq *= (long long)Q * g.T[k];
    for (int idx = threadIdx.x; idx < nq; idx += blockDim.x) {
        QpLoc L = tile_qp(g, t, d, Q, idx);
        double xi[3], wq, x[3];
        qp_param(P, g, L, xi, wq);
        patch_point(P.patch[g.patch], xi, x);
        fout[natural_index(g, d, Q, L)] = builtin_source(src, d, x);
    }
}

cudaError_t launch_source_qp(const DevPlan& P, int source, double* fout, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_source_qp<<<P.ntiles, 256, 0, s>>>(P, source, fout);
    return cudaGetLastError();
}

cudaError_t launch_rhs_density_builtin(const DevPlan& P, int source, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_rhs_density<<<P.ntiles, 256, 0, s>>>(P, source, nullptr);
    return cudaGetLastError();
}

// rho = f * mw from a user f in natural order. One block per tile walks the
// tile's box of quadrature points in natural order (direction 0 fastest), so
// the reads of f are rows of Q*T_0 contiguous values, and writes rho at the
// tile-major position, inside the tile's own contiguous range (the L2 merges
// those writes before they reach DRAM).
__global__ void k_rhs_density_nat(DevPlan P, const double* __restrict__ fnat) {
    const TileDesc t = P.tiles[blockIdx.x];
    const GridDesc& g = P.grids[t.grid];
    const int d = P.d, Q = P.Q;
    const int B0 = Q * g.T[0], B1 = d > 1 ? Q * g.T[1] : 1, B2 = d > 2 ? Q * g.T[2] : 1;
    const int pa = g.perm[0], pb = g.perm[1], pc = g.perm[2];
    const int QTb = Q * g.T[pb];
    const int npen = d == 3 ? QTb * Q * g.T[pc] : QTb;
    const long long n0 = (long long)Q * g.E[0], n1 = d > 1 ? (long long)Q * g.E[1] : 1;
    const long long base = g.qp_off + Q * t.e0[0] + n0 * ((long long)Q * t.e0[1] + n1 * (long long)Q * t.e0[2]);
    const FastDiv dB0(B0), dB1(B1);
    const int nq = B0 * B1 * B2;
    for (int j = threadIdx.x; j < nq; j += blockDim.x) {
        int l[3];
        const int r = dB0.div(j);
        l[0] = j - r * B0;
        l[2] = dB1.div(r);
        l[1] = r - l[2] * B1;
        const int idx = l[pa] * npen + l[pb] + (d == 3 ? QTb * l[pc] : 0);
        const long long o = t.g_off + idx;
        P.rho[o] = fnat[base + l[0] + n0 * (l[1] + n1 * l[2])] * P.mw[o];
    }
}

cudaError_t launch_rhs_density_user(const DevPlan& P, const double* f_nat, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_rhs_density_nat<<<P.ntiles, 256, 0, s>>>(P, f_nat);
    return cudaGetLastError();
}

// Densities of the learned scaling's features at every quadrature point
// (tile-major, the layout of rho): mode 0 the trace of G_q (its diagonal
// planes; the trace does not depend on the tile's axis order), mode 1 d times
// the parametric Gauss weight w_q. Their load vectors give
// c_i = sum_q R_i tr(G_q) / (d sum_q R_i w_q).
__global__ void k_feature_density(DevPlan P, double* __restrict__ out, int mode) {
    const TileDesc t = P.tiles[blockIdx.x];
    const GridDesc g = P.grids[t.grid];
    const int d = P.d, Q = P.Q;
    long long nq = 1;
    for (int k = 0; k < d; ++k) nq *= (long long)Q * g.T[k];
    for (int idx = threadIdx.x; idx < nq; idx += blockDim.x) {
        const long long o = t.g_off + idx;
        double v;
        if (mode == 0) {
            v = d == 3 ? P.G[o] + P.G[3 * P.nqp + o] + P.G[5 * P.nqp + o] : P.G[o] + P.G[2 * P.nqp + o];
        } else {
            QpLoc L = tile_qp(g, t, d, Q, idx);
            double xi[3], wq;
            qp_param(P, g, L, xi, wq);
            v = d * wq;
        }
        out[o] = v;
    }
}

cudaError_t launch_feature_density(const DevPlan& P, double* out, int mode, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_feature_density<<<P.ntiles, 256, 0, s>>>(P, out, mode);
    return cudaGetLastError();
}

// Index of the physical pair (k, l), k <= l, among the d(d+1)/2 entries of a
// symmetric d x d matrix stored row by row (upper triangle).
__device__ __forceinline__ int phys_pair(int d, int k, int l) {
    if (k > l) { const int t = k; k = l; l = t; }
    if (d == 2) return k == 0 ? l : 2;
    return k == 0 ? l : (k == 1 ? 2 + l : 5);
}

// Move the geometry coefficients between the plan's tile-major layout and a
// natural layout (physical component pairs, quadrature points in natural order
// with the plan's natural offsets). EXPORT copies G, mw out of the tile-major
// planes; otherwise they are written back into the tile-major planes of the
// current tiling. The values are the same doubles either way, so a re-tiling
// gathers them instead of evaluating the patch map again.
template <bool EXPORT>
__global__ void k_geometry_move(DevPlan P, double* __restrict__ Gn, double* __restrict__ mwn) {
    const TileDesc t = P.tiles[blockIdx.x];
    const GridDesc g = P.grids[t.grid];
    const int d = P.d, Q = P.Q;
    long long nq = 1;
    for (int k = 0; k < d; ++k) nq *= (long long)Q * g.T[k];
    int cmap[6];
    int nc = 0;
    for (int a = 0; a < d; ++a)
        for (int b = a; b < d; ++b) cmap[nc++] = phys_pair(d, g.perm[a], g.perm[b]);
    for (int idx = threadIdx.x; idx < nq; idx += blockDim.x) {
        const QpLoc L = tile_qp(g, t, d, Q, idx);
        const long long nat = natural_index(g, d, Q, L);
        const long long o = t.g_off + idx;
        for (int c = 0; c < nc; ++c) {
            if (EXPORT) Gn[(long long)cmap[c] * P.nqp + nat] = P.G[(long long)c * P.nqp + o];
            else P.G[(long long)c * P.nqp + o] = Gn[(long long)cmap[c] * P.nqp + nat];
        }
        if (EXPORT) mwn[nat] = P.mw[o];
        else P.mw[o] = mwn[nat];
    }
}

cudaError_t launch_geometry_export(const DevPlan& P, double* Gn, double* mwn, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_geometry_move<true><<<P.ntiles, 256, 0, s>>>(P, Gn, mwn);
    return cudaGetLastError();
}

cudaError_t launch_geometry_import(const DevPlan& P, double* Gn, double* mwn, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    k_geometry_move<false><<<P.ntiles, 256, 0, s>>>(P, Gn, mwn);
    return cudaGetLastError();
}

// Copy one grid's G (physical component order) and mw into natural order.
__global__ void k_geometry_natural(DevPlan P, int tile0, double* Gnat, double* mwnat) {
    const TileDesc t = P.tiles[tile0 + blockIdx.x];
    const GridDesc g = P.grids[t.grid];
    const int d = P.d, Q = P.Q;
    long long nq = 1;
    for (int k = 0; k < d; ++k) nq *= (long long)Q * g.T[k];
    // logical component index of physical pair (k, l)
    int lidx[3][3];
    {
        int inv[3];
        for (int a = 0; a < d; ++a) inv[g.perm[a]] = a;
        int c = 0, tab[3][3];
        for (int a = 0; a < d; ++a)
            for (int b = a; b < d; ++b) { tab[a][b] = tab[b][a] = c++; }
        for (int k = 0; k < d; ++k)
            for (int l = 0; l < d; ++l) lidx[k][l] = tab[inv[k]][inv[l]];
    }
    for (int idx = threadIdx.x; idx < nq; idx += blockDim.x) {
        QpLoc L = tile_qp(g, t, d, Q, idx);
        long long nat = natural_index(g, d, Q, L) - g.qp_off;
        long long o = t.g_off + idx;
        int c = 0;
        for (int k = 0; k < d; ++k)
            for (int l = k; l < d; ++l) Gnat[(long long)(c++) * g.nqp + nat] = P.G[(long long)lidx[k][l] * P.nqp + o];
        mwnat[nat] = P.mw[o];
    }
}

cudaError_t launch_geometry_natural(const DevPlan& P, int g, const GridDesc& gh, double* Gnat, double* mwnat,
                                    cudaStream_t s) {
    (void)g;
    SGIGA_COUNT_LAUNCH();
    k_geometry_natural<<<gh.ntiles, 256, 0, s>>>(P, gh.tile0, Gnat, mwnat);
    return cudaGetLastError();
}

// patch_eval behind a call boundary. Inlined into k_map_points with the patch
// chosen by a runtime index, this kernel returned non-finite coordinates for
// every point under nvcc 13.0 for sm_103a (the same source built for the host
// under ASan/UBSan, and the same kernel with a compile-time patch index, give
// finite values equal to the oracle's); the out-of-line call gives the oracle's
// values and is what the map-point tests check.
__device__ __noinline__ void patch_eval_call(const Patch& pt, const double* t, double* X, double (*J)[3]) {
    patch_eval(pt, t, X, J);
}

// Physical coordinates and Jacobian determinant of the patch map at
// parametric points (eq. F-B-splines; NURBS with separable weights).
__global__ void k_map_points(DevPlan P, const double* xi, const int* patch, long long npts, int npatch, double* x,
                             double* detj) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= npts) return;
    const int d = P.d;
    int q = patch ? patch[j] : 0;
    if (q < 0 || q >= npatch) { atomicOr(&P.flags[1], 2); q = 0; }
    double t[3] = {0.0, 0.0, 0.0}, X[3] = {0.0, 0.0, 0.0};
    double J[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
    for (int k = 0; k < d; ++k) {
        t[k] = xi[j * d + k];
        if (!(t[k] >= 0.0 && t[k] <= 1.0)) { atomicOr(&P.flags[1], 1); t[k] = t[k] < 0.0 ? 0.0 : 1.0; }
    }
    patch_eval_call(P.patch[q], t, X, J);
    for (int k = 0; k < d; ++k) x[j * d + k] = X[k];
    if (detj) {
        double dt;
        if (d == 2) dt = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        else dt = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                  J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        detj[j] = dt;
    }
}

cudaError_t launch_map_points(const DevPlan& P, const double* xi, const int* patch, long long npts, int npatch,
                              double* x, double* detj, cudaStream_t s) {
    if (npts <= 0) return cudaSuccess;
    SGIGA_COUNT_LAUNCH();
    k_map_points<<<(unsigned)((npts + 255) / 256), 256, 0, s>>>(P, xi, patch, npts, npatch, x, detj);
    return cudaGetLastError();
}

}  // namespace sgiga
