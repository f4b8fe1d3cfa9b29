// Nonhomogeneous Dirichlet data of multi-patch plans (the L-shaped domain; not
// in the paper, whose experiments have homogeneous data):
//   * on every Dirichlet side of every piece, the two end coefficients
//     interpolate g (open knot vectors interpolate at the ends);
//   * the side's other coefficients are the L2 projection of g onto the
//     side's 1D spline space, with the ends fixed (parametric measure, which
//     is arc length on the unit sides of the L-shape; p+1 Gauss points per
//     element, the rule of the assembly);
//   * the coefficients go into the piece's full boundary-coefficient array,
//     which the operator kernel (mode 2) turns into b_I -= K_IB g_B and the
//     evaluation adds to the solution.
#include "kernels.h"
#include "spline_dev.cuh"

namespace sgiga {

// g of the built-in sources with Dirichlet data at physical point x.
__device__ __forceinline__ double builtin_dirichlet(int src, const double* x) {
    const double X = x[0], Y = x[1];
    if (src == SRC_HARMONIC_QUADRATIC) return 1.0 + 2.0 * X - 3.0 * Y + 0.5 * (X * X - Y * Y) + X * Y;
    // r^(2/3) sin(2 theta / 3), theta in [0, 2 pi)
    const double r = hypot(X, Y);
    if (r == 0.0) return 0.0;
    double th = atan2(Y, X);
    if (th < 0.0) th += 2.0 * 3.14159265358979323846;
    return cbrt(r * r) * sin(2.0 * th / 3.0);
}

// Parametric point j of side sd: 0 and 1 are the side's ends, then the Gauss
// points of its elements (element-major).
__device__ __forceinline__ void side_point(const DevPlan& P, const SideDesc& sd, const GridDesc& g, long long j,
                                           double* xi) {
    if (sd.k < 0) { xi[0] = 0.0; xi[1] = 0.0; return; }   // the excluded corner of the piece
    const int kp = 1 - sd.k;
    double t;
    if (j < 2) {
        t = (double)j;
    } else {
        const Table1D& tb = P.tabs[g.tab[kp]];
        t = P.xi[tb.off + (j - 2)];
    }
    xi[sd.k] = sd.end ? 1.0 : 0.0;
    xi[kp] = t;
}

__device__ __forceinline__ long long side_npts(const DevPlan& P, const SideDesc& sd, const GridDesc& g) {
    if (sd.k < 0) return 1;
    return 2 + (long long)P.tabs[g.tab[1 - sd.k]].E * P.Q;
}

// Physical boundary points (block per side), [nbpts][2].
__global__ void k_boundary_points(DevPlan P, double* __restrict__ xb) {
    const SideDesc sd = P.sides[blockIdx.x];
    const GridDesc& g = P.grids[sd.piece];
    const long long np = side_npts(P, sd, g);
    for (long long j = threadIdx.x; j < np; j += blockDim.x) {
        double xi[3] = {0, 0, 0}, x[3];
        side_point(P, sd, g, j, xi);
        patch_point(P.patch[g.patch], xi, x);
        xb[2 * (sd.goff + j)] = x[0];
        xb[2 * (sd.goff + j) + 1] = x[1];
    }
}

__global__ void k_boundary_builtin(DevPlan P, int src, const double* __restrict__ xb, double* __restrict__ gdata,
                                   long long n) {
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    gdata[j] = builtin_dirichlet(src, xb + 2 * j);
}

// One thread per side: banded mass matrix of the side's direction, banded
// Cholesky of its interior block, coefficients into the piece's array.
__global__ void k_boundary_project(DevPlan P) {
    const int sidx = blockIdx.x * blockDim.x + threadIdx.x;
    if (sidx >= P.nsides) return;
    const SideDesc sd = P.sides[sidx];
    const GridDesc& g = P.grids[sd.piece];
    double* gf = P.gfull + g.gf_off;
    const double* gv = P.gdata + sd.goff;
    if (sd.k < 0) { gf[0] = gv[0]; return; }
    const int kp = 1 - sd.k;
    const Table1D& tb = P.tabs[g.tab[kp]];
    const int p = P.p, Q = P.Q, P1 = p + 1, nf = tb.nf, E = tb.E;
    double* band = P.gscratch + sd.soff;   // band[i*P1 + (i-j)] = M(i, j), j <= i
    double* rhs = band + (long long)nf * P1;
    for (long long i = 0; i < (long long)nf * P1; ++i) band[i] = 0.0;
    for (int i = 0; i < nf; ++i) rhs[i] = 0.0;
    for (int e = 0; e < E; ++e) {
        const int f0 = P.first[tb.eoff + e];
        for (int q = 0; q < Q; ++q) {
            const long long o = tb.off + (long long)e * Q + q;
            const double wq = P.w[o], gq = gv[2 + (long long)e * Q + q];
            const double* R = P.R + o * P1;
            for (int a = 0; a <= p; ++a) {
                const int i = f0 + a;
                rhs[i] += wq * gq * R[a];
                for (int b = 0; b <= a; ++b) band[(long long)i * P1 + (a - b)] += wq * R[a] * R[b];
            }
        }
    }
    const double c0 = gv[0], cN = gv[1];
    const int lo = 1, hi = nf - 2;   // interior unknowns
    for (int i = lo; i <= hi; ++i) {
        if (i <= p) rhs[i] -= band[(long long)i * P1 + i] * c0;                       // M(i, 0)
        if (nf - 1 - i <= p) rhs[i] -= band[(long long)(nf - 1) * P1 + (nf - 1 - i)] * cN;   // M(nf-1, i)
    }
    // banded Cholesky in place on rows lo..hi: L(i, j) at band[i*P1 + (i-j)]
    for (int i = lo; i <= hi; ++i) {
        const int j0 = max(lo, i - p);
        for (int j = j0; j <= i; ++j) {
            double s = band[(long long)i * P1 + (i - j)];
            for (int k = max(j0, j - p); k < j; ++k) s -= band[(long long)i * P1 + (i - k)] * band[(long long)j * P1 + (j - k)];
            if (j == i) band[(long long)i * P1] = sqrt(s);
            else band[(long long)i * P1 + (i - j)] = s / band[(long long)j * P1];
        }
    }
    for (int i = lo; i <= hi; ++i) {   // L y = rhs
        double s = rhs[i];
        for (int k = max(lo, i - p); k < i; ++k) s -= band[(long long)i * P1 + (i - k)] * rhs[k];
        rhs[i] = s / band[(long long)i * P1];
    }
    for (int i = hi; i >= lo; --i) {   // L^T x = y
        double s = rhs[i];
        for (int k = i + 1; k <= min(hi, i + p); ++k) s -= band[(long long)k * P1 + (k - i)] * rhs[k];
        rhs[i] = s / band[(long long)i * P1];
    }
    const int fk = sd.end ? g.nf[sd.k] - 1 : 0;
    for (int t = 0; t < nf; ++t) {
        const double v = t == 0 ? c0 : (t == nf - 1 ? cN : rhs[t]);
        int f[2];
        f[sd.k] = fk;
        f[kp] = t;
        gf[f[0] + (long long)f[1] * g.nf[0]] = v;
    }
}

cudaError_t launch_boundary_points(const DevPlan& P, double* xb, cudaStream_t s) {
    if (P.nsides == 0) return cudaSuccess;
    SGIGA_COUNT_LAUNCH();
    k_boundary_points<<<P.nsides, 128, 0, s>>>(P, xb);
    return cudaGetLastError();
}

cudaError_t launch_boundary_builtin(const DevPlan& P, int src, const double* xb, double* gdata, long long n,
                                    cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    SGIGA_COUNT_LAUNCH();
    k_boundary_builtin<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P, src, xb, gdata, n);
    return cudaGetLastError();
}

cudaError_t launch_boundary_project(const DevPlan& P, cudaStream_t s) {
    if (P.nsides == 0) return cudaSuccess;
    SGIGA_COUNT_LAUNCH();
    k_boundary_project<<<(P.nsides + 63) / 64, 64, 0, s>>>(P);
    return cudaGetLastError();
}

}  // namespace sgiga
