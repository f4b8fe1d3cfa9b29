// Device-side B-spline evaluation (paper Sec. 2.2, eq. Bsp) and geometry patch
// evaluation (eq. F-B-splines, NURBS with separable weights).
#pragma once
#include "internal.h"

namespace sgiga {

// Knot span s with kn[s] <= t < kn[s+1], restricted to p <= s <= nb-1 (nb basis
// functions); t at the right end maps to the last non-degenerate span.
__device__ __forceinline__ int find_span(const double* kn, int nb, int p, double t) {
    if (t >= kn[nb]) return nb - 1;
    if (t <= kn[p]) return p;
    int lo = p, hi = nb;           // kn[lo] <= t < kn[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (t < kn[mid]) hi = mid; else lo = mid;
    }
    return lo;
}

// The p+1 B-splines nonzero on span s, B_{s-p..s,p}(t), and their first
// derivatives, by the triangular form of the Cox-de Boor recursion (eq. Bsp,
// 0/0 = 0). dN may be null.
template <int MAXP>
__device__ __forceinline__ void basis_funs(const double* kn, int s, int p, double t, double* N, double* dN) {
    double left[MAXP + 1], right[MAXP + 1], Nm1[MAXP + 1];
    N[0] = 1.0;
    Nm1[0] = 1.0;
#pragma unroll
    for (int j = 1; j <= MAXP; ++j) {
        if (j > p) break;
        left[j] = t - kn[s + 1 - j];
        right[j] = kn[s + j] - t;
        double saved = 0.0;
#pragma unroll
        for (int r = 0; r < MAXP; ++r) {
            if (r >= j) break;
            double den = right[r + 1] + left[j - r];
            double tmp = den != 0.0 ? N[r] / den : 0.0;
            N[r] = saved + right[r + 1] * tmp;
            saved = left[j - r] * tmp;
        }
        N[j] = saved;
        if (j == p - 1) {
#pragma unroll
            for (int r = 0; r <= MAXP; ++r) if (r <= j) Nm1[r] = N[r];
        }
    }
    if (!dN) return;
    // B'_{i,p} = p/(k_{i+p}-k_i) B_{i,p-1} - p/(k_{i+p+1}-k_{i+1}) B_{i+1,p-1}, i = s-p+r
#pragma unroll
    for (int r = 0; r <= MAXP; ++r) {
        if (r > p) break;
        int i = s - p + r;
        double v = 0.0;
        if (r >= 1) {
            double den = kn[i + p] - kn[i];
            if (den != 0.0) v += p * Nm1[r - 1] / den;
        }
        if (r <= p - 1) {
            double den = kn[i + p + 1] - kn[i + 1];
            if (den != 0.0) v -= p * Nm1[r] / den;
        }
        dN[r] = v;
    }
}

// 1D rational weight function W_k(t) = sum_i w_i N_i(t) of patch direction k
// and its derivative (1, 0 for polynomial directions).
__device__ __forceinline__ void patch_weight_1d(const Patch& P, int k, double t, double& W, double& dW) {
    if (!P.rational[k]) { W = 1.0; dW = 0.0; return; }
    int deg = P.deg[k], nb = P.nc[k];
    int s = find_span(P.knots[k], nb, deg, t);
    double N[4], dN[4];
    basis_funs<3>(P.knots[k], s, deg, t, N, dN);
    W = 0.0; dW = 0.0;
    for (int r = 0; r <= deg; ++r) {
        W += P.w[k][s - deg + r] * N[r];
        dW += P.w[k][s - deg + r] * dN[r];
    }
}

// x = F(xi) and J[i][k] = dx_i/dxi_k of the patch (NURBS with weights
// prod_k w_k[i_k]): F = A / W with A = sum w N P, W = sum w N.
__device__ __forceinline__ void patch_eval(const Patch& P, const double* xi, double* x, double J[3][3]) {
    const int d = P.d;
    double N[3][4], dN[3][4];
    int s[3], deg[3];
    for (int k = 0; k < 3; ++k) {
        deg[k] = 0; s[k] = 0; N[k][0] = 1.0; dN[k][0] = 0.0;
        if (k >= d) continue;
        deg[k] = P.deg[k];
        s[k] = find_span(P.knots[k], P.nc[k], deg[k], xi[k]);
        basis_funs<3>(P.knots[k], s[k], deg[k], xi[k], N[k], dN[k]);
    }
    if (!(P.rational[0] || P.rational[1] || P.rational[2])) {
        // Polynomial patch: all weights are 1 and W = 1, so F = A and J = dA.
        // x = sum (prod N) cp; the derivative sums below give J.
        double A[3] = {0, 0, 0};
        for (int c = 0; c <= deg[2]; ++c)
            for (int b = 0; b <= deg[1]; ++b)
                for (int a = 0; a <= deg[0]; ++a) {
                    int i0 = s[0] - deg[0] + a, i1 = s[1] - deg[1] + b, i2 = s[2] - deg[2] + c;
                    int ci = i0 + P.nc[0] * (i1 + (d > 1 ? P.nc[1] : 1) * i2);
                    double v = N[0][a] * N[1][b] * N[2][c] * 1.0;
                    for (int i = 0; i < d; ++i) A[i] += v * P.cp[ci][i];
                }
        // Column k of J is summed with direction k innermost,
        //   J[i][k] = sum_{other dirs} (prod N) * sum_{a_k} dN_k[a_k] cp_i,
        // so a coordinate that is constant along direction k (an axis-aligned
        // box) gets an exactly zero derivative there instead of a sum of
        // cancelling products that leaves rounding residues.
        for (int i = 0; i < d; ++i) x[i] = A[i];
        for (int k = 0; k < d; ++k) {
            const int m1 = k == 0 ? 1 : 0, m2 = k == 2 ? 1 : 2;
            double Jk[3] = {0, 0, 0};
            for (int u2 = 0; u2 <= deg[m2]; ++u2)
                for (int u1 = 0; u1 <= deg[m1]; ++u1) {
                    double sk[3] = {0, 0, 0};
                    for (int uk = 0; uk <= deg[k]; ++uk) {
                        int id[3];
                        id[m1] = u1; id[m2] = u2; id[k] = uk;
                        int i0 = s[0] - deg[0] + id[0], i1 = s[1] - deg[1] + id[1], i2 = s[2] - deg[2] + id[2];
                        int ci = i0 + P.nc[0] * (i1 + (d > 1 ? P.nc[1] : 1) * i2);
                        for (int i = 0; i < d; ++i) sk[i] += dN[k][uk] * P.cp[ci][i];
                    }
                    const double outer = N[m1][u1] * N[m2][u2];
                    for (int i = 0; i < d; ++i) Jk[i] += outer * sk[i];
                }
            for (int i = 0; i < d; ++i) J[i][k] = Jk[i];
        }
        return;
    }
    // Rational patch: F = A / W, J = (dA W - A dW^T) / W^2.
    double A[3] = {0, 0, 0}, dA[3][3] = {{0}}, W = 0, dW[3] = {0, 0, 0};
    for (int c = 0; c <= deg[2]; ++c)
        for (int b = 0; b <= deg[1]; ++b)
            for (int a = 0; a <= deg[0]; ++a) {
                int i0 = s[0] - deg[0] + a, i1 = s[1] - deg[1] + b, i2 = s[2] - deg[2] + c;
                double wt = P.w[0][i0] * (d > 1 ? P.w[1][i1] : 1.0) * (d > 2 ? P.w[2][i2] : 1.0);
                int ci = i0 + P.nc[0] * (i1 + (d > 1 ? P.nc[1] : 1) * i2);
                double v = N[0][a] * N[1][b] * N[2][c] * wt;
                double g[3] = {dN[0][a] * N[1][b] * N[2][c] * wt,
                               N[0][a] * dN[1][b] * N[2][c] * wt,
                               N[0][a] * N[1][b] * dN[2][c] * wt};
                W += v;
                for (int k = 0; k < d; ++k) dW[k] += g[k];
                for (int i = 0; i < d; ++i) {
                    A[i] += v * P.cp[ci][i];
                    for (int k = 0; k < d; ++k) dA[i][k] += g[k] * P.cp[ci][i];
                }
            }
    for (int i = 0; i < d; ++i) {
        x[i] = A[i] / W;
        for (int k = 0; k < d; ++k) J[i][k] = (dA[i][k] * W - A[i] * dW[k]) / (W * W);
    }
}

// x = F(xi) alone (no Jacobian): the same sums as patch_eval's, so the same
// doubles.
__device__ __forceinline__ void patch_point(const Patch& P, const double* xi, double* x) {
    const int d = P.d;
    double N[3][4];
    int s[3], deg[3];
    for (int k = 0; k < 3; ++k) {
        deg[k] = 0; s[k] = 0; N[k][0] = 1.0;
        if (k >= d) continue;
        deg[k] = P.deg[k];
        s[k] = find_span(P.knots[k], P.nc[k], deg[k], xi[k]);
        basis_funs<3>(P.knots[k], s[k], deg[k], xi[k], N[k], nullptr);
    }
    const bool rat = P.rational[0] || P.rational[1] || P.rational[2];
    double A[3] = {0, 0, 0}, W = 0;
    for (int c = 0; c <= deg[2]; ++c)
        for (int b = 0; b <= deg[1]; ++b)
            for (int a = 0; a <= deg[0]; ++a) {
                int i0 = s[0] - deg[0] + a, i1 = s[1] - deg[1] + b, i2 = s[2] - deg[2] + c;
                double wt = rat ? P.w[0][i0] * (d > 1 ? P.w[1][i1] : 1.0) * (d > 2 ? P.w[2][i2] : 1.0) : 1.0;
                int ci = i0 + P.nc[0] * (i1 + (d > 1 ? P.nc[1] : 1) * i2);
                double v = N[0][a] * N[1][b] * N[2][c] * wt;
                W += v;
                for (int i = 0; i < d; ++i) A[i] += v * P.cp[ci][i];
            }
    for (int i = 0; i < d; ++i) x[i] = rat ? A[i] / W : A[i];
}

}  // namespace sgiga
