// Evaluation of every component at parametric points and the combination sum
// (paper Sec. 3, eq. TD-combi-tec; post-processing of Sec. 4.1).
//
//   u_g(xi) = sum_i c_i prod_k R_{i_k}(xi_k),  R = B / W_k  (eq. u-IGA-approx)
//   u(xi)   = sum_g c_g u_g(xi), FP64 with Neumaier compensation.
#include "kernels.h"
#include "spline_dev.cuh"

namespace sgiga {

// Basis values of every 1D table at every point: vals[(t*npts + j)*(p+1) + r]
// = R_{first+r}(xi_j[dir_t]) of table t, first[t*npts + j] = first function.
// Shared by all components that use the table.
__global__ void k_eval_basis(DevPlan P, const double* __restrict__ xi, long long npts, double* __restrict__ vals,
                             int* __restrict__ first) {
    const int t = blockIdx.y;
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= npts) return;
    const Table1D& tb = P.tabs[t];
    const int d = P.d, p = P.p;
    const double* kn = P.knots + tb.koff;
    double x = xi[j * d + tb.dir];
    if (!(x >= 0.0 && x <= 1.0)) {  // outside the parametric domain: report, clamp
        atomicOr(&P.flags[1], 1);
        x = x < 0.0 ? 0.0 : 1.0;
    }
    int s = find_span(kn, tb.nf, p, x);
    double N[SGIGA_MAXP + 1];
    basis_funs<SGIGA_MAXP>(kn, s, p, x, N, nullptr);
    double W, dW;
    patch_weight_1d(*P.patch, tb.dir, x, W, dW);
    const long long o = (long long)t * npts + j;
    for (int r = 0; r <= p; ++r) vals[o * (p + 1) + r] = N[r] / W;
    first[o] = s - p;
}

__global__ void k_eval(DevPlan P, const double* __restrict__ coeffs, long long npts,
                       const double* __restrict__ vals, const int* __restrict__ first, double* __restrict__ ucomp) {
    const int g = blockIdx.y;
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= npts) return;
    const GridDesc& gd = P.grids[g];
    const int d = P.d, p = P.p;
    double Rv[3][SGIGA_MAXP + 1];
    int f0[3];
    for (int k = 0; k < 3; ++k) {
        if (k >= d) { Rv[k][0] = 1.0; f0[k] = 1; continue; }
        const long long o = (long long)gd.tab[k] * npts + j;
        f0[k] = first[o];
        for (int r = 0; r <= p; ++r) Rv[k][r] = vals[o * (p + 1) + r];
    }
    const long long st1 = gd.n[0], st2 = (long long)gd.n[0] * gd.n[1];
    const double* c = coeffs + gd.dof_off;
    double u = 0.0;
    const int pc = d == 3 ? p : 0;
    for (int rc = 0; rc <= pc; ++rc) {
        int i2 = d == 3 ? f0[2] + rc : 1;
        if (d == 3 && (i2 < 1 || i2 > gd.nf[2] - 2)) continue;
        for (int rb = 0; rb <= p; ++rb) {
            int i1 = f0[1] + rb;
            if (i1 < 1 || i1 > gd.nf[1] - 2) continue;
            double wbc = Rv[1][rb] * Rv[2][rc];
            double acc = 0.0;
            for (int ra = 0; ra <= p; ++ra) {
                int i0 = f0[0] + ra;
                if (i0 < 1 || i0 > gd.nf[0] - 2) continue;
                acc += Rv[0][ra] * c[(i0 - 1) + (i1 - 1) * st1 + (d == 3 ? (i2 - 1) * st2 : 0)];
            }
            u += wbc * acc;
        }
    }
    ucomp[(long long)g * npts + j] = u;
}

cudaError_t launch_eval(const DevPlan& P, const double* coeffs, const double* xi, long long npts, double* vals,
                        int* first, double* ucomp, cudaStream_t s) {
    if (npts <= 0) return cudaSuccess;
    dim3 gb((unsigned)((npts + 127) / 128), P.ntabs);
    SGIGA_COUNT_LAUNCH();
    k_eval_basis<<<gb, 128, 0, s>>>(P, xi, npts, vals, first);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((npts + 127) / 128), P.ngrids);
    SGIGA_COUNT_LAUNCH();
    k_eval<<<grid, 128, 0, s>>>(P, coeffs, npts, vals, first, ucomp);
    return cudaGetLastError();
}

// u[j] = sum_g coef[g] ucomp[g][j] with Neumaier compensation. A block
// handles 32 points x 8 groups of components: each thread compensates the sum
// of its group (components k, k+8, ...), then one thread per point combines the
// 8 (sum, compensation) pairs, again compensated. Coalesced: a warp reads 32
// consecutive points of one component.
__global__ void k_combine(int ng, const double* __restrict__ ucomp, long long npts, const double* __restrict__ coef,
                          double* __restrict__ u) {
    __shared__ double ps[8][33], pc[8][33];
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const long long j = (long long)blockIdx.x * 32 + lane;
    double sum = 0.0, comp = 0.0;
    if (j < npts) {
        for (int g = grp; g < ng; g += 8) {
            const double t = coef[g] * ucomp[(long long)g * npts + j];
            const double v = sum + t;
            comp += fabs(sum) >= fabs(t) ? (sum - v) + t : (t - v) + sum;
            sum = v;
        }
    }
    ps[grp][lane] = sum;
    pc[grp][lane] = comp;
    __syncthreads();
    if (grp == 0 && j < npts) {
        double s = 0.0, c = 0.0;
        for (int k = 0; k < 8; ++k) {
            const double t = ps[k][lane];
            const double v = s + t;
            c += fabs(s) >= fabs(t) ? (s - v) + t : (t - v) + s;
            s = v;
            c += pc[k][lane];
        }
        u[j] = s + c;
    }
}

cudaError_t launch_combine(const DevPlan& P, const double* ucomp, long long npts, const double* coef, double* u,
                           cudaStream_t s) {
    if (npts <= 0) return cudaSuccess;
    SGIGA_COUNT_LAUNCH();
    k_combine<<<(unsigned)((npts + 31) / 32), 256, 0, s>>>(P.ncomps, ucomp, npts, coef, u);
    return cudaGetLastError();
}

cudaError_t launch_combine_n(int ng, const double* ucomp, long long npts, const double* coef, double* u,
                             cudaStream_t s) {
    if (npts <= 0) return cudaSuccess;
    SGIGA_COUNT_LAUNCH();
    k_combine<<<(unsigned)((npts + 31) / 32), 256, 0, s>>>(ng, ucomp, npts, coef, u);
    return cudaGetLastError();
}

}  // namespace sgiga

namespace sgiga {

// Values and physical gradients of every component at (patch, xi) points.
// Block (x: points, y: component). The point's patch selects the component's
// piece; a coefficient is the packed solution for a kept function, the
// boundary array (Dirichlet lifting) otherwise. 3D plans are single-patch:
// every kept function is interior and there is no lifting.
//   u = sum_abc R_a(xi_0) R_b(xi_1) R_c(xi_2) c_abc,
//   d u / d xi_k = the same sum with R' in direction k,
//   grad_x u = J^{-T} grad_xi u,  R = B / W_k (eq. u-IGA-approx).
template <int D>
__global__ void k_eval_grad(DevPlan P, const double* __restrict__ coeffs, const double* __restrict__ xi,
                            const int* __restrict__ patch, long long npts, double* __restrict__ ucomp,
                            double* __restrict__ gcomp, int lifting) {
    const int c = blockIdx.y;
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= npts) return;
    const CompDesc& cd = P.comps[c];
    int pa = patch ? patch[j] : 0;
    if (pa < 0 || pa >= cd.npieces) {
        atomicOr(&P.flags[1], 2);
        pa = 0;
    }
    const GridDesc& g = P.grids[cd.piece0 + pa];
    const int p = P.p;
    double x[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < D; ++k) x[k] = xi[D * j + k];
    double N[D][SGIGA_MAXP + 1], dN[D][SGIGA_MAXP + 1];
    int f0[D];
    for (int k = 0; k < D; ++k) {
        if (!(x[k] >= 0.0 && x[k] <= 1.0)) {
            atomicOr(&P.flags[1], 1);
            x[k] = x[k] < 0.0 ? 0.0 : 1.0;
        }
        const Table1D& tb = P.tabs[g.tab[k]];
        const double* kn = P.knots + tb.koff;
        const int s = find_span(kn, tb.nf, p, x[k]);
        double B[SGIGA_MAXP + 1], dB[SGIGA_MAXP + 1];
        basis_funs<SGIGA_MAXP>(kn, s, p, x[k], B, dB);
        double W, dW;
        patch_weight_1d(P.patch[g.patch], k, x[k], W, dW);
        for (int r = 0; r <= p; ++r) {
            N[k][r] = B[r] / W;
            dN[k][r] = (dB[r] * W - B[r] * dW) / (W * W);
        }
        f0[k] = s - p;
    }
    double u = 0.0, gxi[3] = {0.0, 0.0, 0.0};
    if (D == 2) {
        const double* gf = (lifting && g.gf_off >= 0) ? P.gfull + g.gf_off : nullptr;
        for (int b = 0; b <= p; ++b) {
            const int i1 = f0[1] + b;
            double v = 0.0, dv = 0.0;
            for (int a = 0; a <= p; ++a) {
                const int i0 = f0[0] + a;
                double cv;
                if (piece_kept2(g, i0, i1)) cv = coeffs[piece_addr2(P.grids, g, i0, i1)];
                else cv = gf ? gf[i0 + (long long)i1 * g.nf[0]] : 0.0;
                v += N[0][a] * cv;
                dv += dN[0][a] * cv;
            }
            u += N[1][b] * v;
            gxi[0] += N[1][b] * dv;
            gxi[1] += dN[1][b] * v;
        }
    } else {
        const long long st1 = g.n[0], st2 = (long long)g.n[0] * g.n[1];
        const double* cg = coeffs + g.dof_off;
        for (int cc = 0; cc <= p; ++cc) {
            const int i2 = f0[D - 1] + cc;
            if (i2 < 1 || i2 > g.nf[D - 1] - 2) continue;
            double w = 0.0, w0 = 0.0, w1 = 0.0;
            for (int b = 0; b <= p; ++b) {
                const int i1 = f0[1] + b;
                if (i1 < 1 || i1 > g.nf[1] - 2) continue;
                double v = 0.0, dv = 0.0;
                for (int a = 0; a <= p; ++a) {
                    const int i0 = f0[0] + a;
                    if (i0 < 1 || i0 > g.nf[0] - 2) continue;
                    const double cv = cg[(i0 - 1) + (i1 - 1) * st1 + (i2 - 1) * st2];
                    v += N[0][a] * cv;
                    dv += dN[0][a] * cv;
                }
                w += N[1][b] * v;
                w0 += N[1][b] * dv;
                w1 += dN[1][b] * v;
            }
            u += N[D - 1][cc] * w;
            gxi[0] += N[D - 1][cc] * w0;
            gxi[1] += N[D - 1][cc] * w1;
            gxi[2] += dN[D - 1][cc] * w;
        }
    }
    ucomp[(long long)c * npts + j] = u;
    if (gcomp) {
        double X[3], J[3][3];
        patch_eval(P.patch[g.patch], x, X, J);
        // J^T grad_x = grad_xi, J[i][k] = d x_i / d xi_k
        if (D == 2) {
            const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
            gcomp[(long long)c * npts + j] = (J[1][1] * gxi[0] - J[1][0] * gxi[1]) / det;
            gcomp[((long long)P.ncomps + c) * npts + j] = (-J[0][1] * gxi[0] + J[0][0] * gxi[1]) / det;
        } else {
            // grad_x = adj(J)^T grad_xi / det J, with adj(J)^T = the cofactor matrix of J
            double C[3][3];
            for (int r = 0; r < 3; ++r)
                for (int k = 0; k < 3; ++k) {
                    const int r1 = (r + 1) % 3, r2 = (r + 2) % 3, k1 = (k + 1) % 3, k2 = (k + 2) % 3;
                    C[r][k] = J[r1][k1] * J[r2][k2] - J[r1][k2] * J[r2][k1];
                }
            const double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
            for (int r = 0; r < 3; ++r)
                gcomp[((long long)r * P.ncomps + c) * npts + j] =
                    (C[r][0] * gxi[0] + C[r][1] * gxi[1] + C[r][2] * gxi[2]) / det;
        }
    }
}

cudaError_t launch_eval_grad(const DevPlan& P, const double* coeffs, const double* xi, const int* patch,
                             long long npts, double* ucomp, double* gcomp, int lifting, cudaStream_t s) {
    if (npts <= 0) return cudaSuccess;
    dim3 grid((unsigned)((npts + 127) / 128), P.ncomps);
    SGIGA_COUNT_LAUNCH();
    if (P.d == 3) k_eval_grad<3><<<grid, 128, 0, s>>>(P, coeffs, xi, patch, npts, ucomp, gcomp, lifting);
    else k_eval_grad<2><<<grid, 128, 0, s>>>(P, coeffs, xi, patch, npts, ucomp, gcomp, lifting);
    return cudaGetLastError();
}

}  // namespace sgiga
