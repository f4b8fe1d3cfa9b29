// 1D basis tables at Gauss points (paper Sec. 2.2, eq. Bsp; NURBS "verbatim").
//
// For every (direction, level) table and every element e, Gauss point q:
//   xi = z_e + (1 + t_q) h_e / 2,  w = omega_q h_e / 2,
//   R_r = B_{first+r,p}(xi) / W(xi),  R'_r = (B' W - B W') / W^2,  r = 0..p,
// with W the direction's rational weight function of the geometry (1 for
// B-spline directions) and first = s - p for the knot span s of element e.
#include "kernels.h"
#include "spline_dev.cuh"

namespace sgiga {

__global__ void k_basis_tables(const Table1D* __restrict__ tabs, const double* __restrict__ knots,
                               const double* __restrict__ bp, const double* __restrict__ gauss,
                               const Patch* __restrict__ patch, int p, int Q, double* xi_out,
                               double* w_out, double* R_out, double* dR_out, int* first_out) {
    const Table1D tb = tabs[blockIdx.y];
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= tb.E * Q) return;
    int e = idx / Q, q = idx % Q;
    const double* kn = knots + tb.koff;
    double z0 = bp[tb.eoff + e], z1 = bp[tb.eoff + e + 1];
    double h = z1 - z0;
    double t = z0 + 0.5 * (1.0 + gauss[q]) * h;
    double wq = 0.5 * h * gauss[Q + q];
    int nb = tb.nf;
    int s = find_span(kn, nb, p, t);
    double N[SGIGA_MAXP + 1], dN[SGIGA_MAXP + 1];
    basis_funs<SGIGA_MAXP>(kn, s, p, t, N, dN);
    double W, dW;
    patch_weight_1d(*patch, tb.dir, t, W, dW);
    long long o = tb.off + idx;
    xi_out[o] = t;
    w_out[o] = wq;
    for (int r = 0; r <= p; ++r) {
        R_out[o * (p + 1) + r] = N[r] / W;
        dR_out[o * (p + 1) + r] = (dN[r] * W - N[r] * dW) / (W * W);
    }
    if (q == 0) first_out[tb.eoff + e] = s - p;
}

cudaError_t launch_basis_tables(const DevPlan& P, int maxE, cudaStream_t s) {
    dim3 block(128);
    dim3 grid((maxE * P.Q + block.x - 1) / block.x, P.ntabs);
    SGIGA_COUNT_LAUNCH();
    k_basis_tables<<<grid, block, 0, s>>>(P.tabs, P.knots, P.bp, P.gauss, P.patch, P.p, P.Q, P.xi, P.w,
                                          P.R, P.dR, P.first);
    return cudaGetLastError();
}

}  // namespace sgiga
