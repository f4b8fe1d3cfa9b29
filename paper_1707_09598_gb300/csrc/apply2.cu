// 2D matrix-free operator kernel: y = K x (MODE 0), the load vector (MODE 1)
// or the boundary lifting y -= K_IB g_B (MODE 2: the input is each piece's
// array of boundary coefficients over all of its functions) for every
// component at once (Problem 1, Sec. 2.2, pulled back to the parametric
// square). Multi-patch pieces read and add their interface functions at the
// address of the piece that stores them (GridDesc), so y is the glued
// (assembled) result.
//
//   grad u(q) = (D_a B_b x, B_a D_b x),  v = G_q grad u,
//   y = (D_a B_b)^T v_a + (B_a D_b)^T v_b.
// Stages: X --b--> S1 = {B_b X, D_b X} (pencil-major, shared); pencil a in
// registers (gradients, G from HBM, backward along a, in place); S1 --b^T--> Y,
// atomically added to the packed output.
#include "op_common.cuh"

namespace sgiga {

template <typename Real, int P, int MODE, bool DIAG>
__global__ void __launch_bounds__(256, sizeof(Real) == 4 ? 3 : 2)
k_op2(DevPlan Pl, const Real* __restrict__ x, Real* __restrict__ y, const int* __restrict__ active) {
    constexpr int Q = P + 1, P1 = P + 1;
    extern __shared__ double sm_raw[];
    Real* sm = reinterpret_cast<Real*>(sm_raw);
    const int tid = threadIdx.x, nth = blockDim.x;
    const TileDesc td = Pl.tiles[Pl.sched[blockIdx.x]];
    const GridDesc& g = Pl.grids[td.grid];
    if (active && !active[g.comp]) return;
    const int M = Pl.m;
    int ax[2], T[2], L[2], E0[2], NF[2], KLO[2], SLO[2];
    long long ST[2];
    const long long stp[2] = {1, (long long)g.n[0]};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        ax[k] = g.perm[k];
        T[k] = g.T[ax[k]];
        L[k] = (T[k] - 1) * M + P1;
        E0[k] = td.e0[ax[k]];
        NF[k] = g.nf[ax[k]];
        ST[k] = stp[ax[k]];
        KLO[k] = g.klo[ax[k]];
        SLO[k] = g.slo[ax[k]];
    }
    // kept function (logical indices) and its packed address
    const bool plain = g.alias[0] < 0 && g.alias[1] < 0 && !g.xcorner;
    auto kept = [&](int fa, int fb) {
        if (fa < KLO[0] || fa > NF[0] - 2 || fb < KLO[1] || fb > NF[1] - 2) return false;
        if (plain) return true;
        return !(fa == 0 && fb == 0);   // the excluded corner of a piece is (0,0) in any axis order
    };
    auto addr = [&](int fa, int fb) -> long long {
        if (plain) return g.dof_off + (fa - SLO[0]) * ST[0] + (fb - SLO[1]) * ST[1];
        int f[2];
        f[ax[0]] = fa;
        f[ax[1]] = fb;
        return piece_addr2(Pl.grids, g, f[0], f[1]);
    };
    const int Ta = T[0], Tb = T[1], La = L[0], Lb = L[1];
    const int QTb = Q * Tb, npen = QTb, LaP = La | 1;
    const FastDiv dLa(La);
    Real* tb[2];
    Real* tdv[2];
    Real* cur = sm;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        tb[k] = cur; cur += T[k] * Q * P1;
        tdv[k] = cur; cur += T[k] * Q * P1;
    }
    Real* X = cur; cur += La * Lb;
    Real* S1 = cur;
    const int S1n = npen * LaP;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const Table1D& tt = Pl.tabs[g.tab[ax[k]]];
        const long long base = (tt.off + (long long)E0[k] * Q) * P1;
        const int cnt = T[k] * Q * P1;
        for (int i = tid; i < cnt; i += nth) { tb[k][i] = OpData<Real>::R(Pl)[base + i]; tdv[k][i] = OpData<Real>::dR(Pl)[base + i]; }
    }
    __syncthreads();   // tables visible to every thread before any stage reads them
    if (MODE != 1) {
        const int nX = La * Lb;
        for (int idx = tid; idx < nX; idx += nth) {
            const int jb = dLa.div(idx), ja = idx - jb * La;
            int fa = E0[0] * M + ja, fb = E0[1] * M + jb;
            Real v = 0.0;
            if (MODE == 2) {   // every function: boundary coefficients (zero on kept functions)
                int f[2];
                f[ax[0]] = fa;
                f[ax[1]] = fb;
                v = (Real)Pl.gfull[g.gf_off + f[0] + (long long)f[1] * g.nf[0]];
            } else if (kept(fa, fb)) {
                if (SGIGA_GUARD(Pl, addr(fa, fb) >= 0 && addr(fa, fb) < Pl.ndof, CHK_OP2_X)) v = x[addr(fa, fb)];
            }
            X[idx] = v;
        }
        __syncthreads();
        const int n1 = npen * La;
        for (int idx = tid; idx < n1; idx += nth) {
            const int qb = dLa.div(idx), ja = idx - qb * La;
            int eb = qb / Q;
            const Real* bt = tb[1] + qb * P1;
            const Real* dt = tdv[1] + qb * P1;
            const Real* xp = X + (eb * M) * La + ja;
            Real sB = 0.0, sD = 0.0;
#pragma unroll
            for (int t = 0; t < P1; ++t) {
                Real v = xp[t * La];
                sB += bt[t] * v;
                sD += dt[t] * v;
            }
            S1[qb * LaP + ja] = sB;
            S1[S1n + qb * LaP + ja] = sD;
        }
        __syncthreads();
    }
    const long long nqp = Pl.nqp;
    const Real* __restrict__ G = OpData<Real>::G(Pl);
    const double* __restrict__ rho = Pl.rho;
    for (int pid = tid; pid < npen; pid += nth) {
        Real* c0 = S1 + pid * LaP;
        Real* c1 = c0 + S1n;
        Real a0[P1], a1[P1];
#pragma unroll
        for (int t = 0; t < P1; ++t) a0[t] = a1[t] = 0.0;
        long long gi = td.g_off + pid;
        for (int ea = 0; ea < Ta; ++ea) {
            const int base = ea * M;
            Real i0[P1], i1[P1];
            if (MODE != 1) {
#pragma unroll
                for (int t = 0; t < P1; ++t) { i0[t] = c0[base + t]; i1[t] = c1[base + t]; }
            }
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int qa = ea * Q + q;
                const Real* bt = tb[0] + qa * P1;
                const Real* dt = tdv[0] + qa * P1;
                if (MODE != 1) {
                    Real ga = 0.0, gb = 0.0;
#pragma unroll
                    for (int t = 0; t < P1; ++t) { ga += dt[t] * i0[t]; gb += bt[t] * i1[t]; }
                    Real va, vb;
                    if (DIAG) {   // metric with zero off-diagonal entry: only G_aa, G_bb
                        va = G[gi] * ga;
                        vb = G[2 * nqp + gi] * gb;
                    } else {
                        const Real G00 = G[gi], G01 = G[nqp + gi], G11 = G[2 * nqp + gi];
                        va = G00 * ga + G01 * gb;
                        vb = G01 * ga + G11 * gb;
                    }
#pragma unroll
                    for (int t = 0; t < P1; ++t) { a0[t] += dt[t] * va; a1[t] += bt[t] * vb; }
                } else {
                    const Real rv = (Real)rho[gi];
#pragma unroll
                    for (int t = 0; t < P1; ++t) a0[t] += bt[t] * rv;
                }
                gi += npen;
            }
            for (int u = 0; u < M; ++u) {
                c0[base + u] = a0[0];
                if (MODE != 1) c1[base + u] = a1[0];
#pragma unroll
                for (int t = 0; t < P; ++t) { a0[t] = a0[t + 1]; a1[t] = a1[t + 1]; }
                a0[P] = a1[P] = 0.0;
            }
        }
        const int base = Ta * M;
        for (int u = 0; u <= P - M; ++u) {
            c0[base + u] = a0[0];
            if (MODE != 1) c1[base + u] = a1[0];
#pragma unroll
            for (int t = 0; t < P; ++t) { a0[t] = a0[t + 1]; a1[t] = a1[t + 1]; }
            a0[P] = a1[P] = 0.0;
        }
    }
    __syncthreads();
    const int nX = La * Lb;
    for (int idx = tid; idx < nX; idx += nth) {
        const int jb = dLa.div(idx), ja = idx - jb * La;
        int fa = E0[0] * M + ja, fb = E0[1] * M + jb;
        if (!kept(fa, fb)) continue;
        int lo = elem_lo(jb, P, M), hi = elem_hi(jb, M, Tb);
        Real yv = 0.0;
        for (int eb = lo; eb <= hi; ++eb) {
            const int t = jb - eb * M;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int qb = eb * Q + q;
                const int o = qb * LaP + ja;
                yv += tb[1][qb * P1 + t] * S1[o];
                if (MODE != 1) yv += tdv[1][qb * P1 + t] * S1[S1n + o];
            }
        }
        if (SGIGA_GUARD(Pl, addr(fa, fb) >= 0 && addr(fa, fb) < Pl.ndof, CHK_OP2_Y))
            atomicAdd(&y[addr(fa, fb)], MODE == 2 ? -yv : yv);
    }
}

template <int P>
static cudaError_t launch2(const DevPlan& Pl, const double* x, double* y, const int* active, int mode,
                           cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    if (mode == 1)
        k_op2<double, P, 1, false><<<Pl.ntiles, 256, Pl.smem_op, s>>>(Pl, x, y, active);
    else if (mode == 2)
        k_op2<double, P, 2, false><<<Pl.ntiles, 256, Pl.smem_op, s>>>(Pl, x, y, active);
    else if (Pl.diag)
        k_op2<double, P, 0, true><<<Pl.ntiles, 256, Pl.smem_op, s>>>(Pl, x, y, active);
    else
        k_op2<double, P, 0, false><<<Pl.ntiles, 256, Pl.smem_op, s>>>(Pl, x, y, active);
    return cudaGetLastError();
}

cudaError_t launch_op2(const DevPlan& Pl, const double* x, double* y, const int* active, int mode,
                       cudaStream_t s) {
    switch (Pl.p) {
    case 1: return launch2<1>(Pl, x, y, active, mode, s);
    case 2: return launch2<2>(Pl, x, y, active, mode, s);
    case 3: return launch2<3>(Pl, x, y, active, mode, s);
    case 4: return launch2<4>(Pl, x, y, active, mode, s);
    }
    return cudaErrorInvalidValue;
}

// FP32 stiffness apply (FP32 geometry planes and tables, FP32 accumulation).
template <int P>
static cudaError_t launch2f(const DevPlan& Pl, const float* x, float* y, const int* active, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    if (Pl.diag)
        k_op2<float, P, 0, true><<<Pl.ntiles, 256, Pl.smem_op / 2, s>>>(Pl, x, y, active);
    else
        k_op2<float, P, 0, false><<<Pl.ntiles, 256, Pl.smem_op / 2, s>>>(Pl, x, y, active);
    return cudaGetLastError();
}

cudaError_t launch_op2_f32(const DevPlan& Pl, const float* x, float* y, const int* active, cudaStream_t s) {
    switch (Pl.p) {
    case 1: return launch2f<1>(Pl, x, y, active, s);
    case 2: return launch2f<2>(Pl, x, y, active, s);
    case 3: return launch2f<3>(Pl, x, y, active, s);
    case 4: return launch2f<4>(Pl, x, y, active, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t set_op2_smem(int p, size_t bytes) {
    cudaError_t e = cudaSuccess;
#define SET(PP)                                                                                          \
    if (p == PP) {                                                                                       \
        e = cudaFuncSetAttribute(k_op2<double, PP, 0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes); \
        if (e == cudaSuccess)                                                                            \
            e = cudaFuncSetAttribute(k_op2<double, PP, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes); \
        if (e == cudaSuccess)                                                                            \
            e = cudaFuncSetAttribute(k_op2<double, PP, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes); \
        if (e == cudaSuccess)                                                                            \
            e = cudaFuncSetAttribute(k_op2<double, PP, 2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes); \
        if (e == cudaSuccess)                                                                            \
            e = cudaFuncSetAttribute(k_op2<float, PP, 0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(bytes / 2)); \
        if (e == cudaSuccess)                                                                            \
            e = cudaFuncSetAttribute(k_op2<float, PP, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(bytes / 2)); \
    }
    SET(1) SET(2) SET(3) SET(4)
#undef SET
    return e;
}

}  // namespace sgiga
