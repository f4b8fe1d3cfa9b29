// 3D matrix-free operator kernel: y = K x (MODE 0) or b = load vector (MODE 1)
// for every component at once (Galerkin stiffness / right-hand side of
// Problem 1 pulled back to the parametric cube, Sec. 2.2).
//
//   grad u(q) = (D_a B_b B_c x, B_a D_b B_c x, B_a B_b D_c x)   (forward)
//   v(q)      = G_q grad u(q)                                  (pointwise)
//   y         = (D_a B_b B_c)^T v_a + (B_a D_b B_c)^T v_b + (B_a B_b D_c)^T v_c
//
// B_x / D_x are the 1D tables of values / derivatives at Gauss points. Stages:
//   X  --c-->  S1 = {B_c X, D_c X}                       (shared)
//   S1 --b-->  S2 = {B_b S1_B, D_b S1_B, B_b S1_D}       (shared, pencil-major)
//   pencil a (registers): gradients, G from HBM, backward along a, in place
//   S2 --b^T--> S1 = {B_b^T W0 + D_b^T W1, B_b^T W2}
//   S1 --c^T--> Y, atomically added to the packed output vector.
#include "op_common.cuh"

namespace sgiga {

// NT threads per block: 256 (FP64, and FP32 with large tiles) or 128 (FP32:
// more, smaller blocks per SM, so that one block's warps waiting at a stage
// barrier overlap with other blocks' work; chosen by the autotuner).
// A metric value of the FP32 apply: streamed (read once per apply), loaded
// with the evict-first policy so that it does not push the tile's x and y
// entries, which neighbouring tiles reuse, out of L2.
__device__ __forceinline__ float ldg_stream(const float* p) { return __ldcs(p); }

template <typename Real, int P, int MODE, bool DIAG, int NT = 256>
__global__ void __launch_bounds__(NT, sizeof(Real) == 4 ? (NT == 128 ? 6 : 3) : 2)
k_op3(DevPlan Pl, const Real* __restrict__ x, Real* __restrict__ y, const int* __restrict__ active) {
    constexpr int Q = P + 1, P1 = P + 1;
    // FP32 stiffness: the b-direction stages run as register-window pencils
    // (fewer index divisions and shared loads per FMA; FP64 is FMA-bound and
    // keeps the per-output form)
    constexpr bool PB = sizeof(Real) == 4 && MODE == 0;
    extern __shared__ double sm_raw[];
    Real* sm = reinterpret_cast<Real*>(sm_raw);
    const int tid = threadIdx.x, nth = blockDim.x;
    const TileDesc td = Pl.tiles[Pl.sched[blockIdx.x]];
    const GridDesc& g = Pl.grids[td.grid];
    if (active && !active[g.comp]) return;
    const int M = Pl.m;
    int ax[3], T[3], L[3], E0[3], NF[3];
    long long ST[3];
    const long long stp[3] = {1, (long long)g.n[0], (long long)g.n[0] * g.n[1]};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        ax[k] = g.perm[k];
        T[k] = g.T[ax[k]];
        L[k] = (T[k] - 1) * M + P1;
        E0[k] = td.e0[ax[k]];
        NF[k] = g.nf[ax[k]];
        ST[k] = stp[ax[k]];
    }
    const int Ta = T[0], Tb = T[1], Tc = T[2], La = L[0], Lb = L[1], Lc = L[2];
    const int QTb = Q * Tb, QTc = Q * Tc, npen = QTb * QTc, LaP = La | 1;
    const FastDiv dLa(La), dLb(Lb), dQTb(QTb);
    Real* tb[3];
    Real* tdv[3];
    Real* cur = sm;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        tb[k] = cur; cur += T[k] * Q * P1;
        tdv[k] = cur; cur += T[k] * Q * P1;
    }
    Real* X = cur; cur += (long long)La * Lb * Lc;
    Real* S1 = cur; cur += 2LL * QTc * Lb * La;
    Real* S2 = cur;
    const int S1n = QTc * Lb * La;
    const int S2n = npen * LaP;

#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const Table1D& tt = Pl.tabs[g.tab[ax[k]]];
        const long long base = (tt.off + (long long)E0[k] * Q) * P1;
        const int cnt = T[k] * Q * P1;
        for (int i = tid; i < cnt; i += nth) { tb[k][i] = OpData<Real>::R(Pl)[base + i]; tdv[k][i] = OpData<Real>::dR(Pl)[base + i]; }
    }
    const long long doff = g.dof_off;
    if constexpr (sizeof(Real) == 4 && MODE == 0) {
        // FP32: start moving this tile's metric planes from HBM to L2 now, so
        // that the pencil stage, which follows the two forward contractions,
        // reads them from L2. Each plane's tile segment is contiguous; with an
        // even number of quadrature points per direction (p odd) an element
        // holds a multiple of 8 points, so every segment starts and ends on a
        // 32-byte boundary, as the bulk prefetch needs (16). Pl.op_pf caps the
        // bytes per plane so that the segments in flight on all SMs stay well
        // inside L2: prefetched lines evicted before the pencil stage reads
        // them would be fetched from HBM twice.
        if constexpr ((P1 & 1) == 0) {
            if (Pl.op_pf >= 0 && tid < (DIAG ? 3 : 6)) {
                const int c = DIAG ? (tid == 0 ? 0 : 2 * tid + 1) : tid;    // diagonal planes 0, 3, 5
                const float* src = OpData<Real>::G(Pl) + (long long)c * Pl.nqp + td.g_off;
                long long bytes = (long long)QTb * QTc * Q * Ta * 4;
                if (Pl.op_pf > 0 && bytes > Pl.op_pf) bytes = Pl.op_pf & ~15;
                if (bytes >= 16) {
                    // evict-first: the planes are read once; x and y stay in L2
                    unsigned long long pol;
                    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
                    asm volatile("cp.async.bulk.prefetch.L2.global.L2::cache_hint [%0], %1, %2;\n" ::"l"(src),
                                 "r"((unsigned)bytes), "l"(pol) : "memory");
                }
            }
        }
    }
    __syncthreads();   // tables visible to every thread before any stage reads them
    if (MODE == 0) {
        const int nX = La * Lb * Lc;
        for (int idx = tid; idx < nX; idx += nth) {
            const int r = dLa.div(idx), ja = idx - r * La, jc = dLb.div(r), jb = r - jc * Lb;
            int fa = E0[0] * M + ja, fb = E0[1] * M + jb, fc = E0[2] * M + jc;
            Real v = 0.0;
            if (fa >= 1 && fa <= NF[0] - 2 && fb >= 1 && fb <= NF[1] - 2 && fc >= 1 && fc <= NF[2] - 2) {
                const long long xi = doff + (fa - 1) * ST[0] + (fb - 1) * ST[1] + (fc - 1) * ST[2];
                if (SGIGA_GUARD(Pl, xi >= 0 && xi < Pl.ndof, CHK_OP3_X)) v = x[xi];
            }
            X[idx] = v;
        }
        __syncthreads();
        // stage 1: contract c (DoF -> qp)
        for (int idx = tid; idx < S1n; idx += nth) {
            const int r = dLa.div(idx), ja = idx - r * La, qc = dLb.div(r), jb = r - qc * Lb;
            int ec = qc / Q;
            Real bt[P1], dt[P1];
            load_row<Real, P1>(tb[2] + qc * P1, bt);
            load_row<Real, P1>(tdv[2] + qc * P1, dt);
            const Real* xp = X + ((ec * M) * Lb + jb) * La + ja;
            Real sB = 0.0, sD = 0.0;
#pragma unroll
            for (int t = 0; t < P1; ++t) {
                Real v = xp[t * Lb * La];
                sB += bt[t] * v;
                sD += dt[t] * v;
            }
            S1[idx] = sB;
            S1[S1n + idx] = sD;
        }
        __syncthreads();
        // stage 2: contract b
        if constexpr (PB) {
            // FP32: one thread per (ja, qc) pencil walks along b with a
            // register window of the p+1 functions the current element touches
            // (M new ones loaded per element), writing Q qp per element
            for (int k = tid; k < La * QTc; k += nth) {
                const int qc = dLa.div(k), ja = k - qc * La;
                const Real* s1v = S1 + (long long)qc * Lb * La + ja;
                const Real* s1d = s1v + S1n;
                Real wv[P1], wd[P1];
#pragma unroll
                for (int t = 0; t < P1; ++t) { wv[t] = s1v[t * La]; wd[t] = s1d[t * La]; }
                for (int eb = 0; eb < Tb; ++eb) {
#pragma unroll
                    for (int q = 0; q < Q; ++q) {
                        const int qb = eb * Q + q;
                        Real bt[P1], dt[P1];
                        load_row<Real, P1>(tb[1] + qb * P1, bt);
                        load_row<Real, P1>(tdv[1] + qb * P1, dt);
                        Real s0 = 0.0, s1 = 0.0, s2 = 0.0;
#pragma unroll
                        for (int t = 0; t < P1; ++t) {
                            s0 += bt[t] * wv[t];
                            s1 += dt[t] * wv[t];
                            s2 += bt[t] * wd[t];
                        }
                        const int o = (qb + QTb * qc) * LaP + ja;
                        S2[o] = s0;
                        S2[S2n + o] = s1;
                        S2[2 * S2n + o] = s2;
                    }
                    if (eb + 1 < Tb) {
                        for (int u = 0; u < M; ++u) {
#pragma unroll
                            for (int t = 0; t < P; ++t) { wv[t] = wv[t + 1]; wd[t] = wd[t + 1]; }
                            const int jn = eb * M + P1 + u;   // <= (Tb - 1) * M + P = Lb - 1
                            wv[P] = s1v[jn * La];
                            wd[P] = s1d[jn * La];
                        }
                    }
                }
            }
        } else {
            const int n2 = npen * La;
            for (int idx = tid; idx < n2; idx += nth) {
                const int r = dLa.div(idx), ja = idx - r * La, qc = dQTb.div(r), qb = r - qc * QTb;
                int eb = qb / Q;
                Real bt[P1], dt[P1];
                load_row<Real, P1>(tb[1] + qb * P1, bt);
                load_row<Real, P1>(tdv[1] + qb * P1, dt);
                const Real* s1b = S1 + (qc * Lb + eb * M) * La + ja;
                const Real* s1d = s1b + S1n;
                Real s0 = 0.0, s1 = 0.0, s2 = 0.0;
    #pragma unroll
                for (int t = 0; t < P1; ++t) {
                    Real vb = s1b[t * La], vd = s1d[t * La];
                    s0 += bt[t] * vb;
                    s1 += dt[t] * vb;
                    s2 += bt[t] * vd;
                }
                int pid = qb + QTb * qc;
                S2[pid * LaP + ja] = s0;
                S2[S2n + pid * LaP + ja] = s1;
                S2[2 * S2n + pid * LaP + ja] = s2;
            }
        }
        __syncthreads();
    }
    // pencil stage along a
    const long long nqp = Pl.nqp;
    const Real* __restrict__ G = OpData<Real>::G(Pl);
    const double* __restrict__ rho = Pl.rho;
    for (int pid = tid; pid < npen; pid += nth) {
        Real* c0 = S2 + pid * LaP;
        Real* c1 = c0 + S2n;
        Real* c2 = c1 + S2n;
        Real a0[P1], a1[P1], a2[P1];
#pragma unroll
        for (int t = 0; t < P1; ++t) a0[t] = a1[t] = a2[t] = 0.0;
        long long gi = td.g_off + pid;
        // FP32: the metric values of the element's Q quadrature points are
        // loaded before any is used, so that their loads are in flight together
        // (the FP32 instance is latency-bound on them; the FP64 one is bound by
        // its FMA pipe and keeps its registers)
        constexpr bool PRE = sizeof(Real) == 4 && MODE == 0;
        constexpr int NGP = DIAG ? 3 : 6;
        Real gpre[PRE ? Q : 1][PRE ? NGP : 1];
        for (int ea = 0; ea < Ta; ++ea) {
            const int base = ea * M;
            Real i0[P1], i1[P1], i2[P1];
            if (MODE == 0) {
#pragma unroll
                for (int t = 0; t < P1; ++t) { i0[t] = c0[base + t]; i1[t] = c1[base + t]; i2[t] = c2[base + t]; }
            }
            if constexpr (PRE) {
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    long long gq = gi + (long long)q * npen;
                    if (!SGIGA_GUARD(Pl, gq >= 0 && gq < nqp, CHK_OP3_G)) gq = 0;
                    if (DIAG) {
                        gpre[q][0] = ldg_stream(G + gq);
                        gpre[q][1] = ldg_stream(G + 3 * nqp + gq);
                        gpre[q][2] = ldg_stream(G + 5 * nqp + gq);
                    } else {
#pragma unroll
                        for (int c = 0; c < NGP; ++c) gpre[q][c] = ldg_stream(G + c * nqp + gq);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int qa = ea * Q + q;
                Real bt[P1], dt[P1];
                load_row<Real, P1>(tb[0] + qa * P1, bt);
                load_row<Real, P1>(tdv[0] + qa * P1, dt);
                if (MODE == 0) {
                    Real ga = 0.0, gb = 0.0, gc = 0.0;
#pragma unroll
                    for (int t = 0; t < P1; ++t) { ga += dt[t] * i0[t]; gb += bt[t] * i1[t]; gc += bt[t] * i2[t]; }
                    Real va, vb, vc;
                    if constexpr (PRE) {
                        if (DIAG) {
                            va = gpre[q][0] * ga;
                            vb = gpre[q][1] * gb;
                            vc = gpre[q][2] * gc;
                        } else {
                            const Real G00 = gpre[q][0], G01 = gpre[q][1], G02 = gpre[q][2];
                            const Real G11 = gpre[q][3], G12 = gpre[q][4], G22 = gpre[q][NGP - 1];
                            va = G00 * ga + G01 * gb + G02 * gc;
                            vb = G01 * ga + G11 * gb + G12 * gc;
                            vc = G02 * ga + G12 * gb + G22 * gc;
                        }
                    } else if (DIAG) {   // metric with zero off-diagonal entries: only G_aa, G_bb, G_cc
                        va = G[gi] * ga;
                        vb = G[3 * nqp + gi] * gb;
                        vc = G[5 * nqp + gi] * gc;
                    } else {
                        const Real G00 = G[gi], G01 = G[nqp + gi], G02 = G[2 * nqp + gi];
                        const Real G11 = G[3 * nqp + gi], G12 = G[4 * nqp + gi], G22 = G[5 * nqp + gi];
                        va = G00 * ga + G01 * gb + G02 * gc;
                        vb = G01 * ga + G11 * gb + G12 * gc;
                        vc = G02 * ga + G12 * gb + G22 * gc;
                    }
#pragma unroll
                    for (int t = 0; t < P1; ++t) { a0[t] += dt[t] * va; a1[t] += bt[t] * vb; a2[t] += bt[t] * vc; }
                } else {
                    const Real rv = (Real)rho[gi];
#pragma unroll
                    for (int t = 0; t < P1; ++t) a0[t] += bt[t] * rv;
                }
                gi += npen;
            }
            for (int u = 0; u < M; ++u) {
                c0[base + u] = a0[0];
                if (MODE == 0) { c1[base + u] = a1[0]; c2[base + u] = a2[0]; }
#pragma unroll
                for (int t = 0; t < P; ++t) { a0[t] = a0[t + 1]; a1[t] = a1[t + 1]; a2[t] = a2[t + 1]; }
                a0[P] = a1[P] = a2[P] = 0.0;
            }
        }
        const int base = Ta * M;
        for (int u = 0; u <= P - M; ++u) {
            c0[base + u] = a0[0];
            if (MODE == 0) { c1[base + u] = a1[0]; c2[base + u] = a2[0]; }
#pragma unroll
            for (int t = 0; t < P; ++t) { a0[t] = a0[t + 1]; a1[t] = a1[t + 1]; a2[t] = a2[t + 1]; }
            a0[P] = a1[P] = a2[P] = 0.0;
        }
    }
    __syncthreads();
    // backward b: S2 -> S1
    if constexpr (PB) {
        // FP32: one thread per (ja, qc) pencil along b, accumulating the p+1
        // functions of the current element in registers; the lowest M are
        // complete after each element and are written out (as the a pencils)
        for (int k = tid; k < La * QTc; k += nth) {
            const int qc = dLa.div(k), ja = k - qc * La;
            Real* o1v = S1 + (long long)qc * Lb * La + ja;
            Real* o1d = o1v + S1n;
            Real aB[P1], aD[P1];
#pragma unroll
            for (int t = 0; t < P1; ++t) aB[t] = aD[t] = 0.0;
            for (int eb = 0; eb < Tb; ++eb) {
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const int qb = eb * Q + q;
                    const int o = (qb + QTb * qc) * LaP + ja;
                    const Real v0 = S2[o], v1 = S2[S2n + o], v2 = S2[2 * S2n + o];
                    Real bt[P1], dt[P1];
                    load_row<Real, P1>(tb[1] + qb * P1, bt);
                    load_row<Real, P1>(tdv[1] + qb * P1, dt);
#pragma unroll
                    for (int t = 0; t < P1; ++t) {
                        aB[t] += bt[t] * v0 + dt[t] * v1;
                        aD[t] += bt[t] * v2;
                    }
                }
                const int base = eb * M;
                for (int u = 0; u < M; ++u) {
                    o1v[(base + u) * La] = aB[0];
                    o1d[(base + u) * La] = aD[0];
#pragma unroll
                    for (int t = 0; t < P; ++t) { aB[t] = aB[t + 1]; aD[t] = aD[t + 1]; }
                    aB[P] = aD[P] = 0.0;
                }
            }
            const int base = Tb * M;
            for (int u = 0; u <= P - M; ++u) {
                o1v[(base + u) * La] = aB[0];
                o1d[(base + u) * La] = aD[0];
#pragma unroll
                for (int t = 0; t < P; ++t) { aB[t] = aB[t + 1]; aD[t] = aD[t + 1]; }
                aB[P] = aD[P] = 0.0;
            }
        }
    } else {
        for (int idx = tid; idx < S1n; idx += nth) {
            const int r = dLa.div(idx), ja = idx - r * La, qc = dLb.div(r), jb = r - qc * Lb;
            int lo = elem_lo(jb, P, M), hi = elem_hi(jb, M, Tb);
            Real rB = 0.0, rD = 0.0;
            for (int eb = lo; eb <= hi; ++eb) {
                const int t = jb - eb * M;
    #pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const int qb = eb * Q + q;
                    const int o = (qb + QTb * qc) * LaP + ja;
                    const Real bv = tb[1][qb * P1 + t];
                    if (MODE == 0) {
                        rB += bv * S2[o] + tdv[1][qb * P1 + t] * S2[S2n + o];
                        rD += bv * S2[2 * S2n + o];
                    } else {
                        rB += bv * S2[o];
                    }
                }
            }
            S1[idx] = rB;
            if (MODE == 0) S1[S1n + idx] = rD;
        }
    }
    __syncthreads();
    // backward c and scatter
    const int nX = La * Lb * Lc;
    for (int idx = tid; idx < nX; idx += nth) {
        const int r = dLa.div(idx), ja = idx - r * La, jc = dLb.div(r), jb = r - jc * Lb;
        int fa = E0[0] * M + ja, fb = E0[1] * M + jb, fc = E0[2] * M + jc;
        if (!(fa >= 1 && fa <= NF[0] - 2 && fb >= 1 && fb <= NF[1] - 2 && fc >= 1 && fc <= NF[2] - 2)) continue;
        int lo = elem_lo(jc, P, M), hi = elem_hi(jc, M, Tc);
        Real yv = 0.0;
        for (int ec = lo; ec <= hi; ++ec) {
            const int t = jc - ec * M;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int qc = ec * Q + q;
                const int o = (qc * Lb + jb) * La + ja;
                yv += tb[2][qc * P1 + t] * S1[o];
                if (MODE == 0) yv += tdv[2][qc * P1 + t] * S1[S1n + o];
            }
        }
        const long long yi = doff + (fa - 1) * ST[0] + (fb - 1) * ST[1] + (fc - 1) * ST[2];
        if (SGIGA_GUARD(Pl, yi >= 0 && yi < Pl.ndof, CHK_OP3_Y)) atomicAdd(&y[yi], yv);
    }
}

template <int P>
static cudaError_t launch3(const DevPlan& Pl, const double* x, double* y, const int* active, int mode,
                           cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    if (mode == 1)
        k_op3<double, P, 1, false><<<Pl.ntiles, 256, Pl.smem_op, s>>>(Pl, x, y, active);
    else if (Pl.diag)
        k_op3<double, P, 0, true><<<Pl.ntiles, 256, Pl.smem_op, s>>>(Pl, x, y, active);
    else
        k_op3<double, P, 0, false><<<Pl.ntiles, 256, Pl.smem_op, s>>>(Pl, x, y, active);
    return cudaGetLastError();
}

cudaError_t launch_op3(const DevPlan& Pl, const double* x, double* y, const int* active, int mode,
                       cudaStream_t s) {
    switch (Pl.p) {
    case 1: return launch3<1>(Pl, x, y, active, mode, s);
    case 2: return launch3<2>(Pl, x, y, active, mode, s);
    case 3: return launch3<3>(Pl, x, y, active, mode, s);
    case 4: return launch3<4>(Pl, x, y, active, mode, s);
    }
    return cudaErrorInvalidValue;
}

// FP32 stiffness apply (FP32 geometry planes and tables, FP32 accumulation).
template <int P>
static cudaError_t launch3f(const DevPlan& Pl, const float* x, float* y, const int* active, cudaStream_t s) {
    SGIGA_COUNT_LAUNCH();
    if (Pl.op_nth == 128) {
        if (Pl.diag)
            k_op3<float, P, 0, true, 128><<<Pl.ntiles, 128, Pl.smem_op / 2, s>>>(Pl, x, y, active);
        else
            k_op3<float, P, 0, false, 128><<<Pl.ntiles, 128, Pl.smem_op / 2, s>>>(Pl, x, y, active);
    } else if (Pl.diag) {
        k_op3<float, P, 0, true><<<Pl.ntiles, 256, Pl.smem_op / 2, s>>>(Pl, x, y, active);
    } else {
        k_op3<float, P, 0, false><<<Pl.ntiles, 256, Pl.smem_op / 2, s>>>(Pl, x, y, active);
    }
    return cudaGetLastError();
}

cudaError_t launch_op3_f32(const DevPlan& Pl, const float* x, float* y, const int* active, cudaStream_t s) {
    switch (Pl.p) {
    case 1: return launch3f<1>(Pl, x, y, active, s);
    case 2: return launch3f<2>(Pl, x, y, active, s);
    case 3: return launch3f<3>(Pl, x, y, active, s);
    case 4: return launch3f<4>(Pl, x, y, active, s);
    }
    return cudaErrorInvalidValue;
}

template <int P>
static int resident3f(const DevPlan& Pl) {
    int nb = 0;
    const int nth = Pl.op_nth == 128 ? 128 : 256;
    const size_t smem = Pl.smem_op / 2;
    cudaError_t e;
    if (nth == 128)
        e = Pl.diag ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_op3<float, P, 0, true, 128>, 128, smem)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_op3<float, P, 0, false, 128>, 128, smem);
    else
        e = Pl.diag ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_op3<float, P, 0, true>, 256, smem)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_op3<float, P, 0, false>, 256, smem);
    if (e != cudaSuccess) { cudaGetLastError(); return 1; }
    return nb > 0 ? nb : 1;
}

int op3_f32_resident(const DevPlan& Pl) {
    switch (Pl.p) {
    case 1: return resident3f<1>(Pl);
    case 2: return resident3f<2>(Pl);
    case 3: return resident3f<3>(Pl);
    case 4: return resident3f<4>(Pl);
    }
    return 1;
}

cudaError_t set_op3_smem(int p, size_t bytes) {
    cudaError_t e = cudaSuccess;
#define SET(PP)                                                                                          \
    if (p == PP) {                                                                                       \
        e = cudaFuncSetAttribute(k_op3<double, PP, 0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes); \
        if (e == cudaSuccess)                                                                            \
            e = cudaFuncSetAttribute(k_op3<double, PP, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes); \
        if (e == cudaSuccess)                                                                            \
            e = cudaFuncSetAttribute(k_op3<double, PP, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes); \
        if (e == cudaSuccess)                                                                            \
            e = cudaFuncSetAttribute(k_op3<float, PP, 0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(bytes / 2)); \
        if (e == cudaSuccess)                                                                            \
            e = cudaFuncSetAttribute(k_op3<float, PP, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(bytes / 2)); \
        if (e == cudaSuccess)                                                                            \
            e = cudaFuncSetAttribute(k_op3<float, PP, 0, false, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(bytes / 2)); \
        if (e == cudaSuccess)                                                                            \
            e = cudaFuncSetAttribute(k_op3<float, PP, 0, true, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(bytes / 2)); \
    }
    SET(1) SET(2) SET(3) SET(4)
#undef SET
    return e;
}

}  // namespace sgiga
