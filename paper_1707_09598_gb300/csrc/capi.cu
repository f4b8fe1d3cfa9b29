// Host planner and C ABI (include/sgiga.h).
//
// sgiga_plan builds, once per (domain, p, r, w, grading):
//   - the index set and coefficients of the combination technique (Sec. 3,
//     eq. TD-combi-tec);
//   - per (direction, level) the open knot vector of 2^level elements with
//     graded breakpoints (Sec. 2.2, Sec. 4.4) and the Gauss rule;
//   - the tile decomposition of every component and its launch order (largest
//     tiles first, the greedy longest-processing-time order of Sec. 4.1);
//   - device tables (basis, geometry coefficients) through the CUDA kernels;
//   - the 1D generalised eigenpairs of the preconditioner (on the device, eig.cu).
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "plan.h"
#include "op_common.cuh"

namespace sgiga {
}

using namespace sgiga;

std::atomic<long long> sgiga::g_launches{0};

static thread_local std::string g_last_error = "";

void sgiga::set_last_error(const char* msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}


// ---------------------------------------------------------------------------
// 1D ingredients
// ---------------------------------------------------------------------------

// Gauss-Legendre nodes/weights on [-1,1] by Newton's method on P_Q.
static void gauss_legendre(int Q, double* x, double* w) {
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < Q; ++i) {
        double z = std::cos(pi * (i + 0.75) / (Q + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= Q; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (Q == 1) { p1 = z; p0 = 1.0; }
            dp = Q * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-17) break;
        }
        {   // final derivative at the converged root
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= Q; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (Q == 1) { p1 = z; p0 = 1.0; }
            dp = Q * (z * p1 - p0) / (z * z - 1.0);
        }
        x[Q - 1 - i] = z;                       // ascending
        w[Q - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

static double grading(int kind, double gamma, double t) {
    if (kind == SGIGA_GRADING_RADICAL) {
        double c = std::pow(2.0, gamma - 1.0);
        return t <= 0.5 ? c * std::pow(t, gamma) : 1.0 - c * std::pow(1.0 - t, gamma);
    }
    if (kind == SGIGA_GRADING_ONESIDED) return std::pow(t, gamma);
    return t;
}

static int make_user_patch(const sgiga_patch* up, int d, Patch& pt) {
    std::memset(&pt, 0, sizeof(pt));
    pt.d = d;
    int tot = 1;
    for (int k = 0; k < 3; ++k) {
        if (k >= d) { pt.deg[k] = 0; pt.nc[k] = 1; pt.nk[k] = 2; pt.knots[k][0] = 0; pt.knots[k][1] = 1;
                      pt.w[k][0] = 1.0; continue; }
        if (up->deg[k] < 1 || up->deg[k] > 3 || up->nknots[k] > 12 || up->ncp[k] > 8 || !up->knots[k] ||
            up->nknots[k] != up->ncp[k] + up->deg[k] + 1)
            return -1;
        pt.deg[k] = up->deg[k];
        pt.nk[k] = up->nknots[k];
        pt.nc[k] = up->ncp[k];
        for (int i = 0; i < pt.nk[k]; ++i) pt.knots[k][i] = up->knots[k][i];
        for (int i = 0; i < pt.nc[k]; ++i) pt.w[k][i] = up->weights[k] ? up->weights[k][i] : 1.0;
        pt.rational[k] = up->weights[k] ? 1 : 0;
        tot *= pt.nc[k];
    }
    if (tot > 128 || !up->cp) return -1;
    for (int i = 0; i < tot; ++i)
        for (int k = 0; k < d; ++k) pt.cp[i][k] = up->cp[(size_t)i * d + k];
    return 0;
}

static void make_patch(int domain, int d, Patch& pt) {
    std::memset(&pt, 0, sizeof(pt));
    pt.d = d;
    for (int k = 0; k < 3; ++k) {
        pt.deg[k] = 1;
        pt.nk[k] = 4;
        pt.nc[k] = 2;
        pt.knots[k][0] = pt.knots[k][1] = 0.0;
        pt.knots[k][2] = pt.knots[k][3] = 1.0;
        for (int i = 0; i < 8; ++i) pt.w[k][i] = 1.0;
    }
    if (domain == SGIGA_DOMAIN_UNIT) {
        int nc = 1 << d;
        for (int c = 0; c < nc; ++c)
            for (int k = 0; k < d; ++k) pt.cp[c][k] = (c >> k) & 1;
        return;
    }
    // quarter annulus: direction 0 radial (degree 1), direction 1 angular (degree 2)
    pt.deg[1] = 2;
    pt.nk[1] = 6;
    pt.nc[1] = 3;
    double kn[6] = {0, 0, 0, 1, 1, 1};
    for (int i = 0; i < 6; ++i) pt.knots[1][i] = kn[i];
    pt.w[1][0] = 1.0;
    pt.w[1][1] = std::sqrt(2.0) / 2.0;
    pt.w[1][2] = 1.0;
    pt.rational[1] = 1;
    const double rad[2] = {1.0, 2.0};
    const double ang[3][2] = {{1, 0}, {1, 1}, {0, 1}};
    int nz = d == 3 ? 2 : 1;
    for (int c = 0; c < nz; ++c)
        for (int j = 0; j < 3; ++j)
            for (int i = 0; i < 2; ++i) {
                int ci = i + 2 * (j + 3 * c);
                pt.cp[ci][0] = rad[i] * ang[j][0];
                pt.cp[ci][1] = rad[i] * ang[j][1];
                if (d == 3) pt.cp[ci][2] = c;
            }
}

static long long binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    long long r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

// Tile choice: power-of-two element extents per direction and the pencil
// axis, minimising a per-quadrature-point cost model within the
// shared-memory budget.
static void choose_tile(int d, int P, int M, const int* E, size_t budget, long long qpcap, int* Tphys, int* perm) {
    const int Q = P + 1, P1 = P + 1;
    double best = 1e300;
    int lim[3] = {1, 1, 1};
    for (int k = 0; k < d; ++k) lim[k] = std::min(E[k], 64);
    for (int t0 = 1; t0 <= lim[0]; t0 *= 2)
        for (int t1 = 1; t1 <= lim[1]; t1 *= 2)
            for (int t2 = 1; t2 <= lim[2]; t2 *= 2) {
                int Tp[3] = {t0, t1, t2};
                // all pencil choices; b, c in the remaining order by size
                for (int a = 0; a < d; ++a) {
                    int pr[3] = {a, -1, -1};
                    int o = 1;
                    for (int k = 0; k < d; ++k) if (k != a) pr[o++] = k;
                    if (d == 3 && Tp[pr[2]] > Tp[pr[1]]) std::swap(pr[1], pr[2]);
                    int Tl[3] = {Tp[pr[0]], d > 1 ? Tp[pr[1]] : 1, d > 2 ? Tp[pr[2]] : 1};
                    long long sm = op_smem_doubles(d, P, M, Tl) * 8;
                    if ((size_t)sm > budget) continue;
                    double La = (Tl[0] - 1) * M + P1, Lb = (Tl[1] - 1) * M + P1, Lc = (Tl[2] - 1) * M + P1;
                    double QTa = Q * Tl[0], QTb = Q * Tl[1], QTc = Q * Tl[2];
                    double cost, qp, npen;
                    if (d == 3) {
                        npen = QTb * QTc;
                        qp = QTa * npen;
                        double s1 = 2.0 * P1 * QTc * Lb * La, s2 = 3.0 * P1 * npen * La;
                        double pen = (6.0 * P1 + 9.0) * npen * QTa;
                        if (npen < 256) pen *= 1.0 + 0.25 * (256.0 / npen - 1.0);
                        cost = 2 * (s1 + s2) + pen + 10.0 * La * Lb * Lc + 6 * 256;
                    } else {
                        npen = QTb;
                        qp = QTa * npen;
                        double s1 = 2.0 * P1 * QTb * La;
                        double pen = (4.0 * P1 + 4.0) * npen * QTa;
                        if (npen < 256) pen *= 1.0 + 0.25 * (256.0 / npen - 1.0);
                        cost = 2 * s1 + pen + 10.0 * La * Lb + 4 * 256;
                    }
                    if (qp > qpcap) continue;
                    double c = cost / qp;
                    if (c < best - 1e-12) {
                        best = c;
                        for (int k = 0; k < 3; ++k) { Tphys[k] = Tp[k]; perm[k] = pr[k] < 0 ? k : pr[k]; }
                    }
                }
                if (d < 3) break;
            }
}

// 1D interior matrices of a table, from the device-computed tables: the
// upper bands [n][p+1] (entry (i, t) = matrix(i, i+t)) of the stiffness and
// mass matrices of the functions klo .. klo+n-1 (klo = 1: both ends
// Dirichlet; klo = 0: natural condition at the low end), appended to Kb, Mb.
static void assemble_band(int E, int Q, int p, int n, int klo, const double* w, const double* R, const double* dR,
                          const int* first, std::vector<double>& Kb, std::vector<double>& Mb) {
    const size_t b0 = Kb.size();
    Kb.resize(b0 + (size_t)n * (p + 1), 0.0);
    Mb.resize(b0 + (size_t)n * (p + 1), 0.0);
    for (int e = 0; e < E; ++e)
        for (int q = 0; q < Q; ++q) {
            long long o = (long long)e * Q + q;
            for (int a = 0; a <= p; ++a) {
                int i = first[e] + a - klo;
                if (i < 0 || i >= n) continue;
                for (int b = a; b <= p; ++b) {
                    int j = first[e] + b - klo;
                    if (j < 0 || j >= n) continue;
                    const size_t at = b0 + (size_t)i * (p + 1) + (j - i);
                    Kb[at] += w[o] * dR[o * (p + 1) + a] * dR[o * (p + 1) + b];
                    Mb[at] += w[o] * R[o * (p + 1) + a] * R[o * (p + 1) + b];
                }
            }
        }
}

static void free_plan(sgiga_plan_s* P) {
    if (!P) return;
    free_net(P);
    free_ct(P);
    destroy_loop_graph(P->loop64);
    destroy_loop_graph(P->loop32);
    if (P->own_stream) cudaStreamDestroy(P->own_stream);
    if (P->fds_ok) {
        for (int i = 0; i < 3; ++i) {
            cudaStreamDestroy(P->fds.aux[i]);
            cudaEventDestroy(P->fds.join[i]);
        }
        cudaEventDestroy(P->fds.fork);
    }
    if (P->d_eval_vals) cudaFree(P->d_eval_vals);
    if (P->d_eval_first) cudaFree(P->d_eval_first);
    for (void* a : P->allocs) cudaFree(a);
    if (P->stage) cudaFree(P->stage);
    if (P->acoef) cudaFree(P->acoef);
    if (P->h_nactive) cudaFreeHost(P->h_nactive);
    delete P;
}

// After the geometry planes change: is the metric diagonal everywhere?
// Preconditioner work items per direction. Short directions (n <= 64): SMALL
// items of one piece. Longer ones: the pieces whose direction k uses the same
// eigen table form one segment (a GEMM over all their fibres), cut into 64 x 64
// output tiles and ks-deep contraction ranges whose partial sums add
// atomically. Items are ordered by estimated FMAs, largest first (greedy
// longest-processing-time order), so that the short ones fill the tail.
static void make_fd_items(sgiga_plan_s* P, int ks, bool grouped) {
    const int d = P->d;
    P->fd_ks = ks;
    P->fd_grouped = grouped;
    P->fdsegs.clear();
    P->fdcb.clear();
    P->fdcs.clear();
    P->fdcc.clear();
    auto lpt = [](std::vector<FDItem>& v, const std::vector<long long>& cost) {
        std::vector<size_t> ord(v.size());
        for (size_t i = 0; i < ord.size(); ++i) ord[i] = i;
        std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
        std::vector<FDItem> sorted(v.size());
        for (size_t i = 0; i < ord.size(); ++i) sorted[i] = v[ord[i]];
        v.swap(sorted);
    };
    for (int k = 0; k < d; ++k) {
        std::vector<FDItem>& v = P->fd[k];
        v.clear();
        for (int t = 0; t < 3; ++t) P->fdl[k][t].clear();
        std::vector<long long> cost, lcost[3];
        std::map<int, std::vector<int>> by_eig;
        for (size_t gi = 0; gi < P->grids.size(); ++gi) {
            const GridDesc& g = P->grids[gi];
            const long long n = g.fn[k];
            if (g.fd_n == 0) continue;
            const long long ncol = g.fd_n / n;
            auto depth = [&](int j0) { return (int)std::min<long long>(n, j0 + ks); };
            if (n <= 64) {
                const int tc = fd_small_cols((int)n);
                for (long long c0 = 0; c0 < ncol; c0 += tc) {
                    v.push_back(FDItem{(int)gi, FD_SMALL, 0, 0, c0, 0, (int)n});
                    cost.push_back(std::min<long long>(tc, ncol - c0) * n * n);
                }
            } else if (grouped) {
                by_eig[g.eig[k]].push_back((int)gi);
            } else if (ncol >= 64) {
                for (long long i0 = 0; i0 < n; i0 += 32)
                    for (long long c0 = 0; c0 < ncol; c0 += 64)
                        for (int j0 = 0; j0 < n; j0 += ks) {
                            v.push_back(FDItem{(int)gi, FD_TILE, 0, (int)i0, c0, j0, depth(j0)});
                            cost.push_back(std::min<long long>(32, n - i0) * std::min<long long>(64, ncol - c0) *
                                           (depth(j0) - j0));
                        }
            } else {
                const long long ngr = (ncol + 7) / 8, per = (ncol + ngr - 1) / ngr;
                for (long long i0 = 0; i0 < n; i0 += 256)
                    for (long long c0 = 0; c0 < ncol; c0 += per)
                        for (int j0 = 0; j0 < n; j0 += ks) {
                            const int nc = (int)std::min(per, ncol - c0);
                            v.push_back(FDItem{(int)gi, FD_ROWS, nc, (int)i0, c0, j0, depth(j0)});
                            cost.push_back(std::min<long long>(256, n - i0) * nc * (depth(j0) - j0));
                        }
            }
        }
        for (auto& kv : by_eig) {
            FDSeg sg{};
            sg.eig = kv.first;
            sg.n = P->grids[kv.second[0]].fn[k];
            sg.unit = k == 0 ? 1 : 0;
            sg.col0 = (long long)P->fdcb.size();
            for (int gi : kv.second) {
                const GridDesc& g = P->grids[gi];
                long long B = 1;
                for (int j = 0; j < k; ++j) B *= g.fn[j];
                const long long n = g.fn[k], ncol = g.fd_n / n;
                for (long long c = 0; c < ncol; ++c) {
                    const long long a = c / B, b = c - a * B;
                    P->fdcb.push_back(g.fd_off + a * n * B + b);
                    P->fdcs.push_back((int)B);
                    P->fdcc.push_back(g.comp);
                }
            }
            sg.ncols = (int)((long long)P->fdcb.size() - sg.col0);
            // output tile class: 64 columns from 64 columns on (the 64 x 64 tile
            // re-reads U least: measured 0.736 against 0.780 ms per FP32
            // application on the perturbed cube), else the fewest padded
            // columns, ties to the wider tile
            int cls = 2;
            long long best = -1;
            for (int t = 2; t >= 0; --t) {
                const long long tn = 16LL << t, padded = (sg.ncols + tn - 1) / tn * tn;
                if (best < 0 || padded < best) { best = padded; cls = t; }
            }
            if (sg.ncols >= 64) cls = 2;
            sg.tn = 16 << cls;
            const int tm = 4096 / sg.tn;
            const int seg = (int)P->fdsegs.size();
            P->fdsegs.push_back(sg);
            for (int i0 = 0; i0 < sg.n; i0 += tm)
                for (int c0 = 0; c0 < sg.ncols; c0 += sg.tn)
                    for (int j0 = 0; j0 < sg.n; j0 += ks) {
                        const int j1 = std::min(sg.n, j0 + ks);
                        P->fdl[k][cls].push_back(FDItem{seg, FD_LEVEL, 0, i0, c0, j0, j1});
                        lcost[cls].push_back((long long)std::min(tm, sg.n - i0) * std::min(sg.tn, sg.ncols - c0) *
                                             (j1 - j0));
                    }
        }
        lpt(v, cost);
        for (int t = 0; t < 3; ++t) lpt(P->fdl[k][t], lcost[t]);
    }
}

// Upload the preconditioner work lists (host vectors -> plan device arrays).
static int upload_fd(sgiga_plan_s* P) {
    auto drop = [&](void* old) {
        if (!old) return;
        auto it = std::find(P->allocs.begin(), P->allocs.end(), old);
        if (it != P->allocs.end()) P->allocs.erase(it);
        cudaFree(old);
    };
    int rc;
    for (int k = 0; k < P->d; ++k) {
        drop(P->d_fd[k]);
        P->d_fd[k] = nullptr;
        if ((rc = upload(P, &P->d_fd[k], P->fd[k]))) return rc;
        for (int t = 0; t < 3; ++t) {
            drop(P->d_fdl[k][t]);
            P->d_fdl[k][t] = nullptr;
            if ((rc = upload(P, &P->d_fdl[k][t], P->fdl[k][t]))) return rc;
        }
    }
    drop(P->d_fdsegs); drop(P->d_fdcb); drop(P->d_fdcs); drop(P->d_fdcc);
    if ((rc = upload(P, &P->d_fdsegs, P->fdsegs)) || (rc = upload(P, &P->d_fdcb, P->fdcb)) ||
        (rc = upload(P, &P->d_fdcs, P->fdcs)) || (rc = upload(P, &P->d_fdcc, P->fdcc)))
        return rc;
    DevPlan& D = P->dp;
    D.fdsegs = P->d_fdsegs;
    D.fdcb = P->d_fdcb;
    D.fdcs = P->d_fdcs;
    D.fdcc = P->d_fdcc;
    return SGIGA_OK;
}

// Re-split the preconditioner work items (depth ks, layout) and upload them.
static int refd(sgiga_plan_s* P, int ks, bool grouped) {
    CUDA_TRY(cudaStreamSynchronize(P->stream));
    make_fd_items(P, ks, grouped);
    int rc = upload_fd(P);
    if (rc) return rc;
    destroy_loop_graph(P->loop64);   // the captured loops hold the old item arrays
    destroy_loop_graph(P->loop32);
    return SGIGA_OK;
}

static int update_diag(sgiga_plan_s* P) {
    CUDA_TRY(launch_offdiag_check(P->dp, P->dp.flags + 2, P->stream));
    int h = 1;
    CUDA_TRY(cudaMemcpyAsync(&h, P->dp.flags + 2, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
    CUDA_TRY(cudaStreamSynchronize(P->stream));
    P->dp.diag = h ? 0 : 1;
    destroy_loop_graph(P->loop64);
    destroy_loop_graph(P->loop32);
    return SGIGA_OK;
}

// Dynamic shared-memory attribute of the operator kernels; it only grows, so
// plans that coexist keep working.
static int grant_op_smem(sgiga_plan_s* P) {
    static size_t granted[2][SGIGA_MAXP + 1] = {{0}};
    size_t& gr = granted[P->d - 2][P->p];
    if (P->smem > gr) {
        if (P->d == 3) CUDA_TRY(set_op3_smem(P->p, P->smem)); else CUDA_TRY(set_op2_smem(P->p, P->smem));
        gr = P->smem;
    }
    return SGIGA_OK;
}

// Tile decomposition of every component under a shared-memory budget and a
// cap on quadrature points per tile; launch order = largest tiles first (the
// greedy longest-processing-time order of Sec. 4.1). Fills P->tiles, P->sched,
// the grids' tile fields and P->smem (host side only).
static void make_tiles(sgiga_plan_s* P, size_t budget, long long qpcap) {
    const int d = P->d, p = P->p, M = P->m, Q = P->Q;
    P->tiles.clear();
    P->smem = 0;
    long long tqp = 0;
    for (size_t gi = 0; gi < P->grids.size(); ++gi) {
        GridDesc& g = P->grids[gi];
        choose_tile(d, p, M, g.E, budget, qpcap, g.T, g.perm);
        int Tl[3] = {g.T[g.perm[0]], d > 1 ? g.T[g.perm[1]] : 1, d > 2 ? g.T[g.perm[2]] : 1};
        P->smem = std::max(P->smem, (size_t)op_smem_doubles(d, p, M, Tl) * 8);
        g.tile0 = (int)P->tiles.size();
        g.tqp_off = tqp;
        int nt[3] = {1, 1, 1};
        for (int k = 0; k < d; ++k) nt[k] = g.E[k] / g.T[k];
        long long tile_qp = 1;
        for (int k = 0; k < d; ++k) tile_qp *= (long long)Q * g.T[k];
        for (int z = 0; z < nt[2]; ++z)
            for (int y = 0; y < nt[1]; ++y)
                for (int x = 0; x < nt[0]; ++x) {
                    TileDesc td{};
                    td.grid = (int)gi;
                    td.e0[0] = x * g.T[0];
                    td.e0[1] = y * g.T[1];
                    td.e0[2] = z * g.T[2];
                    td.g_off = tqp;
                    tqp += tile_qp;
                    P->tiles.push_back(td);
                }
        g.ntiles = (int)P->tiles.size() - g.tile0;
    }
    P->sched.resize(P->tiles.size());
    for (size_t i = 0; i < P->tiles.size(); ++i) P->sched[i] = (int)i;
    std::vector<double> tcost(P->tiles.size());
    for (size_t i = 0; i < P->tiles.size(); ++i) {
        const GridDesc& g = P->grids[P->tiles[i].grid];
        double qp = 1;
        for (int k = 0; k < d; ++k) qp *= Q * g.T[k];
        tcost[i] = qp;
    }
    std::stable_sort(P->sched.begin(), P->sched.end(), [&](int a, int b) { return tcost[a] > tcost[b]; });
}

static double since(std::chrono::steady_clock::time_point t) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t).count();
}

static int build(sgiga_plan_s* P) {
    const auto tb0 = std::chrono::steady_clock::now();
    const sgiga_config& c = P->cfg;
    const int d = P->d, p = P->p, M = P->m, Q = P->Q;
    // index set
    const int mn = c.min_level, w = c.w;
    const int hi = w + d - 1 - (d - 1) * mn;
    std::vector<std::array<int, 3>> idx;
    int lv[3] = {mn, mn, mn};
    for (lv[2] = (d == 3 ? mn : 0); lv[2] <= (d == 3 ? hi : 0); ++lv[2])
        for (lv[1] = mn; lv[1] <= hi; ++lv[1])
            for (lv[0] = mn; lv[0] <= hi; ++lv[0]) {
                int s = lv[0] + lv[1] + (d == 3 ? lv[2] : 0);
                if (s < w || s > w + d - 1) continue;
                idx.push_back({lv[0], lv[1], d == 3 ? lv[2] : 0});
            }
    std::sort(idx.begin(), idx.end(), [&](const std::array<int, 3>& a, const std::array<int, 3>& b) {
        int sa = a[0] + a[1] + a[2], sb = b[0] + b[1] + b[2];
        if (sa != sb) return sa > sb;
        for (int k = 0; k < d; ++k) if (a[k] != b[k]) return a[k] < b[k];
        return false;
    });
    std::map<std::array<int, 3>, double> given_coef;
    if (c.ncomponents > 0 && c.coefficients) {   // an arbitrary index set with given coefficients
        if (!c.components) return fail(SGIGA_ERR_ARG, "components is NULL");
        idx.clear();
        for (int i = 0; i < c.ncomponents; ++i) {
            std::array<int, 3> lv3 = {0, 0, 0};
            for (int k = 0; k < d; ++k) {
                lv3[k] = c.components[i * d + k];
                if (lv3[k] < mn || lv3[k] > 20) return fail(SGIGA_ERR_ARG, "component level outside [min_level, 20]");
            }
            if (given_coef.count(lv3)) return fail(SGIGA_ERR_ARG, "a component is listed twice");
            given_coef[lv3] = c.coefficients[i];
            idx.push_back(lv3);
        }
    } else if (c.ncomponents > 0) {   // keep only the listed components (in index-set order)
        if (!c.components) return fail(SGIGA_ERR_ARG, "components is NULL");
        std::vector<std::array<int, 3>> keep;
        for (int i = 0; i < c.ncomponents; ++i) {
            std::array<int, 3> lv3 = {0, 0, 0};
            for (int k = 0; k < d; ++k) lv3[k] = c.components[i * d + k];
            if (std::find(idx.begin(), idx.end(), lv3) == idx.end())
                return fail(SGIGA_ERR_ARG, "a listed component is not in the index set of w");
        }
        for (auto& iv : idx)
            for (int i = 0; i < c.ncomponents; ++i) {
                bool same = true;
                for (int k = 0; k < d; ++k) same = same && iv[k] == c.components[i * d + k];
                if (same) { keep.push_back(iv); break; }
            }
        idx.swap(keep);
    }
    if (idx.empty()) return fail(SGIGA_ERR_ARG, "empty index set");
    for (auto& iv : idx)
        for (int k = 0; k < d; ++k) if (iv[k] > 20) return fail(SGIGA_ERR_ARG, "level above 20");
    // tables
    for (auto& iv : idx)
        for (int k = 0; k < d; ++k) {
            auto key = std::make_pair(k, iv[k]);
            if (P->tab_of.count(key)) continue;
            Table1D t{};
            t.dir = k;
            t.level = iv[k];
            t.E = 1 << iv[k];
            t.nf = t.E * M + P->r + 1;
            t.off = P->tab_entries;
            P->tab_entries += (long long)t.E * Q;
            t.eoff = (int)P->bp.size();
            for (int j = 0; j <= t.E; ++j) P->bp.push_back(grading(c.grading, c.gamma, (double)j / t.E));
            P->bp[t.eoff] = 0.0;
            P->bp[t.eoff + t.E] = 1.0;
            t.koff = (int)P->knots.size();
            for (int j = 0; j <= p; ++j) P->knots.push_back(0.0);
            for (int e = 1; e < t.E; ++e)
                for (int j = 0; j < M; ++j) P->knots.push_back(P->bp[t.eoff + e]);
            for (int j = 0; j <= p; ++j) P->knots.push_back(1.0);
            t.nk = (int)P->knots.size() - t.koff;
            P->maxE = std::max(P->maxE, t.E);
            P->tab_of[key] = (int)P->tabs.size();
            P->tabs.push_back(t);
        }
    // components and their pieces (one per geometry patch)
    const bool mp = c.domain == SGIGA_DOMAIN_LSHAPE;
    const int npatch = mp ? 3 : 1;
    P->multipatch = mp;
    for (size_t gi = 0; gi < idx.size(); ++gi) {
        CompDesc cd{};
        cd.piece0 = (int)P->grids.size();
        cd.npieces = npatch;
        cd.dof_off = P->ndof;
        cd.chunk0 = (int)P->chunks.size();
        int s = 0;
        for (int k = 0; k < d; ++k) s += idx[gi][k];
        const int t = w + d - 1 - s;
        cd.coeff = given_coef.empty() ? (double)((t % 2) ? -1 : 1) * (double)binom(d - 1, t) : given_coef[idx[gi]];
        for (int q = 0; q < npatch; ++q) {
            GridDesc g{};
            g.comp = (int)gi;
            g.patch = q;
            g.coeff = cd.coeff;
            g.gf_off = -1;
            for (int k = 0; k < 3; ++k) { g.klo[k] = 1; g.slo[k] = 1; g.alias[k] = -1; }
            if (mp) {
                // L-shape pieces (GridDesc): patch 0 stores the x = 0 interface (its
                // xi_1 = 0 side), patch 1 the y = 0 interface (its xi_2 = 0 side);
                // patch 1's (0,0) function sits at the corner, a Dirichlet point
                const int base = cd.piece0;
                if (q == 0) { g.klo[0] = 0; g.slo[0] = 0; }
                if (q == 1) { g.klo[0] = 0; g.slo[0] = 1; g.alias[0] = base + 0; g.klo[1] = 0; g.slo[1] = 0; g.xcorner = 1; }
                if (q == 2) { g.klo[1] = 0; g.slo[1] = 1; g.alias[1] = base + 1; }
            }
            for (int k = 0; k < 3; ++k) {
                if (k < d) {
                    g.lev[k] = idx[gi][k];
                    g.E[k] = 1 << g.lev[k];
                    g.nf[k] = g.E[k] * M + P->r + 1;
                    g.n[k] = g.nf[k] - 1 - g.slo[k];
                    g.fn[k] = g.nf[k] - 1 - g.klo[k];
                    g.tab[k] = P->tab_of[std::make_pair(k, g.lev[k])];
                } else {
                    g.lev[k] = 0; g.E[k] = 1; g.nf[k] = 3; g.n[k] = 1; g.fn[k] = 1; g.tab[k] = 0;
                }
            }
            g.ndof = 1;
            g.fd_n = 1;
            g.nqp = 1;
            for (int k = 0; k < d; ++k) { g.ndof *= g.n[k]; g.fd_n *= g.fn[k]; g.nqp *= (long long)Q * g.E[k]; }
            g.dof_off = P->ndof;
            g.fd_off = P->nfd;
            g.qp_off = P->nqp;
            P->ndof += g.ndof;
            P->nfd += g.fd_n;
            P->nqp += g.nqp;
            if (mp) { g.gf_off = P->ngf; P->ngf += (long long)g.nf[0] * g.nf[1]; }
            // chunks of the packed vector (component scalars) and of the local layout
            const int piece = (int)P->grids.size();
            g.chunk0 = (int)P->chunks.size();
            for (long long o = 0; o < g.ndof; o += 4096) {
                Chunk ch{};
                ch.grid = (int)gi;
                ch.piece = piece;
                ch.start = g.dof_off + o;
                ch.len = (int)std::min<long long>(4096, g.ndof - o);
                P->chunks.push_back(ch);
            }
            g.nchunk = (int)P->chunks.size() - g.chunk0;
            for (long long o = 0; o < g.fd_n; o += 4096) {
                Chunk ch{};
                ch.grid = (int)gi;
                ch.piece = piece;
                ch.start = g.fd_off + o;
                ch.len = (int)std::min<long long>(4096, g.fd_n - o);
                P->fdchunks.push_back(ch);
            }
            P->grids.push_back(g);
        }
        cd.ndof = P->ndof - cd.dof_off;
        cd.nchunk = (int)P->chunks.size() - cd.chunk0;
        P->comps.push_back(cd);
    }
    // Dirichlet sides of the pieces (multi-patch): (direction, end) per patch
    if (mp) {
        static const int dir_sides[3][3][2] = {{{1, 0}, {0, 1}, {1, 1}}, {{0, 1}, {1, 1}, {-1, -1}},
                                               {{0, 0}, {0, 1}, {1, 1}}};
        for (size_t pi = 0; pi < P->grids.size(); ++pi) {
            const GridDesc& g = P->grids[pi];
            for (int k = 0; k < 3; ++k) {
                const int dk = dir_sides[g.patch][k][0], end = dir_sides[g.patch][k][1];
                if (dk < 0) continue;
                SideDesc sd{};
                sd.piece = (int)pi;
                sd.k = dk;
                sd.end = end;
                sd.goff = P->ngdata;
                sd.soff = P->nscratch;
                const int kp = 1 - dk;
                P->ngdata += 2 + (long long)g.E[kp] * Q;
                P->nscratch += (long long)g.nf[kp] * (p + 1) + g.nf[kp];
                P->sides.push_back(sd);
            }
            if (g.xcorner) {
                SideDesc sd{};
                sd.piece = (int)pi;
                sd.k = -1;
                sd.goff = P->ngdata;
                P->ngdata += 1;
                P->sides.push_back(sd);
            }
        }
    }
    make_tiles(P, 110 * 1024, 16384);
    P->t_host = since(tb0);
    // device data
    if (c.domain == SGIGA_DOMAIN_PATCH) {
        if (!c.patch || make_user_patch(c.patch, d, P->patch) != 0)
            return fail(SGIGA_ERR_ARG, "invalid patch (degree <= 3, <= 12 knots, <= 8 control points per direction, "
                                       "<= 128 in total, nknots = ncp + deg + 1)");
    } else if (mp) {
        for (int q = 0; q < 3; ++q) {   // x = s * xi: bilinear unit squares with the origin at the corner
            static const double sg[3][2] = {{1, 1}, {-1, 1}, {-1, -1}};
            Patch pt;
            make_patch(SGIGA_DOMAIN_UNIT, 2, pt);
            for (int cc = 0; cc < 4; ++cc)
                for (int k = 0; k < 2; ++k) pt.cp[cc][k] *= sg[q][k];
            pt.orient = sg[q][0] * sg[q][1] < 0 ? -1 : 1;
            P->patches.push_back(pt);
        }
        P->patch = P->patches[0];
    } else {
        make_patch(c.domain, d, P->patch);
    }
    if (P->patches.empty()) P->patches.push_back(P->patch);
    std::vector<double> gauss(2 * Q);
    gauss_legendre(Q, gauss.data(), gauss.data() + Q);
    DevPlan& D = P->dp;
    std::memset(&D, 0, sizeof(D));
    D.d = d; D.p = p; D.m = M; D.Q = Q;
    D.ngrids = (int)P->grids.size();
    D.ntiles = (int)P->tiles.size();
    D.ntabs = (int)P->tabs.size();
    D.nchunks = (int)P->chunks.size();
    D.ndof = P->ndof;
    D.nqp = P->nqp;
    D.smem_op = P->smem;
    int rc;
    GridDesc* dg; TileDesc* dt; int* ds; Table1D* dtab; Chunk* dch; Patch* dpatch;
    double *dkn, *dbp, *dgauss;
    CompDesc* dcomps; Chunk* dfdch; SideDesc* dsides;
    if ((rc = upload(P, &dtab, P->tabs)) || (rc = upload(P, &dt, P->tiles)) || (rc = upload(P, &ds, P->sched)) ||
        (rc = upload(P, &dch, P->chunks)) || (rc = upload(P, &dpatch, P->patches)) ||
        (rc = upload(P, &dkn, P->knots)) || (rc = upload(P, &dbp, P->bp)) || (rc = upload(P, &dgauss, gauss)) ||
        (rc = upload(P, &dcomps, P->comps)) || (rc = upload(P, &dfdch, P->fdchunks)) ||
        (rc = upload(P, &dsides, P->sides)))
        return rc;
    D.comps = dcomps; D.ncomps = (int)P->comps.size();
    D.fdchunks = dfdch; D.nfdchunks = (int)P->fdchunks.size(); D.nfd = P->nfd;
    D.sides = dsides; D.nsides = (int)P->sides.size();
    D.multipatch = mp ? 1 : 0;
    if (mp) {
        if ((rc = dalloc(P, &D.gfull, P->ngf)) || (rc = dalloc(P, &D.gdata, P->ngdata)) ||
            (rc = dalloc(P, &D.gscratch, P->nscratch)) || (rc = dalloc(P, &P->d_xb, 2 * P->ngdata)))
            return rc;
        CUDA_TRY(cudaMemset(D.gfull, 0, (size_t)P->ngf * 8));
        CUDA_TRY(cudaMemset(D.gdata, 0, (size_t)P->ngdata * 8));
    }

    D.tiles = dt; D.sched = ds; D.tabs = dtab; D.chunks = dch; D.patch = dpatch;
    P->d_tiles = dt;
    P->d_sched = ds;
    D.knots = dkn; D.bp = dbp; D.gauss = dgauss;
    int* dfirst; int* dflags;
    if ((rc = dalloc(P, &D.xi, P->tab_entries)) || (rc = dalloc(P, &D.w, P->tab_entries)) ||
        (rc = dalloc(P, &D.R, P->tab_entries * (p + 1))) || (rc = dalloc(P, &D.dR, P->tab_entries * (p + 1))) ||
        (rc = dalloc(P, &dfirst, P->bp.size())) || (rc = dalloc(P, &dflags, 4)))
        return rc;
    D.first = dfirst; D.flags = dflags;
    CUDA_TRY(cudaMemset(dflags, 0, 4 * sizeof(int)));
    const int ncomp = d * (d + 1) / 2;
    P->ncomp = ncomp;
    if ((rc = dalloc(P, &D.G, (size_t)ncomp * P->nqp)) || (rc = dalloc(P, &D.mw, P->nqp)) ||
        (rc = dalloc(P, &D.rho, P->nqp)))
        return rc;
    cudaStream_t s = P->stream;
    const auto tbasis = std::chrono::steady_clock::now();
    CUDA_TRY(launch_basis_tables(D, P->maxE, s));
    // eigen tables: one per (level, rational direction or not)
    std::vector<double> hw(P->tab_entries), hR(P->tab_entries * (p + 1)), hdR(P->tab_entries * (p + 1));
    std::vector<int> hfirst(P->bp.size());
    CUDA_TRY(cudaMemcpyAsync(hw.data(), D.w, hw.size() * 8, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(hR.data(), D.R, hR.size() * 8, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(hdR.data(), D.dR, hdR.size() * 8, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(hfirst.data(), D.first, hfirst.size() * 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    P->t_basis = since(tbasis);
    // one eigen table per (level, rational direction or not, first kept
    // function): klo = 0 keeps the interface end (natural condition there)
    std::map<std::array<int, 3>, int> eig_key;
    std::map<std::pair<int, int>, int> eig_of;   // (table, klo) -> eigen table
    std::vector<EigJob> jobs;
    std::vector<double> hKb, hMb, hlam;
    long long ulen = 0, llen = 0;
    P->eig_of_tab.assign(P->tabs.size(), -1);
    auto eig_for = [&](int ti, int klo) -> int {
        auto f = eig_of.find(std::make_pair(ti, klo));
        if (f != eig_of.end()) return f->second;
        const Table1D& t = P->tabs[ti];
        std::array<int, 3> key = {t.level, P->patch.rational[t.dir] ? t.dir : -1, klo};
        auto it = eig_key.find(key);
        if (it != eig_key.end()) { eig_of[std::make_pair(ti, klo)] = it->second; return it->second; }
        const int n = t.nf - 1 - klo;
        Eig1D e{};
        e.n = n;
        e.uoff = ulen;
        e.loff = llen;
        ulen += (long long)n * n;
        llen += n;
        if (n > 0) {
            EigJob J{};
            J.n = n;
            J.boff = (long long)hKb.size();
            J.uoff = e.uoff;
            J.loff = e.loff;
            assemble_band(t.E, Q, p, n, klo, hw.data() + t.off, hR.data() + t.off * (p + 1),
                          hdR.data() + t.off * (p + 1), hfirst.data() + t.eoff, hKb, hMb);
            jobs.push_back(J);
        }
        const int id = (int)P->eigs.size();
        eig_key[key] = id;
        eig_of[std::make_pair(ti, klo)] = id;
        P->eigs.push_back(e);
        return id;
    };
    for (size_t ti = 0; ti < P->tabs.size(); ++ti) P->eig_of_tab[ti] = eig_for((int)ti, 1);
    for (auto& g : P->grids)
        for (int k = 0; k < 3; ++k) g.eig[k] = k < d ? eig_for(g.tab[k], g.klo[k]) : 0;
    P->ulen = ulen;
    P->llen = llen;
    // the eigenpairs on the device, FP64 (eig.cu)
    Eig1D* deig; double *dU, *dUt, *dlam;
    if ((rc = upload(P, &deig, P->eigs)) || (rc = dalloc(P, &dU, (size_t)ulen)) ||
        (rc = dalloc(P, &dUt, (size_t)ulen)) || (rc = dalloc(P, &dlam, (size_t)llen)))
        return rc;
    {
        const auto te = std::chrono::steady_clock::now();
        std::string msg;
        std::vector<double> jl;
        if (gpu_generalized_eigen(p, jobs, hKb, hMb, dU, dUt, dlam, jl, s, msg) != 0)
            return fail(SGIGA_ERR_CUDA, "1D generalised eigenproblems: " + msg);
        hlam.assign((size_t)llen, 0.0);
        for (const EigJob& J : jobs)
            std::copy(jl.begin() + J.t0, jl.begin() + J.t0 + J.n, hlam.begin() + J.loff);
        P->t_eigen = std::chrono::duration<double>(std::chrono::steady_clock::now() - te).count();
    }
    const auto tfd = std::chrono::steady_clock::now();
    // preconditioner work items (grouped by eigen table)
    // default layout: grouped for FP32 (latency-bound) plans, per piece for FP64
    make_fd_items(P, 32, c.precision == SGIGA_PREC_MIXED_FP32);
    if ((rc = upload_fd(P))) return rc;
    // reciprocal eigenvalue sums of every entry of the preconditioner's local layout
    std::vector<double> hdinv((size_t)P->nfd);
    for (const GridDesc& g : P->grids)
        for (long long idx = 0; idx < g.fd_n; ++idx) {
            long long rem = idx;
            double sum = 0.0;
            for (int k = 0; k < d; ++k) {
                int ik = (int)(rem % g.fn[k]);
                rem /= g.fn[k];
                sum += hlam[P->eigs[g.eig[k]].loff + ik];
            }
            hdinv[g.fd_off + idx] = 1.0 / sum;
        }
    double* ddinv;
    if ((rc = upload(P, &ddinv, hdinv))) return rc;
    D.dinv = ddinv;
    if ((rc = upload(P, &dg, P->grids))) return rc;
    D.eigs = deig; D.U = dU; D.Ut = dUt; D.lam = dlam; D.grids = dg;
    P->t_fd = since(tfd);
    const auto tgeo = std::chrono::steady_clock::now();
    if (mp) CUDA_TRY(launch_boundary_points(D, P->d_xb, s));
    // geometry coefficients
    CUDA_TRY(launch_geometry(D, s));
    int hflags[4];
    CUDA_TRY(cudaMemcpyAsync(hflags, dflags, sizeof(hflags), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (hflags[0] & 1) return fail(SGIGA_ERR_GEOMETRY, "det J <= 0 at a quadrature point");
    if ((rc = update_diag(P))) return rc;
    P->t_geometry = since(tgeo);
    const auto tvec = std::chrono::steady_clock::now();
    // operator kernel shared memory
    if ((rc = grant_op_smem(P))) return rc;
    // solver vectors and scalars
    const size_t nd = (size_t)P->ndof, ng = P->comps.size(), nt = std::max<size_t>(nd, (size_t)P->nfd);
    if ((rc = dalloc(P, &P->d_b, nd)) || (rc = dalloc(P, &P->d_x, nd)) || (rc = dalloc(P, &P->d_r, nd)) ||
        (rc = dalloc(P, &P->d_z, nd)) || (rc = dalloc(P, &P->d_p, nd)) || (rc = dalloc(P, &P->d_q, nd)) ||
        (rc = dalloc(P, &P->d_t1, nt)) || (rc = dalloc(P, &P->d_t2, nt)) ||
        (mp && (rc = dalloc(P, &P->d_l0, (size_t)P->nfd))) ||
        (rc = dalloc(P, &P->d_partial, P->chunks.size())) || (rc = dalloc(P, &P->d_scal, 8 * ng)) ||
        (rc = dalloc(P, &P->d_active, ng)) || (rc = dalloc(P, &P->d_iters, ng)) || (rc = dalloc(P, &P->d_nactive, 1)))
        return rc;
    std::vector<double> coef(ng);
    for (size_t i = 0; i < ng; ++i) coef[i] = P->comps[i].coeff;
    if ((rc = upload(P, &P->d_coef, coef))) return rc;
    CUDA_TRY(cudaMemsetAsync(P->d_b, 0, nd * 8, s));
    CUDA_TRY(cudaMemsetAsync(P->d_x, 0, nd * 8, s));
    CUDA_TRY(cudaMallocHost(&P->h_nactive, 2 * sizeof(int)));
    if ((rc = dalloc(P, &P->d_counter, 1))) return rc;
    if (!P->stream) CUDA_TRY(cudaStreamCreate(&P->own_stream));
    CUDA_TRY(fd_prepare());
    {   // branches for the kernels of a preconditioner pass (all or none)
        FDStreams& f = P->fds;
        const bool fork_ok = cudaEventCreateWithFlags(&f.fork, cudaEventDisableTiming) == cudaSuccess;
        bool ok = fork_ok;
        int ns = 0, ne = 0;
        for (int i = 0; ok && i < 3; ++i) {
            ok = cudaStreamCreateWithFlags(&f.aux[i], cudaStreamNonBlocking) == cudaSuccess;
            ns += ok;
            ok = ok && cudaEventCreateWithFlags(&f.join[i], cudaEventDisableTiming) == cudaSuccess;
            ne += ok;
        }
        if (!ok) {
            for (int i = 0; i < ns; ++i) cudaStreamDestroy(f.aux[i]);
            for (int i = 0; i < ne; ++i) cudaEventDestroy(f.join[i]);
            if (fork_ok) cudaEventDestroy(f.fork);
            cudaGetLastError();
            return fail(SGIGA_ERR_CUDA, "preconditioner streams");
        }
        P->fds_ok = true;
    }
    if (c.precision == SGIGA_PREC_MIXED_FP32) {
        // FP32 copies of the operator and preconditioner data, FP32 work vectors
        float *Gf, *Rf, *dRf, *Uf, *Utf, *dinvf;
        const long long ntab = P->tab_entries * (p + 1);
        if ((rc = dalloc(P, &Gf, (size_t)ncomp * P->nqp)) || (rc = dalloc(P, &Rf, ntab)) ||
            (rc = dalloc(P, &dRf, ntab)) || (rc = dalloc(P, &Uf, (size_t)ulen)) || (rc = dalloc(P, &Utf, (size_t)ulen)) ||
            (rc = dalloc(P, &dinvf, (size_t)P->nfd)) || (rc = dalloc(P, &P->f_b, nd)) || (rc = dalloc(P, &P->f_x, nd)) ||
            (rc = dalloc(P, &P->f_r, nd)) || (rc = dalloc(P, &P->f_z, nd)) || (rc = dalloc(P, &P->f_p, nd)) ||
            (rc = dalloc(P, &P->f_q, nd)) || (rc = dalloc(P, &P->f_t1, nt)) || (rc = dalloc(P, &P->f_t2, nt)) ||
            (mp && (rc = dalloc(P, &P->f_l0, (size_t)P->nfd))) ||
            (rc = dalloc(P, &P->d_active_o, ng)) || (rc = dalloc(P, &P->d_iters_o, ng)) ||
            (rc = dalloc(P, &P->d_scal64o, 8 * ng)) || (rc = dalloc(P, &P->d_d, nd)))
            return rc;
        CUDA_TRY(launch_narrow(Gf, D.G, (long long)ncomp * P->nqp, s));
        CUDA_TRY(launch_narrow(Rf, D.R, ntab, s));
        CUDA_TRY(launch_narrow(dRf, D.dR, ntab, s));
        CUDA_TRY(launch_narrow(Uf, D.U, ulen, s));
        CUDA_TRY(launch_narrow(Utf, D.Ut, ulen, s));
        CUDA_TRY(launch_narrow(dinvf, D.dinv, P->nfd, s));
        D.Gf = Gf; D.Rf = Rf; D.dRf = dRf; D.Uf = Uf; D.Utf = Utf; D.dinvf = dinvf;
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    P->t_vectors = since(tvec);
    P->t_total = since(tb0);
    return SGIGA_OK;
}

// Re-plan the tiles (autotuner): new tile arrays, grids, shared-memory
// attribute, and the tile-major geometry planes in the new layout: gathered
// from a natural-layout copy (Gn, mwn) when the caller holds one, else
// recomputed from the patch map.
static int retile(sgiga_plan_s* P, size_t budget, long long qpcap, double* Gn = nullptr, double* mwn = nullptr) {
    cudaStream_t s = P->stream;
    CUDA_TRY(cudaStreamSynchronize(s));
    make_tiles(P, budget, qpcap);
    for (void* old : {(void*)P->d_tiles, (void*)P->d_sched}) {
        auto it = std::find(P->allocs.begin(), P->allocs.end(), old);
        if (it != P->allocs.end()) P->allocs.erase(it);
        cudaFree(old);
    }
    TileDesc* dt;
    int* ds;
    int rc;
    if ((rc = upload(P, &dt, P->tiles)) || (rc = upload(P, &ds, P->sched))) return rc;
    P->d_tiles = dt;
    P->d_sched = ds;
    DevPlan& D = P->dp;
    D.tiles = dt;
    D.sched = ds;
    D.ntiles = (int)P->tiles.size();
    D.smem_op = P->smem;
    CUDA_TRY(cudaMemcpy((void*)D.grids, P->grids.data(), P->grids.size() * sizeof(GridDesc), cudaMemcpyHostToDevice));
    if ((rc = grant_op_smem(P))) return rc;
    if (Gn) CUDA_TRY(launch_geometry_import(D, Gn, mwn, s));
    else CUDA_TRY(launch_geometry(D, s));
    if (P->cfg.precision == SGIGA_PREC_MIXED_FP32)
        CUDA_TRY(launch_narrow(D.Gf, D.G, (long long)P->ncomp * P->nqp, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    net_invalidate_features(P);
    return update_diag(P);
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int sgiga_build_checked(void) {
#ifdef SGIGA_CHECKED
    return 1;
#else
    return 0;
#endif
}

int sgiga_check_site(sgiga_plan_t P, int* site) {
    if (!P || !site) return fail(SGIGA_ERR_ARG, "null argument");
    int h[2] = {0, 0};
    CUDA_TRY(cudaMemcpyAsync(h, P->dp.flags + 2, sizeof(h), cudaMemcpyDeviceToHost, P->stream));
    CUDA_TRY(cudaStreamSynchronize(P->stream));
    *site = h[0] ? h[1] : 0;
    return SGIGA_OK;
}

const char* sgiga_last_error(void) { return g_last_error.c_str(); }

long long sgiga_launch_count(void) { return g_launches.load(); }

int sgiga_plan(const sgiga_config* cfg, void* stream, sgiga_plan_t* out) {
    NvtxRange nvtx_("sgiga_plan");
    if (!cfg || !out) return fail(SGIGA_ERR_ARG, "null argument");
    *out = nullptr;
    sgiga_config c = *cfg;
    if (c.d != 2 && c.d != 3) return fail(SGIGA_ERR_ARG, "d must be 2 or 3");
    if (c.p < 1 || c.p > SGIGA_MAXP) return fail(SGIGA_ERR_ARG, "p must be in 1..4");
    if (c.continuity < 0) c.continuity = c.p - 1;
    if (c.continuity > c.p - 1) return fail(SGIGA_ERR_ARG, "continuity must be <= p-1");
    if (c.min_level < 0) return fail(SGIGA_ERR_ARG, "min_level must be >= 0");
    if (c.w < c.d * c.min_level - c.d + 1) return fail(SGIGA_ERR_ARG, "w too small for min_level");
    if (c.domain < SGIGA_DOMAIN_UNIT || c.domain > SGIGA_DOMAIN_LSHAPE) return fail(SGIGA_ERR_ARG, "unknown domain");
    if (c.domain == SGIGA_DOMAIN_LSHAPE && c.d != 2) return fail(SGIGA_ERR_ARG, "the L-shaped domain is 2D");
    if (c.domain == SGIGA_DOMAIN_LSHAPE && c.precond == SGIGA_PRECOND_LEARNED)
        return fail(SGIGA_ERR_ARG, "the learned preconditioner needs a single-patch domain");
    if (c.grading < 0 || c.grading > 2 || (c.grading != 0 && !(c.gamma > 0))) return fail(SGIGA_ERR_ARG, "bad grading");
    if (c.precision != SGIGA_PREC_FP64 && c.precision != SGIGA_PREC_MIXED_FP32)
        return fail(SGIGA_ERR_ARG, "unsupported precision");
    if (c.precond != SGIGA_PRECOND_FD && c.precond != SGIGA_PRECOND_NONE && c.precond != SGIGA_PRECOND_LEARNED)
        return fail(SGIGA_ERR_ARG, "bad precond");
    if (c.precond == SGIGA_PRECOND_LEARNED && c.precision != SGIGA_PREC_MIXED_FP32)
        return fail(SGIGA_ERR_ARG, "the learned preconditioner runs inside the MIXED_FP32 inner solve");
    if (c.domain == SGIGA_DOMAIN_ANNULUS && c.p < 2) return fail(SGIGA_ERR_ARG, "annulus needs p >= 2 (exact circle)");
    sgiga_plan_s* P = new sgiga_plan_s();
    P->cfg = c;
    P->d = c.d; P->p = c.p; P->r = c.continuity; P->m = c.p - c.continuity; P->Q = c.p + 1;
    P->stream = (cudaStream_t)stream;
    int rc = build(P);
    if (rc != SGIGA_OK) {
        std::string msg = g_last_error;
        free_plan(P);
        g_last_error = msg;
        return rc;
    }
    *out = P;
    return SGIGA_OK;
}

void sgiga_destroy(sgiga_plan_t plan) {
    if (!plan) return;
    cudaStreamSynchronize(plan->stream);
    if (plan->own_stream) cudaStreamSynchronize(plan->own_stream);
    free_plan(plan);
}

int sgiga_plan_info(sgiga_plan_t P, sgiga_info* out) {
    if (!P || !out) return fail(SGIGA_ERR_ARG, "null argument");
    out->d = P->d; out->p = P->p; out->continuity = P->r;
    out->ngrids = (int)P->comps.size();
    out->ndof = P->ndof;
    out->nqp = P->nqp;
    out->max_tile_smem = (int)P->smem;
    out->ntiles = (int)P->tiles.size();
    out->diag_metric = P->dp.diag;
    out->npatches = (int)P->patches.size();
    out->nbpts = P->ngdata;
    return SGIGA_OK;
}

int sgiga_grid_info(sgiga_plan_t P, int g, sgiga_grid* out) {
    if (!P || !out) return fail(SGIGA_ERR_ARG, "null argument");
    if (g < 0 || g >= (int)P->comps.size()) return fail(SGIGA_ERR_ARG, "grid index out of range");
    const CompDesc& cd = P->comps[g];
    const GridDesc& gd = P->grids[cd.piece0];
    for (int k = 0; k < 3; ++k) {
        out->levels[k] = k < P->d ? gd.lev[k] : 0;
        out->n[k] = k < P->d ? gd.n[k] : 1;
    }
    out->coeff = (int)cd.coeff;
    out->ndof = cd.ndof; out->dof_off = cd.dof_off; out->qp_off = gd.qp_off;
    out->nqp = 0;
    out->ntiles = 0;
    for (int q = 0; q < cd.npieces; ++q) {
        out->nqp += P->grids[cd.piece0 + q].nqp;
        out->ntiles += P->grids[cd.piece0 + q].ntiles;
    }
    for (int k = 0; k < 3; ++k) out->tile[k] = k < P->d ? gd.T[k] : 1;
    out->pencil_dir = gd.perm[0];
    return SGIGA_OK;
}

int sgiga_qp_coords(sgiga_plan_t P, double* xq) {
    if (!P || !xq) return fail(SGIGA_ERR_ARG, "null argument");
    const size_t bytes = (size_t)P->d * P->nqp * 8;
    double* out = xq;
    if (!is_device(xq)) {   // host buffer: through the staging area
        int rc = ensure_stage(P, bytes);
        if (rc) return rc;
        out = (double*)P->stage;
    }
    CUDA_TRY(launch_qp_coords(P->dp, out, P->stream));
    if (out != xq) CUDA_TRY(cudaMemcpyAsync(xq, out, bytes, cudaMemcpyDeviceToHost, P->stream));
    CUDA_TRY(cudaStreamSynchronize(P->stream));
    return SGIGA_OK;
}

int sgiga_set_rhs(sgiga_plan_t P, const double* f) {
    if (!P || !f) return fail(SGIGA_ERR_ARG, "null argument");
    const double* fd = f;
    const bool host = !is_device(f);
    if (host) {
        // page-locked: the density kernel reads f over the host link, once per
        // value, in place of a staging copy; pageable: staged
        fd = (const double*)mapped_host_alias(f);
        if (!fd) {
            int rc = ensure_stage(P, (size_t)P->nqp * 8);
            if (rc) return rc;
            CUDA_TRY(cudaMemcpyAsync(P->stage, f, (size_t)P->nqp * 8, cudaMemcpyHostToDevice, P->stream));
            fd = (const double*)P->stage;
        }
    }
    CUDA_TRY(launch_rhs_density_user(P->dp, fd, P->stream));
    int rc = run_rhs_operator(P);
    if (rc) return rc;
    if (host) CUDA_TRY(cudaStreamSynchronize(P->stream));   // host buffer may be reused on return
    return SGIGA_OK;
}

// Project the boundary data in P->dp.gdata onto every Dirichlet side.
static int project_boundary(sgiga_plan_s* P) {
    CUDA_TRY(cudaMemsetAsync(P->dp.gfull, 0, (size_t)P->ngf * 8, P->stream));
    CUDA_TRY(launch_boundary_project(P->dp, P->stream));
    P->lifting = true;
    return SGIGA_OK;
}

int sgiga_set_rhs_builtin(sgiga_plan_t P, int source) {
    if (!P) return fail(SGIGA_ERR_ARG, "null argument");
    if (source < 0 || source > SGIGA_SRC_HARMONIC_QUADRATIC) return fail(SGIGA_ERR_ARG, "unknown source");
    if ((source == SGIGA_SRC_ANNULUS) && P->d != 2) return fail(SGIGA_ERR_ARG, "source needs d = 2");
    if (source >= SGIGA_SRC_LSHAPE_CORNER) {   // harmonic u with Dirichlet data g = u
        if (!P->multipatch) return fail(SGIGA_ERR_ARG, "sources with Dirichlet data need an LSHAPE plan");
        CUDA_TRY(launch_boundary_builtin(P->dp, source, P->d_xb, P->dp.gdata, P->ngdata, P->stream));
        int rc = project_boundary(P);
        if (rc) return rc;
    }
    CUDA_TRY(launch_rhs_density_builtin(P->dp, source, P->stream));
    int rc = run_rhs_operator(P);
    if (rc) return rc;
    CUDA_TRY(cudaGetLastError());
    return SGIGA_OK;
}

int sgiga_boundary_points(sgiga_plan_t P, double* xb) {
    if (!P || !xb) return fail(SGIGA_ERR_ARG, "null argument");
    if (!P->multipatch) return fail(SGIGA_ERR_ARG, "plan has no boundary data points (LSHAPE plans only)");
    const size_t bytes = (size_t)P->ngdata * 2 * 8;
    CUDA_TRY(cudaMemcpyAsync(xb, P->d_xb, bytes, cudaMemcpyDefault, P->stream));
    CUDA_TRY(cudaStreamSynchronize(P->stream));
    return SGIGA_OK;
}

int sgiga_set_dirichlet(sgiga_plan_t P, const double* g) {
    if (!P) return fail(SGIGA_ERR_ARG, "null argument");
    if (!P->multipatch) return fail(SGIGA_ERR_ARG, "plan has no Dirichlet data (LSHAPE plans only)");
    if (!g) {
        P->lifting = false;
        CUDA_TRY(cudaMemsetAsync(P->dp.gfull, 0, (size_t)P->ngf * 8, P->stream));
        return SGIGA_OK;
    }
    CUDA_TRY(cudaMemcpyAsync(P->dp.gdata, g, (size_t)P->ngdata * 8, cudaMemcpyDefault, P->stream));
    int rc = project_boundary(P);
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(P->stream));
    return SGIGA_OK;
}

int sgiga_eval_grad(sgiga_plan_t P, const double* xi, const int* patch, long long npts, double* ucomp,
                    double* gcomp) {
    if (!P || (!xi && npts > 0) || (!ucomp && npts > 0)) return fail(SGIGA_ERR_ARG, "null argument");
    if (npts < 0) return fail(SGIGA_ERR_ARG, "npts < 0");
    if (npts == 0) return SGIGA_OK;
    const size_t ng = P->comps.size();
    const size_t xb = (size_t)npts * P->d * 8, pb = patch ? (size_t)npts * 4 : 0;
    const size_t ub = (size_t)npts * ng * 8, gb = gcomp ? (size_t)P->d * ub : 0;
    const bool xdev = is_device(xi), pdev = !patch || is_device(patch), udev = is_device(ucomp);
    const bool gdev = !gcomp || is_device(gcomp);
    int rc = ensure_stage(P, (xdev ? 0 : xb) + (pdev ? 0 : (pb + 15) / 16 * 16) + (udev ? 0 : ub) + (gdev ? 0 : gb));
    if (rc) return rc;
    char* st = (char*)P->stage;
    const double* xd = xi;
    const int* pd = patch;
    if (!xdev) {
        CUDA_TRY(cudaMemcpyAsync(st, xi, xb, cudaMemcpyHostToDevice, P->stream));
        xd = (const double*)st;
        st += xb;
    }
    double* ud = udev ? ucomp : (double*)st;
    if (!udev) st += ub;
    double* gd = gdev ? gcomp : (double*)st;
    if (!gdev) st += gb;
    if (!pdev) {
        CUDA_TRY(cudaMemcpyAsync(st, patch, pb, cudaMemcpyHostToDevice, P->stream));
        pd = (const int*)st;
    }
    CUDA_TRY(cudaMemsetAsync(P->dp.flags + 1, 0, sizeof(int), P->stream));
    CUDA_TRY(launch_eval_grad(P->dp, P->d_x, xd, pd, npts, ud, gd, P->lifting ? 1 : 0, P->stream));
    CUDA_TRY(cudaMemcpyAsync(P->h_nactive, P->dp.flags + 1, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
    if (!udev) CUDA_TRY(cudaMemcpyAsync(ucomp, ud, ub, cudaMemcpyDeviceToHost, P->stream));
    if (!gdev) CUDA_TRY(cudaMemcpyAsync(gcomp, gd, gb, cudaMemcpyDeviceToHost, P->stream));
    CUDA_TRY(cudaStreamSynchronize(P->stream));
    const int hflag = *P->h_nactive;
    if (hflag & 2) return fail(SGIGA_ERR_ARG, "patch id out of range");
    if (hflag) return fail(SGIGA_ERR_ARG, "evaluation point outside [0,1]^d");
    return SGIGA_OK;
}

int sgiga_functional(sgiga_plan_t P, const double* q, double* comp, double* combined) {
    if (!P || !q || !combined) return fail(SGIGA_ERR_ARG, "null argument");
    if (P->lifting) return fail(SGIGA_ERR_ARG, "functional: plans with Dirichlet data are not supported");
    cudaStream_t s = P->stream;
    const DevPlan& D = P->dp;
    const double* qd = q;
    if (!is_device(q)) {
        int rc = ensure_stage(P, (size_t)P->nqp * 8);
        if (rc) return rc;
        CUDA_TRY(cudaMemcpyAsync(P->stage, q, (size_t)P->nqp * 8, cudaMemcpyHostToDevice, s));
        qd = (const double*)P->stage;
    }
    const int ng = (int)P->comps.size();
    // b_q into a work vector (the density buffer is an intermediate of the load vector only)
    CUDA_TRY(launch_rhs_density_user(D, qd, s));
    CUDA_TRY(cudaMemsetAsync(P->d_t1, 0, (size_t)P->ndof * 8, s));
    if (P->d == 3) CUDA_TRY(launch_op3(D, nullptr, P->d_t1, nullptr, 1, s));
    else CUDA_TRY(launch_op2(D, nullptr, P->d_t1, nullptr, 1, s));
    double* vals = P->d_scal + 7 * ng;        // scratch slot of the CG scalars
    CUDA_TRY(launch_dot<double>(D, P->d_t1, P->d_x, P->d_partial, vals, s));
    CUDA_TRY(launch_combine(D, vals, 1, P->d_coef, P->d_scal + 6 * ng, s));
    if (comp) CUDA_TRY(cudaMemcpyAsync(comp, vals, (size_t)ng * 8, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(combined, P->d_scal + 6 * ng, 8, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return SGIGA_OK;
}

int sgiga_map_points(sgiga_plan_t P, const double* xi, const int* patch, long long npts, double* x, double* detj) {
    if (!P || (npts > 0 && (!xi || !x))) return fail(SGIGA_ERR_ARG, "null argument");
    if (npts < 0) return fail(SGIGA_ERR_ARG, "npts < 0");
    if (npts == 0) return SGIGA_OK;
    const int d = P->d;
    const size_t xb = (size_t)npts * d * 8, pb = patch ? ((size_t)npts * 4 + 15) / 16 * 16 : 0, db = (size_t)npts * 8;
    const bool xidev = is_device(xi), pdev = !patch || is_device(patch), xdev = is_device(x);
    const bool ddev = !detj || is_device(detj);
    int rc = ensure_stage(P, (xidev ? 0 : xb) + (pdev ? 0 : pb) + (xdev ? 0 : xb) + (ddev ? 0 : db));
    if (rc) return rc;
    char* st = (char*)P->stage;
    cudaStream_t s = P->stream;
    const double* xid = xi;
    if (!xidev) { CUDA_TRY(cudaMemcpyAsync(st, xi, xb, cudaMemcpyHostToDevice, s)); xid = (const double*)st; st += xb; }
    const int* pd = patch;
    if (!pdev) { CUDA_TRY(cudaMemcpyAsync(st, patch, (size_t)npts * 4, cudaMemcpyHostToDevice, s)); pd = (const int*)st; st += pb; }
    double* xd = xdev ? x : (double*)st;
    if (!xdev) st += xb;
    double* dd = ddev ? detj : (double*)st;
    CUDA_TRY(cudaMemsetAsync(P->dp.flags + 1, 0, sizeof(int), s));
    CUDA_TRY(launch_map_points(P->dp, xid, pd, npts, (int)P->patches.size(), xd, dd, s));
    CUDA_TRY(cudaMemcpyAsync(P->h_nactive, P->dp.flags + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (!xdev) CUDA_TRY(cudaMemcpyAsync(x, xd, xb, cudaMemcpyDeviceToHost, s));
    if (!ddev) CUDA_TRY(cudaMemcpyAsync(detj, dd, db, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    const int hflag = *P->h_nactive;
    if (hflag & 2) return fail(SGIGA_ERR_ARG, "patch id out of range");
    if (hflag) return fail(SGIGA_ERR_ARG, "point outside [0,1]^d");
    return SGIGA_OK;
}

int sgiga_source_at_qp(sgiga_plan_t P, int source, double* f) {
    if (!P || !f) return fail(SGIGA_ERR_ARG, "null argument");
    if (source < 0 || source > SGIGA_SRC_HARMONIC_QUADRATIC) return fail(SGIGA_ERR_ARG, "unknown source");
    if ((source == SGIGA_SRC_ANNULUS) && P->d != 2) return fail(SGIGA_ERR_ARG, "source needs d = 2");
    double* fd = f;
    const bool dev = is_device(f);
    if (!dev) {
        int rc = ensure_stage(P, (size_t)P->nqp * 8);
        if (rc) return rc;
        fd = (double*)P->stage;
    }
    CUDA_TRY(launch_source_qp(P->dp, source, fd, P->stream));
    if (!dev) CUDA_TRY(cudaMemcpyAsync(f, fd, (size_t)P->nqp * 8, cudaMemcpyDeviceToHost, P->stream));
    CUDA_TRY(cudaStreamSynchronize(P->stream));
    return SGIGA_OK;
}

// Recompute the geometry coefficients with the plan's current coefficient
// plane; SGIGA_ERR_ARG if some a(x_q) is not positive and finite.
static int refresh_geometry(sgiga_plan_s* P) {
    cudaStream_t s = P->stream;
    CUDA_TRY(cudaMemsetAsync(P->dp.flags, 0, sizeof(int), s));
    CUDA_TRY(launch_geometry(P->dp, s));
    int hf = 0;
    CUDA_TRY(cudaMemcpyAsync(&hf, P->dp.flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (hf & 2) {   // leave the plan with a = 1 rather than with non-finite coefficients
        if (P->acoef) { cudaFree(P->acoef); P->acoef = nullptr; }
        P->dp.acoef = nullptr;
        CUDA_TRY(launch_geometry(P->dp, s));
        if (P->cfg.precision == SGIGA_PREC_MIXED_FP32)
            CUDA_TRY(launch_narrow(P->dp.Gf, P->dp.G, (long long)P->ncomp * P->nqp, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        net_invalidate_features(P);
        update_diag(P);
        return fail(SGIGA_ERR_ARG, "the diffusion coefficient must be positive and finite at every quadrature "
                                   "point (the plan keeps a = 1)");
    }
    if (P->cfg.precision == SGIGA_PREC_MIXED_FP32)
        CUDA_TRY(launch_narrow(P->dp.Gf, P->dp.G, (long long)P->ncomp * P->nqp, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    net_invalidate_features(P);
    return update_diag(P);
}

static int ensure_acoef(sgiga_plan_s* P) {
    if (P->acoef) return SGIGA_OK;
    cudaError_t e = cudaMalloc(&P->acoef, (size_t)P->nqp * 8);
    if (e != cudaSuccess) {
        cudaGetLastError();
        P->acoef = nullptr;
        return fail(SGIGA_ERR_NOMEM, "coefficient plane allocation failed");
    }
    return SGIGA_OK;
}

int sgiga_set_coefficient(sgiga_plan_t P, int nfeat, const double* omega, const double* phase, double amp) {
    NvtxRange nvtx_("sgiga_set_coefficient");
    if (!P) return fail(SGIGA_ERR_ARG, "null argument");
    if (nfeat < 0 || (nfeat > 0 && (!omega || !phase))) return fail(SGIGA_ERR_ARG, "bad coefficient features");
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = P->stream;
    const int d = P->d;
    int rc;
    if (nfeat == 0) {
        if (P->acoef) { cudaFree(P->acoef); P->acoef = nullptr; }
        P->dp.acoef = nullptr;
    } else {
        std::vector<double> f((size_t)nfeat * 4, 0.0);
        for (int i = 0; i < nfeat; ++i) {
            for (int k = 0; k < d; ++k) f[(size_t)i * 4 + k] = omega[(size_t)i * d + k];
            f[(size_t)i * 4 + 3] = phase[i];
        }
        double* feat = nullptr;
        if (cudaMalloc(&feat, f.size() * 8) != cudaSuccess) {
            cudaGetLastError();
            return fail(SGIGA_ERR_NOMEM, "feature table allocation failed");
        }
        if ((rc = ensure_acoef(P))) { cudaFree(feat); return rc; }
        cudaError_t e = cudaMemcpy(feat, f.data(), f.size() * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = launch_coef_features(P->dp, feat, nfeat, amp, P->acoef, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(feat);
        if (e != cudaSuccess) return fail(SGIGA_ERR_CUDA, std::string("coefficient: ") + cudaGetErrorString(e));
        P->dp.acoef = P->acoef;
    }
    rc = refresh_geometry(P);
    P->t_coefficient = since(t0);
    return rc;
}

int sgiga_set_coefficient_qp(sgiga_plan_t P, const double* a_qp) {
    if (!P) return fail(SGIGA_ERR_ARG, "null argument");
    const auto t0 = std::chrono::steady_clock::now();
    int rc;
    if (!a_qp) {
        if (P->acoef) { cudaFree(P->acoef); P->acoef = nullptr; }
        P->dp.acoef = nullptr;
    } else {
        if ((rc = ensure_acoef(P))) return rc;
        CUDA_TRY(cudaMemcpyAsync(P->acoef, a_qp, (size_t)P->nqp * 8, cudaMemcpyDefault, P->stream));
        CUDA_TRY(cudaStreamSynchronize(P->stream));
        P->dp.acoef = P->acoef;
    }
    rc = refresh_geometry(P);
    P->t_coefficient = since(t0);
    return rc;
}

int sgiga_get_rhs(sgiga_plan_t P, double* b) {
    if (!P || !b) return fail(SGIGA_ERR_ARG, "null argument");
    CUDA_TRY(cudaMemcpyAsync(b, P->d_b, (size_t)P->ndof * 8, cudaMemcpyDefault, P->stream));
    CUDA_TRY(cudaStreamSynchronize(P->stream));
    return SGIGA_OK;
}

int sgiga_apply(sgiga_plan_t P, const double* x, double* y) {
    if (!P || !x || !y) return fail(SGIGA_ERR_ARG, "null argument");
    if (!is_device(x) || !is_device(y)) return fail(SGIGA_ERR_ARG, "x and y must be device buffers");
    int rc = apply_op(P, x, y, nullptr);
    if (rc) return rc;
    CUDA_TRY(cudaGetLastError());
    return SGIGA_OK;
}

int sgiga_apply_f32(sgiga_plan_t P, const float* x, float* y) {
    if (!P || !x || !y) return fail(SGIGA_ERR_ARG, "null argument");
    if (!is_device(x) || !is_device(y)) return fail(SGIGA_ERR_ARG, "x and y must be device buffers");
    if (P->cfg.precision != SGIGA_PREC_MIXED_FP32) return fail(SGIGA_ERR_ARG, "plan has no FP32 data (precision)");
    int rc = apply_op(P, x, y, nullptr);
    if (rc) return rc;
    CUDA_TRY(cudaGetLastError());
    return SGIGA_OK;
}

int sgiga_precond(sgiga_plan_t P, const double* r, double* z) {
    if (!P || !r || !z) return fail(SGIGA_ERR_ARG, "null argument");
    if (!is_device(r) || !is_device(z)) return fail(SGIGA_ERR_ARG, "r and z must be device buffers");
    return precond_fd<double>(P, r, z, nullptr, P->d_t1, P->d_t2);
}

int sgiga_precond_f32(sgiga_plan_t P, const float* r, float* z) {
    if (!P || !r || !z) return fail(SGIGA_ERR_ARG, "null argument");
    if (!is_device(r) || !is_device(z)) return fail(SGIGA_ERR_ARG, "r and z must be device buffers");
    if (P->cfg.precision != SGIGA_PREC_MIXED_FP32) return fail(SGIGA_ERR_ARG, "plan has no FP32 data (precision)");
    return precond_fd<float>(P, r, z, nullptr, P->f_t1, P->f_t2);
}

// MIXED_FP32 plans with the FD preconditioner: the mixed solve against plain
// FP64 PCG, both to a relative residual of 1e-8 on a probe load vector (the
// plan's own if it is set, else that of f = 1), each timed after one run that
// captures its graphs; sgiga_solve then runs the faster. FP64 PCG gets at most
// the iterations that fit in the mixed solve's time. FP64 PCG with the FP32
// preconditioner is kept only if it is also not slower than with the FP64 one
// to 1e-12: the FP32 rounding of z limits how much each flexible-CG step can
// gain, so a tie at 1e-8 (the unit cube, where FD is exact) turns into extra
// iterations at FP64 tolerances. The plan's load vector and solution are
// restored.
static int choose_precision(sgiga_plan_s* P, double* ms64, double* msmx, double* ms6432) {
    *ms64 = *msmx = *ms6432 = 0.0;
    P->solve_fp64 = false;
    P->fp64_fd32 = false;
    const size_t n = (size_t)P->ndof;
    cudaStream_t s = P->stream;
    double* save = nullptr;
    if (cudaMalloc(&save, 2 * n * 8) != cudaSuccess) { cudaGetLastError(); return SGIGA_OK; }   // keep MIXED
    int rc = SGIGA_OK;
    auto body = [&]() -> int {
        CUDA_TRY(cudaMemcpyAsync(save, P->d_b, n * 8, cudaMemcpyDeviceToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(save + n, P->d_x, n * 8, cudaMemcpyDeviceToDevice, s));
        const int ng = (int)P->comps.size();
        CUDA_TRY(launch_dot<double>(P->dp, P->d_b, P->d_b, P->d_partial, P->d_scal, s));
        std::vector<double> hb(ng);
        CUDA_TRY(cudaMemcpyAsync(hb.data(), P->d_scal, ng * 8, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        bool zero = true;
        for (double v : hb) zero = zero && v == 0.0;
        if (zero) {
            CUDA_TRY(launch_rhs_density_builtin(P->dp, SGIGA_SRC_ONE, s));
            int r = run_rhs_operator(P);
            if (r) return r;
        }
        sgiga_solve_stats st{};
        auto timed = [&](int maxit, int& code, double tol = 1e-8) {
            const auto t0 = std::chrono::steady_clock::now();
            code = sgiga_solve(P, tol, maxit, &st);
            return since(t0) * 1e3;
        };
        int c = 0;
        timed(50, c);
        double tm = timed(50, c);
        if (c != SGIGA_OK && c != SGIGA_ERR_NOT_CONVERGED) return c;
        if (c != SGIGA_OK) tm = 1e30;
        // FP64 PCG with the FP64, then with the FP32 preconditioner
        double best = tm, tfp[2] = {0.0, 0.0};
        int pick = -1, its[2] = {0, 0};
        for (int v = 0; v < 2; ++v) {
            P->solve_fp64 = true;
            P->fp64_fd32 = v == 1;
            timed(1, c);
            const double t1 = timed(1, c);
            if (c != SGIGA_OK && c != SGIGA_ERR_NOT_CONVERGED) { P->solve_fp64 = P->fp64_fd32 = false; return c; }
            // iterations that fit in twice the fastest time so far (one timed
            // iteration includes the per-solve overhead), at least 4
            const int cap = (int)std::min(1000.0, std::max(4.0, 2.0 * best / std::max(t1, 1e-3)));
            const double t64 = timed(cap, c);
            if (c != SGIGA_OK && c != SGIGA_ERR_NOT_CONVERGED) { P->solve_fp64 = P->fp64_fd32 = false; return c; }
            if (c == SGIGA_OK) {
                tfp[v] = t64;
                its[v] = st.iterations;
                if (t64 < best) { best = t64; pick = v; }
            }
        }
        if (pick == 1 && tfp[0] > 0.0) {
            // both FP64 variants converged to 1e-8: the FP32 preconditioner
            // must keep up to 1e-12 as well (each gets three times its 1e-8
            // iterations, plus four, after one untimed run)
            double t12[2] = {1e30, 1e30};
            for (int v = 0; v < 2; ++v) {
                P->fp64_fd32 = v == 1;
                const int cap = 3 * its[v] + 4;
                timed(cap, c, 1e-12);
                const double t = timed(cap, c, 1e-12);
                if (c != SGIGA_OK && c != SGIGA_ERR_NOT_CONVERGED) { P->solve_fp64 = P->fp64_fd32 = false; return c; }
                if (c == SGIGA_OK) t12[v] = t;
            }
            if (t12[1] >= t12[0]) pick = 0;
        }
        *msmx = tm;
        *ms64 = tfp[0];
        *ms6432 = tfp[1];
        P->solve_fp64 = pick >= 0;
        P->fp64_fd32 = pick == 1;
        g_last_error.clear();
        return SGIGA_OK;
    };
    rc = body();
    cudaMemcpyAsync(P->d_b, save, n * 8, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(P->d_x, save + n, n * 8, cudaMemcpyDeviceToDevice, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == SGIGA_OK) rc = fail(SGIGA_ERR_CUDA, "autotune: restore failed");
    cudaFree(save);
    return rc;
}

// Operator tile policy (and, for FP32 3D plans, threads per block and the
// metric planes' L2 prefetch), timed with the FP32 (f32) or FP64 operator, and
// preconditioner layout, timed with the FP32 (fd32) or FP64 preconditioner:
// the kernels the plan's CG runs.
static int tune_decomposition(sgiga_plan_s* P, int reps, bool f32, bool fd32, sgiga_tune_result* out) {
    struct Cand { size_t budget; long long qpcap; };
    const Cand cands[] = {{48 * 1024, 4096}, {48 * 1024, 16384}, {110 * 1024, 8192},
                          {110 * 1024, 16384}, {200 * 1024, 16384}, {200 * 1024, 32768}};
    const int nc = (int)(sizeof(cands) / sizeof(cands[0]));
    cudaStream_t s = P->stream;
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    // probe vector: the plan's direction vector p (overwritten), output q
    CUDA_TRY(cudaMemsetAsync(P->d_p, 0, (size_t)P->ndof * 8, s));
    double best = 1e30;
    int bi = 3;
    int rc = SGIGA_OK;
    // the operator the plan's CG runs: FP32 in mixed plans (inner solve), else FP64
    if (f32) CUDA_TRY(cudaMemsetAsync(P->f_p, 0, (size_t)P->ndof * 4, s));
    auto apply_once = [&]() {
        return f32 ? apply_op(P, P->f_p, P->f_q, nullptr) : apply_op(P, P->d_b, P->d_q, nullptr);
    };
    // FP32 3D plans: each tile policy with 256 and with 128 threads per block
    const int nth_opts = (f32 && P->d == 3) ? 2 : 1;
    // the geometry planes in natural layout, gathered into each candidate's
    // tiling (the map is not evaluated again); without the memory for the
    // copy every candidate recomputes them
    double* Gn = nullptr;
    if (cudaMalloc(&Gn, (size_t)(P->ncomp + 1) * P->nqp * 8) != cudaSuccess) {
        cudaGetLastError();
        Gn = nullptr;
    }
    double* mwn = Gn ? Gn + (size_t)P->ncomp * P->nqp : nullptr;
    if (Gn) {
        cudaError_t e = launch_geometry_export(P->dp, Gn, mwn, s);
        if (e != cudaSuccess) { cudaFree(Gn); return fail(SGIGA_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e)); }
    }
    // FP32 3D plans with p odd (the metric planes' tile segments are 32-byte
    // aligned): L2 prefetch of the tile's planes, whole, capped so that the
    // segments in flight on all SMs total at most 48 MB or 16 MB, or none
    const int npf = (f32 && P->d == 3 && (P->p & 1)) ? 4 : 1;
    int nsm = 152;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess) { cudaGetLastError(); nsm = 152; }
    auto pf_value = [&](int f) -> int {
        if (f == 0) return 0;
        if (f == 3) return -1;
        const long long total = (f == 1 ? 48LL : 16LL) << 20;
        const long long per = total / ((long long)nsm * op3_f32_resident(P->dp) * (P->dp.diag ? 3 : 6));
        return (int)std::max(16LL, per & ~15LL);
    };
    int bnth = 256, bpf = 0, ci = 0;
    for (int i = 0; i < nc && rc == SGIGA_OK; ++i) {
        if ((rc = retile(P, cands[i].budget, cands[i].qpcap, Gn, mwn))) break;
        for (int o = 0; o < nth_opts && rc == SGIGA_OK; ++o, ++ci) {
            P->dp.op_nth = o == 0 ? 256 : 128;
            double cbest = 1e30;
            int cpf = 0;
            for (int f = 0; f < npf && rc == SGIGA_OK; ++f) {
                P->dp.op_pf = pf_value(f);
                if ((rc = apply_once())) break;   // warm-up
                cudaEventRecord(e0, s);
                for (int r = 0; r < reps && rc == SGIGA_OK; ++r) rc = apply_once();
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) { rc = fail(SGIGA_ERR_CUDA, "autotune timing failed"); break; }
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                const double per = ms / reps;
                if (per < cbest) { cbest = per; cpf = P->dp.op_pf; }
            }
            if (out && ci < 16) {
                out->ms[ci] = cbest; out->budget[ci] = (int)cands[i].budget; out->qpcap[ci] = (int)cands[i].qpcap;
                out->nthreads[ci] = P->dp.op_nth;
                out->prefetch[ci] = cpf;
            }
            if (cbest < best) { best = cbest; bi = i; bnth = P->dp.op_nth; bpf = cpf; }
        }
    }
    P->dp.op_nth = bnth;
    P->dp.op_pf = bpf;
    if (rc == SGIGA_OK) rc = retile(P, cands[bi].budget, cands[bi].qpcap, Gn, mwn);
    if (Gn) cudaFree(Gn);
    // preconditioner item depth
    const int ks_v[] = {16, 32, 64, 128};
    const int nksv = (int)(sizeof(ks_v) / sizeof(ks_v[0]));
    const int nks = 2 * nksv;   // per-piece layout, then grouped layout
    double fbest = 1e30;
    int fbi = 1;
    for (int i = 0; i < nks && rc == SGIGA_OK; ++i) {
        const int ksi = ks_v[i % nksv];
        const bool grp = i >= nksv;
        if ((rc = refd(P, ksi, grp))) break;
        // the precision the plan's CG runs in; plain FD (no learned correction)
        auto fd_once = [&]() {
            if (fd32)
                return precond_fd<float>(P, P->f_b, P->f_z, nullptr, P->f_t1, P->f_t2);
            return precond_fd<double>(P, P->d_b, P->d_z, nullptr, P->d_t1, P->d_t2);
        };
        if ((rc = fd_once())) break;   // warm-up
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && rc == SGIGA_OK; ++r) rc = fd_once();
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = fail(SGIGA_ERR_CUDA, "autotune timing failed"); break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        double per = ms / reps;
        if (out) { out->fd_ms[i] = per; out->fd_ks[i] = ksi; out->fd_grouped[i] = grp ? 1 : 0; }
        if (per < fbest) { fbest = per; fbi = i; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if ((rc = refd(P, ks_v[fbi % nksv], fbi >= nksv))) return rc;
    if (out) {
        out->ncand = ci;
        out->best = bi * nth_opts + (bnth == 128 ? 1 : 0);
        out->best_ms = best;
        out->best_prefetch = bpf;
        out->ntiles = (int)P->tiles.size();
        out->fd_ncand = nks;
        out->fd_best = fbi;
        size_t items = 0;
        for (int k = 0; k < P->d; ++k) {
            items += P->fd[k].size();
            for (int t = 0; t < 3; ++t) items += P->fdl[k][t].size();
        }
        out->fd_nitems = (int)items;
    }
    return SGIGA_OK;
}

int sgiga_autotune(sgiga_plan_t P, int reps, sgiga_tune_result* out) {
    NvtxRange nvtx_("sgiga_autotune");
    if (!P || reps < 1) return fail(SGIGA_ERR_ARG, "null plan or reps < 1");
    const auto tt0 = std::chrono::steady_clock::now();
    // the kernels the plan's CG runs: FP32 in mixed plans (inner solve), else FP64
    const bool mixed = P->cfg.precision == SGIGA_PREC_MIXED_FP32;
    int rc = tune_decomposition(P, reps, mixed, mixed, out);
    if (rc) return rc;
    double ms64 = 0.0, msmx = 0.0, ms6432 = 0.0;
    if (mixed && P->cfg.precond == SGIGA_PRECOND_FD)
        if ((rc = choose_precision(P, &ms64, &msmx, &ms6432))) return rc;
    // a mixed plan that now solves in FP64: its decomposition tuned for the
    // kernels of that solve (FP64 operator; FP64 or FP32 preconditioner)
    if (P->solve_fp64 && (rc = tune_decomposition(P, reps, false, P->fp64_fd32, out))) return rc;
    if (out) {
        out->solve_precision = mixed && !P->solve_fp64 ? SGIGA_PREC_MIXED_FP32 : SGIGA_PREC_FP64;
        out->solve_ms_fp64 = ms64;
        out->solve_ms_mixed = msmx;
        out->solve_ms_fp64_fd32 = ms6432;
        out->solve_fp32_precond = P->fp64_fd32 ? 1 : 0;
    }
    P->t_autotune = since(tt0);
    return SGIGA_OK;
}

int sgiga_set_tiling(sgiga_plan_t P, int budget, int qpcap, int nthreads, int prefetch) {
    if (!P) return fail(SGIGA_ERR_ARG, "null argument");
    if (budget < 16 * 1024 || budget > 227 * 1024 || qpcap < 64 || qpcap > (1 << 20))
        return fail(SGIGA_ERR_ARG, "budget must be in [16 KB, 227 KB] and qpcap in [64, 2^20]");
    if (nthreads != 256 && nthreads != 128) return fail(SGIGA_ERR_ARG, "nthreads must be 256 or 128");
    if (prefetch > 0 && prefetch % 16) return fail(SGIGA_ERR_ARG, "prefetch must be a multiple of 16 bytes");
    int rc = retile(P, (size_t)budget, qpcap);
    if (rc) return rc;
    P->dp.op_nth = nthreads;
    P->dp.op_pf = prefetch;
    return SGIGA_OK;
}

int sgiga_plan_times(sgiga_plan_t P, sgiga_plan_times_t* out) {
    if (!P || !out) return fail(SGIGA_ERR_ARG, "null argument");
    out->total = P->t_total;
    out->host = P->t_host;
    out->basis = P->t_basis;
    out->eigen = P->t_eigen;
    out->fd = P->t_fd;
    out->geometry = P->t_geometry;
    out->vectors = P->t_vectors;
    out->coefficient = P->t_coefficient;
    out->autotune = P->t_autotune;
    return SGIGA_OK;
}

int sgiga_set_precond_split(sgiga_plan_t P, int ks, int grouped) {
    if (!P) return fail(SGIGA_ERR_ARG, "null argument");
    if (ks < 16 || ks > 4096 || ks % 16) return fail(SGIGA_ERR_ARG, "ks must be a multiple of 16 in [16, 4096]");
    return refd(P, ks, grouped != 0);
}

int sgiga_set_solver_options(sgiga_plan_t P, int use_graph, double inner_tol, int inner_max) {
    if (!P) return fail(SGIGA_ERR_ARG, "null argument");
    if (!(inner_tol > 0) || inner_max < 1) return fail(SGIGA_ERR_ARG, "inner_tol must be > 0 and inner_max >= 1");
    P->use_graph = use_graph != 0;
    P->inner_tol = inner_tol;
    P->inner_max = inner_max;
    return SGIGA_OK;
}

int sgiga_solve(sgiga_plan_t P, double rel_tol, int max_iter, sgiga_solve_stats* stats) {
    NvtxRange nvtx_("sgiga_solve");
    if (!P) return fail(SGIGA_ERR_ARG, "null argument");
    if (!(rel_tol > 0) || max_iter < 1) return fail(SGIGA_ERR_ARG, "rel_tol must be > 0 and max_iter >= 1");
    auto t0 = std::chrono::steady_clock::now();
    const int ng = (int)P->comps.size();
    P->last_inner_iters = 0;
    {   // a right-hand side with a NaN or an infinity is an input error, not a divergence
        CUDA_TRY(launch_dot<double>(P->dp, P->d_b, P->d_b, P->d_partial, P->d_scal, P->stream));
        std::vector<double> hb(ng);
        CUDA_TRY(cudaMemcpyAsync(hb.data(), P->d_scal, ng * 8, cudaMemcpyDeviceToHost, P->stream));
        CUDA_TRY(cudaStreamSynchronize(P->stream));
        for (int g = 0; g < ng; ++g)
            if (!std::isfinite(hb[g]))
                return fail(SGIGA_ERR_ARG, "the load vector of component " + std::to_string(g) +
                                               " is not finite (a NaN or infinity in f or the boundary data)");
    }
    if (P->cfg.precision == SGIGA_PREC_FP64 || P->solve_fp64) {
        ct_inner_iterations(P, true);
        int nact = pcg<double>(P, P->d_b, vecs64(P), rel_tol, max_iter, nullptr, P->d_active, P->d_iters, P->d_scal,
                               nullptr);
        if (nact < 0) return nact;
        int rc = solve_stats(P, P->d_scal + 3 * ng, P->d_scal, P->d_iters, nact, stats, t0);
        if (rc) return rc;
        if (stats && P->ct) stats->inner_iterations = (int)ct_inner_iterations(P, false);
        if (nact > 0) return fail(SGIGA_ERR_NOT_CONVERGED, std::to_string(nact) + " components did not converge");
        return SGIGA_OK;
    }
    // Mixed precision: FP64 iterative refinement around an FP32 inner solve.
    //   x = 0, r = b;  repeat: d = (inner FP32 PCG) K^{-1} r;  x += d;  r = b - K x (FP64)
    // until ||r_g|| <= rel_tol ||b_g|| for every component (max_iter outer steps).
    const DevPlan& D = P->dp;
    cudaStream_t s = P->stream;
    double* bb = P->d_scal64o + 0 * ng;
    double* rr = P->d_scal64o + 3 * ng;
    CUDA_TRY(launch_pcg_init<double>(D, P->d_b, P->d_x, P->d_r, P->d_partial, bb, s));
    CUDA_TRY(launch_copy<double>(rr, bb, ng, s));
    CUDA_TRY(launch_pcg_start(D, bb, nullptr, P->d_active_o, P->d_iters_o, s));
    int nact = ng, outer = 0, inner_total = 0, stalls = 0;
    bool fp64_fallback = false;
    P->learned_off = false;
    if (int rc0 = learned_prepare(P)) return rc0;
    double prev_worst = 0.0;
    std::vector<double> hrr(ng), hbb(ng), prev_rr(ng, 0.0);
    std::vector<int> hact(ng);
    for (outer = 0; outer <= max_iter; ++outer) {
        // convergence of the FP64 residual (also counts outer steps per grid)
        CUDA_TRY(launch_pcg_check(D, rr, bb, rel_tol * rel_tol, P->d_active_o, P->d_iters_o, P->d_nactive, s));
        CUDA_TRY(cudaMemcpyAsync(P->h_nactive, P->d_nactive, sizeof(int), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaMemcpyAsync(hrr.data(), rr, ng * 8, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaMemcpyAsync(hbb.data(), bb, ng * 8, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaMemcpyAsync(hact.data(), P->d_active_o, ng * 4, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        nact = *P->h_nactive;
        if (nact == 0 || outer == max_iter) break;
        // A refinement step that does not halve an active component's residual
        // means the FP32 inner operator is too far from the FP64 one for this
        // system (its error times the condition number is not small). After two
        // such steps the remaining components are finished by FP64 PCG on the
        // current residual: d = K^{-1} r, x += d (the plain method).
        bool stalled = false, broken = false;
        for (int g = 0; g < ng; ++g) {
            if (!hact[g]) continue;
            if (!std::isfinite(hrr[g])) broken = true;   // the FP32 inner solve broke down
            if (outer > 0 && !(hrr[g] <= 0.25 * prev_rr[g])) stalled = true;
        }
        prev_rr = hrr;
        stalls = stalled ? stalls + 1 : 0;
        if ((stalls >= 2 || broken) && P->cfg.precond != SGIGA_PRECOND_LEARNED) {
            if (broken) {   // restart the active components from x = 0, r = b
                int rc = SGIGA_OK;
                CUDA_TRY(launch_zero_active(D, P->d_x, P->d_active_o, s));
                if ((rc = apply_op(P, P->d_x, P->d_q, P->d_active_o))) return rc;
                CUDA_TRY(launch_ir_residual(D, P->d_b, P->d_q, P->d_r, P->d_active_o, P->d_partial, rr, s));
                CUDA_TRY(cudaMemcpyAsync(hrr.data(), rr, ng * 8, cudaMemcpyDeviceToHost, s));
                CUDA_TRY(cudaStreamSynchronize(s));
            }
            double ratio = 1.0;   // tightest ||b_g|| / ||r_g|| over the active components
            for (int g = 0; g < ng; ++g)
                if (hact[g] && hrr[g] > 0) ratio = std::min(ratio, std::sqrt(hbb[g] / hrr[g]));
            const double tol64 = std::max(0.5 * rel_tol * ratio, 1e-15);
            Vecs<double> v{P->d_d, P->d_r, P->d_z, P->d_p, P->d_q, P->d_t1, P->d_t2};
            int it64 = 0;
            int rc = pcg<double>(P, P->d_r, v, tol64, max_iter * 10, P->d_active_o, P->d_active, P->d_iters,
                                 P->d_scal, &it64);
            if (rc < 0) return rc;
            inner_total += it64;
            CUDA_TRY(launch_ir_up64(D, P->d_x, P->d_d, P->d_active_o, s));
            if ((rc = apply_op(P, P->d_x, P->d_q, P->d_active_o))) return rc;
            CUDA_TRY(launch_ir_residual(D, P->d_b, P->d_q, P->d_r, P->d_active_o, P->d_partial, rr, s));
            fp64_fallback = true;
            stalls = 0;
            continue;
        }
        if (P->cfg.precond == SGIGA_PRECOND_LEARNED) {
            // fall back to FD for the rest of the solve when a refinement step
            // with the learned scaling does not cut the worst residual by 10
            double worst = 0.0;
            for (int g = 0; g < ng; ++g)
                if (hbb[g] > 0) worst = std::max(worst, std::sqrt(hrr[g] / hbb[g]));
            if (outer > 0 && worst > 0.1 * prev_worst) P->learned_off = true;
            prev_worst = worst;
        }
        CUDA_TRY(launch_ir_down(D, P->d_r, P->f_b, P->d_active_o, s));
        int inner = 0;
        int rc = pcg<float>(P, P->f_b, vecs32(P), P->inner_tol, P->inner_max, P->d_active_o, P->d_active,
                            P->d_iters, P->d_scal, &inner);
        if (rc < 0) return rc;
        inner_total += inner;
        CUDA_TRY(launch_ir_up(D, P->d_x, P->f_x, P->d_active_o, s));
        if ((rc = apply_op(P, P->d_x, P->d_q, P->d_active_o))) return rc;
        CUDA_TRY(launch_ir_residual(D, P->d_b, P->d_q, P->d_r, P->d_active_o, P->d_partial, rr, s));
    }
    P->last_inner_iters = inner_total;
    int rc = solve_stats(P, rr, bb, P->d_iters_o, nact, stats, t0);
    if (rc) return rc;
    if (stats) {
        stats->iterations = outer;
        stats->inner_iterations = inner_total;
        stats->fallback = (P->learned_off ? 1 : 0) | (fp64_fallback ? 2 : 0);
    }
    P->learned_off = false;
    if (nact > 0) return fail(SGIGA_ERR_NOT_CONVERGED, std::to_string(nact) + " components did not converge");
    return SGIGA_OK;
}

int sgiga_get_solution(sgiga_plan_t P, double* u) {
    if (!P || !u) return fail(SGIGA_ERR_ARG, "null argument");
    CUDA_TRY(cudaMemcpyAsync(u, P->d_x, (size_t)P->ndof * 8, cudaMemcpyDefault, P->stream));
    CUDA_TRY(cudaStreamSynchronize(P->stream));
    return SGIGA_OK;
}

int sgiga_set_solution(sgiga_plan_t P, const double* u) {
    if (!P || !u) return fail(SGIGA_ERR_ARG, "null argument");
    CUDA_TRY(cudaMemcpyAsync(P->d_x, u, (size_t)P->ndof * 8, cudaMemcpyDefault, P->stream));
    CUDA_TRY(cudaStreamSynchronize(P->stream));
    return SGIGA_OK;
}

int sgiga_eval(sgiga_plan_t P, const double* xi, long long npts, double* ucomp) {
    NvtxRange nvtx_("sgiga_eval");
    if (!P || (!xi && npts > 0) || (!ucomp && npts > 0)) return fail(SGIGA_ERR_ARG, "null argument");
    if (npts < 0) return fail(SGIGA_ERR_ARG, "npts < 0");
    if (P->multipatch) return fail(SGIGA_ERR_ARG, "multi-patch plan: evaluate with sgiga_eval_grad (patch ids)");
    if (npts == 0) return SGIGA_OK;
    const size_t ng = P->comps.size();
    const size_t xb = (size_t)npts * P->d * 8, ub = (size_t)npts * ng * 8;
    const bool xdev = is_device(xi), udev = is_device(ucomp);
    size_t need = (xdev ? 0 : xb) + (udev ? 0 : ub);
    int rc = ensure_stage(P, need);
    if (rc) return rc;
    char* st = (char*)P->stage;
    const double* xd = xi;
    if (!xdev) {
        CUDA_TRY(cudaMemcpyAsync(st, xi, xb, cudaMemcpyHostToDevice, P->stream));
        xd = (const double*)st;
        st += xb;
    }
    double* ud = udev ? ucomp : (double*)st;
    // per-(table, point) basis values, shared by the components (plan-owned, grown on demand)
    const size_t need_vals = (size_t)P->tabs.size() * npts;
    if (need_vals > P->eval_cap) {
        if (P->d_eval_vals) cudaFree(P->d_eval_vals);
        if (P->d_eval_first) cudaFree(P->d_eval_first);
        P->d_eval_vals = nullptr;
        P->d_eval_first = nullptr;
        P->eval_cap = 0;
        if (cudaMalloc(&P->d_eval_vals, need_vals * (P->p + 1) * 8) != cudaSuccess ||
            cudaMalloc(&P->d_eval_first, need_vals * 4) != cudaSuccess) {
            cudaGetLastError();
            return fail(SGIGA_ERR_NOMEM, "evaluation basis buffer allocation failed");
        }
        P->eval_cap = need_vals;
    }
    CUDA_TRY(cudaMemsetAsync(P->dp.flags + 1, 0, sizeof(int), P->stream));
    CUDA_TRY(launch_eval(P->dp, P->d_x, xd, npts, P->d_eval_vals, P->d_eval_first, ud, P->stream));
    int hflag = 0;
    CUDA_TRY(cudaMemcpyAsync(P->h_nactive, P->dp.flags + 1, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
    if (!udev) CUDA_TRY(cudaMemcpyAsync(ucomp, ud, ub, cudaMemcpyDeviceToHost, P->stream));
    CUDA_TRY(cudaStreamSynchronize(P->stream));
    hflag = *P->h_nactive;
    if (hflag) return fail(SGIGA_ERR_ARG, "evaluation point outside [0,1]^d");
    return SGIGA_OK;
}

int sgiga_combine(sgiga_plan_t P, const double* ucomp, long long npts, double* u) {
    if (!P || (!ucomp && npts > 0) || (!u && npts > 0)) return fail(SGIGA_ERR_ARG, "null argument");
    if (npts < 0) return fail(SGIGA_ERR_ARG, "npts < 0");
    if (npts == 0) return SGIGA_OK;
    const size_t ng = P->comps.size();
    const size_t ub = (size_t)npts * ng * 8, ob = (size_t)npts * 8;
    const bool idev = is_device(ucomp), odev = is_device(u);
    int rc = ensure_stage(P, (idev ? 0 : ub) + (odev ? 0 : ob));
    if (rc) return rc;
    char* st = (char*)P->stage;
    const double* ud = ucomp;
    if (!idev) {
        CUDA_TRY(cudaMemcpyAsync(st, ucomp, ub, cudaMemcpyHostToDevice, P->stream));
        ud = (const double*)st;
        st += ub;
    }
    double* od = odev ? u : (double*)st;
    CUDA_TRY(launch_combine(P->dp, ud, npts, P->d_coef, od, P->stream));
    if (!odev) CUDA_TRY(cudaMemcpyAsync(u, od, ob, cudaMemcpyDeviceToHost, P->stream));
    CUDA_TRY(cudaStreamSynchronize(P->stream));
    return SGIGA_OK;
}

int sgiga_combine_plans(int nplans, const sgiga_plan_t* plans, const double* ucomp, long long npts, double* u) {
    NvtxRange nvtx_("sgiga_combine_plans");
    if (nplans < 1 || !plans) return fail(SGIGA_ERR_ARG, "nplans must be >= 1 with the plans given");
    if (npts < 0) return fail(SGIGA_ERR_ARG, "npts < 0");
    size_t ng = 0;
    for (int k = 0; k < nplans; ++k) {
        if (!plans[k]) return fail(SGIGA_ERR_ARG, "null plan");
        if (plans[k]->d != plans[0]->d) return fail(SGIGA_ERR_ARG, "plans differ in dimension");
        if (plans[k]->stream != plans[0]->stream) return fail(SGIGA_ERR_ARG, "plans must share one stream");
        ng += plans[k]->comps.size();
    }
    if (ng > (size_t)INT32_MAX) return fail(SGIGA_ERR_ARG, "too many components");
    if (npts == 0) return SGIGA_OK;
    if (!ucomp || !u) return fail(SGIGA_ERR_ARG, "null argument");
    sgiga_plan_s* P = plans[0];
    const size_t cb = (ng * 8 + 15) / 16 * 16, ub = (size_t)npts * ng * 8, ob = (size_t)npts * 8;
    const bool idev = is_device(ucomp), odev = is_device(u);
    int rc = ensure_stage(P, cb + (idev ? 0 : ub) + (odev ? 0 : ob));
    if (rc) return rc;
    char* st = (char*)P->stage;
    // every plan's coefficients, in plan order, as one device array
    double* coef = (double*)st;
    st += cb;
    size_t off = 0;
    for (int k = 0; k < nplans; ++k) {
        const size_t n = plans[k]->comps.size();
        if (n) CUDA_TRY(cudaMemcpyAsync(coef + off, plans[k]->d_coef, n * 8, cudaMemcpyDeviceToDevice, P->stream));
        off += n;
    }
    const double* ud = ucomp;
    if (!idev) {
        CUDA_TRY(cudaMemcpyAsync(st, ucomp, ub, cudaMemcpyHostToDevice, P->stream));
        ud = (const double*)st;
        st += ub;
    }
    double* od = odev ? u : (double*)st;
    CUDA_TRY(launch_combine_n((int)ng, ud, npts, coef, od, P->stream));
    if (!odev) CUDA_TRY(cudaMemcpyAsync(u, od, ob, cudaMemcpyDeviceToHost, P->stream));
    CUDA_TRY(cudaStreamSynchronize(P->stream));
    return SGIGA_OK;
}

int sgiga_basis_table(sgiga_plan_t P, int dir, int level, double* xi, double* w, double* R, double* dR,
                      int* first) {
    if (!P) return fail(SGIGA_ERR_ARG, "null argument");
    auto it = P->tab_of.find(std::make_pair(dir, level));
    if (it == P->tab_of.end()) return fail(SGIGA_ERR_ARG, "no table for this direction and level");
    const Table1D& t = P->tabs[it->second];
    const size_t n = (size_t)t.E * P->Q;
    const int p1 = P->p + 1;
    cudaStream_t s = P->stream;
    if (xi) CUDA_TRY(cudaMemcpyAsync(xi, P->dp.xi + t.off, n * 8, cudaMemcpyDeviceToHost, s));
    if (w) CUDA_TRY(cudaMemcpyAsync(w, P->dp.w + t.off, n * 8, cudaMemcpyDeviceToHost, s));
    if (R) CUDA_TRY(cudaMemcpyAsync(R, P->dp.R + t.off * p1, n * p1 * 8, cudaMemcpyDeviceToHost, s));
    if (dR) CUDA_TRY(cudaMemcpyAsync(dR, P->dp.dR + t.off * p1, n * p1 * 8, cudaMemcpyDeviceToHost, s));
    if (first) CUDA_TRY(cudaMemcpyAsync(first, P->dp.first + t.eoff, (size_t)t.E * 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return SGIGA_OK;
}

int sgiga_geometry_coeffs(sgiga_plan_t P, int g, double* G, double* mw) {
    if (!P || !G || !mw) return fail(SGIGA_ERR_ARG, "null argument");
    if (g < 0 || g >= (int)P->grids.size()) return fail(SGIGA_ERR_ARG, "grid index out of range");
    const GridDesc& gd = P->grids[g];
    const size_t nq = (size_t)gd.nqp;
    double* tmp = nullptr;
    cudaError_t e = cudaMalloc(&tmp, (P->ncomp + 1) * nq * 8);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(SGIGA_ERR_NOMEM, "temporary allocation failed"); }
    cudaStream_t s = P->stream;
    e = launch_geometry_natural(P->dp, g, gd, tmp, tmp + P->ncomp * nq, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(G, tmp, P->ncomp * nq * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mw, tmp + P->ncomp * nq, nq * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(tmp);
    if (e != cudaSuccess) return fail(SGIGA_ERR_CUDA, cudaGetErrorString(e));
    return SGIGA_OK;
}

int sgiga_fd_eigen(sgiga_plan_t P, int dir, int level, double* U, double* lam) {
    if (!P) return fail(SGIGA_ERR_ARG, "null argument");
    auto it = P->tab_of.find(std::make_pair(dir, level));
    if (it == P->tab_of.end()) return fail(SGIGA_ERR_ARG, "no table for this direction and level");
    const Eig1D& e = P->eigs[P->eig_of_tab[it->second]];
    if (U) CUDA_TRY(cudaMemcpy(U, P->dp.U + e.uoff, (size_t)e.n * e.n * 8, cudaMemcpyDeviceToHost));
    if (lam) CUDA_TRY(cudaMemcpy(lam, P->dp.lam + e.loff, (size_t)e.n * 8, cudaMemcpyDeviceToHost));
    return SGIGA_OK;
}

}  // extern "C"
