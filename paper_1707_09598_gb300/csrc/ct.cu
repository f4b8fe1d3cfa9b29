// The combination technique as a preconditioner of the full tensor-product
// solve (the paper's closing remark, Sec. 5): an additive two-level method
//
//   z = FD(r) + B_CT r,   B_CT = sum_i c_i P_i K_i^{-1} P_i^T,
//
// where the full plan has one component of levels (J, .., J), the
// combination plan holds the components i of a sparse-grid index set
// (eq. TD-combi-tec), P_i is the prolongation of component i's space into the
// full space (the spaces are nested: uniform knots, the same degree and
// continuity) and K_i^{-1} is the combination plan's batched PCG to an inner
// tolerance. B_CT is not exactly linear (inner solves to a tolerance), so the
// full plan's CG runs flexible.
//
// P_i = P_{i,d-1} x .. x P_{i,0}, each 1D factor the knot-insertion matrix of
// the component's level into level J (computed on the host by inserting the
// fine breakpoints one at a time, Boehm's rule). Restriction P_i^T and
// prolongation P_i run as mode products over all components at once.
#include <algorithm>
#include <cstring>
#include <map>
#include <vector>

#include "plan.h"

namespace sgiga {

// One mode product of one component: out[a][i][b] = sum_j M(i, j) in[a][j][b]
// with b over the directions below `dir` (direction 0 fastest) and a over
// those above. M(i, j) = P[j * pc + i] (trans: restriction, P^T) or
// P[i * pc + j] (prolongation), P row-major with pc columns.
struct CTJob {
    long long in_off, out_off, mat_off;
    int n[3];       // input extents
    int dir, m_out, pc, trans;
};

struct CTPrec {
    sgiga_plan_s* ct = nullptr;     // the combination's components (not owned)
    double inner_tol = 1e-6;
    int inner_max = 200;
    bool ct_only = false;           // sgiga_ct_apply: B_CT without FD
    int npass = 0;                  // mode products per direction sweep (d)
    CTJob* jobs = nullptr;          // device: [2 * d][ncomp] (restriction passes, then prolongation passes)
    double* mats = nullptr;         // device: every 1D prolongation matrix
    double* tmp[2] = {nullptr, nullptr};
    double* Y = nullptr;            // device: [ncomp][nfull] prolonged solutions
    double* coef = nullptr;         // device: combination coefficients
    int ncomp = 0;
    long long nfull = 0, maxout = 0;
    long long inner_total = 0;      // inner CG iterations since the last reset
};

// Knot vector of level l: open ends (p + 1), breakpoints k / 2^l each of
// multiplicity p - r.
static std::vector<double> ct_knots(int p, int r, int l) {
    std::vector<double> t(p + 1, 0.0);
    const int E = 1 << l, m = p - r;
    for (int k = 1; k < E; ++k)
        for (int q = 0; q < m; ++q) t.push_back((double)k / E);
    for (int q = 0; q <= p; ++q) t.push_back(1.0);
    return t;
}

// Interior prolongation matrix [nf - 2][nc - 2] (row-major) of level lc into
// level lf: column j holds the fine coefficients of coarse B-spline j + 1.
// Boehm's rule inserts a knot s with t_k <= s < t_{k+1} into every column:
//   c'_i = c_i (i <= k - p),  (1 - a_i) c_{i-1} + a_i c_i (k - p < i <= k),
//   c_{i-1} (i > k),  a_i = (s - t_i) / (t_{i+p} - t_i).
static std::vector<double> ct_prolongation(int p, int r, int lc, int lf, int& nfi, int& nci) {
    std::vector<double> t = ct_knots(p, r, lc);
    const std::vector<double> tf = ct_knots(p, r, lf);
    const int nc = (int)t.size() - p - 1;
    std::vector<std::vector<double>> C(nc, std::vector<double>(nc, 0.0));   // C[row = basis][col = coarse]
    for (int i = 0; i < nc; ++i) C[i][i] = 1.0;
    // the fine knots the coarse vector lacks (multiset difference)
    std::map<double, int> have, want;
    for (double v : t) have[v]++;
    for (double v : tf) want[v]++;
    std::vector<double> ins;
    for (auto& kv : want)
        for (int q = have[kv.first]; q < kv.second; ++q) ins.push_back(kv.first);
    for (double s : ins) {
        int k = p;
        while (k + 1 < (int)t.size() && t[k + 1] <= s) ++k;   // t_k <= s < t_{k+1}
        const int n = (int)C.size();
        std::vector<std::vector<double>> D(n + 1, std::vector<double>(nc, 0.0));
        for (int i = 0; i <= n; ++i) {
            if (i <= k - p) D[i] = C[i];
            else if (i <= k) {
                const double a = (s - t[i]) / (t[i + p] - t[i]);
                for (int j = 0; j < nc; ++j) D[i][j] = (1.0 - a) * C[i - 1][j] + a * C[i][j];
            } else D[i] = C[i - 1];
        }
        C.swap(D);
        t.insert(t.begin() + k + 1, s);
    }
    const int nf = (int)C.size();
    nfi = nf - 2;
    nci = nc - 2;
    std::vector<double> P((size_t)nfi * nci);
    for (int i = 0; i < nfi; ++i)
        for (int j = 0; j < nci; ++j) P[(size_t)i * nci + j] = C[i + 1][j + 1];
    return P;
}

__global__ void k_ct_mode(const CTJob* __restrict__ jobs, const double* __restrict__ mats,
                          const double* __restrict__ in, double* __restrict__ out) {
    const CTJob J = jobs[blockIdx.y];
    long long B = 1, A = 1;
    for (int k = 0; k < J.dir; ++k) B *= J.n[k];
    for (int k = J.dir + 1; k < 3; ++k) A *= J.n[k];
    const int m_in = J.n[J.dir];
    const long long total = A * J.m_out * B;
    const double* M = mats + J.mat_off;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long b = idx % B, rr = idx / B;
        const int i = (int)(rr % J.m_out);
        const long long a = rr / J.m_out;
        const double* src = in + J.in_off + a * m_in * B + b;
        double acc = 0.0;
        if (J.trans)
            for (int j = 0; j < m_in; ++j) acc += M[(long long)j * J.pc + i] * src[(long long)j * B];
        else
            for (int j = 0; j < m_in; ++j) acc += M[(long long)i * J.pc + j] * src[(long long)j * B];
        out[J.out_off + idx] = acc;
    }
}

// z = base + sum_i c_i Y_i (base may be null: no FD part)
__global__ void k_ct_sum(const double* __restrict__ Y, const double* __restrict__ coef, int ncomp, long long n,
                         const double* __restrict__ base, double* __restrict__ z) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        double acc = base ? base[k] : 0.0;
        for (int i = 0; i < ncomp; ++i) acc += coef[i] * Y[(long long)i * n + k];
        z[k] = acc;
    }
}

static cudaError_t launch_ct_mode(const CTJob* jobs, int njobs, long long maxout, const double* mats,
                                  const double* in, double* out, cudaStream_t s) {
    long long bx = (maxout + 255) / 256;
    if (bx > 1024) bx = 1024;
    if (bx < 1) bx = 1;
    SGIGA_COUNT_LAUNCH();
    k_ct_mode<<<dim3((unsigned)bx, (unsigned)njobs), 256, 0, s>>>(jobs, mats, in, out);
    return cudaGetLastError();
}

// B_CT r (plus FD r unless ct_only) into z.
int precond_ct(sgiga_plan_s* P, const double* r, double* z, const int* active, double* t1, double* t2) {
    CTPrec* C = P->ct;
    sgiga_plan_s* Q = C->ct;
    cudaStream_t s = P->stream;
    const int d = P->d, nc = C->ncomp;
    // restriction: r -> tmp -> .. -> Q's load vector (packed components)
    const double* in = r;
    for (int k = 0; k < d; ++k) {
        double* out = k == d - 1 ? Q->d_b : C->tmp[k & 1];
        CUDA_TRY(launch_ct_mode(C->jobs + (size_t)k * nc, nc, C->maxout, C->mats, in, out, s));
        in = out;
    }
    sgiga_solve_stats st{};
    const int rc = sgiga_solve(Q, C->inner_tol, C->inner_max, &st);
    if (rc != SGIGA_OK && rc != SGIGA_ERR_NOT_CONVERGED) return rc;   // an inexact inner solve is allowed
    C->inner_total += st.iterations;
    // prolongation: Q's solution -> tmp -> .. -> Y_i
    in = Q->d_x;
    for (int k = 0; k < d; ++k) {
        double* out = k == d - 1 ? C->Y : C->tmp[k & 1];
        CUDA_TRY(launch_ct_mode(C->jobs + (size_t)(d + k) * nc, nc, C->maxout, C->mats, in, out, s));
        in = out;
    }
    const double* base = nullptr;
    if (!C->ct_only) {
        int r2 = precond_fd<double>(P, r, z, active, t1, t2);
        if (r2) return r2;
        base = z;
    }
    long long bx = (C->nfull + 255) / 256;
    if (bx > 152 * 16) bx = 152 * 16;
    SGIGA_COUNT_LAUNCH();
    k_ct_sum<<<(unsigned)std::max(1LL, bx), 256, 0, s>>>(C->Y, C->coef, nc, C->nfull, base, z);
    CUDA_TRY(cudaGetLastError());
    return SGIGA_OK;
}

void free_ct(sgiga_plan_s* P) {
    if (!P->ct) return;
    CTPrec* C = P->ct;
    cudaFree(C->jobs);
    cudaFree(C->mats);
    cudaFree(C->tmp[0]);
    cudaFree(C->tmp[1]);
    cudaFree(C->Y);
    cudaFree(C->coef);
    delete C;
    P->ct = nullptr;
}

long long ct_inner_iterations(sgiga_plan_s* P, bool reset) {
    if (!P->ct) return 0;
    const long long v = P->ct->inner_total;
    if (reset) P->ct->inner_total = 0;
    return v;
}

}  // namespace sgiga

using namespace sgiga;

extern "C" {

int sgiga_ct_attach(sgiga_plan_t P, sgiga_plan_t Q, double inner_tol, int inner_max) {
    if (!P) return fail(SGIGA_ERR_ARG, "null plan");
    free_ct(P);
    destroy_loop_graph(P->loop64);
    if (!Q) return SGIGA_OK;
    if (P == Q) return fail(SGIGA_ERR_ARG, "the combination plan must be another plan");
    if (!(inner_tol > 0) || inner_max < 1) return fail(SGIGA_ERR_ARG, "inner_tol must be > 0 and inner_max >= 1");
    const int d = P->d;
    if (P->comps.size() != 1 || P->multipatch || Q->multipatch)
        return fail(SGIGA_ERR_ARG, "the full plan needs exactly one component; single-patch plans only");
    if (P->cfg.precision != SGIGA_PREC_FP64 || Q->cfg.precision != SGIGA_PREC_FP64 ||
        P->cfg.precond != SGIGA_PRECOND_FD)
        return fail(SGIGA_ERR_ARG, "FP64 plans with the FD preconditioner only");
    if (Q->d != d || Q->p != P->p || Q->r != P->r || Q->cfg.domain != P->cfg.domain)
        return fail(SGIGA_ERR_ARG, "the plans differ in dimension, degree, continuity or domain");
    if (P->cfg.grading != SGIGA_GRADING_UNIFORM || Q->cfg.grading != SGIGA_GRADING_UNIFORM)
        return fail(SGIGA_ERR_ARG, "nested spaces need uniform knots");
    if (P->cfg.domain == SGIGA_DOMAIN_PATCH && std::memcmp(&P->patch, &Q->patch, sizeof(Patch)) != 0)
        return fail(SGIGA_ERR_ARG, "the plans have different patches");
    if (P->stream != Q->stream) return fail(SGIGA_ERR_ARG, "the plans must share a stream");
    const GridDesc& F = P->grids[0];
    for (int k = 0; k < d; ++k)
        if (F.lev[k] != F.lev[0]) return fail(SGIGA_ERR_ARG, "the full plan's component must be isotropic");
    const int J = F.lev[0];
    for (const GridDesc& g : Q->grids)
        for (int k = 0; k < d; ++k)
            if (g.lev[k] > J) return fail(SGIGA_ERR_ARG, "a component is finer than the full grid");
    CTPrec* C = new CTPrec();
    C->ct = Q;
    C->inner_tol = inner_tol;
    C->inner_max = inner_max;
    C->ncomp = (int)Q->grids.size();
    C->nfull = F.ndof;
    // 1D prolongations per (coarse level), all directions share them
    std::map<int, std::pair<long long, std::pair<int, int>>> mat_of;   // level -> (offset, (nf, nc))
    std::vector<double> mats;
    auto mat = [&](int lc) {
        auto it = mat_of.find(lc);
        if (it != mat_of.end()) return it->second;
        int nfi = 0, nci = 0;
        std::vector<double> M = ct_prolongation(P->p, P->r, lc, J, nfi, nci);
        const long long off = (long long)mats.size();
        mats.insert(mats.end(), M.begin(), M.end());
        return mat_of[lc] = std::make_pair(off, std::make_pair(nfi, nci));
    };
    std::vector<CTJob> jobs((size_t)2 * d * C->ncomp);
    std::vector<double> coef(C->ncomp);
    long long tmpoff = 0, maxtmp = 0, maxout = 0;
    for (int i = 0; i < C->ncomp; ++i) {
        const GridDesc& g = Q->grids[i];
        coef[i] = g.coeff;
        int nf[3] = {1, 1, 1}, ncv[3] = {1, 1, 1};
        long long moff[3] = {0, 0, 0};
        for (int k = 0; k < d; ++k) {
            auto m = mat(g.lev[k]);
            moff[k] = m.first;
            nf[k] = m.second.first;
            ncv[k] = m.second.second;
            if (nf[k] != F.n[k] || ncv[k] != g.n[k]) {
                delete C;
                return fail(SGIGA_ERR_ARG, "prolongation sizes differ from the plans' function counts");
            }
        }
        // restriction passes k = 0..d-1: shape goes from nf to ncv direction by direction
        long long cur = 0;   // input offset for pass 0: the full vector itself
        int shape[3] = {nf[0], d > 1 ? nf[1] : 1, d > 2 ? nf[2] : 1};
        for (int k = 0; k < d; ++k) {
            CTJob& jb = jobs[(size_t)k * C->ncomp + i];
            jb.in_off = k == 0 ? 0 : cur;
            for (int q = 0; q < 3; ++q) jb.n[q] = shape[q];
            jb.dir = k;
            jb.m_out = ncv[k];
            jb.pc = ncv[k];
            jb.trans = 1;
            jb.mat_off = moff[k];
            shape[k] = ncv[k];
            const long long sz = (long long)shape[0] * shape[1] * shape[2];
            jb.out_off = k == d - 1 ? g.dof_off : tmpoff;
            cur = jb.out_off;
            maxtmp = std::max(maxtmp, sz);
            maxout = std::max(maxout, sz);
        }
        // prolongation passes: ncv -> nf
        int sh2[3] = {ncv[0], d > 1 ? ncv[1] : 1, d > 2 ? ncv[2] : 1};
        cur = g.dof_off;
        for (int k = 0; k < d; ++k) {
            CTJob& jb = jobs[(size_t)(d + k) * C->ncomp + i];
            jb.in_off = cur;
            for (int q = 0; q < 3; ++q) jb.n[q] = sh2[q];
            jb.dir = k;
            jb.m_out = nf[k];
            jb.pc = ncv[k];
            jb.trans = 0;
            jb.mat_off = moff[k];
            sh2[k] = nf[k];
            const long long sz = (long long)sh2[0] * sh2[1] * sh2[2];
            jb.out_off = k == d - 1 ? (long long)i * C->nfull : tmpoff;
            cur = jb.out_off;
            maxtmp = std::max(maxtmp, sz);
            maxout = std::max(maxout, sz);
        }
        tmpoff += maxtmp;
        maxtmp = 0;
    }
    // each component's intermediates sit at its own offset in both buffers
    // (pass k reads buffer (k-1)&1 and writes k&1 at the same offset)
    C->maxout = maxout;
    cudaError_t e = cudaSuccess;
    auto dal = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, std::max<size_t>(bytes, 8));
    };
    dal((void**)&C->jobs, jobs.size() * sizeof(CTJob));
    dal((void**)&C->mats, mats.size() * 8);
    dal((void**)&C->tmp[0], (size_t)tmpoff * 8);
    dal((void**)&C->tmp[1], (size_t)tmpoff * 8);
    dal((void**)&C->Y, (size_t)C->ncomp * C->nfull * 8);
    dal((void**)&C->coef, coef.size() * 8);
    if (e == cudaSuccess) e = cudaMemcpy(C->jobs, jobs.data(), jobs.size() * sizeof(CTJob), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(C->mats, mats.data(), mats.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(C->coef, coef.data(), coef.size() * 8, cudaMemcpyHostToDevice);
    P->ct = C;
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_ct(P);
        return fail(SGIGA_ERR_NOMEM, "combination preconditioner buffers");
    }
    return SGIGA_OK;
}

int sgiga_ct_apply(sgiga_plan_t P, const double* r, double* z) {
    if (!P || !r || !z) return fail(SGIGA_ERR_ARG, "null argument");
    if (!P->ct) return fail(SGIGA_ERR_ARG, "no combination preconditioner attached (sgiga_ct_attach)");
    if (!is_device(r) || !is_device(z)) return fail(SGIGA_ERR_ARG, "r and z must be device buffers");
    P->ct->ct_only = true;
    const int rc = precond_ct(P, r, z, nullptr, P->d_t1, P->d_t2);
    P->ct->ct_only = false;
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(P->stream));
    return SGIGA_OK;
}

}  // extern "C"
