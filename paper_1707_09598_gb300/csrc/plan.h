// Internal plan object and helpers shared by the host translation units.
#pragma once
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/sgiga.h"
#include "internal.h"
#include "kernels.h"

namespace sgiga {
struct Net;   // learned correction network (learned.cu)
struct CTPrec;   // combination technique as a preconditioner of a full solve (ct.cu)
}
using namespace sgiga;

// Records msg for sgiga_last_error() and returns code.
int fail(int code, const std::string& msg);

#define CUDA_TRY(expr)                                                                   \
    do {                                                                                 \
        cudaError_t _e = (expr);                                                         \
        if (_e != cudaSuccess) {                                                         \
            return fail(SGIGA_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
        }                                                                                \
    } while (0)

// A named range on the profiler's timeline for the life of the object (NVTX;
// without an attached tool the calls do nothing).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct sgiga_plan_s {
    sgiga_config cfg;
    int d, p, r, m, Q, ncomp;
    cudaStream_t stream;
    std::vector<GridDesc> grids;
    std::vector<TileDesc> tiles;
    std::vector<int> sched;
    std::vector<Table1D> tabs;
    std::map<std::pair<int, int>, int> tab_of;   // (dir, level) -> table
    std::vector<int> eig_of_tab;
    std::vector<Eig1D> eigs;
    std::vector<Chunk> chunks;
    std::vector<CompDesc> comps;         // components (CG systems); grids are their pieces
    std::vector<Chunk> fdchunks;         // chunks of the preconditioner's local layout
    std::vector<SideDesc> sides;         // Dirichlet sides (multi-patch)
    long long nfd = 0, ngf = 0, ngdata = 0, nscratch = 0;
    bool multipatch = false;
    bool lifting = false;                // boundary data set: the load vector subtracts K_IB g_B
    double* d_l0 = nullptr;              // preconditioner local layout (multi-patch)
    float* f_l0 = nullptr;
    std::vector<FDItem> fd[3];           // SMALL items per direction
    std::vector<FDItem> fdl[3][3];       // LEVEL items per direction and tile class (16, 32, 64 columns)
    std::vector<FDSeg> fdsegs;
    std::vector<long long> fdcb;
    std::vector<int> fdcs, fdcc;
    std::vector<double> knots, bp;
    Patch patch;                         // patch 0 (rational directions of the 1D tables)
    std::vector<Patch> patches;          // every geometry patch
    double* d_xb = nullptr;              // boundary data points [nbpts][2] (multi-patch)
    long long ndof = 0, nqp = 0, tab_entries = 0, ulen = 0, llen = 0;
    // set-up phases, seconds (sgiga_plan_times)
    double t_total = 0, t_host = 0, t_basis = 0, t_eigen = 0, t_fd = 0, t_geometry = 0, t_vectors = 0;
    double t_coefficient = 0, t_autotune = 0;
    int maxE = 1;
    int fd_ks = 32;             // contraction depth per preconditioner work item
    bool fd_grouped = false;    // preconditioner layout: level-grouped GEMMs, else per-piece items
    size_t smem = 0;
    std::vector<void*> allocs;
    DevPlan dp;
    FDItem* d_fd[3] = {nullptr, nullptr, nullptr};
    FDItem* d_fdl[3][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
    FDSeg* d_fdsegs = nullptr;
    long long* d_fdcb = nullptr;
    int* d_fdcs = nullptr;
    int* d_fdcc = nullptr;
    double *d_b = nullptr, *d_x = nullptr, *d_r = nullptr, *d_z = nullptr, *d_p = nullptr, *d_q = nullptr;
    double *d_t1 = nullptr, *d_t2 = nullptr, *d_partial = nullptr, *d_scal = nullptr, *d_coef = nullptr;
    int* d_active = nullptr;
    int* d_active_o = nullptr;  // outer (refinement) mask
    int* d_iters_o = nullptr;
    double* d_scal64o = nullptr;
    double* d_d = nullptr;      // FP64 correction of the refinement's FP64 fallback
    float *f_b = nullptr, *f_x = nullptr, *f_r = nullptr, *f_z = nullptr, *f_p = nullptr, *f_q = nullptr;
    float *f_t1 = nullptr, *f_t2 = nullptr;
    double inner_tol = 1e-5;
    int inner_max = 100;
    int last_inner_iters = 0;
    int* d_iters = nullptr;
    int* d_nactive = nullptr;
    int* h_nactive = nullptr;   // pinned
    void* stage = nullptr;      // device staging for host pointers
    double* acoef = nullptr;    // diffusion coefficient a(x_q) [nqp], natural order (null: a = 1)
    sgiga::Net* net = nullptr;  // learned correction network (allocated by sgiga_net_init)
    sgiga::CTPrec* ct = nullptr;  // two-level combination preconditioner (sgiga_ct_attach)
    bool net_ready = false;
    bool learned_off = false;   // set for the rest of a solve after a refinement step without progress
    bool use_graph = true;      // run CG loops as one captured graph with a device-side while node
    bool solve_fp64 = false;    // MIXED_FP32 plan whose solve the autotuner found faster as plain FP64 PCG
    bool fp64_fd32 = false;     // ... preconditioned by the FP32 FD (flexible CG), also found faster
    cudaStream_t own_stream = nullptr;   // capture/launch stream when the plan's stream is the legacy one
    FDStreams fds{};                     // branches of a preconditioner pass's kernels
    bool fds_ok = false;
    int* d_counter = nullptr;            // iteration counter of the captured loop
    double* d_eval_vals = nullptr;       // evaluation: basis values per (table, point)
    int* d_eval_first = nullptr;
    size_t eval_cap = 0;
    TileDesc* d_tiles = nullptr;         // current tile arrays (replaced by the autotuner)
    int* d_sched = nullptr;
    struct LoopGraph {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        double tol = -1.0;
        int max_iter = -1;
        const void* rhs = nullptr;
        const void* xbuf = nullptr;
        const int* outer = nullptr;
        bool flexible = false;
        bool learned = false;         // the body applies the learned preconditioner
        bool failed = false;
        long long body_kernels = 0;   // kernels per iteration of the captured body
    } loop64, loop32;
    size_t stage_bytes = 0;
};

template <typename T>
inline int dalloc(sgiga_plan_s* P, T** out, size_t count) {
    void* ptr = nullptr;
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SGIGA_ERR_NOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    P->allocs.push_back(ptr);
    *out = (T*)ptr;
    return SGIGA_OK;
}

template <typename T>
inline int upload(sgiga_plan_s* P, T** out, const std::vector<T>& v) {
    int rc = dalloc(P, out, v.size());
    if (rc) return rc;
    if (!v.empty()) CUDA_TRY(cudaMemcpy(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return SGIGA_OK;
}

// ---------------------------------------------------------------------------
// helpers for host-or-device pointers
// ---------------------------------------------------------------------------

inline bool is_device(const void* ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The address at which the current device reads a page-locked host buffer
// (cudaHostAlloc, or cudaHostRegister with mapping: the CUDA runtime reports
// it as devicePointer), or null for any other pointer.
inline const void* mapped_host_alias(const void* ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

inline int ensure_stage(sgiga_plan_s* P, size_t bytes) {
    if (P->stage_bytes >= bytes) return SGIGA_OK;
    if (P->stage) cudaFree(P->stage);
    P->stage = nullptr;
    P->stage_bytes = 0;
    cudaError_t e = cudaMalloc(&P->stage, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SGIGA_ERR_NOMEM, "staging buffer allocation failed");
    }
    P->stage_bytes = bytes;
    return SGIGA_OK;
}

inline int run_rhs_operator(sgiga_plan_s* P) {
    const DevPlan& D = P->dp;
    CUDA_TRY(cudaMemsetAsync(P->d_b, 0, (size_t)P->ndof * 8, P->stream));
    if (P->d == 3) CUDA_TRY(launch_op3(D, nullptr, P->d_b, nullptr, 1, P->stream));
    else CUDA_TRY(launch_op2(D, nullptr, P->d_b, nullptr, 1, P->stream));
    // nonhomogeneous Dirichlet data: b -= K_IB g_B (mode 2 reads the pieces'
    // boundary-coefficient arrays)
    if (P->lifting) CUDA_TRY(launch_op2(D, nullptr, P->d_b, nullptr, 2, P->stream));
    return SGIGA_OK;
}

inline int apply_op(sgiga_plan_s* P, const double* x, double* y, const int* active) {
    CUDA_TRY(cudaMemsetAsync(y, 0, (size_t)P->ndof * 8, P->stream));
    if (P->d == 3) CUDA_TRY(launch_op3(P->dp, x, y, active, 0, P->stream));
    else CUDA_TRY(launch_op2(P->dp, x, y, active, 0, P->stream));
    return SGIGA_OK;
}

inline int apply_op(sgiga_plan_s* P, const float* x, float* y, const int* active) {
    CUDA_TRY(cudaMemsetAsync(y, 0, (size_t)P->ndof * 4, P->stream));
    if (P->d == 3) CUDA_TRY(launch_op3_f32(P->dp, x, y, active, P->stream));
    else CUDA_TRY(launch_op2_f32(P->dp, x, y, active, P->stream));
    return SGIGA_OK;
}

// Work vectors of one precision.
template <typename Real>
struct Vecs {
    Real *x, *r, *z, *p, *q, *t1, *t2;
};

inline Vecs<double> vecs64(sgiga_plan_s* P) {
    return Vecs<double>{P->d_x, P->d_r, P->d_z, P->d_p, P->d_q, P->d_t1, P->d_t2};
}
inline Vecs<float> vecs32(sgiga_plan_s* P) {
    return Vecs<float>{P->f_x, P->f_r, P->f_z, P->f_p, P->f_q, P->f_t1, P->f_t2};
}

inline FDLists fd_lists(const sgiga_plan_s* P, int k) {
    FDLists L{};
    L.small = P->d_fd[k];
    L.nsmall = (int)P->fd[k].size();
    for (int t = 0; t < 3; ++t) {
        L.lvl[t] = P->d_fdl[k][t];
        L.nlvl[t] = (int)P->fdl[k][t].size();
    }
    return L;
}

template <typename Real>
inline int precond_fd(sgiga_plan_s* P, const Real* r, Real* z, const int* active, Real* t1, Real* t2) {
    const DevPlan& D = P->dp;
    cudaStream_t s = P->stream;
    if (P->cfg.precond == SGIGA_PRECOND_NONE) {
        CUDA_TRY(launch_copy(z, r, P->ndof, s));
        return SGIGA_OK;
    }
    const int d = P->d;
    const Real* in = r;
    Real* bufs[2] = {t1, t2};
    Real* loc = nullptr;
    int cur = 0;
    const size_t bytes = (size_t)P->nfd * sizeof(Real);
    if (P->multipatch) {   // additive Schwarz: gather each piece's kept functions
        loc = sizeof(Real) == 8 ? (Real*)P->d_l0 : (Real*)P->f_l0;
        CUDA_TRY(launch_fd_gather<Real>(D, r, loc, active, s));
        in = loc;
    }
    for (int k = 0; k < d; ++k) {
        Real* out = bufs[cur];
        CUDA_TRY(cudaMemsetAsync(out, 0, bytes, s));     // split contractions accumulate
        CUDA_TRY(launch_fd_pass<Real>(D, fd_lists(P, k), k, 1, in, out, active, s, P->fds_ok ? &P->fds : nullptr));
        in = out;
        cur ^= 1;
    }
    CUDA_TRY(launch_fd_scale<Real>(D, (Real*)in, active, s));
    for (int k = 0; k < d; ++k) {
        Real* out = (k == d - 1) ? (loc ? loc : z) : bufs[cur];
        CUDA_TRY(cudaMemsetAsync(out, 0, bytes, s));
        CUDA_TRY(launch_fd_pass<Real>(D, fd_lists(P, k), k, 0, in, out, active, s, P->fds_ok ? &P->fds : nullptr));
        in = out;
        cur ^= 1;
    }
    if (loc) {
        CUDA_TRY(cudaMemsetAsync(z, 0, (size_t)P->ndof * sizeof(Real), s));
        CUDA_TRY(launch_fd_scatter<Real>(D, loc, z, active, s));
    }
    return SGIGA_OK;
}

// Batched preconditioned CG on K_g x_g = rhs_g for the grids allowed by
// `outer` (all when null), each with its own scalars, until
// ||r_g|| <= tol ||rhs_g|| or max_iter iterations. Scalars: scal[0..6].
// Returns the number of grids still active (or a negative status).
// Learned preconditioner (learned.cu): z = S * FD(S * r),
// S = exp(-phi / 2 + 4 tanh(N(phi) / 4)), FP32.
namespace sgiga {
int precond_learned(sgiga_plan_s* P, const float* r, float* z, const int* active);
void free_net(sgiga_plan_s* P);
// FD(r) + sum_i c_i P_i K_i^{-1} P_i^T r (ct.cu)
int precond_ct(sgiga_plan_s* P, const double* r, double* z, const int* active, double* t1, double* t2);
void free_ct(sgiga_plan_s* P);
long long ct_inner_iterations(sgiga_plan_s* P, bool reset);
// the geometry planes changed: the network's features (and S) are stale
void net_invalidate_features(sgiga_plan_s* P);
// before a solve: S up to date (network evaluated once if needed)
int learned_prepare(sgiga_plan_s* P);
}

inline int precond_any(sgiga_plan_s* P, const double* r, double* z, const int* active, double* t1, double* t2) {
    if (P->ct) return precond_ct(P, r, z, active, t1, t2);
    if (P->fp64_fd32) {
        // FP32 FD as the preconditioner of FP64 CG (a MIXED_FP32 plan solving in
        // FP64): r narrowed, FD in FP32, z widened; the FP32 work vectors are
        // free while the solve runs in FP64
        CUDA_TRY(launch_narrow(P->f_r, r, P->ndof, P->stream));
        const int rc = precond_fd<float>(P, P->f_r, P->f_z, active, P->f_t1, P->f_t2);
        if (rc) return rc;
        CUDA_TRY(launch_widen_active(P->dp, z, P->f_z, active, P->stream));
        return SGIGA_OK;
    }
    return precond_fd<double>(P, r, z, active, t1, t2);
}
inline int precond_any(sgiga_plan_s* P, const float* r, float* z, const int* active, float* t1, float* t2) {
    if (P->cfg.precond == SGIGA_PRECOND_LEARNED && P->net_ready) return precond_learned(P, r, z, active);
    return precond_fd<float>(P, r, z, active, t1, t2);
}


inline void destroy_loop_graph(sgiga_plan_s::LoopGraph& L) {
    if (L.exec) cudaGraphExecDestroy(L.exec);
    if (L.graph) cudaGraphDestroy(L.graph);
    L.exec = nullptr;
    L.graph = nullptr;
}

// One CG iteration after the initialisation, in two parts (shared by the host
// loop and the captured graph body). A: q = K p, alpha, x/r update,
// convergence check; B: z = M r, beta, p update.
template <typename Real>
inline int pcg_body_a(sgiga_plan_s* P, Vecs<Real> v, double tol, int* active, int* iters, double* scal) {
    const DevPlan& D = P->dp;
    cudaStream_t s = P->stream;
    const int ng = (int)P->comps.size();
    double* bb = scal + 0 * ng;
    double* rz = scal + 1 * ng;
    double* pq = scal + 2 * ng;
    double* rr = scal + 3 * ng;
    double* alpha = scal + 4 * ng;
    int rc;
    if ((rc = apply_op(P, v.p, v.q, active))) return rc;
    CUDA_TRY(launch_dot<Real>(D, v.p, v.q, P->d_partial, pq, s));
    CUDA_TRY(launch_pcg_alpha(D, rz, pq, alpha, active, s));
    CUDA_TRY(launch_pcg_update_xr<Real>(D, v.x, v.r, v.p, v.q, alpha, active, P->d_partial, rr, s));
    CUDA_TRY(launch_pcg_check(D, rr, bb, tol * tol, active, iters, P->d_nactive, s));
    return SGIGA_OK;
}

template <typename Real>
inline int pcg_body_b(sgiga_plan_s* P, Vecs<Real> v, int* active, double* scal, bool flexible) {
    const DevPlan& D = P->dp;
    cudaStream_t s = P->stream;
    const int ng = (int)P->comps.size();
    double* rz = scal + 1 * ng;
    double* beta = scal + 5 * ng;
    double* rznew = scal + 6 * ng;
    double* rzmid = scal + 7 * ng;
    int rc;
    if (flexible) CUDA_TRY(launch_dot<Real>(D, v.r, v.z, P->d_partial, rzmid, s));
    if ((rc = precond_any(P, v.r, v.z, active, v.t1, v.t2))) return rc;
    CUDA_TRY(launch_dot<Real>(D, v.r, v.z, P->d_partial, rznew, s));
    CUDA_TRY(launch_pcg_beta(D, rz, rznew, flexible ? rzmid : nullptr, beta, s));
    CUDA_TRY(launch_pcg_update_p<Real>(D, v.p, v.z, beta, active, s));
    return SGIGA_OK;
}

// The CG loop as one graph: a while-conditional node whose body is one
// iteration and whose condition the last kernel of the body sets on the device.
// Built on first use and reused while (tol, max_iter, buffers) stay the same.
template <typename Real>
inline int pcg_graph_loop(sgiga_plan_s* P, sgiga_plan_s::LoopGraph& L, Vecs<Real> v, const void* rhs, double tol,
                          int max_iter, const int* outer, int* active, int* iters, double* scal, bool flexible) {
    cudaStream_t ls = P->stream ? P->stream : P->own_stream;
    const bool learned = sizeof(Real) == 4 && P->cfg.precond == SGIGA_PRECOND_LEARNED && P->net_ready &&
                         !P->learned_off;
    const bool same = L.exec && L.tol == tol && L.max_iter == max_iter && L.rhs == rhs && L.outer == outer &&
                      L.flexible == flexible && L.learned == learned && L.xbuf == (const void*)v.x;
    if (!same) {
        destroy_loop_graph(L);
        cudaGraph_t g = nullptr;
        CUDA_TRY(cudaGraphCreate(&g, 0));
        L.graph = g;
        cudaGraphConditionalHandle h;
        CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        CUDA_TRY(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
        cudaGraph_t body = np.conditional.phGraph_out[0];
        cudaStream_t saved = P->stream;
        P->stream = ls;
        cudaError_t e = cudaStreamBeginCaptureToGraph(ls, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        int rc = SGIGA_OK;
        const long long count0 = g_launches.load();
        if (e == cudaSuccess) {
            rc = pcg_body_a<Real>(P, v, tol, active, iters, scal);
            if (rc == SGIGA_OK) rc = pcg_body_b<Real>(P, v, active, scal, flexible);
            if (rc == SGIGA_OK) {
                cudaError_t e2 = launch_loop_cond(P->d_counter, P->d_nactive, max_iter, h, ls);
                if (e2 != cudaSuccess) rc = fail(SGIGA_ERR_CUDA, cudaGetErrorString(e2));
            }
            cudaGraph_t out = nullptr;
            cudaError_t e3 = cudaStreamEndCapture(ls, &out);
            if (rc == SGIGA_OK && e3 != cudaSuccess) rc = fail(SGIGA_ERR_CUDA, cudaGetErrorString(e3));
        } else {
            rc = fail(SGIGA_ERR_CUDA, cudaGetErrorString(e));
        }
        P->stream = saved;
        // capture only records the kernels; they are counted when the graph runs
        L.body_kernels = g_launches.load() - count0;
        g_launches.fetch_sub(L.body_kernels);
        if (rc) { cudaGetLastError(); destroy_loop_graph(L); return rc; }
        CUDA_TRY(cudaGraphInstantiate(&L.exec, g, 0));
        L.tol = tol;
        L.max_iter = max_iter;
        L.rhs = rhs;
        L.xbuf = v.x;
        L.outer = outer;
        L.flexible = flexible;
        L.learned = learned;
    }
    CUDA_TRY(cudaGraphLaunch(L.exec, ls));
    return SGIGA_OK;
}

// Called after every iteration of pcg (with the iteration index) when given;
// a nonzero return stops the solve with that status.
struct PcgHook {
    virtual int after_iteration(int it) = 0;
    virtual ~PcgHook() {}
};

template <typename Real>
inline int pcg(sgiga_plan_s* P, const Real* rhs, Vecs<Real> v, double tol, int max_iter, const int* outer,
               int* active, int* iters, double* scal, int* iters_run, PcgHook* hook = nullptr) {
    const DevPlan& D = P->dp;
    cudaStream_t s = P->stream;
    const int ng = (int)P->comps.size();
    double* bb = scal + 0 * ng;
    double* rz = scal + 1 * ng;
    // the learned preconditioner, and the FP32 FD inside FP64 CG, run in
    // flexible CG (Polak-Ribiere beta), which tolerates a preconditioner that
    // FP32 rounding leaves not exactly symmetric
    const bool flexible = (sizeof(Real) == 4 && P->cfg.precond == SGIGA_PRECOND_LEARNED && P->net_ready &&
                           !P->learned_off) ||
                          (sizeof(Real) == 8 && (P->fp64_fd32 || P->ct));
    auto init = [&]() -> int {
        CUDA_TRY(launch_pcg_init<Real>(D, rhs, v.x, v.r, P->d_partial, bb, s));
        CUDA_TRY(launch_pcg_start(D, bb, outer, active, iters, s));
        int rc = precond_any(P, v.r, v.z, active, v.t1, v.t2);
        if (rc) return rc;
        CUDA_TRY(launch_copy<Real>(v.p, v.z, P->ndof, s));
        CUDA_TRY(launch_dot<Real>(D, v.r, v.z, P->d_partial, rz, s));
        return SGIGA_OK;
    };
    int rc = init();
    if (rc) return rc;
    sgiga_plan_s::LoopGraph& L = sizeof(Real) == 8 ? P->loop64 : P->loop32;
    // (the combination preconditioner runs inner solves from the host: host loop)
    if (P->use_graph && !hook && !L.failed && !(sizeof(Real) == 8 && P->ct)) {
        // whole loop on the device: one graph launch, no host round trip per iteration
        CUDA_TRY(cudaMemsetAsync(P->d_counter, 0, sizeof(int), s));
        rc = pcg_graph_loop<Real>(P, L, v, rhs, tol, max_iter, outer, active, iters, scal, flexible);
        if (rc == SGIGA_OK) {
            CUDA_TRY(cudaMemcpyAsync(P->h_nactive, P->d_counter, sizeof(int), cudaMemcpyDeviceToHost,
                                     P->stream ? P->stream : P->own_stream));
            CUDA_TRY(cudaMemcpyAsync(P->h_nactive + 1, P->d_nactive, sizeof(int), cudaMemcpyDeviceToHost,
                                     P->stream ? P->stream : P->own_stream));
            CUDA_TRY(cudaStreamSynchronize(P->stream ? P->stream : P->own_stream));
            if (iters_run) *iters_run = P->h_nactive[0];
            g_launches.fetch_add((long long)P->h_nactive[0] * L.body_kernels);
            return P->h_nactive[1];
        }
        L.failed = true;   // this device/driver cannot run the captured loop: host loop from now on
        cudaGetLastError();
        if ((rc = init())) return rc;
    }
    int it = 0, nact = ng;
    for (it = 0; it < max_iter; ++it) {
        if ((rc = pcg_body_a<Real>(P, v, tol, active, iters, scal))) return rc;
        if (hook) {
            int hr = hook->after_iteration(it);
            if (hr) return hr;
        }
        CUDA_TRY(cudaMemcpyAsync(P->h_nactive, P->d_nactive, sizeof(int), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        nact = *P->h_nactive;
        if (nact == 0) { ++it; break; }
        if ((rc = pcg_body_b<Real>(P, v, active, scal, flexible))) return rc;
    }
    if (iters_run) *iters_run = it;
    return nact;
}

inline int solve_stats(sgiga_plan_s* P, const double* rr, const double* bb, const int* iters, int nact,
                       sgiga_solve_stats* stats, std::chrono::steady_clock::time_point t0) {
    if (!stats) return SGIGA_OK;
    const int ng = (int)P->comps.size();
    cudaStream_t s = P->stream;
    std::vector<double> hrr(ng), hbb(ng);
    std::vector<int> hit(ng);
    CUDA_TRY(cudaMemcpyAsync(hrr.data(), rr, ng * 8, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(hbb.data(), bb, ng * 8, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(hit.data(), iters, ng * 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    double mx = 0.0;
    int mi = 0;
    for (int g = 0; g < ng; ++g) {
        if (hbb[g] > 0) mx = std::max(mx, std::sqrt(hrr[g] / hbb[g]));
        mi = std::max(mi, hit[g]);
    }
    stats->iterations = mi;
    stats->converged = ng - nact;
    stats->max_rel_residual = mx;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    stats->inner_iterations = 0;
    stats->fallback = 0;
    return SGIGA_OK;
}

