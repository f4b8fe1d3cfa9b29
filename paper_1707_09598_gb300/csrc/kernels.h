// Launchers of the CUDA kernels (defined in the *.cu files of this directory).
#pragma once
#include "internal.h"

#include <atomic>
#include <string>
#include <vector>

namespace sgiga {

// Record the message returned by sgiga_last_error() on this thread.
void set_last_error(const char* msg);

// Number of kernels this library has launched (diagnostic, process-wide).
extern std::atomic<long long> g_launches;
#define SGIGA_COUNT_LAUNCH() (::sgiga::g_launches.fetch_add(1, std::memory_order_relaxed))

struct DevPlan {
    int d, p, m, Q, ngrids, ntiles, ntabs, nchunks;
    long long ndof, nqp;
    const GridDesc* grids;
    const TileDesc* tiles;
    const int* sched;        // tile indices in launch (LPT) order
    const Table1D* tabs;
    const Eig1D* eigs;
    const Chunk* chunks;
    const Patch* patch;
    const double* knots;
    const double* bp;        // breakpoints per table
    const double* gauss;     // [Q] nodes on [-1,1] then [Q] weights
    double* xi;              // per-table Gauss points
    double* w;               // per-table Gauss weights (times h/2)
    double* R;               // per-table basis values [E][Q][p+1]
    double* dR;
    int* first;              // per-table first function of each element
    double* G;               // ncomp planes of nqp (tile-major)
    float* Gf;               // FP32 copy of G (mixed precision)
    float* Rf;               // FP32 copies of the basis tables
    float* dRf;
    const float* Uf;         // FP32 copies of U, U^T and dinv
    const float* Utf;
    const float* dinvf;
    double* mw;              // w |det J| (tile-major)
    double* rho;             // f w |det J| (tile-major)
    const double* U;         // eigenvectors, U[j][i] = component j of eigenvector i
    const double* Ut;        // their transposes (same offsets)
    const double* lam;
    const double* dinv;      // [ndof] 1 / sum_k lambda_{k,i_k} of every packed entry
    int* flags;              // [0] = geometry error, [1] = eval error
    const double* acoef;     // diffusion coefficient a(x_q) [nqp], natural order, or null (a = 1)
    size_t smem_op;          // dynamic shared bytes of the operator kernel
    int op_nth;              // threads per block of the FP32 3D operator kernel (256 or 128)
    int op_pf;               // FP32 3D operator: L2 prefetch per metric plane and tile, bytes (0: the whole
                             // segment, > 0: at most this many, < 0: none)
    int diag;                // every geometry plane off the diagonal is exactly zero
    const CompDesc* comps;   // components (CG systems); pieces are grids[]
    int ncomps;
    int multipatch;          // pieces alias interface functions (GridDesc)
    const Chunk* fdchunks;   // chunks of the preconditioner's local layout
    int nfdchunks;
    long long nfd;           // entries of that layout (= ndof for single-patch plans)
    double* gfull;           // boundary-coefficient arrays of the pieces (multi-patch)
    const SideDesc* sides;   // Dirichlet sides (multi-patch)
    int nsides;
    double* gdata;           // boundary data g at the sides' points
    double* gscratch;        // projection scratch
    const FDSeg* fdsegs;     // preconditioner level segments and their columns
    const long long* fdcb;
    const int* fdcs;
    const int* fdcc;
};

// Bounds checks of the checked build (-DSGIGA_CHECKED): a failed check sets
// flags[2], records the first failing site in flags[3] and skips the access;
// the default build compiles them away (SGIGA_GUARD is then `true`).
#ifdef SGIGA_CHECKED
#ifdef __CUDACC__
__device__ __forceinline__ bool sgiga_guard(int* flags, bool ok, int site) {
    if (!ok) {
        atomicOr(flags + 2, 1);
        atomicCAS(flags + 3, 0, site);
    }
    return ok;
}
#endif
#define SGIGA_GUARD(P, cond, site) sgiga_guard((P).flags, (cond), (site))
#else
#define SGIGA_GUARD(P, cond, site) true
#endif
// sites of the checks (flags[3])
enum { CHK_OP3_X = 1, CHK_OP3_Y = 2, CHK_OP3_G = 3, CHK_OP2_X = 4, CHK_OP2_Y = 5, CHK_FD_LEVEL = 6,
       CHK_FD_SMALL = 7 };

// boundary.cu (multi-patch Dirichlet data)
cudaError_t launch_boundary_points(const DevPlan& P, double* xb, cudaStream_t s);
cudaError_t launch_boundary_builtin(const DevPlan& P, int src, const double* xb, double* gdata, long long n,
                                    cudaStream_t s);
cudaError_t launch_boundary_project(const DevPlan& P, cudaStream_t s);
// eval.cu: values and physical gradients (2D)
cudaError_t launch_eval_grad(const DevPlan& P, const double* coeffs, const double* xi, const int* patch,
                             long long npts, double* ucomp, double* gcomp, int lifting, cudaStream_t s);
// basis.cu
cudaError_t launch_basis_tables(const DevPlan& P, int maxE, cudaStream_t s);
// eig.cu: eigenpairs of every job on the device (0, or -1 with msg set)
int gpu_generalized_eigen(int p, std::vector<EigJob>& jobs, const std::vector<double>& Kb,
                          const std::vector<double>& Mb, double* dU, double* dUt, double* dlam,
                          std::vector<double>& hlam, cudaStream_t s, std::string& msg);
// geometry.cu
cudaError_t launch_geometry(const DevPlan& P, cudaStream_t s);
// tile-major <-> natural layout of G and mw (re-tiling without re-evaluating the map)
cudaError_t launch_geometry_export(const DevPlan& P, double* Gn, double* mwn, cudaStream_t s);
cudaError_t launch_geometry_import(const DevPlan& P, double* Gn, double* mwn, cudaStream_t s);
cudaError_t launch_coef_features(const DevPlan& P, const double* feat, int nfeat, double amp, double* a,
                                 cudaStream_t s);
cudaError_t launch_offdiag_check(const DevPlan& P, int* flag, cudaStream_t s);
cudaError_t launch_qp_coords(const DevPlan& P, double* xq, cudaStream_t s);
cudaError_t launch_map_points(const DevPlan& P, const double* xi, const int* patch, long long npts, int npatch,
                              double* x, double* detj, cudaStream_t s);
cudaError_t launch_rhs_density_builtin(const DevPlan& P, int source, cudaStream_t s);
cudaError_t launch_source_qp(const DevPlan& P, int source, double* fout, cudaStream_t s);
cudaError_t launch_rhs_density_user(const DevPlan& P, const double* f_nat, cudaStream_t s);
// learned-scaling features: mode 0 writes tr(G_q), mode 1 d w_q (tile-major)
cudaError_t launch_feature_density(const DevPlan& P, double* out, int mode, cudaStream_t s);
cudaError_t launch_geometry_natural(const DevPlan& P, int g, const GridDesc& gh, double* Gnat,
                                    double* mwnat, cudaStream_t s);
// apply2.cu / apply3.cu: mode 0 = stiffness apply y += K x, mode 1 = load vector y += b
cudaError_t launch_op2(const DevPlan& P, const double* x, double* y, const int* active, int mode, cudaStream_t s);
cudaError_t launch_op3(const DevPlan& P, const double* x, double* y, const int* active, int mode, cudaStream_t s);
cudaError_t set_op2_smem(int p, size_t bytes);
cudaError_t launch_op2_f32(const DevPlan& P, const float* x, float* y, const int* active, cudaStream_t s);
cudaError_t launch_op3_f32(const DevPlan& P, const float* x, float* y, const int* active, cudaStream_t s);
cudaError_t set_op3_smem(int p, size_t bytes);
// resident blocks per SM of the FP32 3D operator kernel at the plan's settings
int op3_f32_resident(const DevPlan& Pl);
// fd.cu
// Work lists of one preconditioner pass: SMALL items, and LEVEL items by
// output-tile class (16, 32, 64 columns).
struct FDLists {
    const FDItem* small;
    int nsmall;
    const FDItem* lvl[3];
    int nlvl[3];
};
// Streams and events on which the kernels of one preconditioner pass (level
// GEMMs of each output-tile width and the small items; they write disjoint
// outputs) run as parallel branches forked from and joined to the caller's
// stream (in a captured graph: parallel nodes).
struct FDStreams {
    cudaStream_t aux[3];
    cudaEvent_t fork;
    cudaEvent_t join[3];
};
template <typename Real>
cudaError_t launch_fd_pass(const DevPlan& P, const FDLists& L, int dir, int forward, const Real* in, Real* out,
                           const int* active, cudaStream_t s, const FDStreams* fs = nullptr);
// shared-memory attributes of the preconditioner kernels (before their first launch)
cudaError_t fd_prepare();
template <typename Real>
cudaError_t launch_fd_gather(const DevPlan& P, const Real* r, Real* loc, const int* active, cudaStream_t s);
template <typename Real>
cudaError_t launch_fd_scatter(const DevPlan& P, const Real* loc, Real* z, const int* active, cudaStream_t s);
template <typename Real>
cudaError_t launch_fd_scale(const DevPlan& P, Real* z, const int* active, cudaStream_t s);
// vec.cu (Real = double or float; scalars and reductions in FP64)
template <typename Real>
cudaError_t launch_dot(const DevPlan& P, const Real* a, const Real* b, double* partial, double* out, cudaStream_t s);
template <typename Real>
cudaError_t launch_pcg_init(const DevPlan& P, const Real* b, Real* x, Real* r, double* partial, double* bb,
                            cudaStream_t s);
template <typename Real>
cudaError_t launch_pcg_update_xr(const DevPlan& P, Real* x, Real* r, const Real* p, const Real* q,
                                 const double* alpha, const int* active, double* partial, double* rr,
                                 cudaStream_t s);
template <typename Real>
cudaError_t launch_pcg_update_p(const DevPlan& P, Real* p, const Real* z, const double* beta, const int* active,
                                cudaStream_t s);
template <typename Real>
cudaError_t launch_copy(Real* dst, const Real* src, long long n, cudaStream_t s);
cudaError_t launch_pcg_alpha(const DevPlan& P, const double* rz, const double* pq, double* alpha,
                             const int* active, cudaStream_t s);
cudaError_t launch_pcg_beta(const DevPlan& P, double* rz, const double* rznew, const double* rzmid, double* beta,
                            cudaStream_t s);
cudaError_t launch_pcg_check(const DevPlan& P, const double* rr, const double* bb, double tol2, int* active,
                             int* iters, int* nactive, cudaStream_t s);
cudaError_t launch_pcg_start(const DevPlan& P, const double* bb, const int* outer, int* active, int* iters,
                             cudaStream_t s);
cudaError_t launch_loop_cond(int* counter, const int* nactive, int max_iter, cudaGraphConditionalHandle h,
                             cudaStream_t s);
cudaError_t launch_ir_down(const DevPlan& P, const double* r64, float* r32, const int* active, cudaStream_t s);
cudaError_t launch_ir_up(const DevPlan& P, double* x64, const float* d32, const int* active, cudaStream_t s);
cudaError_t launch_ir_up64(const DevPlan& P, double* x64, const double* d64, const int* active, cudaStream_t s);
cudaError_t launch_zero_active(const DevPlan& P, double* x, const int* active, cudaStream_t s);
cudaError_t launch_ir_residual(const DevPlan& P, const double* b, const double* q, double* r, const int* active,
                               double* partial, double* rr, cudaStream_t s);
cudaError_t launch_narrow(float* dst, const double* src, long long n, cudaStream_t s);
cudaError_t launch_widen_active(const DevPlan& P, double* dst, const float* src, const int* active, cudaStream_t s);
// net.cu (learned scaling network) and learned.cu
// conv.cu: the network's convolutions (32-channel activations as BF16 rows [N][32])
cudaError_t launch_conv_in(const DevPlan& P, const void* W, const float* b, const float* x, void* out,
                           cudaStream_t s);
cudaError_t launch_conv_out(const DevPlan& P, const void* W, const float* b, const void* A, float* y,
                            cudaStream_t s);
cudaError_t launch_convT_out(const DevPlan& P, const void* W, const float* dy, const void* act, void* dA,
                             cudaStream_t s);
cudaError_t launch_conv_mid(const DevPlan& P, const ConvTile* tiles, int ntiles, const void* Wt, const float* bias,
                            const void* X, const void* gate, int relu, void* out, cudaStream_t s);
cudaError_t launch_wgrad_mid(const DevPlan& P, const ConvTile* tiles, int ntiles, const void* X, const void* dZ,
                             float* dW, float* db, cudaStream_t s);
cudaError_t launch_wgrad_in(const DevPlan& P, const float* x, const void* dZ, float* dW, float* db, cudaStream_t s);
cudaError_t launch_wgrad_out(const DevPlan& P, const float* dy, const void* A, float* dW, float* db, cudaStream_t s);
cudaError_t launch_arrange_mid(const void* W, int T, void* Wf, void* Wb, cudaStream_t s);
cudaError_t launch_fill(float* x, float v, long long n, cudaStream_t s);
cudaError_t launch_log_ratio(const double* num, const double* den, float* out, long long n, cudaStream_t s);
cudaError_t launch_exp_scaling(const DevPlan& P, const float* y, const float* phi, int* ok, float* S,
                               cudaStream_t s);
cudaError_t launch_mul_active(const DevPlan& P, const float* S, const float* in, float* out, const int* active,
                              cudaStream_t s);
cudaError_t launch_pair_residual(const DevPlan& P, const float* S, const float* z1, const float* e, float* res,
                                 cudaStream_t s);
cudaError_t launch_pair_delta(const DevPlan& P, const float* S, const float* res, const double* rr, const double* ee,
                              const int* mask, double* cnt, float* delta, float* t2, double* lossacc, cudaStream_t s);
cudaError_t launch_pair_mask(int ng, const double* rr, const double* bb, double thr2, int* mask, cudaStream_t s);
cudaError_t launch_pair_grad(const DevPlan& P, const float* S, const float* delta, const float* z1, const float* r,
                             const float* z2, float weight, float* dls, cudaStream_t s);
cudaError_t launch_mask_scaled(const DevPlan& P, float* dy, const int* ok, const float* y, cudaStream_t s);
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, void* wb, const int* wmap, int n, float lr,
                        float b1, float b2, float eps, int step, cudaStream_t s);
cudaError_t launch_f2bf(const float* p, const int* wmap, void* wb, int n, cudaStream_t s);
cudaError_t launch_pair_store(const DevPlan& P, const double* r, const double* xstar, const double* x, float* rd,
                              float* ed, cudaStream_t s);

// eval.cu
cudaError_t launch_eval(const DevPlan& P, const double* coeffs, const double* xi, long long npts, double* vals,
                        int* first, double* ucomp, cudaStream_t s);
cudaError_t launch_combine(const DevPlan& P, const double* ucomp, long long npts, const double* coef,
                           double* u, cudaStream_t s);
// the same sum over ng value rows with caller-given coefficients (several plans)
cudaError_t launch_combine_n(int ng, const double* ucomp, long long npts, const double* coef, double* u,
                             cudaStream_t s);

}  // namespace sgiga
