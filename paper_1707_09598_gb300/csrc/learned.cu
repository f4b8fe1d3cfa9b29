// Host side of the learned scaling of the fast-diagonalisation preconditioner:
// features, the network's parameters, the scaled preconditioner used by the
// inner FP32 flexible CG, training-data generation from the solver's own CG
// iterates, the training loop (the library's forward, backward and Adam
// kernels), checkpoints, and the C ABI entry points.
//
// Preconditioner: M(r) = S * FD(S * r) (elementwise products),
// S = exp(-phi / 2 + 4 tanh(N(phi) / 4)) (the network corrects the
// network-free scaling c^(-1/2) by a factor within [e^-4, e^4]),
// phi_i = log c_i with c_i the local effective coefficient of DoF i,
//   c_i = sum_q R_i(xi_q) tr(G_q) / (d sum_q R_i(xi_q) w_q),
// the R_i-weighted mean of the trace of the Galerkin metric G_q relative to the
// parametric Laplacian (G_q = w_q I) that FD inverts exactly. S depends only on
// the operator, so M is a fixed symmetric positive definite operator: the
// network runs once per plan (and once per training step), not per iteration.
//
// Pairs. For a right-hand side b the FP64 FD-preconditioned CG is run twice:
// once to convergence for x*, once more recording after every iteration k the
// residual r_k and the error e_k = x* - x_k of every component. One recorded
// iteration is one training sample (all components at once).
//
// Loss of a sample: the mean over its counted components (those whose
// residual was above 1e-6 of their right-hand side when recorded) of
// ||M(r) - e||^2 / ||e||^2; its
// gradient with respect to log S_i is S_i (delta_i FD(S r)_i + r_i FD(S delta)_i)
// with delta = 2 (M(r) - e) / (||e||^2 ncounted) (FD symmetric).
#include <cstdio>
#include <random>

#include "plan.h"

namespace sgiga {

struct Net {
    int T = 0, np = 0, nw = 0;
    long long N = 0;
    long long oW[3], ob[3], obw[3];   // offsets of W_l and b_l in p; of W_l in the BF16 copy
    int cin[3] = {1, 32, 32}, cout[3] = {32, 32, 1};
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    void* wb = nullptr;               // BF16 weights
    int* wmap = nullptr;
    int step = 0;
    float *A0 = nullptr, *Y = nullptr, *dY = nullptr;
    void *A1 = nullptr, *A2 = nullptr, *dA1 = nullptr, *dA2 = nullptr;   // BF16 [N][32]
    void *wf = nullptr, *wbk = nullptr;   // layer 2's BF16 weights arranged for the tensor cores
    ConvTile* tiles = nullptr;            // 64-voxel tiles of the tensor-core convolutions
    int ntiles = 0;
    float *feat = nullptr;            // phi = log c (the network input)
    float *S = nullptr;               // scaling of the preconditioner
    float *tA = nullptr, *z1 = nullptr, *z2 = nullptr, *res = nullptr, *delta = nullptr;
    float *kres = nullptr, *ke = nullptr;   // K res, K e (energy-norm loss)
    int loss_norm = 0;                       // 0: Euclidean, 1: energy (K) norm
    double *dots = nullptr, *dots2 = nullptr, *lossacc = nullptr, *cnt = nullptr;
    int* ok = nullptr;
    int* masks = nullptr;             // per training sample: [ncomp] components that count
    bool feat_stale = true;           // the geometry planes changed since phi was computed
    bool s_stale = true;              // S must be recomputed from the network
    bool s_override = false;          // S was set by the caller (no network evaluation)
    float* data = nullptr;            // training pairs [S][2][N]
    double* bval = nullptr;           // validation right-hand side
    int nsamples = 0, capacity = 0;
    std::vector<void*> allocs;
};

static int nalloc(Net* n, void** out, size_t bytes) {
    cudaError_t e = cudaMalloc(out, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SGIGA_ERR_NOMEM, "network buffer allocation failed (" + std::to_string(bytes) + " bytes)");
    }
    n->allocs.push_back(*out);
    return SGIGA_OK;
}

void free_net(sgiga_plan_s* P) {
    if (!P || !P->net) return;
    for (void* a : P->net->allocs) cudaFree(a);
    delete P->net;
    P->net = nullptr;
    P->net_ready = false;
}

void net_invalidate_features(sgiga_plan_s* P) {
    if (P && P->net) {
        P->net->feat_stale = true;
        if (!P->net->s_override) P->net->s_stale = true;
    }
}

static int net_create(sgiga_plan_s* P) {
    if (P->net) return SGIGA_OK;
    Net* n = new Net();
    P->net = n;
    n->T = P->d == 3 ? 27 : 9;
    n->N = P->ndof;
    long long o = 0, ow = 0;
    for (int l = 0; l < 3; ++l) {
        n->oW[l] = o;
        n->obw[l] = ow;
        long long w = (long long)n->cout[l] * n->cin[l] * n->T;
        o += w;
        ow += w;
        n->ob[l] = o;
        o += n->cout[l];
    }
    n->np = (int)o;
    n->nw = (int)ow;
    const size_t N = (size_t)n->N, ng = P->comps.size();
    int rc;
    void** bufs1[] = {(void**)&n->A0, (void**)&n->Y, (void**)&n->dY, (void**)&n->feat, (void**)&n->S,
                      (void**)&n->tA, (void**)&n->z1, (void**)&n->z2, (void**)&n->res, (void**)&n->delta,
                      (void**)&n->kres, (void**)&n->ke};
    for (void** b : bufs1)
        if ((rc = nalloc(n, b, N * 4))) return rc;
    void** bufs32[] = {&n->A1, &n->A2, &n->dA1, &n->dA2};
    for (void** b : bufs32)
        if ((rc = nalloc(n, b, 32 * N * 2))) return rc;
    if ((rc = nalloc(n, &n->wf, (size_t)n->T * 32 * 32 * 2)) || (rc = nalloc(n, &n->wbk, (size_t)n->T * 32 * 32 * 2)))
        return rc;
    std::vector<ConvTile> tl;
    for (size_t c = 0; c < P->chunks.size(); ++c)
        for (int o = 0; o < P->chunks[c].len; o += 64) tl.push_back(ConvTile{(int)c, o});
    n->ntiles = (int)tl.size();
    if ((rc = nalloc(n, (void**)&n->tiles, tl.size() * sizeof(ConvTile)))) return rc;
    CUDA_TRY(cudaMemcpy(n->tiles, tl.data(), tl.size() * sizeof(ConvTile), cudaMemcpyHostToDevice));
    if ((rc = nalloc(n, (void**)&n->p, n->np * 4)) || (rc = nalloc(n, (void**)&n->g, n->np * 4)) ||
        (rc = nalloc(n, (void**)&n->m, n->np * 4)) || (rc = nalloc(n, (void**)&n->v, n->np * 4)) ||
        (rc = nalloc(n, &n->wb, n->nw * 2)) || (rc = nalloc(n, (void**)&n->wmap, n->np * 4)) ||
        (rc = nalloc(n, (void**)&n->dots, ng * 8)) || (rc = nalloc(n, (void**)&n->dots2, ng * 8)) ||
        (rc = nalloc(n, (void**)&n->lossacc, 16)) || (rc = nalloc(n, (void**)&n->ok, ng * 4)) ||
        (rc = nalloc(n, (void**)&n->cnt, 8)))
        return rc;
    std::vector<int> wmap(n->np, -1);
    for (int l = 0; l < 3; ++l) {
        long long w = (long long)n->cout[l] * n->cin[l] * n->T;
        for (long long i = 0; i < w; ++i) wmap[n->oW[l] + i] = (int)(n->obw[l] + i);
    }
    CUDA_TRY(cudaMemcpy(n->wmap, wmap.data(), wmap.size() * 4, cudaMemcpyHostToDevice));
    return SGIGA_OK;
}

// phi = log c on the device: two load-vector launches (transposed sum
// factorisation, the load vector's kernel) with the densities tr(G_q) and
// d w_q, then their log ratio.
static int net_features(sgiga_plan_s* P) {
    Net* n = P->net;
    if (!n->feat_stale) return SGIGA_OK;
    cudaStream_t s = P->stream;
    const size_t nd = (size_t)P->ndof;
    double *rho = nullptr, *num = nullptr, *den = nullptr;
    if (cudaMalloc(&rho, (size_t)P->nqp * 8) != cudaSuccess || cudaMalloc(&num, nd * 8) != cudaSuccess ||
        cudaMalloc(&den, nd * 8) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(rho);
        cudaFree(num);
        return fail(SGIGA_ERR_NOMEM, "feature buffers");
    }
    DevPlan D = P->dp;
    D.rho = rho;
    int rc = SGIGA_OK;
    for (int mode = 0; mode < 2 && rc == SGIGA_OK; ++mode) {
        double* out = mode == 0 ? num : den;
        cudaError_t e = launch_feature_density(D, rho, mode, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(out, 0, nd * 8, s);
        if (e == cudaSuccess) e = P->d == 3 ? launch_op3(D, nullptr, out, nullptr, 1, s)
                                            : launch_op2(D, nullptr, out, nullptr, 1, s);
        if (e != cudaSuccess) rc = fail(SGIGA_ERR_CUDA, std::string("features: ") + cudaGetErrorString(e));
    }
    if (rc == SGIGA_OK) {
        cudaError_t e = launch_log_ratio(num, den, n->feat, P->ndof, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = fail(SGIGA_ERR_CUDA, std::string("features: ") + cudaGetErrorString(e));
    }
    cudaFree(rho);
    cudaFree(num);
    cudaFree(den);
    if (rc == SGIGA_OK) n->feat_stale = false;
    return rc;
}

static const void* wl(const Net* n, int l) { return (const char*)n->wb + n->obw[l] * 2; }

static int net_upload(sgiga_plan_s* P, const std::vector<float>& host) {
    Net* n = P->net;
    CUDA_TRY(cudaMemcpy(n->p, host.data(), n->np * 4, cudaMemcpyHostToDevice));
    CUDA_TRY(launch_f2bf(n->p, n->wmap, n->wb, n->np, P->stream));
    CUDA_TRY(launch_arrange_mid(wl(n, 1), n->T, n->wf, n->wbk, P->stream));
    CUDA_TRY(cudaStreamSynchronize(P->stream));
    n->s_stale = true;
    n->s_override = false;
    return SGIGA_OK;
}


// forward: A0 (1 channel) -> A1 -> A2 (BF16 rows) -> Y
static int net_forward(sgiga_plan_s* P) {
    Net* n = P->net;
    const DevPlan& D = P->dp;
    cudaStream_t s = P->stream;
    CUDA_TRY(launch_conv_in(D, wl(n, 0), n->p + n->ob[0], n->A0, n->A1, s));
    CUDA_TRY(launch_conv_mid(D, n->tiles, n->ntiles, n->wf, n->p + n->ob[1], n->A1, nullptr, 1, n->A2, s));
    CUDA_TRY(launch_conv_out(D, wl(n, 2), n->p + n->ob[2], n->A2, n->Y, s));
    return SGIGA_OK;
}

// backward from dY: gradients of every parameter into g (cleared first); the
// data gradients pass the ReLUs through the forward activations
static int net_backward(sgiga_plan_s* P) {
    Net* n = P->net;
    const DevPlan& D = P->dp;
    cudaStream_t s = P->stream;
    CUDA_TRY(cudaMemsetAsync(n->g, 0, n->np * 4, s));
    CUDA_TRY(launch_wgrad_out(D, n->dY, n->A2, n->g + n->oW[2], n->g + n->ob[2], s));
    CUDA_TRY(launch_convT_out(D, wl(n, 2), n->dY, n->A2, n->dA2, s));
    CUDA_TRY(launch_wgrad_mid(D, n->tiles, n->ntiles, n->A1, n->dA2, n->g + n->oW[1], n->g + n->ob[1], s));
    CUDA_TRY(launch_conv_mid(D, n->tiles, n->ntiles, n->wbk, nullptr, n->dA2, n->A1, 0, n->dA1, s));
    CUDA_TRY(launch_wgrad_in(D, n->A0, n->dA1, n->g + n->oW[0], n->g + n->ob[0], s));
    return SGIGA_OK;
}

// S = exp(-phi / 2 + 4 tanh(N(phi) / 4)); a component whose network output is
// not finite keeps S = 1 there (plain FD for that component).
static int net_scaling(sgiga_plan_s* P) {
    Net* n = P->net;
    int rc;
    if ((rc = net_features(P))) return rc;
    CUDA_TRY(launch_copy<float>(n->A0, n->feat, n->N, P->stream));
    if ((rc = net_forward(P))) return rc;
    CUDA_TRY(launch_exp_scaling(P->dp, n->Y, n->feat, n->ok, n->S, P->stream));
    return SGIGA_OK;
}

static int ensure_scaling(sgiga_plan_s* P) {
    Net* n = P->net;
    if (!n || n->s_override || !n->s_stale) return SGIGA_OK;
    int rc = net_scaling(P);
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(P->stream));
    n->s_stale = false;
    return SGIGA_OK;
}

int learned_prepare(sgiga_plan_s* P) {
    if (P->cfg.precond != SGIGA_PRECOND_LEARNED || !P->net_ready) return SGIGA_OK;
    return ensure_scaling(P);
}

int precond_learned(sgiga_plan_s* P, const float* r, float* z, const int* active) {
    Net* n = P->net;
    if (P->learned_off) return precond_fd<float>(P, r, z, active, P->f_t1, P->f_t2);
    const DevPlan& D = P->dp;
    cudaStream_t s = P->stream;
    CUDA_TRY(launch_mul_active(D, n->S, r, n->tA, active, s));
    int rc = precond_fd<float>(P, n->tA, z, active, P->f_t1, P->f_t2);
    if (rc) return rc;
    CUDA_TRY(launch_mul_active(D, n->S, z, z, active, s));
    return SGIGA_OK;
}

// Loss of the pair (r, e) at the current S (accumulated into n->lossacc[0]
// as the mean over the components that count: mask, or all when null) and
// its gradient with respect to log S added to dls scaled by `weight`.
static int pair_loss_grad(sgiga_plan_s* P, const float* r, const float* e, const int* mask, float* dls,
                          float weight) {
    Net* n = P->net;
    const DevPlan& D = P->dp;
    cudaStream_t s = P->stream;
    int rc;
    CUDA_TRY(launch_mul_active(D, n->S, r, n->tA, nullptr, s));
    if ((rc = precond_fd<float>(P, n->tA, n->z1, nullptr, P->f_t1, P->f_t2))) return rc;
    CUDA_TRY(launch_pair_residual(D, n->S, n->z1, e, n->res, s));          // res = S z1 - e
    // the norm of the loss: Euclidean, or the energy norm (K = the plan's FP32
    // operator): L = res^T K res / e^T K e, delta = 2 K res / (e^T K e ncounted)
    const float* kr = n->res;
    const float* kee = e;
    if (n->loss_norm == 1) {
        if ((rc = apply_op(P, n->res, n->kres, nullptr)) || (rc = apply_op(P, e, n->ke, nullptr))) return rc;
        kr = n->kres;
        kee = n->ke;
    }
    CUDA_TRY(launch_dot<float>(D, n->res, kr, P->d_partial, n->dots, s));
    CUDA_TRY(launch_dot<float>(D, e, kee, P->d_partial, n->dots2, s));
    CUDA_TRY(launch_pair_delta(D, n->S, kr, n->dots, n->dots2, mask, n->cnt, n->delta, n->tA, n->lossacc, s));
    if ((rc = precond_fd<float>(P, n->tA, n->z2, nullptr, P->f_t1, P->f_t2))) return rc;
    CUDA_TRY(launch_pair_grad(D, n->S, n->delta, n->z1, r, n->z2, weight, dls, s));
    return SGIGA_OK;
}

// Mean loss over the recorded samples at the current S (no update).
static int dataset_loss(sgiga_plan_s* P, double* out) {
    Net* n = P->net;
    cudaStream_t s = P->stream;
    CUDA_TRY(cudaMemsetAsync(n->lossacc, 0, 16, s));
    for (int k = 0; k < n->nsamples; ++k) {
        const float* r = n->data + (size_t)k * 2 * n->N;
        int rc = pair_loss_grad(P, r, r + n->N, n->masks + (size_t)k * P->comps.size(), n->dY, 0.0f);
        if (rc) return rc;
    }
    double h[2];
    CUDA_TRY(cudaMemcpyAsync(h, n->lossacc, 16, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    *out = n->nsamples ? h[0] / n->nsamples : 0.0;
    return SGIGA_OK;
}

// Records (r_k, x* - x_k) of every CG iterate into the next dataset slot.
struct RecordHook : PcgHook {
    sgiga_plan_s* P;
    const double* xstar;
    int limit;
    int after_iteration(int it) override {
        Net* n = P->net;
        if (n->nsamples >= n->capacity || it >= limit) return 0;
        float* rd = n->data + (size_t)n->nsamples * 2 * n->N;
        cudaError_t e = launch_pair_store(P->dp, P->d_r, xstar, P->d_x, rd, rd + n->N, P->stream);
        // the components that count: not yet at 1e-6 of their right-hand side
        // (x* is converged to 1e-10; below 1e-6 the recorded error would carry
        // x*'s own error, and a converged component's error is rounding noise)
        const int ng = (int)P->comps.size();
        if (e == cudaSuccess)
            e = launch_pair_mask(ng, P->d_scal + 3 * ng, P->d_scal, 1e-12, n->masks + (size_t)n->nsamples * ng,
                                 P->stream);
        if (e != cudaSuccess) return fail(SGIGA_ERR_CUDA, cudaGetErrorString(e));
        n->nsamples++;
        return 0;
    }
};

static int needs_net(sgiga_plan_t P) {
    if (!P) return fail(SGIGA_ERR_ARG, "null argument");
    if (P->cfg.precision != SGIGA_PREC_MIXED_FP32)
        return fail(SGIGA_ERR_ARG, "the network needs a SGIGA_PREC_MIXED_FP32 plan (FP32 preconditioner data)");
    if (P->multipatch) return fail(SGIGA_ERR_ARG, "the learned preconditioner needs a single-patch domain");
    return SGIGA_OK;
}

}  // namespace sgiga

using namespace sgiga;

extern "C" {

int sgiga_net_init(sgiga_plan_t P, unsigned seed) {
    int rc = needs_net(P);
    if (rc) return rc;
    if ((rc = net_create(P))) return rc;
    Net* n = P->net;
    std::mt19937_64 rng(seed);
    std::vector<float> h(n->np, 0.0f);
    for (int l = 0; l < 3; ++l) {
        // Kaiming-uniform for ReLU layers; the last layer starts at zero, so
        // that the untrained N is 0 and S the network-free scaling c^(-1/2)
        const double fan = (double)n->cin[l] * n->T;
        const double b = std::sqrt(6.0 / fan) * (l == 2 ? 0.0 : 1.0);
        std::uniform_real_distribution<double> U(-b, b);
        long long w = (long long)n->cout[l] * n->cin[l] * n->T;
        for (long long i = 0; i < w; ++i) h[n->oW[l] + i] = (float)U(rng);
    }
    if ((rc = net_upload(P, h))) return rc;
    CUDA_TRY(cudaMemset(n->m, 0, n->np * 4));
    CUDA_TRY(cudaMemset(n->v, 0, n->np * 4));
    n->step = 0;
    P->net_ready = true;
    return SGIGA_OK;
}

int sgiga_net_num_params(sgiga_plan_t P) {
    if (!P || !P->net) return fail(SGIGA_ERR_ARG, "no network (call sgiga_net_init)");
    return P->net->np;
}

int sgiga_net_get_params(sgiga_plan_t P, float* host) {
    if (!P || !P->net || !host) return fail(SGIGA_ERR_ARG, "no network or null argument");
    CUDA_TRY(cudaMemcpy(host, P->net->p, P->net->np * 4, cudaMemcpyDeviceToHost));
    return SGIGA_OK;
}

int sgiga_net_set_params(sgiga_plan_t P, const float* host) {
    if (!P || !P->net || !host) return fail(SGIGA_ERR_ARG, "no network or null argument");
    std::vector<float> h(host, host + P->net->np);
    return net_upload(P, h);
}

int sgiga_net_forward(sgiga_plan_t P, const float* in, float* out) {
    if (!P || !P->net || !in || !out) return fail(SGIGA_ERR_ARG, "no network or null argument");
    if (!is_device(in) || !is_device(out)) return fail(SGIGA_ERR_ARG, "in and out must be device buffers");
    Net* n = P->net;
    CUDA_TRY(launch_copy<float>(n->A0, in, n->N, P->stream));
    int rc = net_forward(P);
    if (rc) return rc;
    CUDA_TRY(launch_copy<float>(out, n->Y, n->N, P->stream));
    CUDA_TRY(cudaStreamSynchronize(P->stream));
    return SGIGA_OK;
}

int sgiga_net_backward(sgiga_plan_t P, const float* in, const float* dy, float* grad_host) {
    if (!P || !P->net || !in || !dy || !grad_host) return fail(SGIGA_ERR_ARG, "no network or null argument");
    if (!is_device(in) || !is_device(dy)) return fail(SGIGA_ERR_ARG, "in and dy must be device buffers");
    Net* n = P->net;
    CUDA_TRY(launch_copy<float>(n->A0, in, n->N, P->stream));
    int rc = net_forward(P);
    if (rc) return rc;
    CUDA_TRY(launch_copy<float>(n->dY, dy, n->N, P->stream));
    if ((rc = net_backward(P))) return rc;
    CUDA_TRY(cudaMemcpyAsync(grad_host, n->g, n->np * 4, cudaMemcpyDeviceToHost, P->stream));
    CUDA_TRY(cudaStreamSynchronize(P->stream));
    // the activations no longer belong to the features
    n->s_stale = !n->s_override;
    return SGIGA_OK;
}

int sgiga_net_features(sgiga_plan_t P, float* phi) {
    int rc = needs_net(P);
    if (rc) return rc;
    if (!phi) return fail(SGIGA_ERR_ARG, "null argument");
    if ((rc = net_create(P)) || (rc = net_features(P))) return rc;
    CUDA_TRY(cudaMemcpyAsync(phi, P->net->feat, (size_t)P->ndof * 4, cudaMemcpyDefault, P->stream));
    CUDA_TRY(cudaStreamSynchronize(P->stream));
    return SGIGA_OK;
}

int sgiga_net_scaling(sgiga_plan_t P, float* S) {
    if (!P || !P->net || !P->net_ready || !S) return fail(SGIGA_ERR_ARG, "no network or null argument");
    int rc = ensure_scaling(P);
    if (rc) return rc;
    CUDA_TRY(cudaMemcpyAsync(S, P->net->S, (size_t)P->ndof * 4, cudaMemcpyDefault, P->stream));
    CUDA_TRY(cudaStreamSynchronize(P->stream));
    return SGIGA_OK;
}

int sgiga_net_set_scaling(sgiga_plan_t P, const float* S) {
    int rc = needs_net(P);
    if (rc) return rc;
    if (!S) return fail(SGIGA_ERR_ARG, "null argument");
    if ((rc = net_create(P))) return rc;
    CUDA_TRY(cudaMemcpyAsync(P->net->S, S, (size_t)P->ndof * 4, cudaMemcpyDefault, P->stream));
    CUDA_TRY(cudaStreamSynchronize(P->stream));
    P->net->s_override = true;
    P->net->s_stale = false;
    P->net_ready = true;
    return SGIGA_OK;
}

int sgiga_net_set_loss_norm(sgiga_plan_t P, int norm) {
    if (!P || !P->net) return fail(SGIGA_ERR_ARG, "no network (call sgiga_net_init)");
    if (norm != 0 && norm != 1) return fail(SGIGA_ERR_ARG, "norm must be 0 (Euclidean) or 1 (energy)");
    P->net->loss_norm = norm;
    return SGIGA_OK;
}

int sgiga_net_loss_grad(sgiga_plan_t P, const float* r, const float* e, double* loss, float* grad) {
    if (!P || !P->net || !P->net_ready || !r || !e || !loss || !grad)
        return fail(SGIGA_ERR_ARG, "no network or null argument");
    if (!is_device(r) || !is_device(e) || !is_device(grad))
        return fail(SGIGA_ERR_ARG, "r, e and grad must be device buffers");
    int rc = ensure_scaling(P);
    if (rc) return rc;
    Net* n = P->net;
    cudaStream_t s = P->stream;
    CUDA_TRY(cudaMemsetAsync(n->lossacc, 0, 16, s));
    CUDA_TRY(cudaMemsetAsync(grad, 0, (size_t)P->ndof * 4, s));
    if ((rc = pair_loss_grad(P, r, e, nullptr, grad, 1.0f))) return rc;
    CUDA_TRY(cudaMemcpyAsync(loss, n->lossacc, 8, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return SGIGA_OK;
}

// Total inner FP32 flexible-CG iterations of the plan's own solve (FP64
// refinement to a relative residual of 1e-8, the plan's inner tolerance) with
// the network's current scaling on the validation right-hand side; 1000 more
// when it does not converge in 50 refinement steps.
static int validation_iters(sgiga_plan_s* P, const double* bval, int* iters) {
    Net* n = P->net;
    CUDA_TRY(cudaMemcpyAsync(P->d_b, bval, (size_t)n->N * 8, cudaMemcpyDeviceToDevice, P->stream));
    n->s_stale = true;
    n->s_override = false;
    sgiga_solve_stats st{};
    const int rc = sgiga_solve(P, 1e-8, 50, &st);
    if (rc != SGIGA_OK && rc != SGIGA_ERR_NOT_CONVERGED) return rc;
    *iters = st.inner_iterations + (rc == SGIGA_OK ? 0 : 1000);
    return SGIGA_OK;
}

int sgiga_train_net(sgiga_plan_t P, const sgiga_train_cfg* cfg, sgiga_train_stats* stats) {
    NvtxRange nvtx_("sgiga_train_net");
    if (!P || !cfg) return fail(SGIGA_ERR_ARG, "null argument");
    if (!P->net_ready || !P->net) return fail(SGIGA_ERR_ARG, "no network (call sgiga_net_init)");
    if (cfg->target_pairs < 1 || cfg->epochs < 1 || !(cfg->lr > 0) || cfg->batch < 0)
        return fail(SGIGA_ERR_ARG, "bad training config");
    auto t0 = std::chrono::steady_clock::now();
    Net* n = P->net;
    const DevPlan& D = P->dp;
    cudaStream_t s = P->stream;
    const int ng = (int)P->comps.size();
    const long long N = n->N;
    int rc;
    if ((rc = net_features(P))) return rc;
    // 1. data: samples of all components, ceil(target_pairs / ncomponents) of them
    const int S = (cfg->target_pairs + ng - 1) / ng;
    if (n->capacity < S) {
        if (n->data) { cudaFree(n->data); n->allocs.erase(std::find(n->allocs.begin(), n->allocs.end(), (void*)n->data)); }
        n->data = nullptr;
        n->capacity = 0;
        if (n->masks) { cudaFree(n->masks); n->allocs.erase(std::find(n->allocs.begin(), n->allocs.end(), (void*)n->masks)); }
        n->masks = nullptr;
        if ((rc = nalloc(n, (void**)&n->data, (size_t)S * 2 * N * 4)) ||
            (rc = nalloc(n, (void**)&n->masks, (size_t)S * ng * 4)))
            return rc;
        n->capacity = S;
    }
    n->nsamples = 0;
    double* xstar = nullptr;
    if (cudaMalloc(&xstar, (size_t)N * 8) != cudaSuccess) { cudaGetLastError(); return fail(SGIGA_ERR_NOMEM, "x* buffer"); }
    std::vector<double> hb(N);
    std::mt19937_64 rng(cfg->seed);
    std::normal_distribution<double> gauss(0.0, 1.0);
    const int per_rhs = std::max(1, cfg->max_iter_record);
    int nrhs = 0;
    const int saved_precond = P->cfg.precond;
    P->cfg.precond = SGIGA_PRECOND_FD;    // data come from plain FD-preconditioned CG
    while (n->nsamples < S && nrhs < 10000) {
        for (long long i = 0; i < N; ++i) hb[i] = gauss(rng);
        if (cudaMemcpy(P->d_b, hb.data(), N * 8, cudaMemcpyHostToDevice) != cudaSuccess) { rc = SGIGA_ERR_CUDA; break; }
        if (nrhs % 2 == 1) {
            // smoother right-hand side: b = K FD(xi), xi random (the error FD(xi) is smooth)
            if ((rc = precond_fd<double>(P, P->d_b, P->d_z, nullptr, P->d_t1, P->d_t2))) break;
            if ((rc = apply_op(P, P->d_z, P->d_b, nullptr))) break;
        }
        int it = 0;
        int nact = pcg<double>(P, P->d_b, vecs64(P), 1e-10, 500, nullptr, P->d_active, P->d_iters, P->d_scal, &it);
        if (nact < 0) { rc = nact; break; }
        if (cudaMemcpyAsync(xstar, P->d_x, N * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess) { rc = SGIGA_ERR_CUDA; break; }
        RecordHook hook;
        hook.P = P;
        hook.xstar = xstar;
        hook.limit = per_rhs;
        nact = pcg<double>(P, P->d_b, vecs64(P), 1e-10, per_rhs, nullptr, P->d_active, P->d_iters, P->d_scal, &it,
                           &hook);
        if (nact < 0) { rc = nact; break; }
        ++nrhs;
    }
    // validation right-hand side, held out of the pairs: b = K FD(xi) with its
    // own seed
    if (rc == SGIGA_OK && !n->bval) rc = nalloc(n, (void**)&n->bval, (size_t)N * 8);
    if (rc == SGIGA_OK) {
        std::mt19937_64 vrng(cfg->seed ^ 0x5DEECE66DULL);
        for (long long i = 0; i < N; ++i) hb[i] = gauss(vrng);
        if (cudaMemcpy(P->d_b, hb.data(), N * 8, cudaMemcpyHostToDevice) != cudaSuccess) rc = SGIGA_ERR_CUDA;
        if (rc == SGIGA_OK) rc = precond_fd<double>(P, P->d_b, P->d_z, nullptr, P->d_t1, P->d_t2);
        if (rc == SGIGA_OK) rc = apply_op(P, P->d_z, n->bval, nullptr);
    }
    P->cfg.precond = saved_precond;
    cudaFree(xstar);
    if (rc) return rc;
    CUDA_TRY(cudaMemsetAsync(P->d_b, 0, N * 8, s));   // the load vector was overwritten
    // 2. training: minibatches of `batch` samples, one network evaluation and
    // one Adam step per minibatch; the learning rate ramps up linearly over the
    // first 50 steps (Adam's first steps move every weight by about lr in the
    // same direction). Kept: the parameters (after an epoch, or the initial
    // ones) with which the plan's solve of the validation right-hand side
    // needs the fewest inner iterations, the earliest among equals: a lower
    // loss on the pairs alone does not mean fewer CG iterations
    const int B = cfg->batch > 0 ? cfg->batch : 2;
    n->loss_norm = cfg->loss_norm == 1 ? 1 : 0;
    n->s_override = false;
    std::vector<int> order(n->nsamples);
    for (int i = 0; i < n->nsamples; ++i) order[i] = i;
    double loss_fd = 0.0, loss_init = 0.0;
    CUDA_TRY(launch_fill(n->S, 1.0f, N, s));                  // S = 1: plain FD
    if ((rc = dataset_loss(P, &loss_fd))) return rc;
    if ((rc = net_scaling(P)) || (rc = dataset_loss(P, &loss_init))) return rc;
    int val_init = 0;
    if ((rc = validation_iters(P, n->bval, &val_init))) return rc;
    double first = 0.0, last = 0.0, best = loss_init;
    int best_epoch = -1, best_val = val_init;
    std::vector<double> ep_loss;
    std::vector<float> best_p(n->np);
    CUDA_TRY(cudaMemcpy(best_p.data(), n->p, n->np * 4, cudaMemcpyDeviceToHost));
    int steps = 0;
    for (int ep = 0; ep < cfg->epochs; ++ep) {
        std::shuffle(order.begin(), order.end(), rng);
        CUDA_TRY(cudaMemsetAsync(n->lossacc, 0, 16, s));
        for (int k0 = 0; k0 < n->nsamples; k0 += B) {
            const int nb = std::min(B, n->nsamples - k0);
            if ((rc = net_scaling(P))) return rc;             // S from the current parameters (A0..A2 kept)
            CUDA_TRY(cudaMemsetAsync(n->dY, 0, N * 4, s));
            for (int k = k0; k < k0 + nb; ++k) {
                const float* r = n->data + (size_t)order[k] * 2 * N;
                if ((rc = pair_loss_grad(P, r, r + N, n->masks + (size_t)order[k] * ng, n->dY, 1.0f / nb)))
                    return rc;
            }
            CUDA_TRY(launch_mask_scaled(D, n->dY, n->ok, n->Y, s));    // d/dlog S -> d/dy
            if ((rc = net_backward(P))) return rc;
            n->step++;
            steps++;
            const float lr = cfg->lr * std::min(1.0f, (float)steps / 50.0f);
            CUDA_TRY(launch_adam(n->p, n->g, n->m, n->v, n->wb, n->wmap, n->np, lr, 0.9f, 0.999f, 1e-8f,
                                 n->step, s));
            CUDA_TRY(launch_arrange_mid(wl(n, 1), n->T, n->wf, n->wbk, s));
        }
        double hacc[2];
        CUDA_TRY(cudaMemcpyAsync(hacc, n->lossacc, 16, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        const double mean = n->nsamples ? hacc[0] / n->nsamples : 0.0;
        if (ep == 0) first = mean;
        last = mean;
        ep_loss.push_back(mean);
        // the epoch's mean loss belongs to parameters between the epoch's first
        // and last step; the validation solve uses the parameters after it
        int val = 0;
        if ((rc = net_scaling(P)) || (rc = validation_iters(P, n->bval, &val))) return rc;
        if (val < best_val) {
            best = mean;
            best_val = val;
            best_epoch = ep;
            CUDA_TRY(cudaMemcpy(best_p.data(), n->p, n->np * 4, cudaMemcpyDeviceToHost));
        }
    }
    {
        std::vector<float> keep = best_p;
        const int st = n->step;
        if ((rc = net_upload(P, keep))) return rc;
        n->step = st;
    }
    n->s_stale = true;
    if ((rc = ensure_scaling(P))) return rc;
    if (stats) {
        stats->pairs = n->nsamples * ng;
        stats->samples = n->nsamples;
        stats->rhs = nrhs;
        stats->steps = steps;
        stats->loss_first_epoch = first;
        stats->loss_last_epoch = last;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        stats->loss_initial = loss_init;
        stats->loss_fd = loss_fd;
        for (int e = 0; e < 32; ++e) stats->loss_epoch[e] = e < (int)ep_loss.size() ? ep_loss[e] : 0.0;
        std::vector<float> hS((size_t)N);
        CUDA_TRY(cudaMemcpy(hS.data(), n->S, (size_t)N * 4, cudaMemcpyDeviceToHost));
        double lo = 1e30, hi = -1e30;
        for (float v : hS) { lo = std::min(lo, (double)std::log(v)); hi = std::max(hi, (double)std::log(v)); }
        stats->logs_min = lo;
        stats->logs_max = hi;
        stats->best_epoch = best_epoch;
        stats->val_iters_initial = val_init;
        stats->val_iters_best = best_val;
    }
    return SGIGA_OK;
}

// Checkpoint: "SGIGANET" | version 2 | taps | nparams | step | p | m | v (float32)
int sgiga_net_save(sgiga_plan_t P, const char* path) {
    if (!P || !P->net || !path) return fail(SGIGA_ERR_ARG, "no network or null path");
    Net* n = P->net;
    std::vector<float> p(n->np), m(n->np), v(n->np);
    CUDA_TRY(cudaMemcpy(p.data(), n->p, n->np * 4, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(m.data(), n->m, n->np * 4, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(v.data(), n->v, n->np * 4, cudaMemcpyDeviceToHost));
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(SGIGA_ERR_ARG, std::string("cannot open ") + path);
    const char magic[8] = {'S', 'G', 'I', 'G', 'A', 'N', 'E', 'T'};
    int hdr[4] = {2, n->T, n->np, n->step};
    bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(hdr, 4, 4, f) == 4 &&
              std::fwrite(p.data(), 4, n->np, f) == (size_t)n->np && std::fwrite(m.data(), 4, n->np, f) == (size_t)n->np &&
              std::fwrite(v.data(), 4, n->np, f) == (size_t)n->np;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(SGIGA_ERR_ARG, std::string("write failed: ") + path);
    return SGIGA_OK;
}

int sgiga_net_load(sgiga_plan_t P, const char* path) {
    int rc = needs_net(P);
    if (rc) return rc;
    if (!path) return fail(SGIGA_ERR_ARG, "null argument");
    if ((rc = net_create(P))) return rc;
    Net* n = P->net;
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(SGIGA_ERR_ARG, std::string("cannot open ") + path);
    char magic[8];
    int hdr[4];
    std::vector<float> p(n->np), m(n->np), v(n->np);
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "SGIGANET", 8) == 0 &&
              std::fread(hdr, 4, 4, f) == 4 && hdr[0] == 2 && hdr[1] == n->T && hdr[2] == n->np &&
              std::fread(p.data(), 4, n->np, f) == (size_t)n->np && std::fread(m.data(), 4, n->np, f) == (size_t)n->np &&
              std::fread(v.data(), 4, n->np, f) == (size_t)n->np;
    std::fclose(f);
    if (!ok) return fail(SGIGA_ERR_ARG, std::string("not a compatible network checkpoint: ") + path);
    if ((rc = net_upload(P, p))) return rc;
    CUDA_TRY(cudaMemcpy(n->m, m.data(), n->np * 4, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(n->v, v.data(), n->np * 4, cudaMemcpyHostToDevice));
    n->step = hdr[3];
    P->net_ready = true;
    return SGIGA_OK;
}

}  // extern "C"
