// Generalised symmetric-definite eigenproblems K U = M U diag(lam),
// U^T M U = I, of the banded 1D matrices of the fast-diagonalisation
// preconditioner, solved on the GPU in FP64 without forming a dense matrix.
//
// Both matrices are symmetric with bandwidth p (B-splines of degree p overlap
// p neighbours); M is positive definite and so is K (Dirichlet ends), so every
// eigenvalue is positive. Method (textbook steps, written for this library):
//   1. eigenvalues by bisection, one thread per eigenvalue: by Sylvester's law
//      of inertia, the number of eigenvalues below s equals the number of
//      negative pivots of the LDL^T factorisation of K - s M (M positive
//      definite), computed in one banded sweep;
//   2. units of close eigenvalues (relative gaps below 1e-6, or below 1e-3
//      up to 4 members) found on the host;
//   3. eigenvectors by inverse iteration, one thread per cluster: three
//      solves (K - s M) y = M v with banded LU and partial pivoting, each
//      followed by M-orthogonalisation against the cluster's earlier vectors
//      and M-normalisation. Away from clusters inverse iteration alone leaves
//      an M-orthogonality error of order eps ||K|| / gap, harmless for a
//      preconditioner.
// Cost: O(n p^2) per inertia count and per solve instead of the O(n^3) of a
// dense reduction, and no n x n matrix besides U itself.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <string>
#include <vector>

#include "kernels.h"

namespace sgiga {

// A(i, j) = K(i, j) - s M(i, j) for |i - j| <= P from the upper bands.
template <int P>
__device__ __forceinline__ double band_at(const double* Kb, const double* Mb, double s, int i, int j) {
    const int lo = i < j ? i : j, t = i < j ? j - i : i - j;
    return Kb[(long long)lo * (P + 1) + t] - s * Mb[(long long)lo * (P + 1) + t];
}

// Number of negative pivots of LDL^T(K - s M): a banded sweep keeping the last
// P rows of L and their pivots in registers. A pivot below `floor` in
// magnitude (eps^2 times the entries' scale: an exact or near-exact zero) is
// replaced by -floor, as tridiagonal Sturm counts do with their pivot minimum.
template <int P>
__device__ int inertia_count(const double* __restrict__ Kb, const double* __restrict__ Mb, int n, double s,
                             double floor) {
    double Lr[P + 1][P + 1];   // Lr[r][t] = L(i-r, i-r-t), r, t = 1..P
    double Di[P + 1];          // 1 / D(i-r)
#pragma unroll
    for (int r = 0; r <= P; ++r) {
        Di[r] = 0.0;
#pragma unroll
        for (int t = 0; t <= P; ++t) Lr[r][t] = 0.0;
    }
    int neg = 0;
    for (int i = 0; i < n; ++i) {
        double u[P + 1];
#pragma unroll
        for (int t = P; t >= 1; --t) {
            double v = i - t >= 0 ? Kb[(long long)(i - t) * (P + 1) + t] - s * Mb[(long long)(i - t) * (P + 1) + t] : 0.0;
#pragma unroll
            for (int q = t + 1; q <= P; ++q) v -= u[q] * Lr[t][q - t];
            u[t] = v;
        }
        double D = Kb[(long long)i * (P + 1)] - s * Mb[(long long)i * (P + 1)];
        double l[P + 1];
#pragma unroll
        for (int t = 1; t <= P; ++t) {
            l[t] = u[t] * Di[t];
            D -= u[t] * l[t];
        }
        if (fabs(D) < floor) D = -floor;
        neg += D < 0.0 ? 1 : 0;
#pragma unroll
        for (int r = P; r >= 2; --r) {
            Di[r] = Di[r - 1];
#pragma unroll
            for (int t = 1; t <= P; ++t) Lr[r][t] = Lr[r - 1][t];
        }
        Di[1] = 1.0 / D;
#pragma unroll
        for (int t = 1; t <= P; ++t) Lr[1][t] = l[t];
    }
    return neg;
}

// Eigenvalue j of every job by bisection on the inertia count. Invariant:
// count(lo) <= j < count(hi). Below lo = 0 there is nothing (K positive
// definite); from hi the search first descends geometrically (factor 7) until
// lo > 0, then halves the ratio hi / lo while it exceeds 2, then the interval.
// The first bound (2.17 max K_ii / M_ii, times powers of 4) and the descent
// factor are no powers of 2, so that no bisection point equals some
// K_ii / M_ii (which would make the first pivot of that row vanish exactly).
template <int P>
__global__ void k_eig_bisect(const EigJob* __restrict__ jobs, int njobs, long long nthreads,
                             const double* __restrict__ Kb, const double* __restrict__ Mb, double* __restrict__ lam) {
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gt >= nthreads) return;
    int a = 0, b = njobs - 1;
    while (a < b) {            // last job with t0 <= gt
        const int m = (a + b + 1) >> 1;
        if (jobs[m].t0 <= gt) a = m; else b = m - 1;
    }
    const EigJob J = jobs[a];
    const int j = (int)(gt - J.t0);
    if (j >= J.n) return;
    const double* kb = Kb + J.boff;
    const double* mb = Mb + J.boff;
    const double floor = DBL_EPSILON * DBL_EPSILON * J.anorm;
    double hi = J.hi0;
    for (int it = 0; it < 64 && inertia_count<P>(kb, mb, J.n, hi, floor) <= j; ++it) hi *= 4.0;
    double lo = 0.0;
    for (int it = 0; it < 400; ++it) {
        double mid;
        if (lo == 0.0) mid = hi * (1.0 / 7.0);
        else if (hi > 2.0 * lo) mid = sqrt(lo * hi);
        else mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi) || hi - lo <= 4.0 * DBL_EPSILON * hi) break;
        if (inertia_count<P>(kb, mb, J.n, mid, floor) > j) hi = mid;
        else lo = mid;
    }
    lam[J.loff + j] = lo == 0.0 ? 0.5 * hi : 0.5 * (lo + hi);
}

// Deterministic start vector of inverse iteration (an integer hash of (i, j)
// mapped to [-1/2, 1/2)).
__device__ __forceinline__ double start_entry(int i, int j) {
    unsigned x = (unsigned)(i + 1) * 0x9E3779B1u ^ (unsigned)(j + 1) * 0x85EBCA77u;
    x ^= x >> 15;
    x *= 0x2C1B3C6Du;
    x ^= x >> 12;
    x *= 0x297A2D39u;
    x ^= x >> 15;
    return (double)(x & 0xFFFFFu) / 1048576.0 - 0.5;
}

// (M v)_r from the upper band of M; v read through `vec`.
template <int P, typename F>
__device__ __forceinline__ double band_mv(const double* __restrict__ Mb, int n, int r, F vec) {
    double acc = Mb[(long long)r * (P + 1)] * vec(r);
#pragma unroll
    for (int t = 1; t <= P; ++t) {
        if (r + t < n) acc += Mb[(long long)r * (P + 1) + t] * vec(r + t);
        if (r - t >= 0) acc += Mb[(long long)(r - t) * (P + 1) + t] * vec(r - t);
    }
    return acc;
}

// Eigenvectors of every job by inverse iteration, one thread per unit (a run
// of `cnt` eigenvalues from j0 whose gaps are below the cluster tolerance;
// most units are single eigenvalues), all jobs in one launch (the jobs are
// independent; the largest come first, their threads run longest). Per thread,
// in the job's `scratch` (interleaved by the job's threads: entry e of thread
// t at e * nu + t, so that a warp's accesses to the same row are contiguous):
// the U rows of the banded LU (2P+1 entries and the transformed right-hand
// side per row), then the current vector (n).
template <int P>
__global__ void __launch_bounds__(128)
k_eig_vectors(const EigJob* __restrict__ jobs, int njobs, long long nunits, const int2* __restrict__ units,
              const double* __restrict__ Kb, const double* __restrict__ Mb, const double* __restrict__ lam,
              double* __restrict__ U, double* __restrict__ Ut, double* __restrict__ scratch_all) {
    constexpr int W2 = 2 * P + 1, SL = W2 + 1;
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gt >= nunits) return;
    int a = 0, b = njobs - 1;
    while (a < b) {            // last job with u0 <= gt
        const int m = (a + b + 1) >> 1;
        if (jobs[m].u0 <= gt) a = m; else b = m - 1;
    }
    const EigJob J = jobs[a];
    const int tid = (int)(gt - J.u0);
    const int n = J.n;
    const long long NT = J.nu;
    double* __restrict__ scratch = scratch_all + J.soff;
    const double* kb = Kb + J.boff;
    const double* mb = Mb + J.boff;
    const double* lm = lam + J.loff;
    double* Uo = U + J.uoff;
    double* Uto = Ut + J.uoff;
    auto row = [&](int i, int s) -> double& { return scratch[((long long)i * SL + s) * NT + tid]; };
    double* vecbase = scratch + (long long)n * SL * NT;
    auto vec = [&](int i) -> double& { return vecbase[(long long)i * NT + tid]; };
    const double tiny = DBL_EPSILON * DBL_EPSILON * J.anorm;   // only an exact or near-exact zero pivot
    const int j0 = units[gt].x, cnt = units[gt].y;
    double sprev = 0.0;
    for (int m = 0; m < cnt; ++m) {
        const int j = j0 + m;
        double s = lm[j];
        if (m > 0 && s - sprev < 10.0 * DBL_EPSILON * s) s = sprev + 10.0 * DBL_EPSILON * s;
        sprev = s;
        for (int i = 0; i < n; ++i) vec(i) = start_entry(i, j);
        for (int it = 0; it < 3; ++it) {
            // forward elimination with partial pivoting on the window of rows
            // i..i+P (columns i..i+2P); the right-hand side M v enters row by row
            double Wn[P + 1][W2], bw[P + 1];
#pragma unroll
            for (int k = 0; k <= P; ++k) {
#pragma unroll
                for (int c = 0; c < W2; ++c) {
                    const int dd = c - k;
                    Wn[k][c] = (k < n && c < n && dd <= P && dd >= -P) ? band_at<P>(kb, mb, s, k, c) : 0.0;
                }
                bw[k] = k < n ? band_mv<P>(mb, n, k, vec) : 0.0;
            }
            for (int i = 0; i < n; ++i) {
                int kp = 0;
                double best = fabs(Wn[0][0]);
#pragma unroll
                for (int k = 1; k <= P; ++k)
                    if (fabs(Wn[k][0]) > best) { best = fabs(Wn[k][0]); kp = k; }
#pragma unroll
                for (int k = 1; k <= P; ++k) {
                    if (kp == k) {
#pragma unroll
                        for (int c = 0; c < W2; ++c) { const double t = Wn[0][c]; Wn[0][c] = Wn[k][c]; Wn[k][c] = t; }
                        const double t = bw[0]; bw[0] = bw[k]; bw[k] = t;
                    }
                }
                if (fabs(Wn[0][0]) < tiny) Wn[0][0] = tiny;
                const double pinv = 1.0 / Wn[0][0];
#pragma unroll
                for (int c = 0; c < W2; ++c) row(i, c) = Wn[0][c];
                row(i, W2) = bw[0];
#pragma unroll
                for (int k = 1; k <= P; ++k) {
                    const double f = Wn[k][0] * pinv;
#pragma unroll
                    for (int c = 1; c < W2; ++c) Wn[k][c] -= f * Wn[0][c];
                    bw[k] -= f * bw[0];
                }
                // slide the window: rows up, columns left; row i+P+1 enters
#pragma unroll
                for (int k = 0; k < P; ++k) {
#pragma unroll
                    for (int c = 0; c + 1 < W2; ++c) Wn[k][c] = Wn[k + 1][c + 1];
                    Wn[k][W2 - 1] = 0.0;
                    bw[k] = bw[k + 1];
                }
                const int r = i + P + 1;
#pragma unroll
                for (int c = 0; c < W2; ++c) {
                    const int col = r - P + c;
                    Wn[P][c] = (r < n && col < n) ? band_at<P>(kb, mb, s, r, col) : 0.0;
                }
                bw[P] = r < n ? band_mv<P>(mb, n, r, vec) : 0.0;
            }
            // back substitution; y overwrites v (M v has been consumed)
            double yw[2 * P];
#pragma unroll
            for (int c = 0; c < 2 * P; ++c) yw[c] = 0.0;
            for (int i = n - 1; i >= 0; --i) {
                double t = row(i, W2);
#pragma unroll
                for (int c = 1; c < W2; ++c) t -= row(i, c) * yw[c - 1];
                const double yi = t / row(i, 0);
                vec(i) = yi;
#pragma unroll
                for (int c = 2 * P - 1; c >= 1; --c) yw[c] = yw[c - 1];
                yw[0] = yi;
            }
            // M-orthogonal to the unit's earlier vectors (twice), then M-normalised
            for (int pass = 0; pass < 2; ++pass)
                for (int q = 0; q < m; ++q) {
                    const double* uq = Uto + (long long)(j0 + q) * n;
                    double dot = 0.0;
                    for (int i = 0; i < n; ++i) dot += uq[i] * band_mv<P>(mb, n, i, vec);
                    for (int i = 0; i < n; ++i) vec(i) -= dot * uq[i];
                }
            double nrm = 0.0;
            for (int i = 0; i < n; ++i) nrm += vec(i) * band_mv<P>(mb, n, i, vec);
            const double f = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
            for (int i = 0; i < n; ++i) vec(i) *= f;
        }
        for (int i = 0; i < n; ++i) {
            const double v = vec(i);
            Uo[(long long)i * n + j] = v;
            Uto[(long long)j * n + i] = v;
        }
    }
}

template <int P>
static cudaError_t launch_eig(std::vector<EigJob>& jobs, const std::vector<double>& Kb, const std::vector<double>& Mb,
                              double* dU, double* dUt, double* dlam, std::vector<double>& hlam, cudaStream_t s,
                              std::string& msg) {
    long long nthreads = 0;
    for (EigJob& J : jobs) {
        J.t0 = nthreads;
        nthreads += J.n;
        double hi0 = 0.0, an = 0.0;
        for (int i = 0; i < J.n; ++i)
            hi0 = fmax(hi0, 2.17 * Kb[J.boff + (long long)i * (P + 1)] / Mb[J.boff + (long long)i * (P + 1)]);
        for (int i = 0; i < J.n; ++i) {
            double a = 0.0;
            for (int t = -P; t <= P; ++t) {
                const int lo = t < 0 ? i + t : i, tt = t < 0 ? -t : t;
                if (lo < 0 || lo + tt >= J.n) continue;
                a += fabs(Kb[J.boff + (long long)lo * (P + 1) + tt]) + hi0 * fabs(Mb[J.boff + (long long)lo * (P + 1) + tt]);
            }
            an = fmax(an, a);
        }
        J.hi0 = hi0 > 0.0 ? hi0 : 1.0;
        J.anorm = an > 0.0 ? an : 1.0;
    }
    hlam.assign((size_t)nthreads, 0.0);
    if (nthreads == 0) return cudaSuccess;
    EigJob* djobs = nullptr;
    double *dKb = nullptr, *dMb = nullptr, *scratch = nullptr;
    int2* dunits = nullptr;
    cudaError_t e = cudaSuccess;
    auto cleanup = [&]() {
        cudaFree(djobs); cudaFree(dKb); cudaFree(dMb); cudaFree(scratch); cudaFree(dunits);
    };
    if ((e = cudaMalloc(&djobs, jobs.size() * sizeof(EigJob))) != cudaSuccess ||
        (e = cudaMalloc(&dKb, Kb.size() * 8)) != cudaSuccess || (e = cudaMalloc(&dMb, Mb.size() * 8)) != cudaSuccess ||
        (e = cudaMemcpyAsync(djobs, jobs.data(), jobs.size() * sizeof(EigJob), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dKb, Kb.data(), Kb.size() * 8, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dMb, Mb.data(), Mb.size() * 8, cudaMemcpyHostToDevice, s)) != cudaSuccess) {
        cleanup();
        msg = "eigensolver set-up";
        return e;
    }
    SGIGA_COUNT_LAUNCH();
    k_eig_bisect<P><<<(unsigned)((nthreads + 127) / 128), 128, 0, s>>>(djobs, (int)jobs.size(), nthreads, dKb, dMb,
                                                                        dlam);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(hlam.data(), dlam, (size_t)nthreads * 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
        cleanup();
        msg = "eigenvalue bisection";
        return e;
    }
    // units of eigenvalues whose vectors are M-orthogonalised against each
    // other. Inverse iteration alone leaves two eigenvectors M-orthogonal only
    // to about eps lam / gap. Maximally smooth splines have pairs of modes
    // localised at the two ends of the interval whose eigenvalues agree to
    // many digits (uniform and symmetric graded meshes): neighbours with a
    // relative gap below 1e-6 always share a unit (up to 32 members). The top
    // of the spectrum is dense on fine levels: neighbours with a relative gap
    // below 1e-3 share a unit while it has fewer than 4 members, which keeps
    // each thread's Gram-Schmidt work small; across a cut the gap is above
    // 1e-6 lam.
    std::vector<int2> units;
    std::vector<EigJob> vjobs;   // the jobs in launch order (largest first) with their units and scratch
    std::vector<size_t> ord(jobs.size());
    for (size_t q = 0; q < ord.size(); ++q) ord[q] = q;
    std::stable_sort(ord.begin(), ord.end(), [&](size_t x, size_t y) { return jobs[x].n > jobs[y].n; });
    size_t scratch_doubles = 0;
    for (size_t q : ord) {
        EigJob J = jobs[q];
        const double* l = hlam.data() + J.t0;
        for (int j = 0; j < J.n; ++j)
            if (!(l[j] > 0.0) || !std::isfinite(l[j]) || (j > 0 && l[j] < l[j - 1])) {
                cleanup();
                msg = "eigenvalue bisection produced a non-positive, non-finite or unordered value";
                return cudaErrorInvalidValue;
            }
        J.u0 = (long long)units.size();
        for (int j = 0; j < J.n;) {
            int j1 = j + 1;
            while (j1 < J.n) {
                const double gap = l[j1] - l[j1 - 1], size = j1 - j;
                if ((gap <= 1e-6 * l[j1] && size < 32) || (gap <= 1e-3 * l[j1] && size < 4)) ++j1;
                else break;
            }
            units.push_back(make_int2(j, j1 - j));
            j = j1;
        }
        J.nu = (int)((long long)units.size() - J.u0);
        J.soff = (long long)scratch_doubles;
        scratch_doubles += (size_t)J.n * (2 * P + 3) * J.nu;
        vjobs.push_back(J);
    }
    const long long nunits = (long long)units.size();
    if ((e = cudaMalloc(&dunits, units.size() * sizeof(int2))) != cudaSuccess ||
        (e = cudaMalloc(&scratch, std::max<size_t>(scratch_doubles, 1) * 8)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dunits, units.data(), units.size() * sizeof(int2), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(djobs, vjobs.data(), vjobs.size() * sizeof(EigJob), cudaMemcpyHostToDevice, s)) != cudaSuccess) {
        cleanup();
        msg = "eigenvector scratch (" + std::to_string(scratch_doubles * 8) + " bytes)";
        return e;
    }
    if (nunits > 0) {
        SGIGA_COUNT_LAUNCH();
        k_eig_vectors<P><<<(unsigned)((nunits + 127) / 128), 128, 0, s>>>(djobs, (int)vjobs.size(), nunits, dunits, dKb,
                                                                          dMb, dlam, dU, dUt, scratch);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    if (e != cudaSuccess) msg = "inverse iteration";
    return e;
}

// Every job's eigenpairs: U and U^T (row-major n x n, column j of U = the
// M-normalised eigenvector of the j-th smallest eigenvalue) at uoff, lam at
// loff, in device memory; hlam receives the eigenvalues of all jobs in job
// order. Kb, Mb: the upper bands [n][p+1] of K and M of every job at boff.
int gpu_generalized_eigen(int p, std::vector<EigJob>& jobs, const std::vector<double>& Kb,
                          const std::vector<double>& Mb, double* dU, double* dUt, double* dlam,
                          std::vector<double>& hlam, cudaStream_t s, std::string& msg) {
    cudaError_t e;
    switch (p) {
    case 1: e = launch_eig<1>(jobs, Kb, Mb, dU, dUt, dlam, hlam, s, msg); break;
    case 2: e = launch_eig<2>(jobs, Kb, Mb, dU, dUt, dlam, hlam, s, msg); break;
    case 3: e = launch_eig<3>(jobs, Kb, Mb, dU, dUt, dlam, hlam, s, msg); break;
    case 4: e = launch_eig<4>(jobs, Kb, Mb, dU, dUt, dlam, hlam, s, msg); break;
    default: msg = "degree out of range"; return -1;
    }
    if (e != cudaSuccess) {
        msg += std::string(": ") + cudaGetErrorString(e);
        cudaGetLastError();
        return -1;
    }
    return 0;
}

}  // namespace sgiga
