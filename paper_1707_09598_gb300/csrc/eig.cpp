// Generalised symmetric-definite eigenproblem K U = M U diag(lam), U^T M U = I,
// for the banded 1D matrices of the fast-diagonalisation preconditioner.
//
// Method (textbook, written for this library):
//   1. banded Cholesky M = L L^T (bandwidth p);
//   2. C = L^{-1} K L^{-T} by banded triangular solves;
//   3. Householder reduction of C to tridiagonal form, with the orthogonal
//      factor accumulated;
//   4. implicit QL iterations with Wilkinson shifts on the tridiagonal matrix,
//      rotations applied to the accumulated factor (rows of its transpose,
//      so every rotation touches contiguous memory);
//   5. U = L^{-T} V, eigenpairs sorted by increasing eigenvalue.
// For large n (> 384) steps 3-5 run on a pool of host threads, and the
// eigenvectors of the tridiagonal matrix come from inverse iteration (one
// tridiagonal LU with partial pivoting per eigenvalue, re-orthogonalised by
// modified Gram-Schmidt inside clusters of close eigenvalues), back-transformed
// through the stored Householder reflectors one eigenvector at a time.
#include <algorithm>
#include <atomic>
#include <thread>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

namespace sgiga {

// K, M: dense row-major n x n (symmetric, M SPD with bandwidth bw).
// U: row-major n x n, column j = eigenvector j. Returns 0 on success.
static int generalized_eigen_large(int n, int bw, const double* K, const double* M, double* U, double* lam);

int generalized_eigen(int n, int bw, const double* K, const double* M, double* U, double* lam) {
    if (n <= 0) return 0;
    if (n > 384) return generalized_eigen_large(n, bw, K, M, U, lam);
    std::vector<double> L((size_t)n * n, 0.0);
    // 1. banded Cholesky
    for (int j = 0; j < n; ++j) {
        double s = M[(size_t)j * n + j];
        int k0 = std::max(0, j - bw);
        for (int k = k0; k < j; ++k) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(s > 0.0)) return -1;
        double ljj = std::sqrt(s);
        L[(size_t)j * n + j] = ljj;
        int i1 = std::min(n - 1, j + bw);
        for (int i = j + 1; i <= i1; ++i) {
            double t = M[(size_t)i * n + j];
            int kk = std::max(0, i - bw);
            for (int k = std::max(k0, kk); k < j; ++k) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = t / ljj;
        }
    }
    // 2. Y = L^{-1} K (column by column: forward substitution), then C = L^{-1} Y^T
    std::vector<double> Y((size_t)n * n);
    std::vector<double> col(n);
    for (int c = 0; c < n; ++c) {
        for (int i = 0; i < n; ++i) {
            double t = K[(size_t)i * n + c];
            for (int k = std::max(0, i - bw); k < i; ++k) t -= L[(size_t)i * n + k] * col[k];
            col[i] = t / L[(size_t)i * n + i];
        }
        for (int i = 0; i < n; ++i) Y[(size_t)i * n + c] = col[i];
    }
    std::vector<double> A((size_t)n * n);
    for (int c = 0; c < n; ++c) {          // column c of C = L^{-1} (row c of Y)^T
        for (int i = 0; i < n; ++i) {
            double t = Y[(size_t)c * n + i];
            for (int k = std::max(0, i - bw); k < i; ++k) t -= L[(size_t)i * n + k] * col[k];
            col[i] = t / L[(size_t)i * n + i];
        }
        for (int i = 0; i < n; ++i) A[(size_t)i * n + c] = col[i];
    }
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double s = 0.5 * (A[(size_t)i * n + j] + A[(size_t)j * n + i]);
            A[(size_t)i * n + j] = A[(size_t)j * n + i] = s;
        }
    // 3. Householder tridiagonalisation: A = Q T Q^T. Reflector k acts on k+1..n-1.
    std::vector<double> d(n), e(n, 0.0);
    std::vector<double> V((size_t)n * n, 0.0);   // reflector vectors, row k = v_k
    std::vector<double> tau(n, 0.0), pv(n), qv(n);
    for (int k = 0; k + 2 < n; ++k) {
        int m = n - k - 1;
        double* x = &pv[0];
        for (int i = 0; i < m; ++i) x[i] = A[(size_t)(k + 1 + i) * n + k];
        double nrm = 0.0;
        for (int i = 0; i < m; ++i) nrm += x[i] * x[i];
        nrm = std::sqrt(nrm);
        double alpha = x[0] > 0 ? -nrm : nrm;
        double* v = &V[(size_t)k * n];
        for (int i = 0; i < m; ++i) v[i] = x[i];
        v[0] -= alpha;
        double beta = 0.0;
        for (int i = 0; i < m; ++i) beta += v[i] * v[i];
        d[k] = A[(size_t)k * n + k];
        e[k] = alpha;
        if (beta == 0.0) { tau[k] = 0.0; e[k] = x[0]; continue; }
        double t = 2.0 / beta;
        tau[k] = t;
        // p = t * A22 v
        for (int i = 0; i < m; ++i) {
            const double* row = &A[(size_t)(k + 1 + i) * n + k + 1];
            double s = 0.0;
            for (int j = 0; j < m; ++j) s += row[j] * v[j];
            qv[i] = t * s;
        }
        double kk = 0.0;
        for (int i = 0; i < m; ++i) kk += qv[i] * v[i];
        kk *= 0.5 * t;
        for (int i = 0; i < m; ++i) qv[i] -= kk * v[i];
        // A22 -= v q^T + q v^T
        for (int i = 0; i < m; ++i) {
            double* row = &A[(size_t)(k + 1 + i) * n + k + 1];
            double vi = v[i], qi = qv[i];
            for (int j = 0; j < m; ++j) row[j] -= vi * qv[j] + qi * v[j];
        }
    }
    if (n >= 2) {
        d[n - 2] = A[(size_t)(n - 2) * n + (n - 2)];
        e[n - 2] = A[(size_t)(n - 1) * n + (n - 2)];
    }
    d[n - 1] = A[(size_t)(n - 1) * n + (n - 1)];
    e[n - 1] = 0.0;
    // Accumulate Z^T = Q^T with Q = H_0 H_1 ... ; rows of Zt are columns of Q.
    // Build Q explicitly (row-major) then transpose into Zt.
    std::vector<double> Qm((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Qm[(size_t)i * n + i] = 1.0;
    for (int k = n - 3; k >= 0; --k) {
        if (tau[k] == 0.0) continue;
        int m = n - k - 1;
        const double* v = &V[(size_t)k * n];
        // Q[k+1:, k+1:] = (I - t v v^T) Q[k+1:, k+1:]
        std::fill(qv.begin(), qv.end(), 0.0);
        for (int i = 0; i < m; ++i) {
            const double* row = &Qm[(size_t)(k + 1 + i) * n + k + 1];
            double vi = v[i];
            for (int j = 0; j < m; ++j) qv[j] += vi * row[j];
        }
        for (int i = 0; i < m; ++i) {
            double* row = &Qm[(size_t)(k + 1 + i) * n + k + 1];
            double s = tau[k] * v[i];
            for (int j = 0; j < m; ++j) row[j] -= s * qv[j];
        }
    }
    std::vector<double> Zt((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Zt[(size_t)j * n + i] = Qm[(size_t)i * n + j];
    // 4. implicit QL with Wilkinson shifts; e[i] couples d[i] and d[i+1]
    const double eps = 2.220446049250313e-16;
    for (int l = 0; l < n; ++l) {
        int iter = 0;
        for (;;) {
            int m = l;
            for (; m < n - 1; ++m) {
                double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
                if (std::fabs(e[m]) <= eps * dd) break;
            }
            if (m == l) break;
            if (++iter > 60) return -2;
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = std::hypot(g, 1.0);
            g = d[m] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
            double s = 1.0, c = 1.0, p = 0.0;
            int i = m - 1;
            bool deflated = false;
            for (; i >= l; --i) {
                double f = s * e[i];
                double b = c * e[i];
                r = std::hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) {
                    d[i + 1] -= p;
                    e[m] = 0.0;
                    deflated = true;
                    break;
                }
                s = f / r;
                c = g / r;
                g = d[i + 1] - p;
                r = (d[i] - g) * s + 2.0 * c * b;
                p = s * r;
                d[i + 1] = g + p;
                g = c * r - b;
                double* zi = &Zt[(size_t)i * n];
                double* zj = &Zt[(size_t)(i + 1) * n];
                for (int k = 0; k < n; ++k) {
                    double fk = zj[k];
                    zj[k] = s * zi[k] + c * fk;
                    zi[k] = c * zi[k] - s * fk;
                }
            }
            if (deflated) continue;
            d[l] -= p;
            e[l] = g;
            e[m] = 0.0;
        }
    }
    // 5. sort and back-transform: U = L^{-T} V, column j of V = row j of Zt
    std::vector<int> ord(n);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return d[a] < d[b]; });
    for (int jj = 0; jj < n; ++jj) {
        int j = ord[jj];
        lam[jj] = d[j];
        const double* v = &Zt[(size_t)j * n];
        // solve L^T u = v (backward substitution, banded)
        for (int i = n - 1; i >= 0; --i) {
            double t = v[i];
            int i1 = std::min(n - 1, i + bw);
            for (int k = i + 1; k <= i1; ++k) t -= L[(size_t)k * n + i] * col[k];
            col[i] = t / L[(size_t)i * n + i];
        }
        for (int i = 0; i < n; ++i) U[(size_t)i * n + jj] = col[i];
    }
    return 0;
}

// ---------------------------------------------------------------------------
// Large-n path
// ---------------------------------------------------------------------------

namespace {

struct Pool {
    int nt;
    explicit Pool(int n) : nt(n) {}
    // run f(t, nt) on nt threads and join
    template <typename F>
    void run(F f) {
        std::vector<std::thread> th;
        for (int t = 1; t < nt; ++t) th.emplace_back(f, t, nt);
        f(0, nt);
        for (auto& x : th) x.join();
    }
};

// Sense-reversing spin barrier for a fixed team.
struct SpinBarrier {
    std::atomic<int> count{0};
    std::atomic<int> gen{0};
    int n;
    explicit SpinBarrier(int nn) : n(nn) {}
    void wait() {
        int g = gen.load(std::memory_order_acquire);
        if (count.fetch_add(1, std::memory_order_acq_rel) == n - 1) {
            count.store(0, std::memory_order_relaxed);
            gen.store(g + 1, std::memory_order_release);
        } else {
            while (gen.load(std::memory_order_acquire) == g) std::this_thread::yield();
        }
    }
};

int nthreads() {
    unsigned h = std::thread::hardware_concurrency();
    if (h == 0) h = 4;
    return (int)std::min<unsigned>(h, 16);
}

// eigenvalues of the symmetric tridiagonal (d, e) by implicit QL, no vectors
int tridiag_eigenvalues(int n, std::vector<double> d, std::vector<double> e, std::vector<double>& out) {
    const double eps = 2.220446049250313e-16;
    e[n - 1] = 0.0;
    for (int l = 0; l < n; ++l) {
        int iter = 0;
        for (;;) {
            int m = l;
            for (; m < n - 1; ++m)
                if (std::fabs(e[m]) <= eps * (std::fabs(d[m]) + std::fabs(d[m + 1]))) break;
            if (m == l) break;
            if (++iter > 60) return -2;
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = std::hypot(g, 1.0);
            g = d[m] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
            double s = 1.0, c = 1.0, p = 0.0;
            bool deflated = false;
            for (int i = m - 1; i >= l; --i) {
                double f = s * e[i], b = c * e[i];
                r = std::hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) { d[i + 1] -= p; e[m] = 0.0; deflated = true; break; }
                s = f / r; c = g / r;
                g = d[i + 1] - p;
                r = (d[i] - g) * s + 2.0 * c * b;
                p = s * r;
                d[i + 1] = g + p;
                g = c * r - b;
            }
            if (deflated) continue;
            d[l] -= p; e[l] = g; e[m] = 0.0;
        }
    }
    out = d;
    std::sort(out.begin(), out.end());
    return 0;
}

// One eigenvector of the tridiagonal (d, e) for eigenvalue lam by inverse
// iteration with a tridiagonal LU (partial pivoting); v has length n.
void inverse_iteration(int n, const double* d, const double* e, double lam, double tnorm, unsigned seed,
                       double* v, std::vector<double>& w) {
    // LU of T - lam I with pivoting: rows of U have three entries (u0, u1, u2)
    w.resize((size_t)6 * n);
    double* u0 = w.data();
    double* u1 = u0 + n;
    double* u2 = u1 + n;
    double* lm = u2 + n;
    int* piv = reinterpret_cast<int*>(lm + n);
    const double tiny = 2.220446049250313e-16 * tnorm;
    // current row (a0 diag, a1 super) and carry
    double a0 = d[0] - lam, a1 = n > 1 ? e[0] : 0.0, a2 = 0.0;
    for (int i = 0; i < n - 1; ++i) {
        double b0 = e[i], b1 = d[i + 1] - lam, b2 = (i + 2 < n) ? e[i + 1] : 0.0;  // next row: (e_i, d_{i+1}, e_{i+1})
        if (std::fabs(b0) > std::fabs(a0)) {       // swap rows
            piv[i] = 1;
            u0[i] = b0; u1[i] = b1; u2[i] = b2;
            double l = a0 / b0;
            lm[i] = l;
            a0 = a1 - l * b1;
            a1 = a2 - l * b2;
            a2 = 0.0;
        } else {
            piv[i] = 0;
            if (a0 == 0.0) a0 = tiny;
            u0[i] = a0; u1[i] = a1; u2[i] = a2;
            double l = b0 / a0;
            lm[i] = l;
            a0 = b1 - l * a1;
            a1 = b2 - l * a2;
            a2 = 0.0;
        }
    }
    if (a0 == 0.0) a0 = tiny;
    u0[n - 1] = a0; u1[n - 1] = 0.0; u2[n - 1] = 0.0;
    // start vector: deterministic pseudo-random
    unsigned st = seed * 2654435761u + 12345u;
    for (int i = 0; i < n; ++i) {
        st = st * 1664525u + 1013904223u;
        v[i] = ((st >> 8) & 0xFFFF) / 65536.0 - 0.5 + 1e-3;
    }
    for (int it = 0; it < 3; ++it) {
        // forward: apply the row operations of the elimination to v
        for (int i = 0; i < n - 1; ++i) {
            if (piv[i]) { double t = v[i]; v[i] = v[i + 1]; v[i + 1] = t - lm[i] * v[i]; }
            else v[i + 1] -= lm[i] * v[i];
        }
        // back substitution with U
        for (int i = n - 1; i >= 0; --i) {
            double t = v[i];
            if (i + 1 < n) t -= u1[i] * v[i + 1];
            if (i + 2 < n) t -= u2[i] * v[i + 2];
            v[i] = t / u0[i];
        }
        double nr = 0.0;
        for (int i = 0; i < n; ++i) nr += v[i] * v[i];
        nr = 1.0 / std::sqrt(nr);
        for (int i = 0; i < n; ++i) v[i] *= nr;
    }
}

}  // namespace

static int generalized_eigen_large(int n, int bw, const double* K, const double* M, double* U, double* lam) {
    const int NT = nthreads();
    Pool pool(NT);
    std::vector<double> L((size_t)n * n, 0.0);
    // 1. banded Cholesky of M
    for (int j = 0; j < n; ++j) {
        double s = M[(size_t)j * n + j];
        int k0 = std::max(0, j - bw);
        for (int k = k0; k < j; ++k) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(s > 0.0)) return -1;
        double ljj = std::sqrt(s);
        L[(size_t)j * n + j] = ljj;
        int i1 = std::min(n - 1, j + bw);
        for (int i = j + 1; i <= i1; ++i) {
            double t = M[(size_t)i * n + j];
            for (int k = std::max(k0, i - bw); k < j; ++k) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = t / ljj;
        }
    }
    // 2. A = L^{-1} K L^{-T}: rows of Y = L^{-1} K (column solves in parallel), then A = L^{-1} Y^T
    std::vector<double> Y((size_t)n * n), A((size_t)n * n);
    pool.run([&](int t, int nt) {
        std::vector<double> col(n);
        for (int c = t; c < n; c += nt) {
            for (int i = 0; i < n; ++i) {
                double v = K[(size_t)i * n + c];
                for (int k = std::max(0, i - bw); k < i; ++k) v -= L[(size_t)i * n + k] * col[k];
                col[i] = v / L[(size_t)i * n + i];
            }
            for (int i = 0; i < n; ++i) Y[(size_t)i * n + c] = col[i];
        }
    });
    pool.run([&](int t, int nt) {
        std::vector<double> col(n);
        for (int c = t; c < n; c += nt) {
            for (int i = 0; i < n; ++i) {
                double v = Y[(size_t)c * n + i];
                for (int k = std::max(0, i - bw); k < i; ++k) v -= L[(size_t)i * n + k] * col[k];
                col[i] = v / L[(size_t)i * n + i];
            }
            for (int i = 0; i < n; ++i) A[(size_t)i * n + c] = col[i];
        }
    });
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double s = 0.5 * (A[(size_t)i * n + j] + A[(size_t)j * n + i]);
            A[(size_t)i * n + j] = A[(size_t)j * n + i] = s;
        }
    std::vector<double>().swap(Y);
    // 3. Householder tridiagonalisation (team of threads, two barriers per step)
    std::vector<double> d(n), e(n, 0.0), V((size_t)n * n, 0.0), tau(n, 0.0), qv(n);
    std::vector<double> partial((size_t)NT * 2, 0.0);
    SpinBarrier bar(NT);
    std::atomic<int> failed{0};
    pool.run([&](int t, int nt) {
        for (int k = 0; k + 2 < n; ++k) {
            const int m = n - k - 1;
            double* v = &V[(size_t)k * n];
            bar.wait();   // previous step's rank-2 updates are complete
            if (t == 0) {
                double nrm = 0.0;
                for (int i = 0; i < m; ++i) { v[i] = A[(size_t)(k + 1 + i) * n + k]; nrm += v[i] * v[i]; }
                nrm = std::sqrt(nrm);
                double x0 = v[0];
                double alpha = x0 > 0 ? -nrm : nrm;
                v[0] -= alpha;
                double beta = 0.0;
                for (int i = 0; i < m; ++i) beta += v[i] * v[i];
                d[k] = A[(size_t)k * n + k];
                if (beta == 0.0) { tau[k] = 0.0; e[k] = x0; }
                else { tau[k] = 2.0 / beta; e[k] = alpha; }
            }
            bar.wait();
            const double tk = tau[k];
            if (tk == 0.0) { bar.wait(); bar.wait(); continue; }
            // q = t A22 v (rows split across threads), partial q.v
            double pv = 0.0;
            for (int i = t; i < m; i += nt) {
                const double* row = &A[(size_t)(k + 1 + i) * n + k + 1];
                double s = 0.0;
                for (int j = 0; j < m; ++j) s += row[j] * v[j];
                qv[i] = tk * s;
                pv += qv[i] * v[i];
            }
            partial[t] = pv;
            bar.wait();
            double kk = 0.0;
            for (int u = 0; u < nt; ++u) kk += partial[u];
            kk *= 0.5 * tk;
            // q -= kk v (each thread its rows' entries), then rank-2 update of its rows
            for (int i = t; i < m; i += nt) qv[i] -= kk * v[i];
            bar.wait();
            for (int i = t; i < m; i += nt) {
                double* row = &A[(size_t)(k + 1 + i) * n + k + 1];
                const double vi = v[i], qi = qv[i];
                for (int j = 0; j < m; ++j) row[j] -= vi * qv[j] + qi * v[j];
            }
        }
    });
    (void)failed;
    if (n >= 2) {
        d[n - 2] = A[(size_t)(n - 2) * n + (n - 2)];
        e[n - 2] = A[(size_t)(n - 1) * n + (n - 2)];
    }
    d[n - 1] = A[(size_t)(n - 1) * n + (n - 1)];
    e[n - 1] = 0.0;
    std::vector<double>().swap(A);
    // 4. eigenvalues, then eigenvectors of T by inverse iteration
    std::vector<double> ev;
    if (tridiag_eigenvalues(n, d, e, ev) != 0) return -2;
    double tnorm = 0.0;
    for (int i = 0; i < n; ++i)
        tnorm = std::max(tnorm, std::fabs(d[i]) + std::fabs(e[i]) + (i ? std::fabs(e[i - 1]) : 0.0));
    std::vector<double> W((size_t)n * n);   // row j = eigenvector j of T
    pool.run([&](int t, int nt) {
        std::vector<double> work;
        for (int j = t; j < n; j += nt) inverse_iteration(n, d.data(), e.data(), ev[j], tnorm, (unsigned)j + 1,
                                                          &W[(size_t)j * n], work);
    });
    // clusters of (numerically) coincident eigenvalues: modified Gram-Schmidt
    // inside each cluster. Elsewhere inverse iteration alone leaves an
    // orthogonality error of order eps ||T|| / gap, harmless for a preconditioner.
    const double ctol = 1e-10 * tnorm;
    std::vector<std::pair<int, int>> clusters;
    for (int j = 0; j < n;) {
        int j1 = j + 1;
        while (j1 < n && ev[j1] - ev[j1 - 1] <= ctol) ++j1;
        if (j1 - j > 1) clusters.push_back({j, j1});
        j = j1;
    }
    pool.run([&](int t, int nt) {
        for (size_t c = t; c < clusters.size(); c += nt) {
            for (int a = clusters[c].first; a < clusters[c].second; ++a) {
                double* va = &W[(size_t)a * n];
                for (int pass = 0; pass < 2; ++pass)
                    for (int b = clusters[c].first; b < a; ++b) {
                        const double* vb = &W[(size_t)b * n];
                        double dot = 0.0;
                        for (int i = 0; i < n; ++i) dot += va[i] * vb[i];
                        for (int i = 0; i < n; ++i) va[i] -= dot * vb[i];
                    }
                double nr = 0.0;
                for (int i = 0; i < n; ++i) nr += va[i] * va[i];
                nr = 1.0 / std::sqrt(nr);
                for (int i = 0; i < n; ++i) va[i] *= nr;
            }
        }
    });
    // 5. back-transform blocks of eigenvectors through the reflectors (last to
    //    first; each reflector is read once per block), then U = L^{-T} v
    const int JB = 32;
    const int nblk = (n + JB - 1) / JB;
    pool.run([&](int t, int nt) {
        std::vector<double> col(n);
        for (int blk = t; blk < nblk; blk += nt) {
            const int j0 = blk * JB, j1 = std::min(n, j0 + JB);
            for (int k = n - 3; k >= 0; --k) {
                if (tau[k] == 0.0) continue;
                const double* v = &V[(size_t)k * n];
                const int m = n - k - 1;
                for (int j = j0; j < j1; ++j) {
                    double* w = &W[(size_t)j * n + k + 1];
                    double s = 0.0;
                    for (int i = 0; i < m; ++i) s += v[i] * w[i];
                    s *= tau[k];
                    for (int i = 0; i < m; ++i) w[i] -= s * v[i];
                }
            }
            for (int j = j0; j < j1; ++j) {
                const double* w = &W[(size_t)j * n];
                for (int i = n - 1; i >= 0; --i) {
                    double v = w[i];
                    int i1 = std::min(n - 1, i + bw);
                    for (int k = i + 1; k <= i1; ++k) v -= L[(size_t)k * n + i] * col[k];
                    col[i] = v / L[(size_t)i * n + i];
                }
                for (int i = 0; i < n; ++i) U[(size_t)i * n + j] = col[i];
                lam[j] = ev[j];
            }
        }
    });
    return 0;
}

}  // namespace sgiga
