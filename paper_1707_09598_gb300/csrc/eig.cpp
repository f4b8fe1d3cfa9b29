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
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

namespace sgiga {

// K, M: dense row-major n x n (symmetric, M SPD with bandwidth bw).
// U: row-major n x n, column j = eigenvector j. Returns 0 on success.
int generalized_eigen(int n, int bw, const double* K, const double* M, double* U, double* lam) {
    if (n <= 0) return 0;
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

}  // namespace sgiga
