// Shared pieces of the matrix-free operator kernels (sum factorisation of the
// Galerkin stiffness and load vector of Problem 1, Sec. 2.2).
//
// A thread block owns one tile of T_a x T_b (x T_c) elements of one component.
// Logical axes: a = the "pencil" axis processed per thread in registers, b and
// c the axes contracted through shared memory. Local DoF j of a tile along an
// axis with first element E0 is the full 1D index E0*m + j (m = p - r = knot
// multiplicity; element e's functions are e*m .. e*m + p). Dirichlet DoFs
// (full index 0 and nf-1) read as zero and are never written.
#pragma once
#include "internal.h"
#include "kernels.h"

namespace sgiga {

// Plan arrays of the operator kernels in the kernel's arithmetic type.
template <typename Real> struct OpData;
template <> struct OpData<double> {
    static __device__ __forceinline__ const double* G(const DevPlan& P) { return P.G; }
    static __device__ __forceinline__ const double* R(const DevPlan& P) { return P.R; }
    static __device__ __forceinline__ const double* dR(const DevPlan& P) { return P.dR; }
};
template <> struct OpData<float> {
    static __device__ __forceinline__ const float* G(const DevPlan& P) { return P.Gf; }
    static __device__ __forceinline__ const float* R(const DevPlan& P) { return P.Rf; }
    static __device__ __forceinline__ const float* dR(const DevPlan& P) { return P.dRf; }
};

// Exact n / d for 0 <= n < 2^21 with 1 <= d <= 256, and for 0 <= n < 2^17
// with 1 <= d <= 4096: a float reciprocal estimate is off by at most one there
// and one correction step fixes it (checked exhaustively over both ranges). Replaces runtime integer division
// in the staging loops, where it cost more instructions than the FMAs.
struct FastDiv {
    int d;
    float inv;
    __device__ explicit FastDiv(int dd) : d(dd), inv(1.0f / (float)dd) {}
    __device__ __forceinline__ int div(int n) const {
        int q = __float2int_rz((float)n * inv);
        const int r = n - q * d;
        if (r >= d) ++q;
        else if (r < 0) --q;
        return q;
    }
};

// A table row of N values from shared memory into registers: 128-bit loads
// for FP32 rows of 4 (the rows start at multiples of 4 floats: every table
// region holds T*Q rows of P+1 = 4 values), scalar loads otherwise.
template <typename Real, int N>
__device__ __forceinline__ void load_row(const Real* p, Real (&v)[N]) {
#pragma unroll
    for (int t = 0; t < N; ++t) v[t] = p[t];
}
template <>
__device__ __forceinline__ void load_row<float, 4>(const float* p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}

__device__ __forceinline__ int elem_lo(int j, int P, int M) { return j >= P ? (j - P + M - 1) / M : 0; }
__device__ __forceinline__ int elem_hi(int j, int M, int T) { int e = j / M; return e < T - 1 ? e : T - 1; }

// Shared-memory footprint (doubles) of one tile; T are logical extents.
__host__ __device__ inline long long op_smem_doubles(int d, int P, int M, const int* T) {
    const int Q = P + 1, P1 = P + 1;
    long long L[3], tab = 0;
    for (int x = 0; x < d; ++x) { L[x] = (long long)(T[x] - 1) * M + P1; tab += 2LL * P1 * Q * T[x]; }
    long long LaP = L[0] | 1;
    if (d == 2) return tab + L[0] * L[1] + 2LL * Q * T[1] * LaP;
    return tab + L[0] * L[1] * L[2] + 2LL * Q * T[2] * L[1] * L[0] + 3LL * (Q * T[1]) * (Q * T[2]) * LaP;
}

}  // namespace sgiga
