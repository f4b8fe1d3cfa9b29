// Internal data layout shared by the host planner and the CUDA kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define SGIGA_MAXP 4
#define SGIGA_MAXQ (SGIGA_MAXP + 1)

// Built-in sources with Dirichlet data (values of SGIGA_SRC_* in sgiga.h).
enum { SRC_LSHAPE_CORNER = 5, SRC_HARMONIC_QUADRATIC = 6 };

// One piece of a component grid: the component's tensor-product space on one
// geometry patch (single-patch domains: the whole component). Physical
// directions are 0..d-1 (direction 0 fastest in every packed or natural
// array).
//
// Function (f_0, f_1, ..) of the piece (full 1D indices 0..nf-1) is kept (a
// degree of freedom) if klo[k] <= f_k <= nf[k]-2 in every direction and it is
// not the excluded (0,0) corner (xcorner). It is stored at
//   dof_off + sum_k (f_k - slo[k]) * stride_k   (strides from n[]),
// except where f_k = 0 < slo[k] with alias[k] >= 0: that function is the same
// global function as (.., 0, ..) of piece alias[k] and is stored there. The
// high end of every direction is a Dirichlet end.
struct GridDesc {
    int lev[3];        // i_k
    int E[3];          // elements 2^{i_k}
    int nf[3];         // B-splines incl. the end functions
    int n[3];          // stored DoFs per direction: nf - 1 - slo
    int tab[3];        // 1D table id per direction
    int eig[3];        // 1D eigen table id per direction
    int perm[3];       // logical axis (a = pencil, b, c) -> physical direction
    int T[3];          // tile extent in elements per PHYSICAL direction
    int tile0, ntiles; // tiles of this grid: tile0 .. tile0+ntiles-1 (plan order)
    int chunk0, nchunk;// vector chunks of this grid (reductions)
    long long dof_off, ndof;
    long long qp_off, nqp;   // natural qp numbering
    long long tqp_off;       // first qp of this grid in tile-major numbering
    double coeff;
    int comp;                // component (CG system) of this piece
    int patch;               // geometry patch
    int klo[3];              // first kept function: 1 after a Dirichlet end, 0 at a patch interface
    int slo[3];              // first stored function (klo, or 1 where alias[k] stores f_k = 0)
    int alias[3];            // piece that stores the f_k = 0 functions, or -1
    int xcorner;             // the (0,0) function is a Dirichlet function of a neighbouring patch
    int fn[3];               // kept functions per direction, nf - 1 - klo (preconditioner tensor)
    long long fd_off, fd_n;  // that tensor in the preconditioner's local layout
    long long gf_off;        // full boundary-coefficient array [nf_1][nf_0] (multi-patch), else -1
};

// One component (CG system): its pieces are consecutive, and so are its
// stored DoFs and its vector chunks.
struct CompDesc {
    int piece0, npieces;
    int chunk0, nchunk;
    long long dof_off, ndof;
    double coeff;
};

// One Dirichlet side of one piece (multi-patch boundary data): direction k
// fixed at end (0 or 1); the side's parameter runs along direction 1-k (2D).
// g is given at 2 + E*Q points from goff: the two side ends, then the Gauss
// points of the side's elements.
struct SideDesc {
    int piece, k, end;
    long long goff;          // into the boundary data array
    long long soff;          // scratch of the projection: nf*(p+1) + nf doubles
};

// One tile of elements: the unit of work of the operator kernels.
struct TileDesc {
    int grid;
    int e0[3];          // first element per PHYSICAL direction
    long long g_off;    // first qp of the tile in tile-major numbering
};

// A 1D table: element data of one (direction, level).
struct Table1D {
    int dir, level, E, nf;
    long long off;      // into xi / w: E*Q entries; into R / dR: E*Q*(p+1)
    int eoff;           // into first[] and into breakpoints (E+1 entries at eoff + t)
    int koff, nk;       // into the knot array
};

// 1D eigen table for the fast-diagonalisation preconditioner.
struct Eig1D {
    int n;
    long long uoff;     // U [n][n] row-major at uoff
    long long loff;     // lambda [n] at loff
};

// One 1D generalised eigenproblem of the GPU eigensolver (eig.cu): n interior
// functions; band arrays Kb, Mb [n][p+1] with Kb[i][t] = K(i, i+t) (zero past
// the end) at boff; outputs at uoff (U and U^T, n x n) and loff (lam, n).
struct EigJob {
    int n;
    long long boff;
    long long uoff;
    long long loff;
    long long t0;          // first global thread of the job (bisection)
    double hi0;            // first upper bound tried for the eigenvalues: 2.17 max_i K_ii / M_ii
    double anorm;          // max_i sum_t |K_it| + hi0 |M_it|: the scale of K - s M's entries
    long long u0;          // first inverse-iteration unit of the job (all jobs' units in one launch)
    int nu;                // its units
    long long soff;        // its inverse-iteration scratch (doubles)
};

// Vector chunk: a contiguous piece of one component's packed vector (or of
// one piece's preconditioner tensor); grid = the component (scalar slot).
struct Chunk {
    int grid;
    int len;
    long long start;
    int piece;
};

// A tile of the network's tensor-core convolutions: 64 consecutive voxels
// (packed DoFs) of one vector chunk, from offset off.
struct ConvTile {
    int chunk;
    int off;
};

// Work item of the batched mode product of the preconditioner.
//   FD_SMALL: grid = piece, c0 = first column (fibre a*B + b) of a tile of
//             fd_small_cols(n) columns
//   FD_ROWS / FD_TILE: grid = piece, rows from i0, columns from c0 (a*B + b)
//   FD_LEVEL: grid = level segment (FDSeg), an output tile at rows i0,
//             columns c0 of the segment, contraction range [j0, j1)
enum { FD_SMALL = 0, FD_ROWS = 1, FD_TILE = 2, FD_LEVEL = 3 };

// Columns per FD_SMALL item for a direction of n <= 64 functions: the n x n
// matrix and an n x cols tile of fibres (rows padded by one) fill at most 48 KB
// of FP64 shared memory (6144 doubles); at most 2048 (for n = 3 a tile of 256
// fibres gave each block only 3 outputs per thread).
#ifdef __CUDACC__
__host__ __device__
#endif
inline int fd_small_cols(int n) {
    const int c = (6144 - n * (n + 1)) / (n + 1) - 1;
    return c < 2048 ? (c < 1 ? 1 : c) : 2048;
}
struct FDItem {
    int grid;
    int mode;
    int nc;             // FD_ROWS: columns of the group (1..8)
    int i0;             // first row (output index along the direction)
    long long c0;       // first column of the segment (FD_SMALL: of the piece's fibres)
    int j0, j1;         // contraction range [j0, j1) (split K: partial sums are added atomically)
};

// All long-direction mode products of one pass that share one eigenvector
// matrix (same direction, level and kind): one GEMM Y = Mat X whose columns
// are the columns of every such piece. Column c of the segment is the fibre
// at fdcb[col0 + c] + j * fdcs[col0 + c], j = 0..n-1, of component fdcc[...].
struct FDSeg {
    int eig;            // eigen table
    int n;              // its size
    int ncols;
    int unit;           // every column has stride 1 (direction 0)
    long long col0;     // first column in the column arrays
    int tn;             // output tile: 4096/tn rows x tn columns (tn = 16, 32 or 64, by column count)
    int pad;
};

// Geometry patch: tensor-product NURBS with separable weights.
struct Patch {
    int d;
    int deg[3];
    int nk[3];
    int nc[3];
    int rational[3];
    double knots[3][12];
    double w[3][8];       // 1D weights per direction (W = prod_k W_k)
    double cp[128][3];    // control points, direction 0 fastest
    int orient;           // -1: the map reverses orientation (det J < 0 everywhere), else +1 (0 reads as +1)
};

// Packed address of function (f0, f1) of a 2D piece (see GridDesc); the
// function must be kept.
#ifdef __CUDACC__
__host__ __device__
#endif
inline long long piece_addr2(const GridDesc* grids, const GridDesc& g, int f0, int f1) {
    if (f0 == 0 && g.slo[0] > 0 && g.alias[0] >= 0) {
        const GridDesc& h = grids[g.alias[0]];
        return h.dof_off + (0 - h.slo[0]) + (long long)(f1 - h.slo[1]) * h.n[0];
    }
    if (f1 == 0 && g.slo[1] > 0 && g.alias[1] >= 0) {
        const GridDesc& h = grids[g.alias[1]];
        return h.dof_off + (f0 - h.slo[0]) + (long long)(0 - h.slo[1]) * h.n[0];
    }
    return g.dof_off + (f0 - g.slo[0]) + (long long)(f1 - g.slo[1]) * g.n[0];
}

// Whether function (f0, f1) of a 2D piece is a degree of freedom.
#ifdef __CUDACC__
__host__ __device__
#endif
inline bool piece_kept2(const GridDesc& g, int f0, int f1) {
    return f0 >= g.klo[0] && f0 <= g.nf[0] - 2 && f1 >= g.klo[1] && f1 <= g.nf[1] - 2 &&
           !(g.xcorner && f0 == 0 && f1 == 0);
}
