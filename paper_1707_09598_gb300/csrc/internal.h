// Internal data layout shared by the host planner and the CUDA kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define SGIGA_MAXP 4
#define SGIGA_MAXQ (SGIGA_MAXP + 1)

// One component grid. Physical directions are 0..d-1 (direction 0 fastest in
// every packed or natural array).
struct GridDesc {
    int lev[3];        // i_k
    int E[3];          // elements 2^{i_k}
    int nf[3];         // B-splines incl. the two Dirichlet ones
    int n[3];          // interior DoFs nf - 2
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

// Vector chunk: a contiguous piece of one grid's packed vector.
struct Chunk {
    int grid;
    int len;
    long long start;
};

// Work item of the batched mode product of the preconditioner.
enum { FD_SMALL = 0, FD_ROWS = 1, FD_TILE = 2 };
struct FDItem {
    int grid;
    int mode;           // FD_SMALL / FD_ROWS / FD_TILE
    int nc;             // FD_ROWS: columns of the group (1..8)
    int i0;             // first row (output index along the direction)
    long long c0;       // first column (a*B + b); FD_SMALL: first packed output
    int j0, j1;         // contraction range [j0, j1) (split K: partial sums are added atomically)
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
};
