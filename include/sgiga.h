/*
 * sgiga.h -- C ABI of the GB300 sparse-grid isogeometric Poisson solver.
 *
 * What it computes (Beck, Sangalli, Tamellini, arXiv:1707.09598):
 *   Problem 1 (Sec. 2.1): -Laplace(u) = f in Omega, u = 0 on the boundary,
 *   discretised on every component grid of the combination technique
 *   (Sec. 3, eq. TD-combi-tec) by tensor-product B-splines/NURBS pulled back
 *   through the geometry map F (Sec. 2.2, eqs. F-B-splines, spline_space_phys,
 *   u-IGA-approx), solved by Galerkin's method, and combined as
 *       u_J(x) = sum_i c_i u_i(x).
 *
 * Index convention. A component is i in N^d with i_k >= min_level and
 * w <= |i| <= w + d - 1; it has 2^{i_k} elements in direction k and the
 * combination coefficient c_i = (-1)^{w+d-1-|i|} binom(d-1, w+d-1-|i|)
 * (Sec. 3, eq. TD-combi-tec with beta = i - min_level). Components are
 * numbered 0..ngrids-1 in the order sgiga_grid_info reports.
 *
 * Vectors. A "packed" vector concatenates the interior (Dirichlet-eliminated)
 * coefficients of every component, component g starting at dof_off[g]; inside
 * a component direction 1 varies fastest. Quadrature points (qp) use a
 * "natural" order: component g's (p+1)E_1 x ... lattice of Gauss points,
 * direction 1 fastest, starting at qp_off[g].
 *
 * Conventions for every call:
 *   - returns SGIGA_OK (0) or a negative sgiga_status; never aborts; the
 *     message of the last failure on the calling thread is sgiga_last_error();
 *   - device pointers unless the parameter says "host or device"; such
 *     pointers are detected with cudaPointerGetAttributes and staged;
 *   - work is ordered on the plan's stream; a call returns once its status is
 *     known (calls that read results back synchronise the stream); a device
 *     buffer written on another stream must be complete, or that stream
 *     ordered before the plan's (an event), when the call is made;
 *   - the caller owns every buffer it passes; the plan owns the device memory
 *     it allocates and frees it in sgiga_destroy.
 */
#ifndef SGIGA_H
#define SGIGA_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sgiga_plan_s* sgiga_plan_t;

typedef enum {
    SGIGA_OK = 0,
    SGIGA_ERR_ARG = -1,           /* invalid argument or unsupported configuration */
    SGIGA_ERR_NOMEM = -2,         /* device or host allocation failed */
    SGIGA_ERR_CUDA = -3,          /* a CUDA runtime call or kernel launch failed */
    SGIGA_ERR_NOT_CONVERGED = -4, /* sgiga_solve reached max_iter before rel_tol */
    SGIGA_ERR_TIMEOUT = -5,       /* a bounded device wait gave up */
    SGIGA_ERR_GEOMETRY = -6       /* det J <= 0 at some quadrature point */
} sgiga_status;

/* Domains. UNIT: identity map on [0,1]^d. ANNULUS: quarter annulus with radii
 * 1 and 2 as a NURBS patch (direction 1 radial, degree 1; direction 2 angular,
 * degree 2, weights 1, sqrt(2)/2, 1), extruded along z in [0,1] when d = 3
 * (Sec. 4.2). LSHAPE (d = 2): (-1,1)^2 minus [0,1] x [-1,0] as three glued
 * bilinear patches x = s * xi with the parametric origin at the re-entrant
 * corner: patch 0 (0,1)x(0,1), s = (1,1); patch 1 (-1,0)x(0,1), s = (-1,1);
 * patch 2 (-1,0)x(-1,0), s = (-1,-1). Interfaces: xi_1 = 0 of patches 0 and
 * 1, xi_2 = 0 of patches 1 and 2 (conforming C^0 gluing); every other side is
 * a Dirichlet side. Every component uses the same knots on the three
 * patches; grading maps toward xi_k = 0 (use ONESIDED for the corner).
 * Packed layout of a component: blocks of patch 0, 1, 2; patch q's block
 * holds its functions (f_0, f_1) (full 1D indices, direction 0 fastest) with
 * s_0 <= f_0 <= nf_0 - 2 and s_1 <= f_1 <= nf_1 - 2, (s_0, s_1) = (0,1), (1,0),
 * (1,1) for q = 0, 1, 2. An interface function is stored once: f_0 = 0 of
 * patches 0 and 1 in patch 0's block, f_1 = 0 of patches 1 and 2 in patch 1's
 * block.
 * Preconditioner: weighted additive Schwarz over the patches (Neumann-Neumann
 * weights 1/2 on interface functions) with one exact fast-diagonalisation
 * solve per patch. The paper's graded-mesh experiments (Sec. 4.4) motivate
 * this domain; it is not among them. */
enum { SGIGA_DOMAIN_UNIT = 0, SGIGA_DOMAIN_ANNULUS = 1, SGIGA_DOMAIN_PATCH = 2, SGIGA_DOMAIN_LSHAPE = 3 };

/* A user geometry for SGIGA_DOMAIN_PATCH (eq. F-B-splines): a tensor-product
 * B-spline/NURBS patch with per-direction degree (<= 3), open knot vector
 * (<= 12 knots), control-point count (<= 8) and optional 1D weights (NULL:
 * polynomial direction; the weight function is their tensor product). cp is
 * [ncp0*ncp1*ncp2][d] (host), direction 0 fastest, at most 128 points. */
typedef struct {
    int deg[3];
    int nknots[3];
    const double* knots[3];
    int ncp[3];
    const double* weights[3];
    const double* cp;
} sgiga_patch;

/* Breakpoint grading g(j/E) (Sec. 4.4): UNIFORM g(t) = t; RADICAL
 * g(t) = 2^(gamma-1) t^gamma for t <= 1/2, 1 - 2^(gamma-1) (1-t)^gamma
 * otherwise; ONESIDED g(t) = t^gamma. */
enum { SGIGA_GRADING_UNIFORM = 0, SGIGA_GRADING_RADICAL = 1, SGIGA_GRADING_ONESIDED = 2 };

/* Arithmetic of the solve. FP64: every step in double precision.
 * MIXED_FP32: FP64 iterative refinement (residual r = b - K x with the FP64
 * operator, x += d) around an inner preconditioned-CG solve K d = r in FP32
 * (FP32 operator apply with FP32 geometry planes and tables, FP32
 * preconditioner), per-component scalars and reductions in FP64. After
 * sgiga_autotune a MIXED_FP32 plan with the FD preconditioner may solve as
 * FP64 PCG (its FP64 data is complete), preconditioned in FP64 or in FP32,
 * when that was faster on the probe (sgiga_tune_result.solve_precision,
 * solve_fp32_precond). */
enum { SGIGA_PREC_FP64 = 0, SGIGA_PREC_MIXED_FP32 = 1 };

/* Preconditioner of the batched conjugate-gradient solve. FD: fast
 * diagonalisation with the 1D generalised eigenpairs; NONE: plain CG;
 * LEARNED: FD with a trained elementwise scaling S * FD(S * r) (sgiga_net_*),
 * used by the inner FP32 solve of SGIGA_PREC_MIXED_FP32 as flexible CG (needs
 * that precision; plain FD until a network is initialised). */
enum { SGIGA_PRECOND_FD = 0, SGIGA_PRECOND_NONE = 1, SGIGA_PRECOND_LEARNED = 2 };

/* Built-in right-hand sides f = -Laplace(u) for manufactured solutions u:
 * SINE      u = prod_k sin(pi x_k)
 * POLY      u = prod_k x_k (1 - x_k)
 * ANNULUS   u = x y (x^2+y^2-1)(x^2+y^2-4) sin(x)        (d = 2)
 * ANNULUS_PAPER u = -(x^2+y^2-1)(x^2+y^2-4) x y^2 [sin(pi z)]  (Sec. 4.2)
 * ONE       f = 1
 * With Dirichlet data (LSHAPE plans; f = 0, u = g on the Dirichlet sides):
 * LSHAPE_CORNER  u = r^(2/3) sin(2 theta / 3), theta in [0, 2 pi) from the
 *                positive x axis (harmonic; singular gradient at the corner)
 * HARMONIC_QUADRATIC u = 1 + 2x - 3y + (x^2 - y^2)/2 + xy (in every p >= 2
 *                space of the L-shape: reproduced exactly) */
enum { SGIGA_SRC_SINE = 0, SGIGA_SRC_POLY = 1, SGIGA_SRC_ANNULUS = 2,
       SGIGA_SRC_ANNULUS_PAPER = 3, SGIGA_SRC_ONE = 4, SGIGA_SRC_LSHAPE_CORNER = 5,
       SGIGA_SRC_HARMONIC_QUADRATIC = 6 };

typedef struct {
    int d;            /* 2 or 3 */
    int p;            /* spline degree, 1..4 */
    int continuity;   /* r of C^r at interior breakpoints, 0..p-1; -1 means p-1 */
    int w;            /* combination level: components with w <= |i| <= w+d-1 */
    int min_level;    /* smallest i_k (>= 0); 1 in the usual setting */
    int domain;       /* SGIGA_DOMAIN_* */
    int grading;      /* SGIGA_GRADING_* */
    double gamma;     /* grading exponent (ignored for UNIFORM) */
    int precision;    /* SGIGA_PREC_* */
    int precond;      /* SGIGA_PRECOND_* */
    const sgiga_patch* patch; /* geometry for SGIGA_DOMAIN_PATCH (host), else NULL */
    int ncomponents;  /* > 0: the plan holds only these components of the index
                         set (e.g. one, to solve the grids one at a time); 0: all */
    const int* components; /* [ncomponents][d] levels (host), each in the index set of w */
    const double* coefficients; /* with ncomponents > 0: the combination coefficient of each
                         listed component (host); the components then form an arbitrary
                         index set (levels >= min_level, w ignored), e.g. one chosen by the
                         profits of the hierarchical surpluses (Sec. 4.2, the knapsack view
                         of the sparse-grid set). NULL: coefficients of eq. TD-combi-tec */
} sgiga_config;

typedef struct {
    int d, p, continuity, ngrids;
    long long ndof;   /* packed vector length */
    long long nqp;    /* total quadrature points */
    int max_tile_smem; /* bytes of dynamic shared memory of the operator kernel */
    int ntiles;
    int diag_metric;   /* 1 if every off-diagonal geometry coefficient is exactly zero
                          (the operator kernels then skip the cross terms) */
    int npatches;      /* geometry patches (3 for LSHAPE, else 1) */
    long long nbpts;   /* boundary data points (sgiga_boundary_points), 0 if none */
} sgiga_info;

typedef struct {
    int levels[3];     /* i_k */
    int n[3];          /* interior DoFs per direction */
    int coeff;         /* combination coefficient c_i */
    long long ndof, dof_off, nqp, qp_off;
    int tile[3];       /* elements per tile of the operator kernels, per direction */
    int pencil_dir;    /* direction processed per thread in registers */
    int ntiles;        /* tiles of this component */
} sgiga_grid;

typedef struct {
    int iterations;          /* outer iterations run (max over components) */
    int converged;           /* number of components that met rel_tol */
    double max_rel_residual; /* max_g ||b_g - K_g x_g|| / ||b_g|| (recursive residual) */
    double seconds;          /* wall time of the call */
    int inner_iterations;    /* MIXED_FP32: inner CG iterations summed over refinement steps */
    int fallback;            /* MIXED_FP32 bit flags. 1 (LEARNED): the learned scaling was
                                switched off for the rest of the solve, after a refinement step
                                without a tenfold residual reduction (FD continues).
                                2: refinement stalled (two steps that did not halve some
                                component's residual: the FP32 operator's error times the
                                condition number is not small) and FP64 PCG finished the
                                remaining components from the current residual */
} sgiga_solve_stats;

/* Build a plan: index set and coefficients (Sec. 3), knot vectors and
 * grading (Sec. 2.2, 4.4), Gauss rule, 1D basis tables (eq. Bsp), geometry
 * coefficients at every quadrature point, 1D generalised eigenpairs of the
 * preconditioner, and the tile schedule. `stream` is a cudaStream_t (NULL:
 * the legacy default stream). On success *out owns its device memory. */
int sgiga_plan(const sgiga_config* cfg, void* stream, sgiga_plan_t* out);

/* Release every resource of the plan (NULL is a no-op). */
void sgiga_destroy(sgiga_plan_t plan);

int sgiga_plan_info(sgiga_plan_t plan, sgiga_info* out /* host */);

/* Wall-clock seconds of the plan's set-up phases (host clock; every phase
 * ends with a stream synchronisation). total = host + basis + eigen + fd +
 * geometry + vectors, the sgiga_plan call (Sec. 4.1 times set-up, here the
 * analogue of the paper's mesh set-up and assembly, together with the solve).
 *   host        index set, coefficients, knots, tiles (host)
 *   basis       1D B-spline/NURBS tables on the device and their copy back
 *   eigen       1D generalised eigenproblems on the device (band assembly on
 *               the host, bisection and inverse iteration on the device)
 *   fd          preconditioner work items and eigenvalue-sum reciprocals
 *   geometry    geometry coefficients at every quadrature point
 *   vectors     solver vectors and FP32 copies
 * coefficient: the last sgiga_set_coefficient; autotune: the last
 * sgiga_autotune (0 if not called). */
typedef struct {
    double total, host, basis, eigen, fd, geometry, vectors;
    double coefficient, autotune;
} sgiga_plan_times_t;
int sgiga_plan_times(sgiga_plan_t plan, sgiga_plan_times_t* out /* host */);
int sgiga_grid_info(sgiga_plan_t plan, int g, sgiga_grid* out /* host */);

/* Physical coordinates x = F(xi_q) of every quadrature point: xq is a host or
 * device buffer [d][nqp] (one plane per coordinate, natural qp order). */
int sgiga_qp_coords(sgiga_plan_t plan, double* xq);

/* Load vector b_i = sum_q w_q |det J_q| f(x_q) R_i(xi_q) (Sec. 2.2, Galerkin
 * right-hand side) from f at the quadrature points: f_qp is [nqp] in natural
 * order, host or device. With a device buffer the call is stream-ordered and
 * returns without synchronising. A host buffer has been read in full when the
 * call returns: page-locked host memory (cudaHostAlloc, cudaHostRegister) is
 * read in place by the kernel over the host link, pageable memory through a
 * staging copy. */
int sgiga_set_rhs(sgiga_plan_t plan, const double* f_qp);

/* Same, with f from a built-in manufactured solution (SGIGA_SRC_*),
 * evaluated on the device. The two sources with Dirichlet data (LSHAPE plans)
 * also set the boundary data g = u (as sgiga_set_dirichlet). */
int sgiga_set_rhs_builtin(sgiga_plan_t plan, int source);

/* Nonhomogeneous Dirichlet data of an LSHAPE plan (not in the paper; the
 * reading of the build): on each Dirichlet side of each component's patch
 * pieces, the two end coefficients interpolate g and the others are the L2
 * projection of g onto the side's 1D spline space (parametric measure = arc
 * length on these unit sides, p+1 Gauss points per element); then the load
 * vector becomes b_I - K_IB g_B and evaluations include the boundary part.
 * sgiga_boundary_points writes the physical points where g is needed, xb
 * [nbpts][2] (host or device; nbpts from sgiga_plan_info): per component,
 * per piece, per Dirichlet side, the side's two ends then the Gauss points of
 * its elements; plus one point (the corner) for a piece whose (0,0) function
 * is fixed by a neighbour's side. sgiga_set_dirichlet takes g at those
 * points, g [nbpts] (host or device), or NULL for homogeneous data. Call it
 * before sgiga_set_rhs. SGIGA_ERR_ARG on a plan without boundary data. */
int sgiga_boundary_points(sgiga_plan_t plan, double* xb);
int sgiga_set_dirichlet(sgiga_plan_t plan, const double* g);

/* f(x_q) of a built-in source (SGIGA_SRC_*) at every quadrature point, in
 * natural qp order: f is [nqp], host or device (input data for sgiga_set_rhs). */
int sgiga_source_at_qp(sgiga_plan_t plan, int source, double* f);

/* Diffusion coefficient a(x) in -div(a grad u) = f: a = exp(amp * sum_f
 * cos(omega_f . x + phase_f)), a random-Fourier-feature sample of a log-normal
 * field (not in the paper, whose coefficient is 1). omega [nfeat][d] and phase
 * [nfeat] are host arrays; nfeat = 0 restores a = 1. The geometry
 * coefficients of every quadrature point are recomputed (K_ij gains the factor
 * a(x_q)); the load vector and the preconditioner are unchanged. */
int sgiga_set_coefficient(sgiga_plan_t plan, int nfeat, const double* omega, const double* phase, double amp);

/* Diffusion coefficient given at the quadrature points: a_qp [nqp] in natural
 * qp order (host or device; values of a(F(xi_q)) > 0), or NULL to restore
 * a = 1. K_ij = sum_q w_q |det J_q| a_q grad R_i^T (J_q^T J_q)^{-1} grad R_j
 * (Galerkin stiffness of -div(a grad u), Sec. 2.2 with a variable
 * coefficient); the geometry coefficients are recomputed, the load vector
 * and the preconditioner are unchanged. sgiga_set_coefficient evaluates its
 * Fourier features into the same plane. The plan keeps the values (a
 * re-tiling by sgiga_autotune reuses them). SGIGA_ERR_ARG if some value is
 * not positive and finite (the plan then keeps a = 1). */
int sgiga_set_coefficient_qp(sgiga_plan_t plan, const double* a_qp);

/* Copy the current packed load vector to b ([ndof], host or device). */
int sgiga_get_rhs(sgiga_plan_t plan, double* b);

/* y = K x for every component at once (matrix-free, sum factorisation of the
 * Galerkin stiffness of Sec. 2.2 with Dirichlet rows and columns removed).
 * x, y: device packed vectors [ndof]; y is overwritten. */
int sgiga_apply(sgiga_plan_t plan, const double* x, double* y);

/* FP32 variant of sgiga_apply (the inner operator of the MIXED_FP32 solve):
 * FP32 geometry planes and basis tables, FP32 accumulation. x, y: device
 * float [ndof]. Needs a plan built with SGIGA_PREC_MIXED_FP32. */
int sgiga_apply_f32(sgiga_plan_t plan, const float* x, float* y);

/* z = P^{-1} r with the fast-diagonalisation preconditioner of every
 * component, z = (U_d x .. x U_1) diag(sum_k lambda_k)^{-1} (U_d x .. x U_1)^T r
 * with the 1D generalised eigenpairs of the parametric stiffness and mass
 * matrices (a preconditioner the paper does not use: it names such fast
 * solvers as future work, Sec. 5). Exact inverse on the unit square/cube.
 * Device packed vectors. */
int sgiga_precond(sgiga_plan_t plan, const double* r, double* z);
/* FP32 variant of sgiga_precond (the preconditioner of the MIXED_FP32 inner
 * solve): FP32 eigenvectors and eigenvalue reciprocals, FP32 accumulation.
 * r, z: device float [ndof]. Needs a plan built with SGIGA_PREC_MIXED_FP32. */
int sgiga_precond_f32(sgiga_plan_t plan, const float* r, float* z);

/* Solve K_g u_g = b_g for every component g (batched preconditioned CG,
 * per-component scalars and convergence) until ||r_g|| <= rel_tol ||b_g|| or
 * max_iter iterations (MIXED_FP32: max_iter refinement steps, each with an
 * inner FP32 solve to relative residual 1e-5 or 100 iterations; the stopping
 * test uses the true FP64 residual). The solution stays in the plan
 * (sgiga_get_solution). Returns SGIGA_ERR_NOT_CONVERGED if some component did
 * not converge, SGIGA_ERR_ARG (before any iteration) if some component's load
 * vector holds a NaN or an infinity. */
int sgiga_solve(sgiga_plan_t plan, double rel_tol, int max_iter,
                sgiga_solve_stats* stats /* host, may be NULL */);

/* Autotuner of the operator and preconditioner work decomposition.
 * (1) Re-plans the tiles of every component under each candidate policy
 * (shared-memory budget per block, cap on quadrature points per tile; the
 * shape within a policy comes from the planner's cost model), times `reps`
 * stiffness applies (FP32 in MIXED_FP32 plans, whose inner solve they
 * dominate; else FP64) on the plan's stream for each (CUDA events; FP32 3D
 * plans time each policy with 256 and with 128 threads per block, and, for p
 * odd, with four settings of the metric planes' L2 prefetch), and keeps the
 * fastest; the geometry planes are computed once and gathered into each
 * candidate's tile layout (recomputed from the patch map when the device has
 * no room for the natural-layout copy, (d(d+1)/2 + 1) * nqp doubles).
 * (2) Re-splits the fast-diagonalisation mode products into work items of
 * each candidate layout (per piece, level-grouped) and contraction depth
 * (fd_ks: entries of a long 1D contraction per item; shorter items balance
 * the SMs better, longer ones need fewer atomic partial sums), times `reps`
 * preconditioner applications for each and keeps the fastest. Overwrites the plan's work vectors (not its load vector
 * or solution). out (host, may be NULL) receives the per-candidate mean
 * times. (3) See solve_precision below. */
typedef struct {
    int ncand, best, ntiles;
    double best_ms;
    double ms[16];
    int budget[16];   /* bytes of shared memory per block */
    int qpcap[16];    /* quadrature points per tile at most */
    int nthreads[16]; /* threads per block of the operator kernel (FP32 3D plans try 256 and 128) */
    int fd_ncand, fd_best, fd_nitems;
    int fd_ks[8];     /* contraction depth per preconditioner work item */
    double fd_ms[8];  /* mean time of one preconditioner application */
    int fd_grouped[8];/* 1: level-grouped layout, 0: per-piece layout */
    int prefetch[16]; /* FP32 3D plans, p odd: the candidate's fastest L2 prefetch of a tile's metric planes at tile
                         start (0: whole segments; > 0: at most this many bytes per plane, so that the segments in
                         flight on all SMs total 48 or 16 MB; -1: none) */
    int best_prefetch;
    /* (3) MIXED_FP32 plans with the FD preconditioner: the precision
     * sgiga_solve uses from now on (SGIGA_PREC_FP64 when FP64 PCG, with the
     * FP64 or the FP32 preconditioner, solved a probe load vector to 1e-8
     * faster than the mixed solve, as where FD is nearly exact; the
     * decomposition is then tuned again with that solve's kernels, and the
     * fields above report that tuning), and the probe solves' wall times (ms;
     * 0: not run or, for FP64, not converged within the iterations that fit
     * in twice the fastest time so far, at least 4).
     * Other plans: their own precision, times 0. */
    int solve_precision;
    double solve_ms_fp64, solve_ms_mixed;
    /* FP64 PCG preconditioned by the FP32 FD (narrowed residual, widened
     * output, flexible CG), the third probe: its time (ms; 0 as above), and 1
     * when it was the fastest and sgiga_solve now runs it. It is run only if
     * it was the fastest to 1e-8 and is also not slower than FP64 PCG with
     * the FP64 preconditioner to 1e-12 (a second pair of probe solves, not
     * reported): the FP32 rounding of the preconditioned residual costs extra
     * iterations near FP64 tolerances. */
    double solve_ms_fp64_fd32;
    int solve_fp32_precond;
} sgiga_tune_result;
int sgiga_autotune(sgiga_plan_t plan, int reps, sgiga_tune_result* out);

/* Sets the operator's work decomposition directly (a setting that
 * sgiga_autotune reported, to reuse it without timing again): the tile policy
 * (budget: shared-memory bytes per block, 16 KB..227 KB; qpcap: quadrature
 * points per tile at most), the FP32 3D kernel's threads per block (256 or
 * 128) and its L2 prefetch of a tile's metric planes (0 whole segments, > 0 at
 * most this many bytes per plane, a multiple of 16; < 0 none). The geometry
 * planes are recomputed in the new tile layout. SGIGA_ERR_ARG on a value out
 * of range. No counterpart in the paper (a GPU work-decomposition setting). */
int sgiga_set_tiling(sgiga_plan_t plan, int budget, int qpcap, int nthreads, int prefetch);

/* Solver options. use_graph != 0 (default): each CG loop runs as one captured
 * CUDA graph whose while-conditional node repeats the iteration body until the
 * device-side convergence test stops it (no host round trip per iteration);
 * 0: a host loop that reads the number of active components back every
 * iteration. inner_tol / inner_max: tolerance and iteration limit of the FP32
 * inner solve of SGIGA_PREC_MIXED_FP32 (defaults 1e-5, 100). */
int sgiga_set_solver_options(sgiga_plan_t plan, int use_graph, double inner_tol, int inner_max);

/* Work layout of the preconditioner's mode products. ks: a 1D contraction
 * longer than ks entries is split into ks-deep items whose partial sums are
 * added atomically. grouped = 0: items of one component piece each (ROWS /
 * TILE shapes; the FP64 default); 1: the long directions of all pieces that
 * share an eigenvector matrix form one GEMM over all their fibres (the FP32
 * default). The autotuner picks both by measurement; default ks = 32. ks
 * must be a multiple of 16 in [16, 4096], else SGIGA_ERR_ARG. The result
 * changes only by summation order. */
int sgiga_set_precond_split(sgiga_plan_t plan, int ks, int grouped);

/* Packed solution coefficients (device [ndof]). */
int sgiga_get_solution(sgiga_plan_t plan, double* u);
/* Replace the plan's packed solution (device [ndof]); used to evaluate
 * arbitrary coefficient vectors. */
int sgiga_set_solution(sgiga_plan_t plan, const double* u);

/* Evaluate every component u_g = sum_i c_i R_i at parametric points
 * (Sec. 4.1: post-processing): xi is [npts][d] (host or device), u_comp is
 * [ngrids][npts] (host or device). A parametric point is the same physical
 * point F(xi) in every component because all share the exact geometry. */
int sgiga_eval(sgiga_plan_t plan, const double* xi, long long npts, double* u_comp);

/* Values and physical gradients of every component (2D and 3D plans, any
 * domain; the one evaluation of multi-patch plans). xi [npts][d] parametric
 * points, patch [npts] the patch of each point (NULL: patch 0), u_comp
 * [ngrids][npts], grad_comp [d][ngrids][npts] (x, y [, z] derivative; NULL to
 * skip), all host or device. grad u = J^{-T} grad_xi u with J the patch's
 * Jacobian (eq. F-B-splines). Values include the Dirichlet lifting where
 * boundary data is set. SGIGA_ERR_ARG for a point outside [0,1]^d or a patch
 * id out of range. */
int sgiga_eval_grad(sgiga_plan_t plan, const double* xi, const int* patch, long long npts, double* u_comp,
                    double* grad_comp);

/* Linear functional of the combined solution without evaluation points:
 * l(u) = sum_g c_g int_Omega q u_g dx = sum_g c_g (b_q . u_g), with b_q the
 * load vector of q in component g's space (the right-hand side's rule,
 * Sec. 2.2) and the combination coefficients of eq. TD-combi-tec. q_qp is q at
 * the quadrature points [nqp] in natural order (as for sgiga_set_rhs), host or
 * device. comp [ngrids] (host, may be NULL) receives the per-component
 * values, *combined (host) the Neumaier-compensated sum. Uses the plan's
 * solution; the load vector is not changed. SGIGA_ERR_ARG on a plan with
 * Dirichlet data. */
int sgiga_functional(sgiga_plan_t plan, const double* q_qp, double* comp, double* combined);

/* The geometry map at parametric points (eq. F-B-splines): x = F(xi)
 * [npts][d] and det J [npts] (signed; NULL to skip), for points xi [npts][d]
 * of the given patches (patch [npts], NULL: patch 0); host or device buffers.
 * Serves error integrals on the physical domain (weights times |det J|).
 * SGIGA_ERR_ARG for a point outside [0,1]^d or a patch id out of range. */
int sgiga_map_points(sgiga_plan_t plan, const double* xi, const int* patch, long long npts, double* x,
                     double* detj);

/* u[j] = sum_g c_g u_comp[g][j], FP64 with Neumaier compensation
 * (eq. TD-combi-tec). u_comp [ngrids][npts], u [npts], host or device. */
int sgiga_combine(sgiga_plan_t plan, const double* u_comp, long long npts, double* u);

/* The same compensated sum over the components of several plans, each with
 * its own combination coefficients: u[j] = sum_k sum_g c_{k,g} u_comp_k[g][j].
 * u_comp holds the plans' sgiga_eval outputs one after the other, in the
 * order of plans[] ([sum_k ngrids_k][npts]); u [npts]; host or device.
 * Serves combinations whose components differ in more than their levels, as
 * the h-p sparse combination does (components of several degrees at one
 * continuity, one plan per degree, coefficients from the combination of a
 * downward-closed set of (levels, degree) indices: eq. Delta-combi-tec with
 * the degree as one more index; the paper names p- and h-p-sparsification as
 * possible in Sec. 2.2 and as an extension in Sec. 5). The plans must have
 * the same dimension d and share one stream (SGIGA_ERR_ARG otherwise); that
 * they discretise the same problem is the caller's responsibility. Runs on
 * that stream and synchronises it; uses the first plan's staging buffer. */
int sgiga_combine_plans(int nplans, const sgiga_plan_t* plans /* host [nplans] */, const double* u_comp,
                        long long npts, double* u);

/* Diagnostics for parity tests (host outputs). The 1D table of direction
 * `dir` (0-based) at level `level`: Gauss points xi [E(p+1)], weights w
 * [E(p+1)] (times h/2), basis values R and derivatives dR [E(p+1)][p+1] of the
 * p+1 functions first[e] .. first[e]+p nonzero on element e, first [E]. */
int sgiga_basis_table(sgiga_plan_t plan, int dir, int level, double* xi, double* w,
                      double* R, double* dR, int* first);
/* Geometry coefficients of component g in natural qp order: G is
 * [d(d+1)/2][nqp_g] with the upper triangle of w |det J| (J^T J)^{-1} row by
 * row ((0,0),(0,1),..), then mw [nqp_g] = w |det J|. Host output. */
int sgiga_geometry_coeffs(sgiga_plan_t plan, int g, double* G, double* mw);
/* Generalised eigenpairs K U = M U diag(lam), U^T M U = I, of the 1D interior
 * matrices of direction `dir` at level `level`: U [n][n] row-major (column j
 * is eigenvector j), lam [n] ascending. Host outputs. */
int sgiga_fd_eigen(sgiga_plan_t plan, int dir, int level, double* U, double* lam);

/* ---------------------------------------------------------------------------
 * The combination technique as a preconditioner of a full tensor-product
 * solve (the paper's closing remark, Sec. 5): the full plan (one component of
 * levels (J, .., J)) is preconditioned by the additive two-level method
 *
 *   z = FD(r) + sum_i c_i P_i K_i^{-1} P_i^T r
 *
 * over the components i of the combination plan (its index set and
 * coefficients, eq. TD-combi-tec), P_i the prolongation of component i's
 * space into the full space by knot insertion, K_i^{-1} the combination
 * plan's batched PCG to inner_tol (at most inner_max iterations; an inexact
 * inner solve is allowed: the full plan's CG runs flexible, from the host).
 * Both plans: FP64, FD preconditioner, single patch, uniform knots, the same
 * dimension, degree, continuity and domain (patch), the same stream; every
 * component at most as fine as the full grid; the same diffusion coefficient
 * is the caller's to set on both. The combination plan must outlive the
 * attachment; its load vector and solution are overwritten by every full
 * solve. Q = NULL detaches. SGIGA_ERR_ARG when a condition fails.
 * sgiga_solve of the full plan then reports the total inner iterations in
 * sgiga_solve_stats.inner_iterations. */
int sgiga_ct_attach(sgiga_plan_t full, sgiga_plan_t ct, double inner_tol, int inner_max);
/* z = sum_i c_i P_i K_i^{-1} P_i^T r alone (no FD), r and z device double
 * [ndof of the full plan]. SGIGA_ERR_ARG without an attachment. */
int sgiga_ct_apply(sgiga_plan_t full, const double* r, double* z);

/* ---------------------------------------------------------------------------
 * Learned scaling of the preconditioner (not in the paper; its conclusions
 * name fast solvers used as preconditioners as future work, Sec. 5).
 *
 *   M(r) = S * FD(S * r)   (elementwise products, FD = sgiga_precond_f32),
 *   S = exp(-phi / 2 + 4 tanh(N(phi) / 4)),  phi_i = log c_i,
 *   c_i = sum_q R_i(xi_q) tr(G_q) / (d sum_q R_i(xi_q) w_q),
 * c_i being the local effective coefficient of DoF i: the R_i-weighted mean of
 * the trace of the Galerkin metric G_q = w_q |det J_q| a(x_q) (J_q^T J_q)^{-1}
 * relative to the parametric Laplacian (G_q = w_q I), which FD inverts
 * exactly. The network corrects the network-free scaling S = c^(-1/2) (the
 * inverse square root of the local coefficient, exact for a constant
 * coefficient on an axis-aligned box), which its untrained state (N = 0)
 * gives; the tanh bounds the correction by a factor e^(+-4). N: three 3^d convolutions over each component's DoF tensor (zero
 * padding), 1 -> 32 -> 32 -> 1 channels, ReLU after the first two; BF16
 * weights with an FP32 master copy, FP32 accumulation. S depends only on the
 * operator, so M is a fixed symmetric positive definite operator: the
 * network runs once per plan (after training, loading or a geometry change),
 * not once per CG iteration. The inner FP32 solve of SGIGA_PREC_MIXED_FP32
 * uses M in flexible CG; a component whose network output is not finite
 * keeps S = 1 there (plain FD), and a refinement step that does not cut the
 * worst residual tenfold switches back to FD for the rest of the solve. Every
 * function below needs a single-patch plan built with SGIGA_PREC_MIXED_FP32.
 * ------------------------------------------------------------------------- */
typedef struct {
    int target_pairs;     /* component-level (residual, error) pairs to record (e.g. 10000) */
    int max_iter_record;  /* CG iterations recorded per random right-hand side */
    int epochs;           /* passes over the recorded samples */
    float lr;             /* Adam learning rate */
    unsigned seed;        /* right-hand sides and sample order */
    int batch;            /* samples per Adam step (0: 2) */
    int loss_norm;        /* 0: Euclidean ||M(r) - e||^2 / ||e||^2; 1: energy norm
                             (M(r) - e)^T K (M(r) - e) / e^T K e, K the FP32 operator */
} sgiga_train_cfg;

typedef struct {
    int pairs, samples, rhs, steps;
    double loss_first_epoch, loss_last_epoch;  /* mean over samples of the mean over components of
                                                  ||M(r) - e||^2 / ||e||^2 */
    double seconds;
    double loss_initial;     /* the same at the initial parameters (before any step) */
    double loss_fd;          /* the same with S = 1 (plain FD) */
    double loss_epoch[32];   /* per epoch (the first 32) */
    double logs_min, logs_max; /* range of log S after training */
    int best_epoch;          /* epoch whose parameters were kept (-1: the initial ones) */
    int val_iters_initial;   /* inner iterations of the validation solve at the initial parameters
                                (1000 more if it did not converge) */
    int val_iters_best;      /* the same at the kept parameters */
} sgiga_train_stats;

/* Allocate the network and initialise it (seeded Kaiming-uniform; the last
 * layer zero, so that the untrained N is 0 and S = c^(-1/2)). */
int sgiga_net_init(sgiga_plan_t plan, unsigned seed);
/* Number of parameters (a negative status if there is no network). Layout of
 * the FP32 vector: W1 [32][1][T], b1 [32], W2 [32][32][T], b2 [32], W3 [1][32][T],
 * b3 [1], T = 3^d taps ordered offset_0 fastest over (-1, 0, 1)^d. */
int sgiga_net_num_params(sgiga_plan_t plan);
int sgiga_net_get_params(sgiga_plan_t plan, float* params /* host [nparams] */);
int sgiga_net_set_params(sgiga_plan_t plan, const float* params /* host [nparams] */);
/* N(in) with in = device float [ndof] (one channel over the packed vector),
 * out = device float [ndof]. */
int sgiga_net_forward(sgiga_plan_t plan, const float* in, float* out);
/* Gradient of sum_v dy_v N(in)_v with respect to every parameter (host
 * [nparams]); in, dy device float [ndof]. */
int sgiga_net_backward(sgiga_plan_t plan, const float* in, const float* dy, float* grad);
/* The network input phi = log c of the plan's current geometry coefficients
 * (float [ndof], host or device). */
int sgiga_net_features(sgiga_plan_t plan, float* phi);
/* The scaling S the preconditioner uses (float [ndof], host or device). */
int sgiga_net_scaling(sgiga_plan_t plan, float* S);
/* Replace S by the caller's positive values (float [ndof], host or device),
 * bypassing the network until the next sgiga_net_init, _set_params, _load or
 * sgiga_train_net (e.g. S = c^{-1/2}, a scaling without a network). */
int sgiga_net_set_scaling(sgiga_plan_t plan, const float* S);
/* Training loss of one sample at the current S, the mean over components of
 * ||M(r) - e||^2 / ||e||^2 (*loss, host), and its gradient with respect to
 * log S (grad, device float [ndof]); r, e device float [ndof]. */
int sgiga_net_loss_grad(sgiga_plan_t plan, const float* r, const float* e, double* loss, float* grad);
/* Norm of that loss for sgiga_net_loss_grad (sgiga_train_net sets it from its
 * config): 0 Euclidean, 1 the energy norm of the plan's FP32 operator K,
 * L = (M(r) - e)^T K (M(r) - e) / e^T K e, whose gradient uses
 * delta = 2 K (M(r) - e) / e^T K e in place of 2 (M(r) - e) / ||e||^2. */
int sgiga_net_set_loss_norm(sgiga_plan_t plan, int norm);
/* Record (residual, error) pairs from the plan's own FD-preconditioned FP64 CG
 * on seeded random right-hand sides and train N by Adam on the loss above,
 * back-propagated through S (above). In a recorded sample only the
 * components whose residual was still above 1e-6 of their right-hand side
 * count (a converged component's recorded error is rounding noise of two
 * solves). Kept: the parameters after an epoch (or the initial ones) with
 * which the plan's own solve (sgiga_solve to 1e-8 with the current solver
 * options) of a validation right-hand side held out of the pairs
 * (b = K FD(xi), own seed) needs the fewest inner FP32 iterations, the
 * earliest among equals. Overwrites the plan's load vector and solution. */
int sgiga_train_net(sgiga_plan_t plan, const sgiga_train_cfg* cfg, sgiga_train_stats* stats /* may be NULL */);
/* Checkpoint: magic "SGIGANET", version 2, taps, nparams, Adam step, then the
 * FP32 parameters and both Adam moments. */
int sgiga_net_save(sgiga_plan_t plan, const char* path);
int sgiga_net_load(sgiga_plan_t plan, const char* path);

/* ---------------------------------------------------------------------------
 * Allocation-free preconditioner apply (the paper has no counterpart; this is
 * a service for callers of the library).
 *
 * For callers that cannot call cudaMalloc where they need it: real-time loops
 * that must not touch the device allocator after start-up, processes whose
 * device memory is owned by another allocator that must account for every
 * byte, and code running where an allocation is not permitted. It needs no
 * plan: the caller passes the 1D eigenpairs.
 *
 * Computes, for ONE tensor-product grid with n[0] x .. x n[d-1] entries
 * (direction 0 fastest),
 *     z = (U_{d-1} x .. x U_0) diag(sum_k lam_k)^{-1} (U_{d-1} x .. x U_0)^T r,
 * the same fast-diagonalisation operator as sgiga_precond.
 *   d        1..3
 *   n        host [d], sizes per direction
 *   U, lam   host arrays of d DEVICE pointers: U[k] is n[k] x n[k] row-major
 *            (column j = eigenvector j, as sgiga_fd_eigen returns it), lam[k]
 *            the n[k] eigenvalues
 *   r, z     device [prod n]; z may alias r
 *   stream   cudaStream_t (NULL: legacy default stream); the call only
 *            enqueues kernels and returns without synchronising
 * Intermediate tensors live in a library-owned device array of
 * 2 * SGIGA_NOALLOC_MAX_DOFS doubles (4 MB on every GPU that loads the
 * library, held until the process exits). Grids with more than
 * SGIGA_NOALLOC_MAX_DOFS entries are rejected with SGIGA_ERR_ARG. The call
 * allocates nothing. The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current. The looked-up
 * address stays valid while the device's primary context lives: after a
 * cudaDeviceReset the entry point must not be called again on that device. All calls share the array, so calls that
 * overlap on the GPU race on it: order them on one stream. Returns SGIGA_OK,
 * SGIGA_ERR_ARG or SGIGA_ERR_CUDA (message in sgiga_last_error()). */
#define SGIGA_NOALLOC_MAX_DOFS 262144
int sgiga_fd_apply_noalloc(int d, const int* n, const double* const* U, const double* const* lam,
                           const double* r, double* z, void* stream);

const char* sgiga_last_error(void);

/* Number of CUDA kernels this library has launched in this process so far
 * (a diagnostic count; memsets and copies are not included). */
long long sgiga_launch_count(void);

/* Checked build (compiled with -DSGIGA_CHECKED, build.build(checked=True)):
 * the operator kernels' vector gathers, scatters and metric loads and the
 * preconditioner's outputs check their indices; a failed check skips the
 * access and records the site (1..7: operator 3D x, y, metric; operator 2D x,
 * y; preconditioner level GEMM, small items). sgiga_build_checked() is 1 in
 * that build, else 0; sgiga_check_site stores the first failed site of the
 * plan (0: none, always 0 in the default build). No counterpart in the paper. */
int sgiga_build_checked(void);
int sgiga_check_site(sgiga_plan_t plan, int* site);

#ifdef __cplusplus
}
#endif
#endif /* SGIGA_H */
