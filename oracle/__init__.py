"""Plain CPU FP64 oracle for the sparse-grid isogeometric Poisson solver.

TEST INFRASTRUCTURE. This package is the independent checker of the CUDA
library: it is written from the paper (Beck, Sangalli, Tamellini, "A
sparse-grid isogeometric solver", arXiv:1707.09598) and shares no code with
the CUDA path. Only the test suite, the smoke check of the entry module and
the CPU-baseline leg of the benchmark may import it; the product path never
does.

Modules
  spline       knot vectors, radical grading, Gauss rule, Cox-de Boor (Sec. 2.2)
  geometry     parametrisations F: unit square/cube, quarter annulus (NURBS)
  galerkin     element-by-element Gauss assembly, Dirichlet elimination,
               sparse direct solve, evaluation (Problem 1, Sec. 2.2)
  combination  index set and combination coefficients (Sec. 3, eqs.
               TD-approx and TD-combi-tec), Neumaier-compensated combine
  fd           fast-diagonalisation preconditioner written from its
               definition (not in the paper; the CUDA preconditioner's
               definition, cross-checked against the direct solve)
  adaptive     hierarchical surpluses, their profits, the coefficients of an
               arbitrary index set and the Dantzig (knapsack) choice of it
               (Sec. 4.2, optimal sets)
  multipatch   the L-shaped domain: three glued bilinear patches, Dirichlet
               lifting by edge L2 projection, L2/H1 errors (not in the
               paper's experiments; its graded-mesh topic, Sec. 4.4)
  net          the learned scaling network's forward and backward (not in
               the paper; the CUDA network's definition)
  learned      features, scaled fast-diagonalisation preconditioner
               S * FD(S * r), and the training loss with its gradient (not
               in the paper; the CUDA learned preconditioner's definition)
  problems     manufactured solutions; f = -Laplace(u) derived symbolically
  driver       whole-method runs: solve every component, evaluate, combine
  hp           h-p sparse combination: the degree as one more combination
               index at one continuity (named as possible in Sec. 2.2 and 5;
               the reading is stated in the module)

Parity status: every function is pinned by tests under tests/ (closed forms,
identities of the paper, brute force, convergence rates); none is unpinned.
"""
