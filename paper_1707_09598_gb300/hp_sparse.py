"""h-p sparse combination: the combination technique with the spline degree
as one more index, through the C ABI.

The paper builds its sparse grids by h-refinement alone and names a
p-sparsification, or a combined h-p version, as possible (Sec. 2.2) and as
a direction for further work (Sec. 5), without fixing a construction. The
reading taken here:
  - component (i, q) is the spline space of degree p0 + q with continuity C^r
    at every interior breakpoint, on the mesh with 2^{i_k} elements in
    direction k; one r <= p0 - 1 serves every degree, so that raising the
    degree keeps each space inside the next one on the same mesh, as
    refining the mesh does (Sec. 3);
  - the set of level w with Q degree steps is every (i, q) with
    i_k >= min_level, 0 <= q <= Q and |i| - d min_level + q <= w + d - 1 -
    d min_level (the h-sparse set of eq. TD-approx with q added to |beta|);
    Q = 0 is the h-sparse set of eq. TD-combi-tec;
  - the approximation is the sum of the set's Delta_{beta,q} (eq.
    Delta-combi-tec in all d + 1 indices), i.e. sum_gamma c_gamma u_gamma with
    c_gamma = sum_{z in {0,1}^{d+1}} (-1)^{|z|} [gamma + z in the set].

Host-side set logic around the library: one plan per degree holds that
degree's components with their coefficients, every plan solves and
evaluates its components on the GPU, and sgiga_combine_plans forms the
compensated sum over all of them.
"""
import itertools

from . import knapsack, sgiga


def index_set(d, w, Q, min_level=1):
    """The set's (i_1, .., i_d, q)."""
    J = w + d - 1 - d * min_level
    if J < 0 or Q < 0:
        raise ValueError("level too small for min_level, or Q < 0")
    out = []
    for beta in itertools.product(range(J + 1), repeat=d):
        for q in range(min(Q, J - sum(beta)) + 1):
            out.append(tuple(b + min_level for b in beta) + (q,))
    return out


def coefficients(d, w, Q, min_level=1):
    """{(i_1, .., i_d, q): c} of the set's components with c != 0."""
    return knapsack.set_coefficients(index_set(d, w, Q, min_level))


class HPCombination:
    """The plans of one h-p sparse combination (degrees p0 .. p0 + Q at
    continuity r) on one stream. Marshalling only: every solve, evaluation
    and the combination run in the library."""

    def __init__(self, d, p0, r, w, Q, domain="unit", min_level=1, stream=None, **kw):
        if not 0 <= r <= p0 - 1:
            raise ValueError("continuity r must satisfy 0 <= r <= p0 - 1")
        if p0 + Q > 4:
            raise ValueError("degrees above 4 are not supported (p0 + Q <= 4)")
        self.d, self.p0 = d, p0
        self.coef = coefficients(d, w, Q, min_level)
        self.plans = []          # (degree, Plan)
        try:
            for q in range(Q + 1):
                comps = sorted(k for k in self.coef if k[d] == q)
                if not comps:
                    continue
                P = sgiga.Plan(d, p0 + q, w, domain=domain, continuity=r, min_level=min_level, stream=stream,
                               components=[k[:d] for k in comps], coefficients=[float(self.coef[k]) for k in comps],
                               **kw)
                self.plans.append((p0 + q, P))
        except Exception:
            self.close()
            raise
        self.ngrids = sum(P.info.ngrids for _, P in self.plans)
        self.ndof = sum(P.info.ndof for _, P in self.plans)

    def set_rhs_builtin(self, source):
        for _, P in self.plans:
            sgiga.sgiga_set_rhs_builtin(P.handle, source)

    def solve(self, rel_tol, max_iter):
        """Every plan's batched solve; the per-plan statistics."""
        return [sgiga.sgiga_solve(P.handle, rel_tol, max_iter)[0] for _, P in self.plans]

    def eval_combine(self, xi, npts, u_comp, u):
        """Component values into u_comp [ngrids][npts] (plan after plan, each
        plan's components in its own order) and their combination into u."""
        off = 0
        for _, P in self.plans:
            n = P.info.ngrids * npts
            sgiga.sgiga_eval(P.handle, xi, npts, u_comp[off:off + n])
            off += n
        sgiga.sgiga_combine_plans([P.handle for _, P in self.plans], u_comp, npts, u)

    def component_keys(self):
        """(i_1, .., i_d, q) of the rows of u_comp, in order."""
        out = []
        for p, P in self.plans:
            for g in P.grids:
                out.append(tuple(g.levels[:self.d]) + (p - self.p0,))
        return out

    def close(self):
        for _, P in self.plans:
            P.close()
        self.plans = []

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
