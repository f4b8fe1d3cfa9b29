"""Write the oracle's stored expected values used by the full-size GPU parity tests.

Calls only the oracle (oracle/) and the shared seeded input module. Run from
the repository root:

    python tests/golden/make_golden.py cube_p3_w10
    python tests/golden/make_golden.py lshape_p2_w11_g2
    python tests/golden/make_golden.py perturbed_p3_w12
    python tests/golden/make_golden.py lshape_sensitivity

Output: tests/golden/<name>.txt with, for each parametric evaluation point,
the combined sparse-grid value sum_i c_i u_i(xi) and the values of a few
selected components (L-shape: the combined value and physical gradient at
points of each patch). The components are solved in parallel worker processes
(started with "spawn").
"""
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

# name -> (domain, d, p, w, problem, eval lattice k, selected components)
CASES = {
    "cube_p3_w10": ("unit", 3, 3, 10, "sine3", 16, [(10, 1, 1), (4, 4, 4), (1, 5, 4), (3, 3, 4)]),
    "annulus_p2_w12": ("annulus", 2, 2, 12, "annulus_sinx", 64, [(12, 1), (6, 6), (1, 12)]),
    "annulus_p3_w12": ("annulus", 2, 3, 12, "annulus_sinx", 64, [(12, 1), (6, 6), (1, 12)]),
    "annulus_p4_w12": ("annulus", 2, 4, 12, "annulus_sinx", 64, [(12, 1), (6, 6), (1, 12)]),
}


# L-shape (three glued patches, Dirichlet data r^(2/3) sin(2 theta/3), one-sided
# grading toward the corner): name -> (p, w, gamma, per-patch lattice k)
LSHAPE = {
    "lshape_p2_w11_g1": (2, 11, 1.0, 8),
    "lshape_p2_w11_g2": (2, 11, 2.0, 8),
    "lshape_p2_w11_g3": (2, 11, 3.0, 8),
}


def _one_lshape(args):
    p, i, gamma, patch, pts = args
    from oracle import multipatch
    comp = multipatch.LShapeComponent(i, p, kind="onesided", gamma=gamma).assemble(g=multipatch.corner_u)
    # the extended-precision refinement: the graded systems (gamma = 3) are
    # beyond what an FP64 solve reaches
    return comp.evaluate(comp.solve_extended(), patch, pts)


def main_lshape(name):
    from oracle import combination
    from paper_1707_09598_gb300.inputs import eval_points
    p, w, gamma, k = LSHAPE[name]
    lat = eval_points(2, k)
    pts = np.concatenate([lat] * 3)
    patch = np.repeat(np.arange(3), len(lat))
    idx = combination.index_set(2, w)
    t0 = time.time()
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(8, os.cpu_count())) as pool:
        res = pool.map(_one_lshape, [(p, i, gamma, patch, pts) for i, _ in idx], chunksize=1)
    coeffs = np.array([c for _, c in idx], dtype=np.float64)
    val = combination.combine(np.stack([r[0] for r in res]), coeffs)
    gx = combination.combine(np.stack([r[1][:, 0] for r in res]), coeffs)
    gy = combination.combine(np.stack([r[1][:, 1] for r in res]), coeffs)
    out = os.path.join(HERE, name + ".txt")
    with open(out, "w") as fh:
        fh.write("# oracle values written by tests/golden/make_golden.py %s\n" % name)
        fh.write("# L-shape, 3 patches, u = r^(2/3) sin(2 theta/3) on the Dirichlet sides, f = 0, p=%d C^%d, "
                 "w=%d, one-sided grading gamma=%g toward the corner; points eval_points(2, %d) on each patch; "
                 "components solved with the extended-precision refinement\n" % (p, p - 1, w, gamma, k))
        fh.write("# columns: patch xi_1 xi_2 combined du/dx du/dy\n")
        for q, x, v, a, b in zip(patch, pts, val, gx, gy):
            fh.write("%d %.17e %.17e %.17e %.17e %.17e\n" % (q, x[0], x[1], v, a, b))
    print("wrote %s in %.1f s" % (out, time.time() - t0))


# The learned-preconditioner workload: the unit cube mapped by the seeded cubic
# B-spline perturbation (amplitude 0.1, seed 1) with the log-normal coefficient
# a = exp(g) (128 random Fourier features, seed 2), f = 1:
# name -> (d, p, w, problem, eval lattice k, selected components)
PERTURBED = {
    "perturbed_p3_w12": (3, 3, 12, "one3", 16, [(12, 1, 1), (1, 1, 12), (4, 5, 5)]),
}


def _perturbed_geometry():
    from oracle import geometry
    from paper_1707_09598_gb300.inputs import lognormal_features, perturbed_cube_patch
    kn, cp = perturbed_cube_patch(1)
    om, ph, amp = lognormal_features(2, nfeat=128)
    return geometry.BSplinePatch([3, 3, 3], kn, cp), geometry.lognormal_coefficient(om, ph, amp)


def _one_sensitivity(args):
    """Values of one L-shape component from its extended-precision solve, and
    from the same solve after a symmetric entrywise relative perturbation of
    its FP64 matrix by 4 units in the last place (random signs)."""
    p, i, gamma, patch, pts, seed = args
    from oracle import multipatch
    comp = multipatch.LShapeComponent(i, p, kind="onesided", gamma=gamma).assemble(g=multipatch.corner_u)
    v0 = comp.evaluate(comp.solve_extended(), patch, pts)[0]
    K0 = comp.K.tocsr()
    Kp = K0.copy()
    rng = np.random.default_rng(seed)
    Kp.data = Kp.data * (1.0 + 4.0 * 2.0 ** -53 * rng.choice([-1.0, 1.0], size=Kp.data.size))
    comp.K = ((Kp + Kp.T) * 0.5).tocsc()
    v1 = comp.evaluate(comp.solve_extended(), patch, pts)[0]
    return v0, v1


def main_lshape_sensitivity():
    """How far the combined L-shape solution moves when every component's
    matrix is perturbed entrywise by 4 units in the last place of FP64 (the
    size of the rounding any FP64 representation of the Galerkin matrix
    carries): the accuracy to which the discrete solution is defined in FP64,
    per grading exponent."""
    from oracle import combination
    from paper_1707_09598_gb300.inputs import eval_points
    out = os.path.join(HERE, "lshape_p2_w11_sensitivity.txt")
    lines = ["# written by tests/golden/make_golden.py lshape_sensitivity (oracle only)\n",
             "# L-shape p=2 C^1 w=11, one-sided grading; combined values on eval_points(2, 8) of each patch\n",
             "# columns: gamma  relative L2 change of the combined values under a 4-ulp entrywise perturbation\n"]
    t0 = time.time()
    ctx = mp.get_context("spawn")
    for gamma in (1.0, 2.0, 3.0):
        p, w, k = 2, 11, 8
        lat = eval_points(2, k)
        pts = np.concatenate([lat] * 3)
        patch = np.repeat(np.arange(3), len(lat))
        idx = combination.index_set(2, w)
        with ctx.Pool(min(8, os.cpu_count())) as pool:
            res = pool.map(_one_sensitivity, [(p, i, gamma, patch, pts, 1000 + n) for n, (i, _) in enumerate(idx)],
                           chunksize=1)
        coeffs = np.array([c for _, c in idx], dtype=np.float64)
        a = combination.combine(np.stack([r[0] for r in res]), coeffs)
        b = combination.combine(np.stack([r[1] for r in res]), coeffs)
        lines.append("%g %.6e\n" % (gamma, np.linalg.norm(a - b) / np.linalg.norm(a)))
    with open(out, "w") as fh:
        fh.writelines(lines)
    print("wrote %s in %.1f s" % (out, time.time() - t0))


def _one(args):
    domain, d, p, i, problem, pts = args
    from oracle import geometry, problems
    from oracle.galerkin import Component
    if domain == "perturbed":
        geom, a = _perturbed_geometry()
        comp = Component(geom, i, p).assemble(f=problems.get(problem).f, diffusion=a)
    else:
        comp = Component(geometry.make(domain, d), i, p).assemble(f=problems.get(problem).f)
    u = comp.solve()
    return comp.evaluate(u, pts)


def main(name):
    from oracle import combination
    from paper_1707_09598_gb300.inputs import eval_points
    if name in PERTURBED:
        d, p, w, problem, k, sel = PERTURBED[name]
        domain = "perturbed"
    else:
        domain, d, p, w, problem, k, sel = CASES[name]
    pts = eval_points(d, k)
    idx = combination.index_set(d, w)
    # largest components first (their assembly and LU take longest)
    order = sorted(range(len(idx)), key=lambda j: -sum(idx[j][0]))
    t0 = time.time()
    ctx = mp.get_context("spawn")
    nproc = int(os.environ.get("GOLDEN_PROCS", min(8, os.cpu_count())))
    with ctx.Pool(nproc) as pool:
        done = pool.map(_one, [(domain, d, p, idx[j][0], problem, pts) for j in order], chunksize=1)
    vals = [None] * len(idx)
    for j, v in zip(order, done):
        vals[j] = v
    vals = np.stack(vals)
    coeffs = np.array([c for _, c in idx], dtype=np.float64)
    comb = combination.combine(vals, coeffs)
    grids = [i for i, _ in idx]
    cols = [comb] + [vals[grids.index(s)] for s in sel]
    out = os.path.join(HERE, name + ".txt")
    with open(out, "w") as fh:
        fh.write("# oracle values written by tests/golden/make_golden.py %s\n" % name)
        if domain == "perturbed":
            fh.write("# unit cube mapped by perturbed_cube_patch(1) (cubic, amplitude 0.1), diffusion "
                     "a = exp(field) of lognormal_features(2, nfeat=128), f = 1\n")
        fh.write("# domain=%s d=%d p=%d C^%d w=%d problem=%s lattice k=%d (eval_points(d, k))\n"
                 % (domain, d, p, p - 1, w, problem, k))
        fh.write("# columns: combined %s\n" % " ".join("u" + "_".join(map(str, s)) for s in sel))
        for row in np.stack(cols, axis=1):
            fh.write(" ".join("%.17e" % v for v in row) + "\n")
    print("wrote %s in %.1f s" % (out, time.time() - t0))


if __name__ == "__main__":
    if sys.argv[1] == "lshape_sensitivity":
        main_lshape_sensitivity()
    elif sys.argv[1] in LSHAPE:
        main_lshape(sys.argv[1])
    else:
        main(sys.argv[1])
