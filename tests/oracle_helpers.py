"""Small helpers shared by the oracle pin tests (test code, not oracle code)."""
import numpy as np
import scipy.sparse.linalg as spla

from oracle import bspline, discretize, geometry


def full_numbering(problem, knots):
    """A numbering that keeps every local DoF (no Dirichlet, no sharing)."""
    shapes = [discretize.shape_of(kn, discretize.degree_of(problem, k)) for k, kn in enumerate(knots)]
    sizes = [int(np.prod(s)) for s in shapes]
    offsets = np.concatenate(([0], np.cumsum(sizes)))
    l2g = [offsets[k] + np.arange(sizes[k]) for k in range(len(sizes))]
    owner = [(k, f) for k in range(len(sizes)) for f in range(sizes[k])]
    return dict(shapes=shapes, offsets=offsets, loc2glob=l2g, ndof=int(offsets[-1]), owner=owner)


def solve_discrete(problem, f):
    kn = problem["knots"]
    num = discretize.numbering(problem, kn)
    A = discretize.assemble_global(problem, kn, num)
    b = discretize.assemble_load(problem, kn, num, f)
    u = spla.spsolve(A.tocsc(), b)
    return num, A, b, u


def patch_values(problem, knots, num, u, k, xi):
    local = discretize.global_to_local_vectors(num, u)[k]
    return discretize.evaluate(problem, knots, local, k, xi)


def l2_error(problem, num, u, exact, nq=None):
    """L2(Omega) error of the discrete solution by per-element Gauss quadrature (2D)."""
    locs = discretize.global_to_local_vectors(num, u)
    err2 = 0.0
    for k, kn in enumerate(problem["knots"]):
        p = discretize.degree_of(problem, k)
        nq = nq or discretize.max_degree(problem) + 3
        xs, ws = [], []
        for t in kn:
            x, w, _ = bspline.element_quadrature(t, nq)
            xs.append(x); ws.append(w)
        B0 = bspline.basis(kn[0], p, xs[0])
        B1 = bspline.basis(kn[1], p, xs[1])
        shape = discretize.shape_of(kn, p)
        C = locs[k].reshape(shape[1], shape[0])
        uh = B1 @ C @ B0.T  # (x1, x0)
        X, J = geometry.eval_grid(problem["geo_degree"], problem["geo_knots"][k],
                                  problem["geo_ctrl"][k], xs)
        ue = exact(X.reshape(-1, 2)).reshape(uh.shape)
        wt = np.outer(ws[1], ws[0]) * np.abs(np.linalg.det(J))
        err2 += np.sum(wt * (uh - ue) ** 2)
    return np.sqrt(err2)
