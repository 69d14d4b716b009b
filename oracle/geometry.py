"""Geometry maps G_k : (0,1)^d -> Omega_k (Sec. 2, Eq. omega:2) -- oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Each patch is a tensor-product B-spline map of degree q with control points
c_I (x-fastest ordering): G(xi) = sum_I c_I prod_delta B_{I_delta}(xi_delta).
A multilinear patch (q = 1, knots [0,0,1,1]) has its 2^d vertices as control
points.  J[a, b] = dG_a / dxi_b.
"""
import numpy as np

from . import bspline


def eval_grid(geo_degree, geo_knots, ctrl, xis):
    """Evaluate G and its Jacobian on the tensor grid xis[0] x ... x xis[d-1].

    ctrl: (prod n_cp, d) control points, index I = I_0 + n_0 (I_1 + n_1 I_2).
    Returns X with shape (len(xis[d-1]), ..., len(xis[0]), d) (xi_0 fastest,
    the last axis the coordinate) and J with shape (..., d, d).
    """
    d = len(xis)
    ncp = [bspline.num_basis(geo_knots[a], geo_degree) for a in range(d)]
    c = np.asarray(ctrl, dtype=np.float64).reshape(tuple(reversed(ncp)) + (d,))
    vals = [bspline.basis(geo_knots[a], geo_degree, xis[a]) for a in range(d)]
    ders = [bspline.basis_deriv(geo_knots[a], geo_degree, xis[a]) for a in range(d)]

    def contract(mats):
        # mats[a]: (npts_a, ncp_a); c axes are (I_{d-1}, ..., I_0, coord)
        out = c
        # contract the control-point axis of direction a with mats[a]
        for a in range(d):
            axis = d - 1 - a
            out = np.tensordot(mats[a], out, axes=([1], [axis]))
            # the new point axis is now first; move it back into place
            out = np.moveaxis(out, 0, axis)
        return out

    X = contract(vals)
    J = np.zeros(X.shape[:-1] + (d, d))
    for b in range(d):
        mats = [ders[a] if a == b else vals[a] for a in range(d)]
        J[..., :, b] = contract(mats)
    return X, J


def eval_points(geo_degree, geo_knots, ctrl, pts):
    """Evaluate G and J at a list of parameter points pts (npts, d)."""
    pts = np.atleast_2d(np.asarray(pts, dtype=np.float64))
    d = pts.shape[1]
    ncp = [bspline.num_basis(geo_knots[a], geo_degree) for a in range(d)]
    c = np.asarray(ctrl, dtype=np.float64).reshape(tuple(reversed(ncp)) + (d,))
    X = np.zeros((len(pts), d))
    J = np.zeros((len(pts), d, d))
    vals = [bspline.basis(geo_knots[a], geo_degree, pts[:, a]) for a in range(d)]
    ders = [bspline.basis_deriv(geo_knots[a], geo_degree, pts[:, a]) for a in range(d)]
    for q in range(len(pts)):
        for b in range(-1, d):
            w = np.ones(())
            for a in reversed(range(d)):
                m = ders[a][q] if a == b else vals[a][q]
                w = np.multiply.outer(w, m)
            val = np.tensordot(w, c, axes=(list(range(d)), list(range(d))))
            if b < 0:
                X[q] = val
            else:
                J[q, :, b] = val
    return X, J
