"""B-spline bases on open knot vectors (Sec. 2, Eq. local) -- oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper uses the standard B-spline basis of S_{p,h} (degree p, maximal
smoothness) without restating its definition.  This module writes out the
textbook definition: the Cox-de Boor recursion with the convention 0/0 := 0,
right-continuous degree-0 functions, and the right end point of the parameter
interval assigned to the last non-empty knot span.
"""
import numpy as np


def breakpoints(t):
    """Distinct knot values of the knot vector t, in increasing order."""
    t = np.asarray(t, dtype=np.float64)
    keep = np.concatenate(([True], np.diff(t) > 0))
    return t[keep]


def num_basis(t, p):
    """Number of B-splines of degree p on knot vector t: len(t) - p - 1."""
    return len(t) - p - 1


def find_span(t, p, x):
    """Index s of the knot span [t_s, t_{s+1}) containing x (integer work).

    s is the largest index with t_s <= x < t_{s+1} and p <= s <= len(t)-p-2;
    x equal to the last knot belongs to the last non-empty span.
    """
    t = np.asarray(t, dtype=np.float64)
    n_basis = num_basis(t, p)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    s = np.searchsorted(t, x, side="right") - 1
    s = np.clip(s, p, n_basis - 1)
    # x == t[-1]: move back to the last span of positive length
    for idx in np.nonzero(x >= t[n_basis])[0]:
        k = n_basis - 1
        while k > p and t[k] == t[k + 1]:
            k -= 1
        s[idx] = k
    return s


def _degree0(t, p, x):
    """Degree-0 B-splines B_{i,0}(x) = 1 on [t_i, t_{i+1}), all i (len(t)-1)."""
    m = len(t) - 1
    out = np.zeros((len(x), m))
    for i in range(m):
        if t[i] < t[i + 1]:
            out[:, i] = (t[i] <= x) & (x < t[i + 1])
    # right end point: assign to the last non-empty interval
    last = max(i for i in range(m) if t[i] < t[i + 1])
    out[x >= t[-1], :] = 0.0
    out[x >= t[-1], last] = 1.0
    return out


def _ratio(num, den):
    """num/den with the Cox-de Boor convention 0/0 := 0 (den == 0 -> 0)."""
    return num / den if den != 0.0 else np.zeros_like(num)


def basis_all_degrees(t, p, x):
    """List [B_{.,0}, ..., B_{.,p}] of all B-splines of each degree at x.

    B_{i,k}(x) = (x - t_i)/(t_{i+k} - t_i) B_{i,k-1}(x)
               + (t_{i+k+1} - x)/(t_{i+k+1} - t_{i+1}) B_{i+1,k-1}(x).
    Entry k has shape (len(x), len(t) - k - 1).
    """
    t = np.asarray(t, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    levels = [_degree0(t, p, x)]
    for k in range(1, p + 1):
        prev = levels[-1]
        m = len(t) - k - 1
        cur = np.zeros((len(x), m))
        for i in range(m):
            left = _ratio(x - t[i], t[i + k] - t[i]) * prev[:, i]
            right = _ratio(t[i + k + 1] - x, t[i + k + 1] - t[i + 1]) * prev[:, i + 1]
            cur[:, i] = left + right
        levels.append(cur)
    return levels


def basis(t, p, x):
    """Values B_{i,p}(x) of all len(t)-p-1 B-splines; shape (len(x), N)."""
    return basis_all_degrees(t, p, x)[p]


def basis_deriv(t, p, x):
    """First derivatives of all B-splines of degree p at x; shape (len(x), N).

    B'_{i,p} = p/(t_{i+p} - t_i) B_{i,p-1} - p/(t_{i+p+1} - t_{i+1}) B_{i+1,p-1}.
    """
    t = np.asarray(t, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n_basis = num_basis(t, p)
    if p == 0:
        return np.zeros((len(x), n_basis))
    low = basis_all_degrees(t, p - 1, x)[p - 1]
    out = np.zeros((len(x), n_basis))
    for i in range(n_basis):
        a = _ratio(np.full(len(x), float(p)), t[i + p] - t[i]) * low[:, i]
        b = _ratio(np.full(len(x), float(p)), t[i + p + 1] - t[i + 1]) * low[:, i + 1]
        out[:, i] = a - b
    return out


def gauss_legendre(m):
    """m-point Gauss-Legendre nodes and weights on [0, 1]."""
    xg, wg = np.polynomial.legendre.leggauss(m)
    return 0.5 * (xg + 1.0), 0.5 * wg


def element_quadrature(t, m):
    """Gauss points/weights with m points on every non-empty knot span of t.

    Returns (x, w, elem) with elem[q] = index of the element (non-empty span,
    counted from 0) that point q lies in.
    """
    z = breakpoints(t)
    xg, wg = gauss_legendre(m)
    xs, ws, es = [], [], []
    for e in range(len(z) - 1):
        a, b = z[e], z[e + 1]
        xs.append(a + (b - a) * xg)
        ws.append((b - a) * wg)
        es.append(np.full(m, e))
    return np.concatenate(xs), np.concatenate(ws), np.concatenate(es)


def greville(t, p):
    """Greville abscissae (t_{i+1} + ... + t_{i+p}) / p (p >= 1)."""
    t = np.asarray(t, dtype=np.float64)
    n_basis = num_basis(t, p)
    if p == 0:
        return 0.5 * (t[:-1] + t[1:])
    return np.array([t[i + 1:i + p + 1].mean() for i in range(n_basis)])


def coarsen_knots(t, p):
    """Knot vector of the next coarser level: drop every other breakpoint.

    Levels are nested by uniform refinement (Sec. 2: h_{l} halves from level
    l-1 to level l), so level l-1 keeps the breakpoints z_0, z_2, ..., z_n of
    level l (n even), with end multiplicity p+1 and simple interior knots.
    """
    z = breakpoints(t)
    n = len(z) - 1
    if n % 2 != 0:
        raise ValueError("cannot coarsen a knot vector with an odd number of spans")
    zc = z[::2]
    return np.concatenate((np.full(p + 1, zc[0]), zc[1:-1], np.full(p + 1, zc[-1])))


def prolongation_1d(t_coarse, t_fine, p):
    """Matrix P (N_fine x N_coarse) of the canonical embedding (Sec. 4).

    Column j holds the coefficients of the coarse B-spline j in the fine basis:
    B^c_j = sum_i P[i, j] B^f_i.  Computed from that definition by collocation
    at the fine Greville points, where the fine collocation matrix is
    non-singular (Schoenberg-Whitney); entries below 1e-13 in magnitude are
    structural zeros and are set to 0.
    """
    g = greville(t_fine, p)
    bf = basis(t_fine, p, g)
    bc = basis(t_coarse, p, g)
    P = np.linalg.solve(bf, bc)
    P[np.abs(P) < 1e-13] = 0.0
    return P
