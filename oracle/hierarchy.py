"""Grid hierarchy, prolongation and coarse operators -- oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Levels l = 0..L come from uniform refinement (Sec. 2, Eq. local); the spaces
are nested, the prolongation I_{l-1}^l is the canonical embedding and the
restriction its transpose (Sec. 4).  Coarse operators are Galerkin products
A_{l-1} = P^T A_l P; with the penalty frozen at the finest grid size this is
the SIPG form on the coarse space itself (Sec. 3, Eq. a:galerkin).
"""
import numpy as np
import scipy.sparse as sp

from . import bspline, discretize


def auto_levels(problem):
    """Number of levels when none is given (reading of Sec. 2).

    Coarsen while every patch has an even number of intervals in every
    direction and halving leaves at least 2 intervals (d = 2) or 3 (d = 3).
    """
    d = problem["dim"]
    nmin = 2 if d == 2 else 3
    counts = [len(bspline.breakpoints(t)) - 1 for kn in problem["knots"] for t in kn]
    levels = 1
    while all(n % 2 == 0 and n // 2 >= nmin for n in counts):
        counts = [n // 2 for n in counts]
        levels += 1
    return levels


def level_knots(problem, levels):
    """knots[l][k][a] for l = 0 (coarsest) .. levels-1 (finest = the problem's)."""
    out = [problem["knots"]]
    for _ in range(levels - 1):
        out.append([[bspline.coarsen_knots(t, discretize.degree_of(problem, k)) for t in kn]
                    for k, kn in enumerate(out[-1])])
    return out[::-1]


def patch_prolongation(knots_c, knots_f, p):
    """Tensor-product prolongation of one patch: kron over directions.

    Local flat index has xi_0 fastest, so P = P_{d-1} (x) ... (x) P_0.
    """
    mats = [sp.csr_matrix(bspline.prolongation_1d(tc, tf, p))
            for tc, tf in zip(knots_c, knots_f)]
    P = mats[0]
    for m in mats[1:]:
        P = sp.kron(m, P, format="csr")
    return P


def global_prolongation(problem, knots_c, knots_f, num_c, num_f):
    """Global prolongation matrix between consecutive levels (N_f x N_c).

    Row of a fine global DoF is taken from the patch that owns it (the copy
    that numbered it); coarse columns of Dirichlet DoFs are dropped: a coarse
    function that vanishes on the boundary is a fine one that does.
    """
    Pk = [patch_prolongation(knots_c[k], knots_f[k], discretize.degree_of(problem, k))
          for k in range(len(knots_f))]
    Pblk = sp.block_diag(Pk, format="csr")
    off_f, off_c = num_f["offsets"], num_c["offsets"]
    # fine global DoF g -> row of its owner copy in the block layout
    own = np.array([off_f[k] + f for (k, f) in num_f["owner"]], dtype=np.int64)
    Rsel = sp.csr_matrix((np.ones(len(own)), (np.arange(len(own)), own)),
                         shape=(num_f["ndof"], int(off_f[-1])))
    # coarse block layout -> coarse global DoF (Dirichlet columns dropped)
    rows, cols = [], []
    for k, l2g in enumerate(num_c["loc2glob"]):
        keep = np.nonzero(l2g >= 0)[0]
        rows.append(off_c[k] + keep)
        cols.append(l2g[keep])
    rows, cols = np.concatenate(rows), np.concatenate(cols)
    Ec = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(int(off_c[-1]), num_c["ndof"]))
    return (Rsel @ Pblk @ Ec).tocsr()


def build(problem, levels=None):
    """The whole hierarchy: knots, numbering, A_l (Galerkin) and P_l per level.

    Returns a dict with lists indexed by level (0 = coarsest): knots, num, A,
    P (P[l] maps level l-1 to level l; P[0] is None).
    """
    if levels is None:
        levels = auto_levels(problem)
    kn = level_knots(problem, levels)
    num = [discretize.numbering(problem, k) for k in kn]
    A = [None] * levels
    A[-1] = discretize.assemble_global(problem, kn[-1], num[-1])
    P = [None] * levels
    for l in range(levels - 1, 0, -1):
        P[l] = global_prolongation(problem, kn[l - 1], kn[l], num[l - 1], num[l])
        A[l - 1] = (P[l].T @ A[l] @ P[l]).tocsr()
        A[l - 1].sum_duplicates()
    return dict(levels=levels, knots=kn, num=num, A=A, P=P)


def rediscretize(problem, hier, l):
    """A on level l assembled directly with the finest-level penalty (test aid)."""
    return discretize.assemble_global(problem, hier["knots"][l], hier["num"][l],
                                      fine_knots=hier["knots"][-1])
