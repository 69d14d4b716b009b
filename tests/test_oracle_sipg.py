"""Pins of the oracle's SIPG coupling (Sec. 3, Eq. model:discr2) and of the
assembled systems end to end (polynomial reproduction, convergence order)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import discretize
from paper_1902_01818_gb300 import workloads as W
from oracle_helpers import full_numbering, solve_discrete, patch_values, l2_error


def _nonmatching(cidx, a):
    return 3 if (cidx[0] + cidx[1]) % 2 == 0 else 4


@pytest.mark.parametrize("p", [1, 2, 3])
def test_sipg_symmetric_kills_constants_spd(p):
    prob = W.grid_problem((2, 2), _nonmatching, p, "sipg", jitter=0.1, seed=5)
    kn = prob["knots"]
    full = full_numbering(prob, kn)
    A = discretize.assemble_global(prob, kn, full).toarray()
    assert np.max(np.abs(A - A.T)) <= 1e-14 * np.max(np.abs(A))
    assert np.max(np.abs(A @ np.ones(len(A)))) <= 1e-12 * np.max(np.abs(A))
    num = discretize.numbering(prob, kn)
    Ad = discretize.assemble_global(prob, kn, num).toarray()
    assert np.linalg.eigvalsh(Ad)[0] > 0


def test_sipg_three_dimensional_symmetric_kills_constants():
    def nn(cidx, a):
        return 2 if sum(cidx) % 2 == 0 else 3
    prob = W.grid_problem((2, 1, 2), nn, 2, "sipg", jitter=0.05, seed=9, flip_patches=(1,),
                          transpose_patches=(2,))
    kn = prob["knots"]
    full = full_numbering(prob, kn)
    A = discretize.assemble_global(prob, kn, full).toarray()
    assert np.max(np.abs(A - A.T)) <= 1e-14 * np.max(np.abs(A))
    assert np.max(np.abs(A @ np.ones(len(A)))) <= 1e-12 * np.max(np.abs(A))


@pytest.mark.parametrize("flip", [(), (1,), (0, 3)])
def test_matching_sipg_restricted_to_continuous_functions_is_conforming(flip):
    p = 2
    probs = {c: W.grid_problem((2, 2), 3, p, c, jitter=0.12, seed=4, flip_patches=flip)
             for c in ("sipg", "conforming")}
    kn = probs["sipg"]["knots"]
    ns = discretize.numbering(probs["sipg"], kn)
    nc = discretize.numbering(probs["conforming"], kn)
    As = discretize.assemble_global(probs["sipg"], kn, ns)
    Ac = discretize.assemble_global(probs["conforming"], kn, nc)
    rows, cols = [], []
    for k in range(4):
        keep = ns["loc2glob"][k] >= 0
        rows.append(ns["loc2glob"][k][keep])
        cols.append(nc["loc2glob"][k][keep])
    E = sp.csr_matrix((np.ones(sum(len(r) for r in rows)),
                       (np.concatenate(rows), np.concatenate(cols))), shape=(ns["ndof"], nc["ndof"]))
    diff = (E.T @ As @ E - Ac).toarray()
    assert np.max(np.abs(diff)) <= 1e-13 * abs(Ac).max()


def _quadratic_bubble(box):
    def u(x):
        return np.prod([x[:, a] * (box[a] - x[:, a]) for a in range(x.shape[1])], axis=0)

    def f(x):
        d = x.shape[1]
        out = np.zeros(len(x))
        for a in range(d):
            others = np.prod([x[:, b] * (box[b] - x[:, b]) for b in range(d) if b != a], axis=0)
            out += 2.0 * others
        return out
    return u, f


@pytest.mark.parametrize("coupling,p", [("sipg", 2), ("sipg", 3), ("conforming", 2)])
def test_polynomial_reproduction_2d(coupling, p):
    # interfaces at x, y in {1, 2}: the bubble's normal derivative is nonzero there
    n = _nonmatching if coupling == "sipg" else 3
    flip = (1, 5) if coupling == "sipg" else (2,)
    prob = W.grid_problem((3, 3), n, p, coupling, box=(4.5, 3.0), flip_patches=flip,
                          transpose_patches=(4,))
    u_ex, f = _quadratic_bubble((4.5, 3.0))
    num, A, b, u = solve_discrete(prob, f)
    xi = np.random.default_rng(0).uniform(0, 1, (30, 2))
    from oracle import geometry
    for k in range(9):
        X, _ = geometry.eval_points(1, prob["geo_knots"][k], prob["geo_ctrl"][k], xi)
        uh = patch_values(prob, prob["knots"], num, u, k, xi)
        assert np.max(np.abs(uh - u_ex(X))) <= 1e-11


def test_polynomial_reproduction_3d_sipg():
    def nn(cidx, a):
        return 2 if sum(cidx) % 2 == 0 else 3
    prob = W.grid_problem((3, 1, 3), nn, 2, "sipg", box=(3.0, 2.0, 4.5), flip_patches=(3,),
                          transpose_patches=(4,))
    u_ex, f = _quadratic_bubble((3.0, 2.0, 4.5))
    num, A, b, u = solve_discrete(prob, f)
    xi = np.random.default_rng(1).uniform(0, 1, (8, 3))
    from oracle import geometry
    for k in range(9):
        X, _ = geometry.eval_points(1, prob["geo_knots"][k], prob["geo_ctrl"][k], xi)
        uh = patch_values(prob, prob["knots"], num, u, k, xi)
        assert np.max(np.abs(uh - u_ex(X))) <= 1e-11


@pytest.mark.parametrize("coupling", ["conforming", "sipg"])
def test_convergence_order_h_to_p_plus_1(coupling):
    p = 2
    errs = []
    for n in (2, 4, 8):
        nn = (lambda c, a, n=n: n if (c[0] + c[1]) % 2 == 0 else 2 * n) if coupling == "sipg" else n
        prob = W.grid_problem((2, 2), nn, p, coupling, box=(1.0, 1.0))
        num, A, b, u = solve_discrete(prob, W.source_sinprod)
        errs.append(l2_error(prob, num, u, W.exact_sinprod))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > p + 1 - 0.35), rates
