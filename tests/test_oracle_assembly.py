"""Pins of the oracle's patch assembly (Sec. 2) against closed forms."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import discretize, bspline
from paper_1902_01818_gb300 import workloads as W


def _shoelace(poly):
    x, y = poly[:, 0], poly[:, 1]
    return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))


def test_param_matrices_p1_closed_form():
    n = 6
    h = 1.0 / n
    K, M = discretize.param_matrices_1d(W.uniform_knots(n, 1), 1)
    Kx = (np.diag(np.full(n + 1, 2.0)) - np.diag(np.ones(n), 1) - np.diag(np.ones(n), -1)) / h
    Kx[0, 0] = Kx[-1, -1] = 1.0 / h
    Mx = (np.diag(np.full(n + 1, 4.0)) + np.diag(np.ones(n), 1) + np.diag(np.ones(n), -1)) * h / 6
    Mx[0, 0] = Mx[-1, -1] = 2.0 * h / 6
    assert np.max(np.abs(K - Kx)) <= 1e-12
    assert np.max(np.abs(M - Mx)) <= 1e-15


@pytest.mark.parametrize("p", [1, 2, 3])
def test_mass_sums_to_patch_area_jittered(p):
    prob = W.grid_problem((2, 2), 5, p, "sipg", jitter=0.15, seed=7)
    for k in range(4):
        Mk = discretize.patch_mass(prob, k, prob["knots"][k])
        c = prob["geo_ctrl"][k]
        area = _shoelace(c[[0, 1, 3, 2]])
        assert abs(Mk.sum() - area) <= 1e-13
        ev = np.linalg.eigvalsh(Mk.toarray())
        assert ev.min() > 0


@pytest.mark.parametrize("p", [1, 2, 4])
def test_stiffness_annihilates_constants_and_is_spsd(p):
    prob = W.grid_problem((2, 1), 4, p, "sipg", jitter=0.2, seed=3)
    prob["geo_ctrl"][0][3] += np.array([0.1, 0.05])  # a non-affine patch
    for k in range(2):
        Kk = discretize.patch_stiffness(prob, k, prob["knots"][k]).toarray()
        assert np.max(np.abs(Kk @ np.ones(len(Kk)))) <= 1e-13 * np.max(np.abs(Kk))
        assert np.max(np.abs(Kk - Kk.T)) <= 1e-14 * np.max(np.abs(Kk))
        ev = np.linalg.eigvalsh(Kk)
        assert ev[0] > -1e-12 * ev[-1] and ev[1] > 1e-10 * ev[-1]


def test_stiffness_kills_linears_on_interior_rows_affine():
    p = 3
    prob = W.grid_problem((1, 1), 5, p, "sipg")
    A = np.array([[1.3, 0.4], [-0.2, 0.9]])
    prob["geo_ctrl"][0] = prob["geo_ctrl"][0] @ A.T + np.array([0.5, -1.0])
    kn = prob["knots"][0]
    Kk = discretize.patch_stiffness(prob, 0, kn).toarray()
    g = [bspline.greville(t, p) for t in kn]
    G1, G0 = np.meshgrid(g[1], g[0], indexing="ij")
    pts = np.stack((G0.ravel(), G1.ravel()), axis=1)
    X = pts @ A.T + np.array([0.5, -1.0])
    shape = discretize.shape_of(kn, p)
    multi = discretize.unflatten(np.arange(len(Kk)), shape)
    inner = (multi[0] > 0) & (multi[0] < shape[0] - 1) & (multi[1] > 0) & (multi[1] < shape[1] - 1)
    for c in range(2):
        r = Kk @ X[:, c]
        assert np.max(np.abs(r[inner])) <= 1e-12 * np.max(np.abs(Kk))


def test_stiffness_of_a_box_is_kronecker():
    # identity-like box [0, a] x [0, b]: K = (b/a) M^_1 (x) K^_0 + (a/b) K^_1 (x) M^_0
    p, n = 2, 4
    prob = W.grid_problem((1, 1), n, p, "sipg", box=(2.0, 0.5))
    Kk = discretize.patch_stiffness(prob, 0, prob["knots"][0]).toarray()
    K1, M1 = discretize.param_matrices_1d(W.uniform_knots(n, p), p)
    a, b = 2.0, 0.5
    ref = (b / a) * np.kron(M1, K1) + (a / b) * np.kron(K1, M1)
    assert np.max(np.abs(Kk - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_load_integrates_source():
    # sum_i (f, B_i) = int f by partition of unity; int over [0,3]^2 of 2 pi^2 sin sin = 8
    prob, _ = W.sipg_3x3(2)
    for k in range(len(prob["knots"])):
        prob["knots"][k] = [W.uniform_knots(12, 2)] * 2
    tot = 0.0
    for k in range(9):
        tot += discretize.patch_load(prob, k, prob["knots"][k], W.source_sinprod).sum()
    assert abs(tot - 8.0) <= 1e-6


def test_dof_counts():
    prob, _ = W.unit_square_2x2()
    num = discretize.numbering(prob, prob["knots"])
    assert num["ndof"] == 4225
    # SIPG: every patch keeps its own DoFs, only boundary sides are removed
    prob = W.grid_problem((2, 2), 4, 2, "sipg")
    num = discretize.numbering(prob, prob["knots"])
    assert num["ndof"] == 4 * 5 * 5


def test_conforming_numbering_order_and_sharing():
    prob = W.grid_problem((2, 1), 2, 1, "conforming")
    num = discretize.numbering(prob, prob["knots"])
    # patch 0: 3x3 local, boundary sides 0, 2, 3 -> only i0 in {1,2}, i1 = 1
    assert list(num["loc2glob"][0]) == [-1, -1, -1, -1, 0, 1, -1, -1, -1]
    # patch 1 shares its xi0 = 0 side with patch 0's xi0 = 1 side
    assert list(num["loc2glob"][1]) == [-1, -1, -1, 1, 2, -1, -1, -1, -1]
    assert num["ndof"] == 3


def test_batched_layout_non_rectangular_problem_is_spd():
    """A batched-layout problem with a partial last row of patches (seed 407:
    3 SIPG patches): the oracle assembles a symmetric positive definite matrix,
    every patch side shared by two patches is an interface, the others Dirichlet."""
    from paper_1902_01818_gb300 import workloads as W
    import scipy.sparse.linalg as spla
    prob, opts, _ = W.batched_problem(407)
    assert len(prob["knots"]) == 3 and len(prob["interfaces"]) == 2
    num = discretize.numbering(prob, prob["knots"])
    A = discretize.assemble_global(prob, prob["knots"], num)
    assert abs(A - A.T).max() <= 1e-12 * abs(A).max()
    lam = spla.eigsh(A, k=1, sigma=0, which="LM", return_eigenvectors=False)
    assert lam[0] > 0
