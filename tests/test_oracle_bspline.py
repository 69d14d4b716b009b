"""Pins of the oracle's B-spline layer against closed forms and brute force."""
import numpy as np
import pytest

from oracle import bspline
from paper_1902_01818_gb300.workloads import uniform_knots


def _nonuniform(n, p, seed):
    rng = np.random.default_rng(seed)
    inner = np.sort(rng.uniform(0.05, 0.95, n - 1))
    return np.concatenate(([0.0] * (p + 1), inner, [1.0] * (p + 1)))


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("kind", ["uniform", "random"])
def test_partition_of_unity_and_nonnegativity(p, kind):
    t = uniform_knots(7, p) if kind == "uniform" else _nonuniform(7, p, 3 + p)
    x = np.random.default_rng(p).uniform(0, 1, 1000)
    x = np.concatenate((x, [0.0, 1.0]))
    B = bspline.basis(t, p, x)
    D = bspline.basis_deriv(t, p, x)
    assert np.max(np.abs(B.sum(axis=1) - 1.0)) <= 1e-15 * 4
    assert np.max(np.abs(D.sum(axis=1))) <= 1e-12
    assert B.min() >= -1e-16
    # at most p+1 nonzero functions at a point
    assert np.max((np.abs(B) > 0).sum(axis=1)) <= p + 1


def test_find_span_brute_force():
    for p in (1, 2, 3):
        t = _nonuniform(9, p, 11)
        xs = np.concatenate((np.random.default_rng(1).uniform(0, 1, 500), t[p:-p], [0.0, 1.0]))
        spans = bspline.find_span(t, p, xs)
        for x, s in zip(xs, spans):
            if x < 1.0:
                cand = [i for i in range(p, len(t) - p - 1) if t[i] <= x < t[i + 1]]
                assert s == cand[-1]
            else:
                assert s == len(t) - p - 2


def test_hat_functions_p1():
    n = 5
    t = uniform_knots(n, 1)
    x = np.linspace(0, 1, 201)
    B = bspline.basis(t, 1, x)
    for i in range(n + 1):
        hat = np.maximum(0.0, 1.0 - np.abs(x * n - i))
        assert np.max(np.abs(B[:, i] - hat)) <= 1e-14


def test_uniform_quadratic_values():
    # interior uniform C^1 quadratics: 1/2, 1/2 at a knot; 1/8, 3/4, 1/8 at a midpoint
    n = 6
    t = uniform_knots(n, 2)
    Bk = bspline.basis(t, 2, np.array([3 / n]))[0]
    nz = Bk[np.abs(Bk) > 0]
    assert np.allclose(sorted(nz), [0.5, 0.5], atol=1e-15)
    Bm = bspline.basis(t, 2, np.array([3.5 / n]))[0]
    nz = Bm[np.abs(Bm) > 0]
    assert np.allclose(nz, [1 / 8, 3 / 4, 1 / 8], atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 4, 6])
def test_derivative_matches_difference_quotient(p):
    t = _nonuniform(6, p, 5)
    x = np.random.default_rng(2).uniform(0.01, 0.99, 200)
    # keep away from knots where derivatives jump
    x = x[np.min(np.abs(x[:, None] - t[None, :]), axis=1) > 1e-4]
    h = 1e-6
    fd = (bspline.basis(t, p, x + h) - bspline.basis(t, p, x - h)) / (2 * h)
    D = bspline.basis_deriv(t, p, x)
    assert np.max(np.abs(fd - D)) <= 1e-5 * max(1.0, np.max(np.abs(D)))


@pytest.mark.parametrize("m", [1, 2, 3, 5, 7])
def test_gauss_exact_for_degree_2m_minus_1(m):
    x, w = bspline.gauss_legendre(m)
    for k in range(2 * m):
        assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) <= 1e-14
    # and not exact one degree higher (it is a genuine m-point rule)
    k = 2 * m
    assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) > 1e-12


@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_prolongation_reproduces_coarse_splines(p):
    tf = uniform_knots(8, p)
    tc = bspline.coarsen_knots(tf, p)
    assert np.array_equal(tc, uniform_knots(4, p))
    P = bspline.prolongation_1d(tc, tf, p)
    x = np.random.default_rng(p).uniform(0, 1, 1000)
    c = np.random.default_rng(10 + p).standard_normal(P.shape[1])
    coarse = bspline.basis(tc, p, x) @ c
    fine = bspline.basis(tf, p, x) @ (P @ c)
    assert np.max(np.abs(coarse - fine)) <= 1e-13 * np.max(np.abs(c))
    # partition of unity is preserved: rows of P sum to one
    assert np.max(np.abs(P.sum(axis=1) - 1.0)) <= 1e-13


def test_two_scale_coefficients_closed_form():
    # p=1 hat: 1/2, 1, 1/2 ; p=2 interior uniform quadratic: 1/4, 3/4, 3/4, 1/4
    P1 = bspline.prolongation_1d(uniform_knots(4, 1), uniform_knots(8, 1), 1)
    assert np.allclose(P1[:, 2][np.abs(P1[:, 2]) > 0], [0.5, 1.0, 0.5], atol=1e-14)
    P2 = bspline.prolongation_1d(uniform_knots(4, 2), uniform_knots(8, 2), 2)
    col = P2[:, 3]
    assert np.allclose(col[np.abs(col) > 0], [0.25, 0.75, 0.75, 0.25], atol=1e-14)


def test_greville_linear_precision():
    # sum_i g_i B_i(x) = x
    for p in (1, 2, 3, 5):
        t = _nonuniform(6, p, 7)
        g = bspline.greville(t, p)
        x = np.random.default_rng(0).uniform(0, 1, 300)
        assert np.max(np.abs(bspline.basis(t, p, x) @ g - x)) <= 1e-14
