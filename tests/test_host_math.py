"""The library's host numerics on the CPU (test-only shim over host_spline.cpp,
compiled here with g++): the set-up's B-spline matrices, knot insertion and
quadrature against the oracle and numpy; its blocked SPD inverse and its
generalised symmetric eigen-solver (Householder tridiagonalisation + implicit
QL after a Cholesky reduction) against numpy/scipy and their defining
identities."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import bspline, discretize

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1902_01818_gb300", "csrc")
OUT = os.path.join(HERE, "_build")
_D = C.POINTER(C.c_double)


@pytest.fixture(scope="module")
def hm():
    os.makedirs(OUT, exist_ok=True)
    so = os.path.join(OUT, "libhostmath.so")
    subprocess.run(["g++", "-std=c++17", "-O2", "-fopenmp", "-fPIC", "-shared", "-I", CSRC,
                    os.path.join(CSRC, "host_spline.cpp"), os.path.join(HERE, "host_math_shim.cpp"), "-o", so],
                   check=True)
    lib = C.CDLL(so)
    for name in ("hm_gauss", "hm_param_matrices", "hm_prolongation", "hm_spd_inverse", "hm_gen_eig",
                 "hm_find_span"):
        getattr(lib, name).restype = C.c_int
    lib.hm_find_span.argtypes = [_D, C.c_int, C.c_int, C.c_double]
    return lib


def _p(a):
    return a.ctypes.data_as(_D)


def _knots(n, p, jitter=0.0, seed=0):
    z = np.linspace(0.0, 1.0, n + 1)
    if jitter:
        z[1:-1] += np.random.default_rng(seed).uniform(-jitter, jitter, n - 1) / n
    return np.concatenate((np.zeros(p), z, np.ones(p)))


@pytest.mark.parametrize("m", [1, 2, 5, 9])
def test_gauss_legendre_nodes_and_weights(hm, m):
    x, w = np.zeros(m), np.zeros(m)
    hm.hm_gauss(m, _p(x), _p(w))
    xr, wr = bspline.gauss_legendre(m)
    assert np.allclose(np.sort(x), np.sort(xr), atol=1e-14) and abs(w.sum() - 1.0) < 1e-14
    assert np.allclose(w[np.argsort(x)], wr[np.argsort(xr)], atol=1e-14)


def test_find_span_against_the_oracle(hm):
    t = _knots(7, 3, jitter=0.3, seed=1)
    for x in np.concatenate((np.linspace(0.0, 1.0, 57), t[3:-3])):
        assert hm.hm_find_span(_p(t), len(t), 3, float(x)) == bspline.find_span(t, 3, x)


@pytest.mark.parametrize("p", [1, 2, 4, 6])
def test_parameter_matrices_match_the_oracle(hm, p):
    t = _knots(12, p)
    n = len(t) - p - 1
    K, M = np.zeros((n, n)), np.zeros((n, n))
    assert hm.hm_param_matrices(_p(t), len(t), p, _p(K), _p(M)) == 0
    Kr, Mr = discretize.param_matrices_1d(t, p)
    assert np.allclose(K, Kr, rtol=1e-12, atol=1e-10 * abs(Kr).max())
    assert np.allclose(M, Mr, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3, 6])
def test_knot_insertion_matches_the_oracle(hm, p):
    tf = _knots(16, p)
    tc = bspline.coarsen_knots(tf, p)
    nf, nc = len(tf) - p - 1, len(tc) - p - 1
    P = np.zeros((nf, nc))
    assert hm.hm_prolongation(_p(tc), len(tc), _p(tf), len(tf), p, _p(P)) == 0
    assert np.allclose(P, bspline.prolongation_1d(tc, tf, p), atol=1e-13)


@pytest.mark.parametrize("n,par", [(1, 0), (7, 0), (300, 1), (300, 0)])
def test_spd_inverse(hm, n, par):
    rng = np.random.default_rng(n)
    B = rng.standard_normal((n, n))
    A = B @ B.T + n * np.eye(n)
    X = np.zeros((n, n))
    assert hm.hm_spd_inverse(_p(A), n, par, _p(X)) == 0
    assert np.abs(X - X.T).max() == 0.0
    assert np.abs(A @ X - np.eye(n)).max() < 1e-12 * np.linalg.cond(A)


def test_spd_inverse_reports_a_breakdown(hm):
    A = np.diag([1.0, -1.0, 2.0])
    X = np.zeros((3, 3))
    assert hm.hm_spd_inverse(_p(A), 3, 0, _p(X)) == 4  # MGIGA_ENOTSPD


@pytest.mark.parametrize("p,n", [(1, 9), (2, 30), (4, 60), (6, 292)])
def test_generalised_eigenproblem_of_the_fast_diagonalisation(hm, p, n):
    """K U = M U diag(lam) with U^T M U = I on the interior 1D matrices (the
    interior piece's pencil), eigenvalues as scipy's generalised eigh; p = 1
    also against the closed form (6/h^2)(1 - cos(j pi h)) / (2 + cos(j pi h))."""
    t = _knots(n - p + 2 if p > 1 else n + 1, p)
    N = len(t) - p - 1
    Kf, Mf = discretize.param_matrices_1d(t, p)
    K, M = Kf[1:-1, 1:-1].copy(), Mf[1:-1, 1:-1].copy()
    m = N - 2
    U, lam = np.zeros((m, m)), np.zeros(m)
    assert hm.hm_gen_eig(_p(K), _p(M), m, _p(U), _p(lam)) == 0
    ref = sla.eigh(K, M, eigvals_only=True)
    assert np.allclose(np.sort(lam), ref, rtol=1e-11, atol=1e-11 * ref.max())
    assert np.abs(U.T @ M @ U - np.eye(m)).max() < 1e-11
    assert np.abs(K @ U - M @ U * lam).max() < 1e-11 * np.abs(K).max()
    if p == 1:
        h = 1.0 / (m + 1)
        j = np.arange(1, m + 1)
        closed = 6.0 / h ** 2 * (1.0 - np.cos(j * np.pi * h)) / (2.0 + np.cos(j * np.pi * h))
        assert np.allclose(np.sort(lam), closed, rtol=1e-11)
