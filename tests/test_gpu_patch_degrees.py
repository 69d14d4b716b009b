"""GPU parity with one spline degree per patch (the non-matching SIPG setting of Sec. 5, Table
SCMS2: S_{p,h}, S_{p+1,2h}, S_{p,2h} on the three patches of the L-shaped domain of Sec. 2), and
mixed degrees on jittered 2D and 3D grids.  The library keeps one band width (the largest degree)
for all patches, a patch's own basis, quadrature, transfers and interior eigenbases for its
degree, and the Gauss-Seidel colours modulo the largest degree + 1 -- the same readings as the
oracle.

Bars as in test_gpu_parity.py: integer work (numbering, colours) bit-exact; single stages 1e-12
(transfers 1e-13), one cycle 1e-11, PCG iterates after 1, 3, 6 iterations 1e-10, iteration counts
to 1e-8 within +-1; the load vector 1e-13; mixed precision meets the FP64 stopping rule.
"""
import numpy as np
import pytest

from oracle import discretize, mg as omg, smoothers
from paper_1902_01818_gb300 import workloads as W
from lib_fixture import binding

pytestmark = pytest.mark.gpu


def _nm(c, a):
    return 4 if sum(c) % 2 == 0 else 8


CASES = {
    # name: (problem factory, levels, options)
    "lshape_p2": (lambda: W.lshape(2, 5)[0], 3, dict(tau=0.9, delta=0.12)),
    "lshape_p4": (lambda: W.lshape(4, 5)[0], 3, dict(tau=0.9, delta=0.12)),
    "grid2d_1232": (lambda: W.with_patch_degrees(
        W.grid_problem((2, 2), _nm, 3, "sipg", jitter=0.1, seed=31, flip_patches=(1,), transpose_patches=(2,)),
        [1, 2, 3, 2]), 3, dict(tau=0.5, delta=0.2)),
    "grid3d_23": (lambda: W.with_patch_degrees(
        W.grid_problem((2, 1, 1), lambda c, a: 4 if c[0] == 0 else 6, 3, "sipg", jitter=0.05, seed=32),
        [2, 3]), 2, dict(tau=0.25, delta=0.12)),
}

_cache = {}


def _pair(name, smoother="hybrid", **extra):
    key = (name, smoother, tuple(sorted(extra.items())))
    if key not in _cache:
        fac, levels, opt = CASES[name]
        prob = fac()
        lib = binding().Solver(prob, levels=levels, smoother=smoother, **opt, **extra)
        base = (name, smoother, ())
        orc = _cache[base][2] if base in _cache else omg.Multigrid(prob, levels=levels, smoother=smoother, **opt)
        _cache[key] = (prob, lib, orc)
    return _cache[key]


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("name", list(CASES))
def test_numbering_colours_and_load_vector(name):
    prob, lib, orc = _pair(name)
    for l in range(lib.levels):
        num = orc.h["num"][l]
        patch, local = lib.dof_map(l)
        owner = np.array(num["owner"])
        assert np.array_equal(patch, owner[:, 0]) and np.array_equal(local, owner[:, 1]), l
        if l >= 1:
            col = smoothers.colouring(prob, orc.h["knots"][l], num)
            assert np.array_equal(lib.colours(l), col), l
    f_ref = discretize.assemble_load(prob, prob["knots"], orc.h["num"][-1], W.source_sinprod)
    assert _rel(lib.load_sinprod(), f_ref) <= 1e-13


@pytest.mark.parametrize("name", list(CASES))
def test_stages_every_level(name):
    prob, lib, orc = _pair(name)
    rng = np.random.default_rng(0)
    for l in range(lib.levels):
        A = orc.h["A"][l]
        n = A.shape[0]
        u, f = rng.standard_normal(n), rng.standard_normal(n)
        assert np.max(np.abs(lib.apply("residual", l, f, u) - (f - A @ u))) <= 1e-12 * np.max(np.abs(A @ u)), l
        if l == 0:
            assert _rel(lib.apply("coarse", 0, f), orc.coarse_solve(f)) <= 1e-11
            continue
        P = orc.h["P"][l]
        r = rng.standard_normal(P.shape[0])
        assert _rel(lib.apply("restrict", l, r), P.T @ r) <= 1e-13, l
        e = rng.standard_normal(P.shape[1])
        assert _rel(lib.apply("prolong", l, e), P @ e) <= 1e-13, l
        ref = u + orc.scms[l].apply(f - A @ u)
        assert _rel(lib.apply("smooth", l, f, u), ref) <= 1e-11, l
        assert _rel(lib.apply("gs_fwd", l, f, u), orc.gs[l].forward(f, u)) <= 1e-12, l
        assert _rel(lib.apply("gs_bwd", l, f, u), orc.gs[l].backward(f, u)) <= 1e-12, l


@pytest.mark.parametrize("smoother", ["scms", "hybrid"])
@pytest.mark.parametrize("name", list(CASES))
def test_cycle_and_pcg_iterates(name, smoother):
    prob, lib, orc = _pair(name, smoother)
    r = np.random.default_rng(5).standard_normal(lib.ndof())
    assert _rel(lib.vcycle(r), orc.precondition(r)) <= 1e-11
    f = lib.load_sinprod()
    for k in (1, 3, 6):
        _, lk, _ = _pair(name, smoother, max_iter=k)
        u_l, it_l, _, _ = lk.solve(f, tol=1e-300, allow_noconv=True)
        u_o, it_o, _ = orc.solve_pcg(f, max_iter=k, tol=1e-300)
        assert it_l == k == it_o
        assert np.linalg.norm(u_l - u_o) <= 1e-10 * np.linalg.norm(u_o), k
    u_l, it_l, rel_l, _ = lib.solve(f, tol=1e-8)
    u_o, it_o, _ = orc.solve_pcg(f, tol=1e-8)
    assert abs(it_l - it_o) <= 1, (it_l, it_o)
    assert np.linalg.norm(orc.A @ u_l - f) <= 1e-8 * np.linalg.norm(f) * 1.0001


@pytest.mark.parametrize("precision", ["tf32", "fp32"])
@pytest.mark.parametrize("name", ["lshape_p2", "grid2d_1232", "grid3d_23"])
def test_mixed_precision_solve(name, precision):
    fac, levels, opt = CASES[name]
    prob = fac()
    orc = _pair(name)[2]
    lib = binding().Solver(prob, levels=levels, smoother="hybrid", precision=precision, **opt)
    f = lib.load_sinprod()
    u, it, rel, _ = lib.solve(f, tol=1e-8)
    _, it_o, _ = orc.solve_pcg(f, tol=1e-8)
    assert np.linalg.norm(orc.A @ u - f) <= 1e-8 * np.linalg.norm(f) * 1.0001
    assert it <= it_o + 3, (it, it_o)
    lib.close()
