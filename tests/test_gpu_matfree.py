"""The matrix-free residual of the finest level against the oracle's assembled matrix.

The library evaluates the patch stiffness action at the Gauss points (p + 1 per element and
direction, the quadrature of the assembly, Sec. 2 Eq. linear:system:0) by sum factorisation, with
the geometric factors computed from the geometry's control points; the SIPG terms (Sec. 3,
Eq. model:discr2) stay stored.  The oracle assembles A element by element (oracle/discretize.py).

Cases span several element tiles per direction with a ragged last tile (tiles of 32/16/16/12/8/8
elements per direction in 2D for p = 1..6; 8/6/4/4/3/3 in 3D (FP32), 6/4/3/2/2/2 (FP64)), 2D and
3D, conforming and SIPG, flipped and transposed patches, multilinear and quadratic geometry maps.

Tolerances.  FP64: 1e-12 of max |A u| (only the summation order differs from the assembled
matrix).  FP32: the result is a tree of sums in FP32 whose depth per output is at most
m = d (p + 1) (p + 2) + 2^d + 16 (d forward contractions of p + 1 terms, the pointwise flux, d
backward contractions over at most (p + 1)^2 points, the window partials); the standard bound
gamma_m = m u / (1 - m u), u = 2^-24, applies to sums of absolute values of the products, which on
these mildly distorted maps stay within a factor 8 of (|A| |u|)_i; the test takes
8 gamma_m max_i (|A| |u|)_i.
"""
import numpy as np
import pytest

from oracle import discretize, mg as omg
from paper_1902_01818_gb300 import workloads as W
from lib_fixture import binding

pytestmark = pytest.mark.gpu


def quadratic_geometry(prob, bulge=0.08, seed=5):
    """The same patches with their multilinear maps raised to degree 2 (control points at the
    Greville points 0, 1/2, 1 of each direction), then the control point in the middle of every
    patch moved by U[-bulge, bulge]^d: a curved map whose boundary (and so every interface) is
    unchanged."""
    d = prob["dim"]
    rng = np.random.default_rng(seed)
    ctrl2 = []
    for c in prob["geo_ctrl"]:
        c = np.asarray(c).reshape(2 ** d, d)
        pts = []
        for idx in np.ndindex(*([3] * d)):
            i = tuple(reversed(idx))  # first index fastest
            x = np.zeros(d)
            for bits in np.ndindex(*([2] * d)):
                b = tuple(reversed(bits))
                w = 1.0
                for a in range(d):
                    t = i[a] / 2.0
                    w *= t if b[a] else 1.0 - t
                x += w * c[sum(b[a] << a for a in range(d))]
            pts.append(x)
        pts = np.array(pts)
        mid = sum(3 ** a for a in range(d))
        pts[mid] += rng.uniform(-bulge, bulge, size=d)
        ctrl2.append(pts)
    out = dict(prob)
    out["geo_degree"] = 2
    out["geo_knots"] = [[np.array([0.0, 0.0, 0.0, 1.0, 1.0, 1.0]) for _ in range(d)] for _ in prob["geo_ctrl"]]
    out["geo_ctrl"] = ctrl2
    return out


def _n2(a, b):
    return lambda c, dd: a if sum(c) % 2 == 0 else b


CASES = {
    "conf2d_p1": lambda: W.grid_problem((2, 2), 40, 1, "conforming", jitter=0.1, seed=11, flip_patches=(3,)),
    "sipg2d_p2": lambda: W.grid_problem((3, 3), _n2(20, 36), 2, "sipg", jitter=0.1, seed=12, flip_patches=(1,),
                                        transpose_patches=(4,)),
    "conf2d_p3": lambda: W.grid_problem((2, 2), 36, 3, "conforming", jitter=0.1, seed=13, transpose_patches=(2,)),
    "sipg2d_p4": lambda: W.grid_problem((2, 2), _n2(14, 26), 4, "sipg", jitter=0.1, seed=14, flip_patches=(2,)),
    "sipg2d_p5": lambda: W.grid_problem((2, 1), _n2(10, 18), 5, "sipg", jitter=0.1, seed=15),
    "conf2d_p6": lambda: W.grid_problem((2, 2), 18, 6, "conforming", jitter=0.1, seed=16),
    "quad2d_p3": lambda: quadratic_geometry(W.grid_problem((1, 1), 20, 3, "sipg", box=(1.0, 1.0))),
    "quad2d_sipg_p2": lambda: quadratic_geometry(W.grid_problem((2, 1), _n2(12, 20), 2, "sipg", jitter=0.0)),
    "conf3d_p2": lambda: W.grid_problem((2, 2, 2), 8, 2, "conforming", jitter=0.05, seed=17,
                                        jitter_boundary_tangential=True, flip_patches=(5,)),
    "sipg3d_p3": lambda: W.grid_problem((2, 1, 2), _n2(6, 10), 3, "sipg", jitter=0.05, seed=18, flip_patches=(1,),
                                        transpose_patches=(2,)),
    "sipg3d_p1": lambda: W.grid_problem((2, 2, 1), 10, 1, "sipg", jitter=0.05, seed=19),
    "conf3d_p4": lambda: W.grid_problem((2, 1, 1), 6, 4, "conforming", jitter=0.05, seed=20),
    "sipg3d_p5": lambda: W.grid_problem((1, 1, 2), _n2(4, 6), 5, "sipg", jitter=0.05, seed=21),
    "sipg3d_p6": lambda: W.grid_problem((1, 2, 1), 4, 6, "sipg", jitter=0.05, seed=22),
    "quad3d_p2": lambda: quadratic_geometry(W.grid_problem((1, 1, 1), 8, 2, "sipg", box=(1.0, 1.0, 1.0)), 0.05),
}

_oracle = {}


def _matrix(name):
    if name not in _oracle:
        prob = CASES[name]()
        num = discretize.numbering(prob, prob["knots"])
        _oracle[name] = (prob, discretize.assemble_global(prob, prob["knots"], num))
    return _oracle[name]


def _fp32_bound(d, p):
    m = d * (p + 1) * (p + 2) + 2 ** d + 16
    unit = 2.0 ** -24
    return 8 * m * unit / (1 - m * unit)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", list(CASES))
def test_matrix_free_residual_against_oracle(name, precision):
    prob, A = _matrix(name)
    lib = binding().Solver(prob, levels=2, smoother="scms", precision=precision, matrix_free=True)
    n = A.shape[0]
    assert lib.ndof() == n
    rng = np.random.default_rng(3)
    for rep in range(2):  # twice: the window partials are rewritten, not accumulated
        u, f = rng.standard_normal(n), rng.standard_normal(n)
        ref = f - A @ u
        got = lib.apply("cycle_residual", -1, f, u)
        err = float(np.max(np.abs(got - ref)))
        if precision == "fp64":
            assert err <= 1e-12 * np.max(np.abs(A @ u)), (rep, err / np.max(np.abs(A @ u)))
        else:
            scale = float(np.max(abs(A) @ np.abs(u)))
            assert err <= _fp32_bound(prob["dim"], prob["degree"]) * scale, (rep, err / scale)
            assert err > 0.0  # FP32 arithmetic really in use
    # the stored-band residual of the same handle is unchanged by the option
    got = lib.apply("residual", -1, f, u)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(A @ u))
    lib.close()


def test_matrix_free_zero_iterate():
    """u = 0 (SIPG: no shared copies): every window partial is 0, so out = f bit for bit, in both
    precisions."""
    prob, A = _matrix("sipg2d_p2")
    n = A.shape[0]
    f = np.random.default_rng(4).standard_normal(n)
    for precision in ("fp64", "fp32"):
        lib = binding().Solver(prob, levels=2, smoother="scms", precision=precision, matrix_free=True)
        got = lib.apply("cycle_residual", -1, f, np.zeros(n))
        assert np.array_equal(got, f), precision
        lib.close()


@pytest.mark.parametrize("name", ["sipg2d_p2", "conf3d_p2", "quad2d_sipg_p2"])
def test_matrix_free_pcg_iterates(name):
    """FP64 PCG with the matrix-free cycle residual: iterates after 1, 3, 6 iterations within 1e-10
    of the oracle's (whose cycle uses the assembled matrix), iteration counts to 1e-8 within +-1."""
    prob, A = _matrix(name)
    opts = dict(levels=2, smoother="hybrid", tau=0.25, delta=0.12)
    orc = omg.Multigrid(prob, **opts)
    f = discretize.assemble_load(prob, prob["knots"], orc.h["num"][-1], W.source_sinprod)
    for k in (1, 3, 6):
        lib = binding().Solver(prob, **opts, precision="fp64", matrix_free=True, max_iter=k)
        u, it, _, _ = lib.solve(f, tol=1e-300, allow_noconv=True)
        ref, _, _ = orc.solve_pcg(f, max_iter=k, tol=1e-300)
        assert np.linalg.norm(u - ref) <= 1e-10 * np.linalg.norm(ref), (k, np.linalg.norm(u - ref) / np.linalg.norm(ref))
        lib.close()
    lib = binding().Solver(prob, **opts, precision="fp64", matrix_free=True)
    u, it, _, _ = lib.solve(f, tol=1e-8)
    _, it_ref, _ = orc.solve_pcg(f, tol=1e-8)
    assert abs(it - it_ref) <= 1
    lib.close()


@pytest.mark.parametrize("precision", ["tf32", "fp32"])
@pytest.mark.parametrize("name", ["sipg2d_p4", "conf3d_p2", "sipg3d_p3"])
def test_matrix_free_mixed_solve(name, precision):
    """Mixed precision with the matrix-free FP32 cycle residual on the finest level: the FP64
    stopping rule holds with the oracle's matrix, within 3 iterations of the oracle's FP64 count."""
    prob, A = _matrix(name)
    opts = dict(levels=2, smoother="hybrid", tau=0.25, delta=0.12)
    orc = omg.Multigrid(prob, **opts)
    f = discretize.assemble_load(prob, prob["knots"], orc.h["num"][-1], W.source_sinprod)
    lib = binding().Solver(prob, **opts, precision=precision, matrix_free=True)
    u, it, _, _ = lib.solve(f, tol=1e-8)
    res = np.linalg.norm(f - A @ u) / np.linalg.norm(f)
    _, it_ref, _ = orc.solve_pcg(f, tol=1e-8)
    assert res <= 1e-8 * 1.0001 and it <= it_ref + 3, (res, it, it_ref)
    lib.close()


def test_matrix_free_unsupported_geometry_is_refused():
    """A geometry map with an interior knot (two polynomial pieces) is refused at assembly."""
    prob = W.grid_problem((1, 1), 8, 2, "sipg", box=(1.0, 1.0))
    c = np.asarray(prob["geo_ctrl"][0]).reshape(4, 2)
    # the same bilinear map with a knot inserted at 1/2 in direction 0
    pts = [c[0], 0.5 * (c[0] + c[1]), c[1], c[2], 0.5 * (c[2] + c[3]), c[3]]
    prob = dict(prob, geo_knots=[[np.array([0.0, 0.0, 0.5, 1.0, 1.0]), np.array([0.0, 0.0, 1.0, 1.0])]],
                geo_ctrl=[np.array(pts)])
    mg = binding()
    with pytest.raises(mg.MgigaError) as e:
        mg.Solver(prob, levels=2, precision="fp32", matrix_free=True)
    assert e.value.status == mg.EINVAL and "one polynomial piece" in str(e.value)


@pytest.mark.parametrize("p", [2, 6])
def test_matrix_free_benchmark_layout_full_size(p):
    """The benchmark layout at 192/288 intervals (0.52-0.54M unknowns): the FP64 matrix-free
    residual equals the FP64 band residual of the same handle within 1e-12 of max |A u|; that band
    is pinned element by element against the oracle at this size by the GPU set-up tests."""
    prob, opts = W.sipg_3x3(p, scale=3, smoother="hybrid")
    mg = binding()
    lib = mg.Solver(prob, smoother="hybrid", tau=opts["tau"], delta=opts["delta"], precision="fp64",
                    matrix_free=True)
    n = lib.ndof()
    rng = np.random.default_rng(9)
    u, f = rng.standard_normal(n), rng.standard_normal(n)
    band = lib.apply("residual", -1, f, u)
    Au = lib.apply("matvec", -1, u)
    got = lib.apply("cycle_residual", -1, f, u)
    assert np.max(np.abs(got - band)) <= 1e-12 * np.max(np.abs(Au))
    lib.close()
