"""Full-size runs of the benchmark layout (2D SIPG 3x3, 192/288 intervals) and
of the 3D cube (2x2x2 patches, 48 intervals), in the launch configuration the
benchmark times (automatic levels, hybrid smoother, V-cycle-preconditioned CG).

At these sizes the oracle does not solve; it supplies what it computes point
by point: the DoF numbering (integer work, bit-exact against the library), the
B-spline basis and the geometry map at sampled parameter points.  The library's
solution must
  (a) meet the FP64 stopping rule ||f - A u|| <= 1e-8 ||f|| (A u by the FP64
      band product, itself pinned element by element at small sizes),
  (b) agree with the exact solution prod sin(pi x_a) of the manufactured
      problem at sampled points within the discretisation error
      (~ (pi h)^{p+1}, here far below the 1e-4 bound; a wrong solution is off
      by O(1)), and
  (c) on the mixed paths take at most a few more iterations than FP64.
"""
import numpy as np
import pytest

from oracle import bspline, discretize, geometry
from paper_1902_01818_gb300 import workloads as W
from lib_fixture import binding

pytestmark = pytest.mark.gpu


def _sample_error(prob, lib, u, npts=6, seed=7):
    """max |u_h - u| over npts random parameter points in every patch."""
    d, p = prob["dim"], prob["degree"]
    knots = prob["knots"]
    patch, local = lib.dof_map()
    rng = np.random.default_rng(seed)
    worst = 0.0
    shapes = [discretize.shape_of(kn, p) for kn in knots]
    coeffs = [np.zeros(int(np.prod(s))) for s in shapes]
    for g in range(len(u)):  # owner copies; conforming copies are filled below
        coeffs[patch[g]][local[g]] = u[g]
    if prob["coupling"] == "conforming":
        num = discretize.numbering(prob, knots)
        coeffs = discretize.global_to_local_vectors(num, u)
    for k in range(len(knots)):
        xi = rng.uniform(0.05, 0.95, size=(npts, d))
        uh = discretize.evaluate(prob, knots, coeffs[k], k, xi)
        X, _ = geometry.eval_points(prob["geo_degree"], prob["geo_knots"][k], prob["geo_ctrl"][k], xi)
        worst = max(worst, float(np.max(np.abs(uh - W.exact_sinprod(X)))))
    return worst


def _numbering_matches(prob, lib):
    num = discretize.numbering(prob, prob["knots"])
    patch, local = lib.dof_map()
    assert lib.ndof() == num["ndof"]
    owner = np.array(num["owner"])
    assert np.array_equal(patch, owner[:, 0]) and np.array_equal(local, owner[:, 1])


def _solve(prob, opts, precision):
    lib = binding().Solver(prob, levels=opts.get("levels", 0), smoother=opts["smoother"], tau=opts["tau"],
                           delta=opts["delta"], precision=precision)
    f = lib.load_sinprod()
    u, it, rel, st = lib.solve(f, tol=1e-8)
    r = f - lib.apply("matvec", -1, u)
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(f) * 1.0001, (precision, np.linalg.norm(r) / np.linalg.norm(f))
    return lib, u, it


@pytest.mark.parametrize("p", [2, 6])
def test_benchmark_layout_full_size(p):
    prob, opts = W.sipg_3x3(p, scale=3, smoother="hybrid")
    lib64, u64, it64 = _solve(prob, opts, "fp64")
    _numbering_matches(prob, lib64)
    assert lib64.ndof() > 500_000
    assert _sample_error(prob, lib64, u64) <= 1e-4
    lib64.close()
    for prec in ("fp32", "tf32"):
        lib32, u32, it32 = _solve(prob, opts, prec)
        assert it32 <= it64 + 2, (prec, it32, it64)
        assert _sample_error(prob, lib32, u32) <= 1e-4
        lib32.close()


@pytest.mark.parametrize("coupling", ["conforming", "sipg"])
def test_cube_full_size(coupling, monkeypatch):
    """Interiors of 49 per direction: MGIGA_FD_TENSOR_MIN_N=1 sends the TF32 and
    BF16 contractions to the tensor cores (by default these sizes take FP32 SIMT)."""
    monkeypatch.setenv("MGIGA_FD_TENSOR_MIN_N", "1")
    prob, opts = W.cube_2x2x2(3, coupling)
    lib64, u64, it64 = _solve(prob, opts, "fp64")
    _numbering_matches(prob, lib64)
    assert lib64.ndof() > 900_000
    assert _sample_error(prob, lib64, u64, npts=4) <= 1e-4
    lib64.close()
    for prec, extra in (("tf32", 3), ("bf16", 6)):
        lib, u, it = _solve(prob, opts, prec)
        assert it <= it64 + extra, (prec, it, it64)
        assert _sample_error(prob, lib, u, npts=4) <= 1e-4
        lib.close()


def _interior_smoother_check(prob, opts, precision, seed):
    """One application of the smoother on the finest level with u = 0 and f
    supported on the patch interiors: the interface pieces receive zero, so the
    result is tau sum_k P_k L_k^{-1} P_k^T f over the interiors (Sec. 5,
    Eq. Ldef), which the oracle evaluates patch by patch in the eigenbasis of the
    1D pencils (LAPACK; pinned against the sparse LU of L_k on small patches).
    Returns the relative 2-norm error."""
    from oracle import smoothers
    lib = binding().Solver(prob, levels=opts.get("levels", 0), smoother=opts["smoother"], tau=opts["tau"],
                           delta=opts["delta"], precision=precision)
    num = discretize.numbering(prob, prob["knots"])
    assert lib.ndof() == num["ndof"]
    rng = np.random.default_rng(seed)
    f = np.zeros(num["ndof"])
    ref = np.zeros(num["ndof"])
    for k in range(len(prob["knots"])):
        idx = smoothers.interior_dofs(num, k)
        f[idx] = rng.standard_normal(len(idx))
        solve = smoothers.interior_solve_eigen(prob["knots"][k], prob["degree"], opts["delta"])
        ref[idx] = opts["tau"] * solve(f[idx])
    got = lib.apply("smooth", lib.levels - 1, f, np.zeros_like(f))
    lib.close()
    return np.linalg.norm(got - ref) / np.linalg.norm(ref)


def _smooth_tol(precision, d):
    # one application's rounding bound (as in test_gpu_mixed.smooth_tol): FP64 at the
    # accuracy of the two eigen-solvers, FP32 summation, 2d truncated / rounded TF32 / BF16 steps
    if precision == "fp64":
        return 1e-10
    if precision == "fp32":
        return 1e-5
    return 4 * d * (2.0 ** -10 if precision == "tf32" else 2.0 ** -8)


@pytest.mark.parametrize("precision,chained", [("fp64", "1"), ("fp32", "1"), ("tf32", "1"), ("tf32", "0"),
                                              ("bf16", "1")])
@pytest.mark.parametrize("p", [2, 6])
def test_benchmark_layout_finest_smoother(p, precision, chained, monkeypatch):
    """The finest level of the benchmark layout (192/288 intervals, interiors of
    190-292 per direction): by default the TF32 / BF16 modes run the tcgen05
    contractions here (TF32: the four separate steps, or the chained passes with
    MGIGA_FD_CHAINED=1), FP32 the SIMT tiles, FP64 the FP64 tiles."""
    monkeypatch.setenv("MGIGA_FD_CHAINED", chained)
    prob, opts = W.sipg_3x3(p, scale=3, smoother="hybrid")
    err = _interior_smoother_check(prob, opts, precision, seed=20 + p)
    assert err <= _smooth_tol(precision, 2), err


@pytest.mark.parametrize("precision", ["tf32", "bf16"])
def test_cube_finest_smoother_tensor_cores(precision, monkeypatch):
    """The 3D contractions (six steps, batched planes) on the tensor cores at the
    cube's full size (48 intervals, p = 3: interiors of 49)."""
    monkeypatch.setenv("MGIGA_FD_TENSOR_MIN_N", "1")
    prob, opts = W.cube_2x2x2(3, "sipg")
    err = _interior_smoother_check(prob, opts, precision, seed=31)
    assert err <= _smooth_tol(precision, 3), err


@pytest.mark.parametrize("p", [2, 6])
def test_benchmark_layout_finest_transfers(p):
    """Restriction and prolongation between the two finest levels of the benchmark
    layout (mode-wise kernels, FP64 apply) against the oracle's knot-insertion
    matrix P (Sec. 4), element by element at 1e-13."""
    from oracle import hierarchy
    prob, opts = W.sipg_3x3(p, scale=3, smoother="hybrid")
    lib = binding().Solver(prob, levels=0, smoother="hybrid", tau=opts["tau"], delta=opts["delta"],
                           precision="fp32")
    kn = hierarchy.level_knots(prob, lib.levels)
    num_c = discretize.numbering(prob, kn[-2])
    num_f = discretize.numbering(prob, kn[-1])
    P = hierarchy.global_prolongation(prob, kn[-2], kn[-1], num_c, num_f)
    rng = np.random.default_rng(40 + p)
    r = rng.standard_normal(P.shape[0])
    ref = P.T @ r
    got = lib.apply("restrict", lib.levels - 1, r)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    e = rng.standard_normal(P.shape[1])
    ref = P @ e
    got = lib.apply("prolong", lib.levels - 1, e)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    lib.close()
