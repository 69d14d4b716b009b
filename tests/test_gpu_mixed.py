"""The mixed-precision cycle (FP32 / TF32 / BF16 smoothers inside FP64 CG) against the oracle.

The FP32 smoothers change the preconditioner, not the problem: PCG must still
meet the FP64 stopping rule ||f - A u|| / ||f|| <= 1e-8 with the oracle's own
matrix, the iteration count stays close to the FP64 one, and the solution
differs from the oracle's by no more than the residual allows:
||u - u*|| <= ||A^{-1}|| (||r|| + ||r*||) (tolerance derived from the two
residuals and the smallest eigenvalue of A, computed densely on these small
problems).  Single smoother applications agree with FP64 to the rounding of
their arithmetic (the Gauss-Seidel sweeps are FP32 in every mixed mode).
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import mg as omg
from paper_1902_01818_gb300 import workloads as W
from lib_fixture import binding

pytestmark = pytest.mark.gpu


def _nm(c, a):
    return 4 if sum(c) % 2 == 0 else 8


CASES = {
    "conf2d_p2": (lambda: W.grid_problem((2, 2), 8, 2, "conforming", jitter=0.1, seed=1, flip_patches=(3,)),
                  3, dict(tau=1.0, delta=0.12)),
    "sipg2d_p3": (lambda: W.grid_problem((3, 3), _nm, 3, "sipg", jitter=0.1, seed=2, flip_patches=(1,),
                                         transpose_patches=(4,)), 3, dict(tau=0.25, delta=0.1)),
    "sipg3d_p2": (lambda: W.grid_problem((2, 1, 2), _nm, 2, "sipg", jitter=0.05, seed=4, flip_patches=(1,),
                                         transpose_patches=(2,)), 2, dict(tau=0.25, delta=0.12)),
    "conf3d_p3": (lambda: W.grid_problem((2, 2, 2), 4, 3, "conforming", jitter=0.05, seed=3,
                                         jitter_boundary_tangential=True), 2, dict(tau=0.25, delta=0.12)),
}


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
@pytest.mark.parametrize("smoother", ["hybrid", "scms"])
@pytest.mark.parametrize("name", list(CASES))
def test_mixed_pcg_meets_fp64_stopping_rule(name, smoother, precision):
    fac, levels, opt = CASES[name]
    prob = fac()
    mgb = binding()
    lib = mgb.Solver(prob, levels=levels, smoother=smoother, precision=precision, **opt)
    orc = omg.Multigrid(prob, levels=levels, smoother=smoother, **opt)
    f = lib.load_sinprod()
    u, it, rel, st = lib.solve(f, tol=1e-8)
    A = orc.A
    r = f - A @ u
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(f) * 1.0001
    u_o, it_o, _ = orc.solve_pcg(f, tol=1e-8)
    assert it <= it_o + (3 if precision != "bf16" else 6), (it, it_o)
    lam_min = sla.eigh(A.toarray(), eigvals_only=True, subset_by_index=[0, 0])[0]
    bound = (np.linalg.norm(r) + np.linalg.norm(f - A @ u_o)) / lam_min
    err = np.linalg.norm(u - u_o)
    assert err <= 1.01 * bound, (err, bound)
    lib.close()


def smooth_tol(precision, d):
    """Relative accuracy bound of one smoother application.

    FP32: rounding (unit 6e-8) accumulated over contraction lengths of a few
    hundred.  Tensor cores: the fast diagonalisation is 2d contractions; each
    truncates (TF32, 10 fraction bits: 2^-10) or rounds (BF16, 7 fraction
    bits: 2^-8) both operands, so each step is accurate to 2 x that unit and
    the chain to 2d x 2 x unit.
    """
    if precision == "fp32":
        return 1e-5
    unit = 2.0 ** -10 if precision == "tf32" else 2.0 ** -8
    return 4 * d * unit


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
@pytest.mark.parametrize("name", list(CASES))
def test_mixed_smoothers_match_fp64_to_their_rounding(name, precision):
    fac, levels, opt = CASES[name]
    prob = fac()
    mgb = binding()
    lib = mgb.Solver(prob, levels=levels, smoother="hybrid", precision=precision, **opt)
    orc = omg.Multigrid(prob, levels=levels, smoother="hybrid", **opt)
    rng = np.random.default_rng(9)
    for l in range(1, levels):
        A = orc.h["A"][l]
        n = A.shape[0]
        u, f = rng.standard_normal(n), rng.standard_normal(n)
        ref = u + orc.scms[l].apply(f - A @ u)
        got = lib.apply("smooth", l, f, u)
        assert np.linalg.norm(got - ref) <= smooth_tol(precision, prob["dim"]) * np.linalg.norm(ref - u), l
        for op, fn in (("gs_fwd", orc.gs[l].forward), ("gs_bwd", orc.gs[l].backward)):
            ref = fn(f, u)
            got = lib.apply(op, l, f, u)
            assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref - u), (l, op)
    lib.close()


@pytest.mark.parametrize("name", list(CASES))
def test_cycle_residual_within_fp32_rounding(name):
    """The residual inside the mixed cycle (FP32 band, FP32 sums) against f - A u.

    Row i sums m = copies x (2p+1)^d products of FP32-rounded coefficients and
    FP32-rounded u; the standard bound for such a sum is
    |fl(s) - s| <= gamma_{m+2} sum_j |a_ij| |u_j|, gamma_k = k u / (1 - k u),
    u = 2^-24 (the SIPG cross-patch terms stay FP64).
    """
    fac, levels, opt = CASES[name]
    prob = fac()
    lib = binding().Solver(prob, levels=levels, smoother="hybrid", precision="fp32", **opt)
    orc = omg.Multigrid(prob, levels=levels, smoother="hybrid", **opt)
    d, p = prob["dim"], prob["degree"]
    copies = 2 ** d if prob["coupling"] == "conforming" else 1
    m = copies * (2 * p + 1) ** d
    unit = 2.0 ** -24
    gamma = (m + 2) * unit / (1 - (m + 2) * unit)
    rng = np.random.default_rng(11)
    for l in range(1, levels):
        A = orc.h["A"][l]
        n = A.shape[0]
        u, f = rng.standard_normal(n), rng.standard_normal(n)
        ref = f - A @ u
        got = lib.apply("cycle_residual", l, f, u)
        bound = gamma * (abs(A) @ np.abs(u)) + 4 * 2.0 ** -53 * (np.abs(f) + abs(A) @ np.abs(u))
        assert np.all(np.abs(got - ref) <= bound), (l, float(np.max(np.abs(got - ref) / bound)))
        # FP64 precision keeps the FP64 residual
    lib.close()


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
@pytest.mark.parametrize("name", ["conf2d_p2", "sipg2d_p3"])
def test_mixed_smoother_batched_contractions(name, precision, monkeypatch):
    """2D interiors this small take the fused one-CTA path; force the batched
    contractions (on TF32: K-major 16-byte-copy tasks with transposed outputs)."""
    monkeypatch.setenv("MGIGA_FD_FUSE", "0")
    fac, levels, opt = CASES[name]
    prob = fac()
    lib = binding().Solver(prob, levels=levels, smoother="hybrid", precision=precision, **opt)
    orc = omg.Multigrid(prob, levels=levels, smoother="hybrid", **opt)
    rng = np.random.default_rng(12)
    for l in range(1, levels):
        A = orc.h["A"][l]
        n = A.shape[0]
        u, f = rng.standard_normal(n), rng.standard_normal(n)
        ref = u + orc.scms[l].apply(f - A @ u)
        got = lib.apply("smooth", l, f, u)
        assert np.linalg.norm(got - ref) <= smooth_tol(precision, prob["dim"]) * np.linalg.norm(ref - u), l
    lib.close()


@pytest.mark.parametrize("cs", [2, 4, 8, 16])
@pytest.mark.parametrize("name", ["sipg2d_p3", "sipg3d_p2", "conf2d_p2"])
def test_gauss_seidel_cluster_sizes(name, cs, monkeypatch):
    """The patch-parallel sweep with its patches cut into 2..16 slabs (one CTA
    each, halos exchanged between runs of colours with one slow residue): both
    directions match the FP64 sweep to FP32 rounding on every level, also where
    a slab is thinner than the band's reach (halos from several neighbours)."""
    monkeypatch.setenv("MGIGA_GS_CS", str(cs))
    fac, levels, opt = CASES[name]
    prob = fac()
    lib = binding().Solver(prob, levels=levels, smoother="hybrid", precision="fp32", **opt)
    orc = omg.Multigrid(prob, levels=levels, smoother="hybrid", **opt)
    rng = np.random.default_rng(13)
    for l in range(1, levels):
        A = orc.h["A"][l]
        n = A.shape[0]
        u, f = rng.standard_normal(n), rng.standard_normal(n)
        for op, fn in (("gs_fwd", orc.gs[l].forward), ("gs_bwd", orc.gs[l].backward)):
            ref = fn(f, u)
            got = lib.apply(op, l, f, u)
            assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref - u), (l, op)
    lib.close()


_STREAMED = {}


def _streamed_case():
    """The benchmark layout at 64/96 intervals, p = 4 (62,180 unknowns): the
    patches' coefficient blocks exceed shared memory, so the sweep streams them
    through its ring of chunk buffers.  Oracle sweeps on the finest level only."""
    if not _STREAMED:
        from oracle import hierarchy, smoothers
        prob, opts = W.sipg_3x3(4, scale=1, smoother="hybrid")
        h = hierarchy.build(prob, 1)
        col = smoothers.colouring(prob, h["knots"][0], h["num"][0])
        _STREAMED.update(prob=prob, opts=opts, A=h["A"][0],
                         gs=smoothers.GaussSeidel(h["A"][0], smoothers.gs_order(col)))
    return _STREAMED


@pytest.mark.parametrize("cs,nbuf", [(1, 2), (1, 8), (16, 2), (16, 3)])
def test_gauss_seidel_streamed_ring(cs, nbuf, monkeypatch):
    """Streamed coefficient blocks through 2..8 chunk buffers, with colours split
    over several chunks: both sweep directions match the FP64 sweep."""
    monkeypatch.setenv("MGIGA_GS_CS", str(cs))
    monkeypatch.setenv("MGIGA_GS_NBUF", str(nbuf))
    c = _streamed_case()
    o = c["opts"]
    lib = binding().Solver(c["prob"], levels=0, smoother="hybrid", tau=o["tau"], delta=o["delta"],
                           precision="fp32")
    rng = np.random.default_rng(14)
    n = c["A"].shape[0]
    u, f = rng.standard_normal(n), rng.standard_normal(n)
    for op, fn in (("gs_fwd", c["gs"].forward), ("gs_bwd", c["gs"].backward)):
        ref = fn(f, u)
        got = lib.apply(op, lib.levels - 1, f, u)
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref - u), op
    lib.close()


@pytest.mark.parametrize("precision,chained", [("tf32", "1"), ("tf32", "0"), ("bf16", "1")])
@pytest.mark.parametrize("name", list(CASES))
def test_tensor_core_smoother_every_level(name, precision, chained, monkeypatch):
    """The tcgen05 contractions on these small interiors: MGIGA_FD_TENSOR_MIN_N=1
    sends every level's fast diagonalisation to the tensor cores (2D TF32: the two
    chained-contraction passes of fd_fused_tf32 with MGIGA_FD_CHAINED=1, else the
    four gemm_umma_tf32 steps; 3D TF32: gemm_umma_tf32; BF16: gemm_umma<BF16>;
    with MGIGA_FD_FUSE=0 the 2D levels leave the one-CTA SIMT path), one smoother
    application against the oracle's explicit interior solves at the rounding
    bound of the arithmetic."""
    monkeypatch.setenv("MGIGA_FD_TENSOR_MIN_N", "1")
    monkeypatch.setenv("MGIGA_FD_FUSE", "0")
    monkeypatch.setenv("MGIGA_FD_CHAINED", chained)
    fac, levels, opt = CASES[name]
    prob = fac()
    lib = binding().Solver(prob, levels=levels, smoother="hybrid", precision=precision, **opt)
    orc = omg.Multigrid(prob, levels=levels, smoother="hybrid", **opt)
    rng = np.random.default_rng(15)
    for l in range(1, levels):
        A = orc.h["A"][l]
        n = A.shape[0]
        u, f = rng.standard_normal(n), rng.standard_normal(n)
        ref = u + orc.scms[l].apply(f - A @ u)
        got = lib.apply("smooth", l, f, u)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref - u)
        assert err <= smooth_tol(precision, prob["dim"]), (l, err)
        # and not exact: the tensor-core arithmetic is really in use
        assert err > 1e-9, (l, err)
    lib.close()


@pytest.mark.parametrize("name", ["sipg2d_p3", "conf3d_p3"])
def test_autotuned_handle(name):
    """autotune: the contraction engine of every level and the residual's row
    blocking chosen by timing; the smoother still matches the oracle at the
    rounding bound of its arithmetic (TF32 at worst) and PCG meets the FP64
    stopping rule; a second handle of the same sizes reuses the decisions."""
    fac, levels, opt = CASES[name]
    prob = fac()
    mgb = binding()
    orc = omg.Multigrid(prob, levels=levels, smoother="hybrid", **opt)
    for rep in range(2):
        lib = mgb.Solver(prob, levels=levels, smoother="hybrid", precision="tf32", autotune=True, **opt)
        rng = np.random.default_rng(16)
        for l in range(1, levels):
            A = orc.h["A"][l]
            n = A.shape[0]
            u, f = rng.standard_normal(n), rng.standard_normal(n)
            ref = u + orc.scms[l].apply(f - A @ u)
            got = lib.apply("smooth", l, f, u)
            assert np.linalg.norm(got - ref) <= smooth_tol("tf32", prob["dim"]) * np.linalg.norm(ref - u), l
        f = lib.load_sinprod()
        u, it, rel, st = lib.solve(f, tol=1e-8)
        assert np.linalg.norm(f - orc.A @ u) <= 1e-8 * np.linalg.norm(f) * 1.0001
        lib.close()
