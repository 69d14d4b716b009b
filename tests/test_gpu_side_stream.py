"""The smoother's interface-piece solves beside its fast diagonalisation.

The pieces T of the subspace-corrected mass smoother (Sec. 5, Eq. Ldef) partition the unknowns into
patch interiors and interface pieces, and each correction P_T L_T^{-1} P_T^T r reads only r.  The
library therefore runs the pieces on a second stream (two parallel branches of the captured graph);
MGIGA_SIDE_STREAM=0 keeps them after the interiors on one stream.  Every entry of u then receives
the same operations in the same order either way, so the two must agree bit for bit: the smoother
alone, one V-cycle, and PCG solves (graph-driven and host-driven loop), on the 2D SIPG layout and
the conforming 3D cube (whose shared DoFs are summed after the join).
"""
import numpy as np
import pytest

from paper_1902_01818_gb300 import workloads as W
from lib_fixture import binding

pytestmark = pytest.mark.gpu


def _solver(monkeypatch, prob, opts, precision, smoother, side):
    monkeypatch.setenv("MGIGA_SIDE_STREAM", "1" if side else "0")  # read when the handle is created
    s = binding().Solver(prob, levels=0, smoother=smoother, tau=opts["tau"], delta=opts["delta"],
                         precision=precision)
    monkeypatch.delenv("MGIGA_SIDE_STREAM")
    return s


CASES = {
    "sipg3x3_p3": lambda: W.sipg_3x3(3, scale=1, smoother="hybrid"),
    "sipg3x3_p6": lambda: W.sipg_3x3(6, scale=1, smoother="hybrid"),
    "cube_conforming_p3": lambda: W.cube_2x2x2(3, "conforming", n=12),
}


@pytest.mark.parametrize("smoother", ["hybrid", "scms"])
@pytest.mark.parametrize("precision", ["fp64", "tf32"])
@pytest.mark.parametrize("name", list(CASES))
def test_pieces_beside_interiors_bit_identical(monkeypatch, name, precision, smoother):
    prob, opts = CASES[name]()
    a = _solver(monkeypatch, prob, opts, precision, smoother, True)
    b = _solver(monkeypatch, prob, opts, precision, smoother, False)
    n = a.ndof()
    rng = np.random.default_rng(11)
    r = rng.standard_normal(n)
    top = a.levels - 1
    nl = a.ndof(top)
    f, u = rng.standard_normal(nl), rng.standard_normal(nl)
    assert np.array_equal(a.apply("smooth", top, f, u), b.apply("smooth", top, f, u))
    assert np.array_equal(a.vcycle(r), b.vcycle(r))
    rhs = a.load_sinprod()
    ua, ita, rela, _ = a.solve(rhs, tol=1e-8)
    ub, itb, relb, _ = b.solve(rhs, tol=1e-8)
    assert ita == itb and np.array_equal(ua, ub), (ita, itb)
    monkeypatch.setenv("MGIGA_DEVICE_LOOP", "0")
    uh, ith, _, _ = a.solve(rhs, tol=1e-8)
    monkeypatch.delenv("MGIGA_DEVICE_LOOP")
    assert ith == ita and np.array_equal(uh, ua)
    a.close()
    b.close()
