"""Failure detection on the GPU without a fault.

A bounded device wait that runs out: every spin-wait of the kernels gives up
after a fixed number of polls, sets a device flag and lets its launch end;
the host reads the flag when the stream drains and the call returns
MGIGA_ETIMEOUT.  Here one such wait runs on a barrier phase that nothing
completes (a flag nothing sets), with a short poll limit: the call must report
the expiry, and the handle (its stream and context) must stay usable -- the
next solve gives the same result as before.

Faults made on the host: an HBM budget too small (MGIGA_ENOMEM), an SIPG
penalty too small for an SPD operator (the set-up's Cholesky breaks down:
MGIGA_ENOTSPD), a NaN in the right-hand side (MGIGA_EBREAKDOWN, the handle
stays usable).
"""
import numpy as np
import pytest

from paper_1902_01818_gb300 import workloads as W
from lib_fixture import binding

pytestmark = pytest.mark.gpu


def test_expired_wait_reports_timeout_and_handle_stays_usable():
    mgb = binding()
    prob, opts = W.unit_square_2x2(n=16, p=2)
    s = mgb.Solver(prob, levels=3, smoother=opts["smoother"], precision="fp32", tau=opts["tau"], delta=opts["delta"])
    f = s.load_sinprod()
    u0, it0, rel0, _ = s.solve(f, tol=1e-8)
    st, ms = s.check_wait_expiry(1 << 12)
    assert st == mgb.ETIMEOUT, mgb.STATUS_NAMES[st]
    assert "expired" in s.last_error()
    assert 0.0 < ms < 5000.0
    # the flag was cleared: the next calls succeed and repeat the earlier solve exactly
    u1, it1, rel1, _ = s.solve(f, tol=1e-8)
    assert it1 == it0 and np.array_equal(u1, u0)
    st2, _ = s.check_wait_expiry(1 << 10)  # the check repeats
    assert st2 == mgb.ETIMEOUT
    s.close()


def test_wait_expiry_argument_checks():
    mgb = binding()
    prob, opts = W.unit_square_2x2(n=8, p=2)
    s = mgb.Solver(prob, levels=2, precision="fp32")
    for bad in (0, -1, (1 << 18) + 1):
        st, _ = s.check_wait_expiry(bad)
        assert st == mgb.EINVAL
    s.close()


def test_budget_too_small_is_refused_and_handle_stays_destroyable():
    """Allocation refused through a tiny HBM budget: MGIGA_ENOMEM from the set-up."""
    mgb = binding()
    prob, _ = W.unit_square_2x2(n=16, p=2)
    s = mgb.Solver(prob, levels=3, precision="fp32", hbm_budget=64 << 10, assemble=False)
    with pytest.raises(mgb.MgigaError) as e:
        s.assemble()
    assert e.value.status == mgb.ENOMEM and "budget" in s.last_error()
    s.close()


def test_penalty_too_small_breaks_the_cholesky_of_the_setup():
    """SIPG with a penalty far below 5 (p+1)^2 / h: the operator is indefinite (the
    oracle's own matrix, checked here), so the set-up's Cholesky factorisations of
    interface pieces / coarse grid break down: MGIGA_ENOTSPD, no device work."""
    from oracle import hierarchy
    mgb = binding()
    prob = W.grid_problem((2, 2), 8, 2, "sipg", jitter=0.1, seed=1, penalty_factor=1e-3)
    A = hierarchy.build(prob, 1)["A"][0].toarray()
    assert np.linalg.eigvalsh(A)[0] < 0.0
    s = mgb.Solver(prob, levels=2, smoother="scms", tau=0.25, delta=0.1, assemble=False)
    with pytest.raises(mgb.MgigaError) as e:
        s.assemble()
    assert e.value.status == mgb.ENOTSPD
    s.close()


def test_nan_right_hand_side_is_a_breakdown_and_the_handle_stays_usable():
    mgb = binding()
    prob, opts = W.unit_square_2x2(n=16, p=2)
    s = mgb.Solver(prob, levels=3, smoother=opts["smoother"], precision="fp32", tau=opts["tau"],
                   delta=opts["delta"])
    f = s.load_sinprod()
    u0, it0, _, _ = s.solve(f, tol=1e-8)
    g = f.copy()
    g[len(g) // 2] = np.nan
    with pytest.raises(mgb.MgigaError) as e:
        s.solve(g, tol=1e-8)
    assert e.value.status == mgb.EBREAKDOWN
    u1, it1, _, _ = s.solve(f, tol=1e-8)
    assert it1 == it0 and np.array_equal(u1, u0)
    s.close()
