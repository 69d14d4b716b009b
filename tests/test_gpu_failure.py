"""Failure detection on the GPU without a fault: a bounded device wait that
runs out.

Every spin-wait of the kernels gives up after a fixed number of polls, sets a
device flag and lets its launch end; the host reads the flag when the stream
drains and the call returns MGIGA_ETIMEOUT.  Here one such wait runs on a
barrier phase that nothing completes (a flag nothing sets), with a short poll
limit: the call must report the expiry, and the handle (its stream and
context) must stay usable -- the next solve gives the same result as a solve
on a fresh handle.
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
    for bad in (0, -1, (1 << 21) + 1):
        st, _ = s.check_wait_expiry(bad)
        assert st == mgb.EINVAL
    s.close()
