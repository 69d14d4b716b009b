"""Host logic of the request loop (paper_1902_01818_gb300.serve) with a fake
solver: operator reuse, admission by the HBM budget (eviction of idle handles,
waiting for busy ones, rejection of what never fits) and concurrent workers."""
import threading
import time

import numpy as np
import pytest

from paper_1902_01818_gb300.serve import Rejected, Server

ENOMEM = 2


class _Err(RuntimeError):
    def __init__(self, status):
        super().__init__("budget")
        self.status = status


class _Fake:
    def __init__(self, nbytes, delay):
        self.nbytes, self.delay, self.closed = nbytes, delay, False

    def solve(self, rhs, tol):
        time.sleep(self.delay)
        return 2.0 * rhs, 3, 0.0, 0

    def device_bytes(self):
        return self.nbytes

    def ndof(self):
        return 5

    def close(self):
        self.closed = True


def _server(budget, workers=1, delay=0.0):
    made = []

    def factory(problem, options, precision, left):
        if problem["bytes"] > left:
            raise _Err(ENOMEM)
        s = _Fake(problem["bytes"], delay)
        made.append(s)
        return s

    return Server(workers=workers, hbm_budget=budget, solver_factory=factory, enomem_status=ENOMEM), made


def test_reuse_and_eviction_and_rejection():
    srv, made = _server(100)
    srv.start()
    a = srv.submit("A", {"bytes": 60}, {}, np.ones(3)).result(timeout=5)
    a2 = srv.submit("A", {"bytes": 60}, {}, np.full(3, 2.0)).result(timeout=5)
    assert np.array_equal(a[0], np.full(3, 2.0)) and np.array_equal(a2[0], np.full(3, 4.0))
    assert srv.stats()["setups"] == 1  # the resident operator was reused
    srv.submit("B", {"bytes": 60}, {}, np.ones(3)).result(timeout=5)
    st = srv.stats()
    assert st["setups"] == 2 and st["evictions"] == 1 and made[0].closed  # A evicted for B
    with pytest.raises(Rejected):
        srv.submit("C", {"bytes": 200}, {}, np.ones(3)).result(timeout=5)
    srv.stop()
    st = srv.stats()
    assert st["rejected"] == 1 and st["solves"] == 3 and st["p99_ms"] >= st["p50_ms"] >= 0.0


def test_busy_handles_are_waited_for_not_evicted():
    # budget for one operator; two workers: the second request waits until the first solve ends
    srv, made = _server(100, workers=2, delay=0.2)
    srv.start()
    f1 = srv.submit("A", {"bytes": 80}, {}, np.ones(2))
    time.sleep(0.05)
    f2 = srv.submit("B", {"bytes": 80}, {}, np.ones(2))
    r1, r2 = f1.result(timeout=5), f2.result(timeout=5)
    assert r2[3] >= 0.2  # B waited for A's solve before its set-up
    assert srv.stats()["evictions"] == 1
    srv.stop()


def test_many_concurrent_requests():
    srv, made = _server(10_000, workers=4, delay=0.01)
    srv.start()
    futs = [srv.submit(k % 5, {"bytes": 100}, {}, np.full(4, float(k))) for k in range(40)]
    for k, f in enumerate(futs):
        assert np.array_equal(f.result(timeout=10)[0], np.full(4, 2.0 * k))
    st = srv.stats()
    srv.stop()
    assert st["solves"] == 40 and st["setups"] == 5 and st["evictions"] == 0


def test_seed_right_hand_sides_and_throughput_statistics():
    """An int right-hand side is a seed: the worker draws N(0, 1) load coefficients of
    the operator's size; the statistics report solves/s and the admission queue."""
    from paper_1902_01818_gb300 import workloads as W
    srv, made = _server(10_000, workers=1, delay=0.02)
    futs = [srv.submit("A", {"bytes": 10}, {}, 7) for _ in range(4)]  # queued before the workers start
    assert srv.stats()["queue"] == 4 and srv.stats()["max_queue"] == 4
    srv.start()
    outs = [f.result(timeout=5) for f in futs]
    expect = 2.0 * W.random_vector(5, 7, kind="normal")
    for u, it, rel, lat in outs:
        assert np.array_equal(u, expect)
    st = srv.stats()
    srv.stop()
    assert st["queue"] == 0 and st["solves"] == 4
    assert 0.0 < st["solves_per_s"] <= 4 / 0.08 * 1.01  # four 20 ms solves one after another
