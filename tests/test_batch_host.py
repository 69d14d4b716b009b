"""Host logic of the batch runner (paper_1902_01818_gb300.batch) with a fake
solver: every problem set up once and solved `reps` times by the worker pool,
seeded right-hand sides of the operator's size, statistics of the passes."""
import time


from paper_1902_01818_gb300 import workloads as W
from paper_1902_01818_gb300.batch import run_batch


class _Fake:
    made = []

    def __init__(self, n):
        self.n, self.calls, self.closed = n, 0, False
        _Fake.made.append(self)

    def ndof(self):
        return self.n

    def solve(self, rhs, tol):
        assert len(rhs) == self.n
        self.calls += 1
        time.sleep(0.01)
        return 2.0 * rhs, 7, 1e-9, 0

    def close(self):
        self.closed = True


def test_batch_runs_every_problem_each_pass_and_reports():
    _Fake.made = []
    probs = [({"n": 10 + i}, {}, 100 + i) for i in range(12)]
    st = run_batch(probs, workers=4, reps=2, solver_factory=lambda pr, o: _Fake(pr["n"]))
    assert st["problems"] == 12 and st["unknowns"] == sum(10 + i for i in range(12))
    assert len(st["pass_s"]) == 2 and st["value"] == st["unknowns"] / min(st["pass_s"])
    assert all(f.calls == 2 and f.closed for f in _Fake.made)
    assert st["iterations_max"] == 7 and st["solve_p99_ms"] >= st["solve_p50_ms"] >= 10.0 * 0.9
    # four workers: a pass over twelve 10 ms solves takes about three rounds, not twelve
    assert min(st["pass_s"]) < 12 * 0.01


def test_batched_layout_generator_is_seeded():
    a, b = W.batched_problem(401), W.batched_problem(401)
    assert a[2] == b[2] and a[0]["degree"] == b[0]["degree"] and len(a[0]["knots"]) == len(b[0]["knots"])
