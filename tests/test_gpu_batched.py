"""The batched layout: independent problems of uneven sizes (1-16 patches in
non-rectangular arrangements, 16-256 intervals, p = 2..5, conforming or SIPG,
random N(0,1) load coefficients), mixed precision (FP32 smoothers) to 1e-8.

Solved concurrently -- one CUDA stream and host thread per problem -- every
result is bit-identical to the same problem solved alone (the library's
reductions have a fixed order, so nothing may depend on what else runs), meets
the FP64 stopping rule with the library's FP64 product, and on the smallest
problems with the oracle's independently assembled matrix.
"""
import threading

import numpy as np
import pytest

from oracle import discretize
from paper_1902_01818_gb300 import workloads as W
from lib_fixture import binding

pytestmark = pytest.mark.gpu

SEEDS = [401 + i for i in range(12)]


def test_batched_layout_concurrent_results_equal_alone():
    torch = pytest.importorskip("torch")
    mgb = binding()
    probs = [W.batched_problem(s) for s in SEEDS]
    streams = [torch.cuda.Stream() for _ in probs]
    solvers = [mgb.Solver(pr, levels=o["levels"], smoother=o["smoother"], tau=o["tau"], delta=o["delta"],
                          precision="fp32", stream=st.cuda_stream)
               for (pr, o, _rs), st in zip(probs, streams)]
    rhs = [W.random_vector(s.ndof(), rs, kind="normal") for s, (_pr, _o, rs) in zip(solvers, probs)]
    alone = [s.solve(f, tol=1e-8) for s, f in zip(solvers, rhs)]
    mixed = [None] * len(solvers)

    def run(i):
        mixed[i] = solvers[i].solve(rhs[i], tol=1e-8)

    threads = [threading.Thread(target=run, args=(i,)) for i in range(len(solvers))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for i, (a, b) in enumerate(zip(alone, mixed)):
        assert a[1] == b[1], (SEEDS[i], a[1], b[1])
        assert np.array_equal(a[0], b[0]), SEEDS[i]
        f = rhs[i]
        r = f - solvers[i].apply("matvec", -1, a[0])
        assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(f) * 1.0001, SEEDS[i]
    # the smallest problems against the oracle's own matrix
    small = sorted(range(len(solvers)), key=lambda i: solvers[i].ndof())[:3]
    for i in small:
        prob = probs[i][0]
        num = discretize.numbering(prob, prob["knots"])
        A = discretize.assemble_global(prob, prob["knots"], num)
        r = rhs[i] - A @ alone[i][0]
        assert np.linalg.norm(r) <= 1.0001e-8 * np.linalg.norm(rhs[i]), SEEDS[i]
    for s in solvers:
        s.close()


@pytest.mark.parametrize("one_graph", [False, True])
def test_batched_entry_point_equals_alone(one_graph):
    """mgiga_solve_batch_d: all problems enqueued from one thread (each solve one
    graph with conditional nodes), or all of them as the branches of a single
    graph launch; every result bit-identical to the problem solved alone, twice
    in a row (the single graph is reused the second time)."""
    torch = pytest.importorskip("torch")
    mgb = binding()
    probs = [W.batched_problem(s) for s in SEEDS]
    streams = [torch.cuda.Stream() for _ in probs]
    solvers = [mgb.Solver(pr, levels=o["levels"], smoother=o["smoother"], tau=o["tau"], delta=o["delta"],
                          precision="tf32", stream=st.cuda_stream)
               for (pr, o, _rs), st in zip(probs, streams)]
    rhs = [W.random_vector(s.ndof(), rs, kind="normal") for s, (_pr, _o, rs) in zip(solvers, probs)]
    alone = [s.solve(f, tol=1e-8) for s, f in zip(solvers, rhs)]
    rd = [torch.from_numpy(f).cuda() for f in rhs]
    for rep in range(2):
        ud = [torch.zeros_like(x) for x in rd]
        torch.cuda.synchronize()
        its, rels, sts = mgb.solve_batch_d(solvers, rd, ud, tol=1e-8, one_graph=one_graph)
        for i, a in enumerate(alone):
            assert sts[i] == mgb.OK and its[i] == a[1] and rels[i] == a[2], (SEEDS[i], its[i], a[1])
            assert np.array_equal(ud[i].cpu().numpy(), a[0]), (rep, SEEDS[i])
            assert solvers[i].residual_history()[-1] == a[2]
    for s in solvers:
        s.close()
