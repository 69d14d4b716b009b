"""The serving layout through the request loop (paper_1902_01818_gb300.serve):
requests of mixed dimension, size, degree and coupling, half of them reusing a
resident operator with a new right-hand side, served concurrently by four
workers (a handle, hence a CUDA stream, per operator).  Every result is
bit-identical to the same request solved alone on a fresh handle, and meets the
FP64 stopping rule; a budget too small for two operators forces evictions and
still serves every request; the loop reports p50/p99 latency.
"""
import numpy as np
import pytest

from paper_1902_01818_gb300 import workloads as W
from lib_fixture import binding

pytestmark = pytest.mark.gpu


def _requests(n, max_entries=4e7):
    """The first n requests of the stream whose band fits a quick test."""
    out = []
    for key, prob, opts, rs in W.serving_stream(200, max_patch_dof=6000):
        nloc = sum(int(np.prod([len(t) - prob["degree"] - 1 for t in kn])) for kn in prob["knots"])
        if nloc * (2 * prob["degree"] + 1) ** prob["dim"] <= max_entries:
            out.append((key, prob, opts, rs))
        if len(out) == n:
            break
    return out


def _alone(mgb, prob, opts, rhs):
    s = mgb.Solver(prob, levels=0, smoother=opts["smoother"], tau=opts["tau"], delta=opts["delta"],
                   precision="tf32", gs_cluster=8)
    u, it, rel, st = s.solve(rhs, tol=1e-8)
    r = rhs - s.apply("matvec", -1, u)
    s.close()
    return u, it, float(np.linalg.norm(r) / np.linalg.norm(rhs))


def test_serving_results_equal_alone_and_budget_evictions():
    from paper_1902_01818_gb300.serve import Server
    mgb = binding()
    reqs = _requests(10)
    dims = {prob["dim"] for _k, prob, _o, _r in reqs}
    assert dims == {2, 3} and len({k for k, *_ in reqs}) < len(reqs)  # both dimensions, some reuse
    srv = Server(workers=4, hbm_budget=64 << 30)
    srv.start()
    futs = []
    for key, prob, opts, rs in reqs:
        n = _ndof_of(mgb, prob, opts)
        f = W.random_vector(n, rs, kind="normal")
        futs.append((key, prob, opts, f, srv.submit(key, prob, opts, f)))
    results = [(key, prob, opts, f, fut.result(timeout=600)) for key, prob, opts, f, fut in futs]
    st = srv.stats()
    srv.stop()
    assert st["solves"] == len(reqs) and st["rejected"] == 0 and st["setups"] == len({k for k, *_ in reqs})
    assert st["p99_ms"] >= st["p50_ms"] > 0.0
    for key, prob, opts, f, (u, it, rel, lat) in results:
        u1, it1, rel1 = _alone(mgb, prob, opts, f)
        assert it == it1 and np.array_equal(u, u1), key
        assert rel1 <= 1.0001e-8, key
    # a budget that holds the largest operator but not two: evictions, every request served
    biggest = max(_bytes_of(mgb, prob, opts) for _k, prob, opts, _r in reqs)
    srv = Server(workers=2, hbm_budget=int(biggest * 1.5))
    srv.start()
    futs = [srv.submit(key, prob, opts, f) for key, prob, opts, f, _res in results]
    for (key, prob, opts, f, (u, it, rel, lat)), fut in zip(results, futs):
        u2, it2, rel2, lat2 = fut.result(timeout=600)
        assert it2 == it and np.array_equal(u2, u), key
    st = srv.stats()
    srv.stop()
    assert st["evictions"] > 0 and st["rejected"] == 0


_cache = {}


def _probe(mgb, prob, opts):
    key = id(prob)
    if key not in _cache:
        s = mgb.Solver(prob, levels=0, smoother=opts["smoother"], tau=opts["tau"], delta=opts["delta"],
                       precision="tf32", gs_cluster=8)
        _cache[key] = (s.ndof(), s.device_bytes())
        s.close()
    return _cache[key]


def _ndof_of(mgb, prob, opts):
    return _probe(mgb, prob, opts)[0]


def _bytes_of(mgb, prob, opts):
    return _probe(mgb, prob, opts)[1]
