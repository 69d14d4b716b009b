"""Oracle runs of the parity layouts in a pool of spawned processes (test code).

The oracle's set-up of the 64/96-interval SIPG layout and of the 12-interval
cube takes seconds to minutes per case on one host core, so the GPU tests that
need them submit every case at collection time (conftest.py) and pick the
results up when they run; the GPU tests of the other files run meanwhile.
Spawned workers, one BLAS thread each: nothing is forked from a process that
has touched the GPU.  Inputs come from the seeded generators of workloads.py
only; the results are the oracle's alone.
"""
import concurrent.futures as cf
import multiprocessing as mp
import os

_pool = None
_futures = {}

# name -> (workload, degree, coupling, intervals)
LAYOUTS = {}
for _p in (2, 3, 4, 5, 6):
    LAYOUTS[f"sipg3x3_6496_p{_p}"] = ("sipg3x3", _p, "sipg", None)
for _p in (3, 4, 5):
    for _c in ("conforming", "sipg"):
        LAYOUTS[f"cube12_{_c}_p{_p}"] = ("cube", _p, _c, 12)

ITERATES = (1, 3, 6)


def _init_worker():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"


def problem_of(spec):
    from paper_1902_01818_gb300 import workloads as W
    kind, p, coupling, n = spec
    if kind == "sipg3x3":
        return W.sipg_3x3(p, scale=1, smoother="hybrid")
    return W.cube_2x2x2(p, coupling, n=n)


def oracle_run(spec):
    """The oracle's load vector, PCG iterates after 1, 3, 6 iterations and its
    solve to 1e-8 (iterations, history) for one layout (hybrid smoother)."""
    from oracle import discretize, mg
    from paper_1902_01818_gb300 import workloads as W
    prob, opts = problem_of(spec)
    M = mg.Multigrid(prob, smoother=opts["smoother"], tau=opts["tau"], delta=opts["delta"])
    f = discretize.assemble_load(prob, prob["knots"], M.h["num"][-1], W.source_sinprod)
    out = dict(ndof=M.ndof, f=f, iterates={})
    for k in ITERATES:
        u, it, _ = M.solve_pcg(f, max_iter=k, tol=1e-300)
        out["iterates"][k] = u
    u, it, hist = M.solve_pcg(f, tol=1e-8)
    out.update(u=u, it=it, hist=hist)
    return out


def start(names):
    """Submit the oracle runs of `names` (idempotent)."""
    global _pool
    todo = [n for n in names if n not in _futures]
    if not todo:
        return
    if _pool is None:
        workers = max(1, min(len(LAYOUTS), os.cpu_count() or 1))
        _pool = cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"),
                                       initializer=_init_worker)
    # the slowest (highest degree, 3D) first
    for n in sorted(todo, key=lambda n: (LAYOUTS[n][0] != "cube", -LAYOUTS[n][1])):
        _futures[n] = _pool.submit(oracle_run, LAYOUTS[n])


def result(name, timeout=3000):
    start([name])
    return _futures[name].result(timeout=timeout)


def stop():
    """Cancel what has not started and end the workers (pytest session end)."""
    global _pool
    if _pool is None:
        return
    procs = list(getattr(_pool, "_processes", {}).values())
    _pool.shutdown(wait=False, cancel_futures=True)
    for pr in procs:  # the exact worker processes this module started
        if pr.is_alive():
            pr.terminate()
    _pool = None
