"""The batched layout: many independent problems of uneven sizes solved together.

Every problem gets its own handle (operators resident on the device) and its own
non-blocking CUDA stream; `workers` host threads drain the batch, so the solves
of different problems overlap on the GPU.  Set-up (host assembly, hierarchy,
upload) is timed separately from the solves; the solve figure is the unknowns
of the whole batch over the wall time of one pass over it (inputs resident),
with the per-problem solve times' p50/p99.

    python -m paper_1902_01818_gb300.batch --problems 256 --workers 16 --reps 3

prints one JSON line.
"""
import concurrent.futures as cf
import time

import numpy as np


def run_batch(problems, workers=16, reps=1, precision="tf32", tol=1e-8, solver_factory=None,
              setup_workers=None):
    """problems: list of (problem, options, rhs seed).  Returns a statistics dict."""
    from . import workloads as W
    if solver_factory is None:
        from . import mgiga

        def solver_factory(prob, opts):
            return mgiga.Solver(prob, levels=opts["levels"], smoother=opts["smoother"], tau=opts["tau"],
                                delta=opts["delta"], precision=precision, gs_cluster=opts.get("gs_cluster", 8))
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=setup_workers or workers) as ex:
        solvers = list(ex.map(lambda pr: solver_factory(pr[0], pr[1]), problems))
    t_setup = time.perf_counter() - t0
    rhs = [W.random_vector(s.ndof(), int(rs), kind="normal") for s, (_p, _o, rs) in zip(solvers, problems)]
    ndof = [s.ndof() for s in solvers]

    def one(i):
        a = time.perf_counter()
        u, it, rel, _st = solvers[i].solve(rhs[i], tol=tol)
        return time.perf_counter() - a, it, rel

    passes, per = [], []
    try:
        with cf.ThreadPoolExecutor(max_workers=workers) as ex:
            for _ in range(reps):
                a = time.perf_counter()
                out = list(ex.map(one, range(len(solvers))))
                passes.append(time.perf_counter() - a)
                per.extend(o[0] for o in out)
    finally:
        for s in solvers:
            s.close()
    iters = [o[1] for o in out]
    rels = [o[2] for o in out]
    best = min(passes)
    return {"problems": len(problems), "unknowns": int(sum(ndof)), "workers": workers, "reps": reps,
            "precision": precision, "setup_s": t_setup, "pass_s": passes,
            "value": sum(ndof) / best, "unit": "DoF/s (best pass, inputs resident)",
            "solve_p50_ms": 1e3 * float(np.percentile(per, 50)), "solve_p99_ms": 1e3 * float(np.percentile(per, 99)),
            "iterations_mean": float(np.mean(iters)), "iterations_max": int(max(iters)),
            "max_final_relres": float(max(rels))}


def main(argv=None):
    """Solve the seeded batched layout; print the statistics as one JSON line."""
    import argparse
    import json

    from . import workloads as W
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--problems", type=int, default=256)
    ap.add_argument("--workers", type=int, default=16)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--precision", default="tf32", choices=["fp64", "fp32", "tf32", "bf16"])
    ap.add_argument("--seed", type=int, default=401)
    args = ap.parse_args(argv)
    probs = [W.batched_problem(args.seed + i) for i in range(args.problems)]
    print(json.dumps(run_batch(probs, workers=args.workers, reps=args.reps, precision=args.precision)), flush=True)


if __name__ == "__main__":
    main()
