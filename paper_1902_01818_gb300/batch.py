"""The batched layout: many independent problems of uneven sizes solved together.

Every problem gets its own handle (operators resident on the device) and its own
non-blocking CUDA stream; `workers` host threads drain the batch, so the solves
of different problems overlap on the GPU.  Set-up (host assembly, hierarchy,
upload) is timed separately from the solves; the solve figure is the unknowns
of the whole batch over the wall time of one pass over it (inputs resident),
with the per-problem solve times' p50/p99.

    python -m paper_1902_01818_gb300.batch --problems 256 --reps 3 [--mode graph|streams|threads]

prints one JSON line.  Modes: the whole batch as one graph launch (each problem's PCG loop a branch
with conditional nodes), a graph per problem enqueued from one host thread, or a host thread per
solve.
"""
import concurrent.futures as cf
import time

import numpy as np


def run_batch_device(problems, reps=1, precision="tf32", tol=1e-8, one_graph=True, setup_workers=16):
    """The batch through mgiga_solve_batch_d: every solve one graph (no host round trip per
    iteration), all enqueued from this thread; one_graph: all of them the branches of a single graph
    launch.  Inputs resident on the device; returns a statistics dict."""
    import torch

    from . import mgiga, workloads as W
    streams = [torch.cuda.Stream() for _ in problems]
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=setup_workers) as ex:
        solvers = list(ex.map(lambda a: mgiga.Solver(a[0][0], levels=a[0][1]["levels"], smoother=a[0][1]["smoother"],
                                                     tau=a[0][1]["tau"], delta=a[0][1]["delta"], precision=precision,
                                                     gs_cluster=a[0][1].get("gs_cluster", 8),
                                                     stream=a[1].cuda_stream),
                              zip(problems, streams)))
    t_setup = time.perf_counter() - t0
    rhs = [torch.from_numpy(W.random_vector(s.ndof(), int(rs), kind="normal")).cuda()
           for s, (_p, _o, rs) in zip(solvers, problems)]
    ndof = [s.ndof() for s in solvers]
    passes = []
    try:
        for _ in range(reps + 1):  # the first pass builds the graphs
            u = [torch.zeros_like(f) for f in rhs]
            torch.cuda.synchronize()
            a = time.perf_counter()
            its, rels, sts = mgiga.solve_batch_d(solvers, rhs, u, tol=tol, one_graph=one_graph)
            torch.cuda.synchronize()
            passes.append(time.perf_counter() - a)
    finally:
        for s in solvers:
            s.close()
    best = min(passes[1:]) if reps > 0 else passes[0]
    return {"problems": len(problems), "unknowns": int(sum(ndof)), "mode": "one graph" if one_graph else
            "one graph per problem, one host thread", "reps": reps, "precision": precision, "setup_s": t_setup,
            "first_pass_s": passes[0], "pass_s": passes[1:], "value": sum(ndof) / best,
            "unit": "DoF/s (best pass, inputs resident)", "iterations_mean": float(np.mean(its)),
            "iterations_max": int(max(its)), "max_final_relres": float(max(rels)),
            "failed": int(sum(1 for x in sts if x != 0))}


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
    ap.add_argument("--mode", default="graph", choices=["graph", "streams", "threads"],
                    help="graph: one graph launch for the whole batch; streams: a graph per problem, all "
                         "enqueued from one thread; threads: a host thread per solve (mgiga_solve)")
    args = ap.parse_args(argv)
    probs = [W.batched_problem(args.seed + i) for i in range(args.problems)]
    if args.mode == "threads":
        out = run_batch(probs, workers=args.workers, reps=args.reps, precision=args.precision)
    else:
        out = run_batch_device(probs, reps=args.reps, precision=args.precision, one_graph=args.mode == "graph")
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
