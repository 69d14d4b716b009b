"""Per-level stage times of the V-cycle on the SIPG 3x3 benchmark layout.

    python -m paper_1902_01818_gb300.stage_timer --degree 6 --precision fp32 \
        [--levels 5] [--stages gs,fd] [--reps 5] [--scale 3]

For every level (finest first) prints the device milliseconds of one
application of each stage (mgiga_time_stage: CUDA events on the handle's
stream, after one warm-up application), plus the algorithmic flops and bytes
of the band product, the fast diagonalisation and a Gauss-Seidel sweep.  Also
the program the ncu captures of single stages run: with --stages gs --levels L
the only kernels launched after set-up are one warm-up and `reps` sweeps of
level L.
"""
import argparse
import json

from . import workloads as W


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--degree", type=int, default=6)
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "tf32", "bf16"])
    ap.add_argument("--smoother", default="hybrid", choices=["hybrid", "scms", "gs"])
    ap.add_argument("--scale", type=int, default=3)
    ap.add_argument("--levels", default="all", help="comma-separated level indices (negative: from the finest)")
    ap.add_argument("--stages", default="band,residual,fd,pieces,gs,restrict,prolong,coarse,vcycle")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--gs-cluster", type=int, default=0, help="0 automatic, or 2/4/8/16 (see mgiga_options)")
    args = ap.parse_args(argv)

    from . import mgiga  # loads libmgiga.so (CUDA)

    prob, opts = W.sipg_3x3(args.degree, scale=args.scale, smoother=args.smoother)
    s = mgiga.Solver(prob, levels=0, smoother=args.smoother, tau=opts["tau"], delta=opts["delta"],
                     precision=args.precision, gs_cluster=args.gs_cluster)
    nl = s.levels
    levels = list(range(nl - 1, -1, -1)) if args.levels == "all" else [int(x) % nl for x in args.levels.split(",")]
    print(f"p={args.degree} {args.precision} levels={nl} ndof={s.ndof()}", flush=True)
    for lvl in levels:
        row = {"level": lvl, "ndof": s.ndof(lvl)}
        for st in args.stages.split(","):
            try:
                row[st] = round(s.time_stage(st, lvl, reps=args.reps), 4)
            except mgiga.MgigaError:
                continue  # stage absent on this level (no smoother on level 0, no coarse solve above it)
            if st in ("band", "residual", "fd", "gs"):
                fl, by = s.stage_work(st, lvl)
                row[st + "_gflop"] = round(fl / 1e9, 4)
                row[st + "_mbytes"] = round(by / 1e6, 2)
        print(json.dumps(row), flush=True)
    s.close()


if __name__ == "__main__":
    main()
