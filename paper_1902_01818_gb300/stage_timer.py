"""Per-level stage times of the V-cycle on the SIPG 3x3 benchmark layout (or the 3D cube).

    python -m paper_1902_01818_gb300.stage_timer --degree 6 --precision fp32 \
        [--levels 5] [--stages gs,fd] [--reps 5] [--scale 3] [--workload cube-sipg] [--matrix-free]

The first line gives the wall time of the handle's set-up (MGIGA_VERBOSE=1
prints its phases on stderr).

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
import time

from . import workloads as W


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="sipg3x3", choices=["sipg3x3", "cube-conforming", "cube-sipg"],
                    help="sipg3x3: [0,3]^2 as 3x3 SIPG patches; cube-*: [0,1]^3 as 2x2x2 patches, 48 intervals")
    ap.add_argument("--degree", type=int, default=6)
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "tf32", "bf16"])
    ap.add_argument("--smoother", default="hybrid", choices=["hybrid", "scms", "gs"])
    ap.add_argument("--scale", type=int, default=3)
    ap.add_argument("--levels", default="all", help="comma-separated level indices (negative: from the finest)")
    ap.add_argument("--stages", default="band,residual,fd,pieces,gs,restrict,prolong,coarse,vcycle")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--gs-cluster", type=int, default=0, help="0 automatic, or 2/4/8/16 (see mgiga_options)")
    ap.add_argument("--matrix-free", action="store_true",
                    help="the finest level's cycle residual by sum factorisation (mgiga_options.matrix_free)")
    args = ap.parse_args(argv)

    from . import mgiga  # loads libmgiga.so (CUDA)

    if args.workload == "sipg3x3":
        prob, opts = W.sipg_3x3(args.degree, scale=args.scale, smoother=args.smoother)
    else:
        prob, opts = W.cube_2x2x2(args.degree, args.workload.split("-")[1])
    t0 = time.perf_counter()
    s = mgiga.Solver(prob, levels=0, smoother=args.smoother, tau=opts["tau"], delta=opts["delta"],
                     precision=args.precision, gs_cluster=args.gs_cluster, matrix_free=args.matrix_free)
    setup = time.perf_counter() - t0
    nl = s.levels
    levels = list(range(nl - 1, -1, -1)) if args.levels == "all" else [int(x) % nl for x in args.levels.split(",")]
    print(f"{args.workload} p={args.degree} {args.precision} levels={nl} ndof={s.ndof()} setup_s={setup:.2f}",
          flush=True)
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
