"""Benchmark: DoF/s of V-cycle-preconditioned CG solves to 1e-8 relative residual.

Workload (default): [0,3]^2 as 3x3 SIPG-coupled bilinear patches with jittered
interior vertices, 192 / 288 intervals per direction (alternating, so the
interface knots do not match), degrees p = 2..6, penalty 5 (p+1)^2 / h, hybrid
smoother (forward Gauss-Seidel + subspace-corrected mass smoother, tau .25,
delta .1), PCG to ||f - A u|| / ||f|| <= 1e-8; mixed precision by default (TF32 tensor-core
contractions on the large levels, FP32 smoothers, FP64 CG and coarse solve).  One step solves all five
degrees once (0.52-0.54M unknowns each), the five independent solves concurrently
(a CUDA stream and a host thread each; --sequential: one after another); value =
unknowns solved / second over the whole job.  Inputs are resident in HBM before the timed region; every
solve starts from u = 0.  The working set (five band matrices, 106 MB-730 MB
each) exceeds L2, so no explicit flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun) runs independent replicas of the workload on every rank
(the solve has no data exchange across problems): weak scaling.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DoF/s to 1e-8 rel. residual (V-cycle-preconditioned CG, SIPG 3x3 patches, p=2..6)"
METRIC_OF = {"sipg3x3": METRIC,
             "cube-conforming": "DoF/s to 1e-8 rel. residual (V-cycle-preconditioned CG, conforming 2x2x2 cube patches)",
             "cube-sipg": "DoF/s to 1e-8 rel. residual (V-cycle-preconditioned CG, SIPG 2x2x2 cube patches)"}
# peaks: derived from unit counts and the maximum SM clock (2.07 GHz, 152 SMs)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12    # 2 DFMA/clk/SM
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # 128 FFMA/clk/SM


def hbm_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "of measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "of fallback"


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one application of a stage on the
# finest level, per degree, from one ncu capture of the current kernels on a GB300 (profiles/
# traffic_sipg3x3_finest_level.md gives the command and the per-kernel figures).  Used only for the
# default configuration (scale 3, hybrid, TF32 contractions, 8-CTA GS clusters; the band, residual
# and GS kernels are the same in the FP32 mode); None elsewhere or when a stage's kernels change.
DRAM_TRAFFIC = {
    ("band", 2): 1.093e+08,
    ("residual", 2): 6.325e+07,
    ("fd", 2): 2.71e+07,
    ("gs", 2): 8.2e+07,
    ("band", 3): 2.139e+08,
    ("residual", 3): 1.153e+08,
    ("fd", 3): 2.75e+07,
    ("gs", 3): 1.351e+08,
    ("band", 4): 3.538e+08,
    ("residual", 4): 1.851e+08,
    ("fd", 4): 2.77e+07,
    ("gs", 4): 2.096e+08,
    ("band", 5): 5.304e+08,
    ("residual", 5): 2.734e+08,
    ("fd", 5): 2.78e+07,
    ("gs", 5): 3.015e+08,
    ("band", 6): 7.443e+08,
    ("residual", 6): 3.804e+08,
    ("fd", 6): 2.8e+07,
    ("gs", 6): 4.305e+08,
}


def dram_traffic(stage, degrees, args, f32):
    if not (args.workload == "sipg3x3" and args.scale == 3 and args.smoother == "hybrid"
            and args.precision in ("fp32", "tf32")
            and not args.sequential):
        return None
    if stage == "fd" and args.precision != "tf32":  # the table's contractions are the TF32 ones
        return None
    vals = [DRAM_TRAFFIC.get((stage, p)) for p in degrees]
    if any(v is None for v in vals):
        return None
    return sum(vals) / len(vals)


def bf16_peak_tflops():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops_sustained"]), "of measured (sustained)"
    except (OSError, KeyError, ValueError):
        return 1700.0, "of fallback (sustained)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sipg3x3", choices=list(WORKLOADS),
                    help="sipg3x3: [0,3]^2 as 3x3 SIPG patches (the headline); cube-*: [0,1]^3 as "
                         "2x2x2 patches, 48 intervals, conforming or SIPG")
    ap.add_argument("--degrees", default=None, help="comma list (default: the workload's)")
    ap.add_argument("--scale", type=int, default=3, help="interval multiplier of 64/96 (3: 192/288)")
    ap.add_argument("--smoother", default="hybrid", choices=["scms", "hybrid"])
    ap.add_argument("--precision", default="tf32", choices=["fp32", "tf32", "bf16", "fp64"],
                    help="smoother arithmetic of the timed path (CG is FP64 either way)")
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip the plain-FP64 comparison solves")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lshape", type=int, default=1,
                    help="1: also solve the paper's non-matching L-shape (one degree per patch; lshape key)")
    ap.add_argument("--matrix-free", type=int, default=1,
                    help="1: also time the matrix-free finest-level residual and a solve with it (matrix_free key)")
    ap.add_argument("--cube", type=int, default=1,
                    help="add the 3D cube configurations (2x2x2 patches, 48 intervals, conforming and SIPG; mixed "
                         "against plain FP64) as the line's 'cube' key: 1 p = 3 (keeps the default run short), "
                         "2 p = 3..5, 0 none")
    ap.add_argument("--sequential", action="store_true",
                    help="solve the degrees one after another (default: concurrently, a stream each)")
    ap.add_argument("--priority", default="degree", choices=["degree", "none"],
                    help="concurrent solves: higher stream priority for higher degrees (the longest solves)")
    ap.add_argument("--autotune", type=int, default=1,
                    help="1: the mixed handles pick their contraction engines and residual row blocking by "
                         "timing at set-up (once per size bucket)")
    ap.add_argument("--mu", type=int, default=1, help="1: V-cycle, 2: W-cycle (Sec. 4)")
    ap.add_argument("--nu", type=int, default=1, help="smoothing steps per level")
    ap.add_argument("--outer", default="pcg", choices=["pcg", "direct"],
                    help="pcg: the cycle preconditions CG; direct: the cycle is the solver")
    ap.add_argument("--gs-cluster", default="8",
                    help="Gauss-Seidel cluster size per degree (one value, or one per degree); "
                         "ignored with --sequential, which lets the library choose")
    return ap.parse_args()


_T0 = time.perf_counter()


def progress(msg):
    """A timestamped progress line on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.perf_counter() - _T0:7.1f} s] {msg}", file=sys.stderr, flush=True)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, world, device="cpu"):
    """The largest value of x over all ranks (the timed region ends with the slowest rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, unknowns_per_rank, steps, ms):
    """Whole-job DoF/s: every rank solves its own replica of the workload (weak scaling)."""
    return world * unknowns_per_rank * steps / (ms / 1e3)


# workload -> (default degrees, oracle sample expression for the CPU legs, description)
WORKLOADS = {
    "sipg3x3": ("2,3,4,5,6", "W.sipg_3x3(2, scale=1, smoother={smoother!r})",
                "sipg-3x3-[0,3]^2-jitter0.1-{a}/{b}-intervals"),
    "cube-conforming": ("3,4,5", "W.cube_2x2x2(3, 'conforming', n=12)",
                        "conforming-2x2x2-[0,1]^3-jitter0.05-48-intervals"),
    "cube-sipg": ("3,4,5", "W.cube_2x2x2(3, 'sipg', n=12)", "sipg-2x2x2-[0,1]^3-jitter0.05-48-intervals"),
}


def workload(p, args):
    from paper_1902_01818_gb300 import workloads as W
    if args.workload == "sipg3x3":
        return W.sipg_3x3(p, scale=args.scale, smoother=args.smoother)
    return W.cube_2x2x2(p, args.workload.split("-")[1])


def workload_name(args):
    return WORKLOADS[args.workload][2].format(a=64 * args.scale, b=96 * args.scale)


# ---------------------------------------------------------------------------
# oracle (CPU) legs
# ---------------------------------------------------------------------------
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
from oracle import discretize, mg
from paper_1902_01818_gb300 import workloads as W
prob, opts = {expr}
M = mg.Multigrid(prob, smoother=opts["smoother"], tau=opts["tau"], delta=opts["delta"])
f = discretize.assemble_load(prob, prob["knots"], M.h["num"][-1], W.source_sinprod)
out = []
for i in range({reps}):
    t0 = time.perf_counter()
    u, it, hist = M.solve_pcg(f, tol=1e-8)
    out.append((time.perf_counter() - t0, it, hist[-1]))
print(json.dumps(dict(ndof=M.ndof, runs=out)))
"""


def run_oracle(expr, reps):
    """Time the oracle's PCG solve of the problem `expr` builds in a fresh single-threaded process."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    code = ORACLE_SNIPPET.format(root=ROOT, expr=expr, reps=reps)
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if res.returncode != 0:
        raise RuntimeError("oracle run failed: " + res.stderr[-2000:])
    return json.loads(res.stdout.strip().splitlines()[-1])


def oracle_sample(args):
    """The bounded sample of the workload the CPU legs time: the 2D layout at 64/96 intervals,
    p = 2 (60k unknowns); the cube at 12 intervals, p = 3 (22k unknowns)."""
    return WORKLOADS[args.workload][1].format(smoother=args.smoother)


class _single_threaded_children:
    """One BLAS / OpenMP thread in the processes spawned inside the block: a spawned child imports
    numpy before any initializer runs, so the limit must be in the environment it inherits.  The
    variables are put back afterwards, so this process's own OpenMP runtime (the library's host
    set-up) keeps every core."""

    KEYS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")

    def __enter__(self):
        self.saved = {k: os.environ.get(k) for k in self.KEYS}
        for k in self.KEYS:
            os.environ[k] = "1"

    def __exit__(self, *exc):
        for k, v in self.saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def _oracle_worker_init():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"


def oracle_job(kind, p, scale, smoother):
    """One oracle job in a spawned single-threaded worker (the oracle is test infrastructure; this
    CPU leg is the one place the benchmark runs it).  kind 'time': a timed PCG solve (set-up
    excluded); kind 'solution': the oracle's load vector and its PCG solution to 1e-8."""
    from oracle import discretize, mg
    from paper_1902_01818_gb300 import workloads as W
    if isinstance(scale, str):  # a cube sample: scale = coupling, 12 intervals
        prob, opts = W.cube_2x2x2(p, scale, n=12)
    else:
        prob, opts = W.sipg_3x3(p, scale=scale, smoother=smoother)
    t0 = time.perf_counter()
    M = mg.Multigrid(prob, smoother=opts["smoother"], tau=opts["tau"], delta=opts["delta"])
    f = discretize.assemble_load(prob, prob["knots"], M.h["num"][-1], W.source_sinprod)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    u, it, hist = M.solve_pcg(f, tol=1e-8)
    t = time.perf_counter() - t0
    out = {"ndof": int(M.ndof), "seconds": t, "setup_s": t_setup, "iterations": int(it), "relres": float(hist[-1])}
    if kind == "solution":
        out.update(f=f, u=u)
    return out


class OracleLegs:
    """CPU legs of the benchmark, started before the process touches the GPU (spawned workers):
      * cpu_baseline: one timed oracle PCG solve of the benchmark's own layout (192/288 intervals)
        at p = 2, one core;
      * the oracle's FP64 solutions of the 64/96-interval sample, p = 2..6, against which both GPU
        arms report their error;
      * afterwards, all host cores: one oracle solve of the 64/96, p = 2 sample per core at once."""

    def __init__(self, args, degrees):
        import concurrent.futures as cf
        import multiprocessing as mp
        self.args = args
        self.ncpu = os.cpu_count() or 1
        # workers are spawned as the jobs are submitted (all of them here, inside the block)
        with _single_threaded_children():
            self.pool = cf.ProcessPoolExecutor(max_workers=max(2, min(self.ncpu, len(degrees) + 7)),
                                               mp_context=mp.get_context("spawn"), initializer=_oracle_worker_init)
            # the slowest first: the cube samples (3D, p up to 5), the 192/288 baseline, the 2D samples
            self.cube = {}
            if args.cube:
                for c in ("conforming", "sipg"):
                    for p in ((5, 4, 3) if args.cube >= 2 else (3,)):
                        self.cube[(c, p)] = self.pool.submit(oracle_job, "solution", p, c, "hybrid")
            self.base = self.pool.submit(oracle_job, "time", 2, args.scale, args.smoother)
            self.sol = {p: self.pool.submit(oracle_job, "solution", p, 1, args.smoother) for p in degrees}

    def baseline(self):
        r = self.base.result()
        return {"value": r["ndof"] / r["seconds"], "unit": "DoF/s", "cores": 1, "kind": "oracle",
                "sample": f"one oracle PCG solve of the benchmark layout at {64 * self.args.scale}/"
                          f"{96 * self.args.scale} intervals, p = 2 ({r['ndof']} unknowns, {r['iterations']} "
                          f"iterations to 1e-8, {r['seconds']:.1f} s; set-up {r['setup_s']:.0f} s excluded; "
                          f"numpy/scipy, 1 thread)", "cpu_model": cpu_model(), "nproc": self.ncpu}

    def solutions(self):
        return {p: fu.result() for p, fu in self.sol.items()}

    def cube_solutions(self):
        return {k: fu.result() for k, fu in self.cube.items()}

    def all_cores(self):
        """One 64/96, p = 2 oracle solve per host core, all at once (after the GPU timing)."""
        import concurrent.futures as cf
        import multiprocessing as mp
        self.pool.shutdown(wait=True)
        n = self.ncpu
        with _single_threaded_children(), cf.ProcessPoolExecutor(
                max_workers=n, mp_context=mp.get_context("spawn"), initializer=_oracle_worker_init) as ex:
            t0 = time.perf_counter()
            rs = list(ex.map(oracle_job, ["time"] * n, [2] * n, [1] * n, [self.args.smoother] * n))
            wall = time.perf_counter() - t0
        slowest = max(r["seconds"] for r in rs)
        return {"value": sum(r["ndof"] for r in rs) / slowest, "unit": "DoF/s", "cores": n, "kind": "oracle",
                "cpu_model": cpu_model(), "nproc": n,
                "sample": f"{n} independent oracle PCG solves of the 64/96-interval layout, p = 2 ({rs[0]['ndof']} "
                          f"unknowns each), one per core at once, 1 thread each; value = unknowns / the slowest "
                          f"solve ({slowest:.1f} s; set-ups excluded, wall {wall:.0f} s)"}


def cpu_model():
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith(("model name", "cpu model")):
                    return ln.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline(args):
    expr = oracle_sample(args)
    r = run_oracle(expr, 1)
    t, it, rel = r["runs"][0]
    return {"value": r["ndof"] / t, "unit": "DoF/s", "cores": 1, "kind": "oracle",
            "sample": f"one PCG solve of {expr} ({r['ndof']} unknowns, {it} iterations, {t:.1f} s, "
                      f"setup excluded; numpy/scipy, 1 thread)"}


def reference_arm(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    # each step: one oracle PCG solve of the bounded sample
    expr = oracle_sample(args)
    r = run_oracle(expr, args.warmup + args.steps)
    runs = r["runs"][args.warmup:]
    times = [x[0] for x in runs]
    total = sum(times)
    value = r["ndof"] * len(runs) / total
    line = {"impl": "reference", "metric": METRIC_OF[args.workload], "value": value, "unit": "DoF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(runs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{expr}: bounded sample of the {workload_name(args)} workload",
                       "smoother": args.smoother, "l2": "inputs larger than L2 n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "DoF/s", "cores": 1, "kind": "oracle",
                             "sample": f"{len(runs)} oracle PCG solves of {expr}, {r['ndof']} unknowns, 1 thread"},
            "e2e": {"value": value, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": smax, "reasons": ["unavailable"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# 3D cube configurations (a key of the default line)
# ---------------------------------------------------------------------------
def cube_leg(args, mgiga, W, torch, oracle_sols, reps=3):
    """For p = 3..5, conforming and SIPG, 48 intervals: the mixed (TF32 contractions, FP32 smoothers, FP64
    CG) and the plain FP64 solves to 1e-8 one after another, each timed with CUDA events over `reps` solves
    after one warm-up (inputs resident); errors of both against the FP64 oracle on the 12-interval sample."""
    out, tot = {}, {"tf32": [0, 0.0], "fp64": [0, 0.0]}
    st = torch.cuda.current_stream()
    for c in ("conforming", "sipg"):
        for p in ((3, 4, 5) if args.cube >= 2 else (3,)):
            prob, o = W.cube_2x2x2(p, c)
            rec = {}
            for pr in ("tf32", "fp64"):
                progress(f"cube {c} p = {p} {pr}")
                t0 = time.perf_counter()
                s = mgiga.Solver(prob, levels=0, smoother=o["smoother"], tau=o["tau"], delta=o["delta"], precision=pr,
                                 stream=st.cuda_stream)
                setup = time.perf_counter() - t0
                f = torch.from_numpy(s.load_sinprod()).cuda()
                u = torch.zeros_like(f)
                times = []
                for i in range(reps + 1):
                    u.zero_()
                    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    ea.record(st)
                    it, rel, _ = s.solve_d(f, u, tol=1e-8)
                    eb.record(st)
                    torch.cuda.synchronize()
                    if i:
                        times.append(ea.elapsed_time(eb))
                fh = f.cpu().numpy()
                r_true = fh - s.apply("matvec", -1, u.cpu().numpy())
                n = s.ndof()
                s.close()
                med = float(np.median(times))
                tot[pr][0] += n
                tot[pr][1] += med
                rec[pr] = {"value": n / (med / 1e3), "solve_ms_p50": round(med, 3),
                           "solve_ms_p99": round(float(np.percentile(times, 99)), 3), "iterations": it,
                           "true_relres": float(np.linalg.norm(r_true) / np.linalg.norm(fh)), "setup_s": round(setup, 1)}
            rec["unknowns"] = n
            ref = oracle_sols.get((c, p)) if oracle_sols else None
            if ref is not None:  # the 12-interval sample, the oracle's load vector
                ps, os_ = W.cube_2x2x2(p, c, n=12)
                for pr in ("tf32", "fp64"):
                    s = mgiga.Solver(ps, levels=0, smoother=os_["smoother"], tau=os_["tau"], delta=os_["delta"],
                                     precision=pr)
                    uu, it, rel, _ = s.solve(ref["f"], tol=1e-8)
                    s.close()
                    rec[pr]["rel_error_vs_oracle"] = float(np.linalg.norm(uu - ref["u"]) / np.linalg.norm(ref["u"]))
                rec["oracle_sample"] = {"intervals": 12, "unknowns": ref["ndof"], "oracle_iterations": ref["iterations"]}
            out[f"{c}_p{p}"] = rec
    return {"workload": "[0,1]^3 as 2x2x2 trilinear patches, jitter 0.05, 48 intervals, hybrid smoother, PCG to 1e-8",
            "solves": f"one at a time, median of {reps} after a warm-up, inputs resident",
            "mixed": {"value": tot["tf32"][0] / (tot["tf32"][1] / 1e3), "unit": "DoF/s",
                      "precision": "tf32 contractions (FP32 SIMT on these 49-51 interiors), fp32 smoothers, fp64 CG"},
            "plain_fp64": {"value": tot["fp64"][0] / (tot["fp64"][1] / 1e3), "unit": "DoF/s"},
            "per_config": out}


def matfree_leg(args, mgiga, W, torch, degrees, solvers, reps=3):
    """The finest level's cycle residual by sum factorisation at the Gauss points (matrix_free) against
    the stored FP32 band, per degree on the benchmark layout: device time of one application (CUDA
    events, mgiga_time_stage), its arithmetic against the FP32 peak (the kernel is bound by its FMAs,
    not by HBM), the FP32 band bytes it makes unnecessary, and a full mixed solve to 1e-8 with it."""
    out = {}
    st = torch.cuda.current_stream()
    for p, s_band in zip(degrees, solvers):
        prob, opts = workload(p, args)
        s = mgiga.Solver(prob, levels=opts["levels"], smoother=opts["smoother"], tau=opts["tau"], delta=opts["delta"],
                         precision=args.precision, matrix_free=True, stream=st.cuda_stream)
        t_mf = s.time_stage("residual", -1, reps=10)
        fl, by = s.stage_work("residual", -1)
        t_band = s_band.time_stage("residual", -1, reps=10)
        _, by_band = s_band.stage_work("residual", -1)
        n = s.ndof()
        f = torch.from_numpy(s.load_sinprod()).cuda()
        u = torch.zeros_like(f)
        times = []
        for i in range(reps + 1):
            u.zero_()
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ea.record(st)
            it, rel, _ = s.solve_d(f, u, tol=1e-8)
            eb.record(st)
            torch.cuda.synchronize()
            if i:
                times.append(ea.elapsed_time(eb))
        fh = f.cpu().numpy()
        r_true = fh - s.apply("matvec", -1, u.cpu().numpy())
        s.close()
        med = float(np.median(times))
        out[str(p)] = {"residual_ms": round(t_mf, 4), "stored_band_residual_ms": round(t_band, 4),
                       "achieved_tflops": round(fl / (t_mf / 1e3) / 1e12, 3), "peak_tflops": FP32_PEAK_TFLOPS,
                       "frac": round(fl / (t_mf / 1e3) / 1e12 / FP32_PEAK_TFLOPS, 4),
                       "band_bytes_saved": int(by_band - 24 * n),
                       "solve": {"value": n / (med / 1e3), "unit": "DoF/s", "solve_ms_p50": round(med, 3),
                                 "iterations": it,
                                 "true_relres": float(np.linalg.norm(r_true) / np.linalg.norm(fh))}}
    return {"what": "finest-level cycle residual matrix-free (sum factorisation at the Gauss points, geometry "
                    "from the control points, FP32) instead of the stored FP32 band; bound: FP32 FMAs "
                    "(peak derived: 152 SMs x 128 FFMA/clk x 2 x 2.07 GHz)",
            "per_degree": out}


# Table SCMS2 (b) of the paper: PCG iterations, V-cycle with the subspace-corrected mass smoother,
# non-conforming L-shape (S_{p,h} / S_{p+1,2h} / S_{p,2h}), refinement L = 4..8 (rows), p = 2..6
PAPER_SCMS2_PCG = {4: [17, 16, 15, 14, 13], 5: [19, 19, 18, 17, 17], 6: [21, 20, 20, 19, 19],
                   7: [22, 22, 21, 21, 21], 8: [23, 23, 22, 22, 22]}


def lshape_leg(args, mgiga, W, torch, refinements=(6, 8), degrees=(2, 3, 4, 5, 6)):
    """The paper's non-matching L-shape (Sec. 5, Table SCMS2): three patches with S_{p,h},
    S_{p+1,2h}, S_{p,2h} (one spline degree per patch), SIPG, the subspace-corrected mass smoother
    with the table's damping .9 and scaling .12, PCG to 1e-8; iterations of the mixed and the plain
    FP64 path beside the paper's count (its hardware and coarsest grid differ: context only)."""
    out = {}
    st = torch.cuda.current_stream()
    for r in refinements:
        for p in degrees:
            prob, o = W.lshape(p, r)
            rec = {"degrees": prob["degrees"], "paper_pcg_iterations": PAPER_SCMS2_PCG.get(r, [None] * 5)[p - 2]}
            for pr in ("tf32", "fp64"):
                s = mgiga.Solver(prob, levels=o["levels"], smoother=o["smoother"], tau=o["tau"], delta=o["delta"],
                                 precision=pr, stream=st.cuda_stream)
                f = torch.from_numpy(s.load_sinprod()).cuda()
                u = torch.zeros_like(f)
                s.solve_d(f, u, tol=1e-8)
                u.zero_()
                ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ea.record(st)
                it, rel, _ = s.solve_d(f, u, tol=1e-8)
                eb.record(st)
                torch.cuda.synchronize()
                fh = f.cpu().numpy()
                r_true = fh - s.apply("matvec", -1, u.cpu().numpy())
                rec[pr] = {"iterations": it, "solve_ms": round(ea.elapsed_time(eb), 3),
                           "true_relres": float(np.linalg.norm(r_true) / np.linalg.norm(fh))}
                rec["unknowns"], rec["levels"] = s.ndof(), s.levels
                s.close()
            out[f"r{r}_p{p}"] = rec
    return {"workload": "L-shape [0,2]^2 without (1,2]^2, 3 patches, S_{p,h} / S_{p+1,2h} / S_{p,2h} (2^r, "
                        "2^(r-1), 2^(r-1) intervals), SIPG C = 5 (p+2)^2, SCMS tau .9 delta .12, PCG to 1e-8",
            "per_config": out}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    world, rank, local = dist_env()
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    degrees = [int(x) for x in (args.degrees or WORKLOADS[args.workload][0]).split(",")]
    # the CPU legs start first (spawned processes, before this process uses the GPU)
    legs, cpu = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if args.workload == "sipg3x3":
            legs = OracleLegs(args, degrees)
        else:
            cpu = cpu_baseline(args)

    import __graft_entry__
    __graft_entry__.build()
    from paper_1902_01818_gb300 import mgiga, workloads as W

    stream = torch.cuda.Stream()  # the timing events live on this stream
    torch.cuda.set_stream(stream)
    # one stream per degree (and precision): the independent solves of a step run concurrently,
    # one host thread each, unless --sequential
    streams = {}
    solvers, rhs_d, u_d, rhs_h, u_h, ndofs, dims = [], [], [], [], [], [], []
    t_setup = time.perf_counter()
    precisions = [args.precision] + ([] if args.no_fp64_compare or args.precision == "fp64" else ["fp64"])
    handles = {pr: [] for pr in precisions}
    cs = [int(x) for x in args.gs_cluster.split(",")]
    cs = cs * len(degrees) if len(cs) == 1 else cs
    if len(cs) != len(degrees):
        raise SystemExit("--gs-cluster: one value, or one per degree")
    # the solve of the highest degree takes the most V-cycles and the longest ones: its stream gets
    # the highest priority, so its blocks are scheduled first and the others fill the gaps
    by_work = sorted(degrees, reverse=True)
    for p, c in zip(degrees, cs):
        prob, opts = workload(p, args)
        dims.append(prob["dim"])
        prio = -max(0, 3 - by_work.index(p)) if args.priority == "degree" and not args.sequential else 0
        for pr in precisions:
            streams[(p, pr)] = torch.cuda.Stream(priority=prio)
            # concurrent solves: 8-CTA clusters on large levels pack better into the processing clusters
            handles[pr].append(mgiga.Solver(prob, levels=opts["levels"], smoother=opts["smoother"],
                                            tau=opts["tau"], delta=opts["delta"], precision=pr,
                                            mu=args.mu, nu=args.nu, outer=args.outer,
                                            autotune=bool(args.autotune) and pr != "fp64",
                                            stream=streams[(p, pr)].cuda_stream,
                                            gs_cluster=0 if args.sequential else c))
        s = handles[args.precision][-1]
        f = s.load_sinprod()
        ndofs.append(len(f))
        rhs_d.append(torch.from_numpy(f).cuda())
        u_d.append(torch.zeros_like(rhs_d[-1]))
        rhs_h.append(torch.from_numpy(f).pin_memory())
        u_h.append(torch.zeros(len(f), dtype=torch.float64).pin_memory())
    solvers = handles[args.precision]
    total_dof = sum(ndofs)
    dev_bytes = sum(s.device_bytes() for s in solvers)
    t_setup = time.perf_counter() - t_setup
    print(f"set-up (assembly, hierarchy, smoother data, upload) of {len(degrees) * len(precisions)} handles: "
          f"{t_setup:.1f} s", file=sys.stderr, flush=True)

    # concurrency is safe when no sweep needs the grid-wide (cooperative) kernel: the base colours
    # cover every DoF on every level (true for this layout; checked, not assumed)
    def coop_free(s, p, d):
        if args.smoother == "scms":
            return True  # no Gauss-Seidel sweep at all
        base = 2 * (p + 1) ** d
        return all(int(s.colours(l).max()) < base for l in range(1, s.levels))

    concurrent = not args.sequential and all(coop_free(s, p, d) for s, p, d in zip(solvers, degrees, dims))

    def solve_one(i, s, host_path, out, ev=None):
        st_ = streams[(degrees[i], s.precision)]
        with torch.cuda.stream(st_):
            if ev is not None:
                ev[i][0].record(st_)
            if host_path:
                u_h[i].zero_()
                u, it, rel, st = s.solve(rhs_h[i].numpy(), u0=u_h[i].numpy(), tol=1e-8)
                u_h[i].copy_(torch.from_numpy(u))
            else:
                u_d[i].zero_()
                it, rel, st = s.solve_d(rhs_d[i], u_d[i], tol=1e-8)
            if ev is not None:
                ev[i][1].record(st_)
        out[i] = (it, rel)

    def step(host_path=False, which=None, ev=None):
        which = which if which is not None else solvers
        out = [None] * len(which)
        # worker streams start after everything enqueued on the timing stream so far
        start = torch.cuda.Event()
        start.record(stream)
        for i, s in enumerate(which):
            streams[(degrees[i], s.precision)].wait_event(start)
        if concurrent and all(s.precision != "fp64" for s in which):
            ths = [threading.Thread(target=solve_one, args=(i, s, host_path, out, ev)) for i, s in enumerate(which)]
            for t in ths:
                t.start()
            for t in ths:
                t.join()
        else:
            for i, s in enumerate(which):
                solve_one(i, s, host_path, out, ev)
        for i, s in enumerate(which):  # the timing stream continues after every solve
            done = torch.cuda.Event()
            done.record(streams[(degrees[i], s.precision)])
            stream.wait_event(done)
        return out

    progress("warm-up")
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    launches0 = sum(s.kernel_launches() for s in solvers)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    per_step = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        barrier()
        ev0.record()
        for _ in range(args.steps):
            e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e_a.record()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in solvers]
            info = step(ev=ev)
            e_b.record()
            per_step.append((e_a, e_b, info, ev))
        ev1.record()
        torch.cuda.synchronize()
        barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, device="cuda")
    progress(f"timed steps done: {ms / args.steps:.2f} ms per step")
    launches = sum(s.kernel_launches() for s in solvers) - launches0
    step_ms = [a.elapsed_time(b) for a, b, _, _ in per_step]
    # per solve (call to result ready on its stream), per degree, over the timed steps
    solve_ms = {p: [ev[i][0].elapsed_time(ev[i][1]) for _, _, _, ev in per_step] for i, p in enumerate(degrees)}
    iters = [x[0] for x in per_step[-1][2]]
    rels = [x[1] for x in per_step[-1][2]]
    value = job_value(world, total_dof, args.steps, ms)

    # end to end: host buffers, H2D and D2H inside the timed region (slowest rank)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps // 2)):
        step(host_path=True)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(1e3 * (time.perf_counter() - t0) / max(1, args.steps // 2), world, device="cuda")
    e2e = {"value": job_value(world, total_dof, 1, e2e_ms), "unit": "DoF/s",
           "h2d_bytes_per_step": int(2 * 8 * total_dof), "d2h_bytes_per_step": int(8 * total_dof)}

    progress("end to end done")
    # plain FP64 comparison: same workload, FP64 smoothers
    plain = None
    if "fp64" in handles and args.precision != "fp64":
        step(which=handles["fp64"])
        torch.cuda.synchronize()
        e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev64 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in degrees]
        e_a.record()
        info64 = step(which=handles["fp64"], ev=ev64)
        e_b.record()
        torch.cuda.synchronize()
        ms64 = e_a.elapsed_time(e_b)
        plain = {"value": total_dof / (ms64 / 1e3), "unit": "DoF/s", "ms_per_step": ms64,
                 "iterations": [x[0] for x in info64], "final_relres": [x[1] for x in info64],
                 "solve_ms": {str(p): round(ev64[i][0].elapsed_time(ev64[i][1]), 3) for i, p in enumerate(degrees)},
                 "solves": "sequential (the FP64 sweep is a grid-wide cooperative launch)"}
    progress("plain FP64 done")
    # the mixed path solved one degree after another, for comparison with the FP64 figure
    mixed_seq = None
    if concurrent:
        concurrent = False
        step()
        torch.cuda.synchronize()
        e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e_a.record()
        step()
        e_b.record()
        torch.cuda.synchronize()
        concurrent = True
        mixed_seq = {"value": total_dof / (e_a.elapsed_time(e_b) / 1e3), "unit": "DoF/s",
                     "ms_per_step": e_a.elapsed_time(e_b), "solves": "sequential"}

    # roofline per stage on the finest level of every degree (times summed over the degrees); the
    # stage with the largest share of a PCG iteration (count x time) is reported.  Per PCG iteration
    # on the finest level: one FP64 band product (CG), three residuals inside the cycle (FP32 band on
    # the mixed path), two fast diagonalisations and, with the hybrid smoother, two Gauss-Seidel sweeps.
    hbm, hbm_src = hbm_peak_gbs()
    f32 = args.precision != "fp64"
    hybrid = args.smoother == "hybrid"
    counts = ({"band": 1, "residual": 3, "fd": 2, "gs": 2 if hybrid else 0} if f32 else
              {"band": 4, "fd": 2, "gs": 2 if hybrid else 0})
    names = {"band": "band_apply (FP64 band product)",
             "residual": "band_residual_f32 + cross_apply (residual inside the cycle, FP32 band)",
             "fd": {"fp32": "gemm_tiled (fast diagonalisation, FP32)",
                    "tf32": ("gather_interior_f32 + gemm_umma_tf32 (fast diagonalisation, TF32 tensor cores)"
                             if args.workload == "sipg3x3" else
                             "gemm_tiled (fast diagonalisation, FP32: interiors below the tensor-core size)"),
                    "bf16": "gemm_umma (fast diagonalisation, BF16 tensor cores)"}.get(
                        args.precision, "gemm_tiled (fast diagonalisation, FP64)"),
             "gs": ("gs_fill_phase + gs_patch_staged (one Gauss-Seidel sweep, FP32)" if f32 else
                    "gs_sweep_coop (one Gauss-Seidel sweep, FP64)")}
    stages = {}
    for st, count in counts.items():
        if count == 0:
            continue
        t_ms = fl = by = 0.0
        for s in solvers:
            t_ms += s.time_stage(st, -1, reps=10)
            a_fl, a_by = s.stage_work(st, -1)
            fl += a_fl
            by += a_by
        if st in ("band", "fd") and not (st == "fd" and f32):
            rec = {"bound": "alu", "achieved": fl / (t_ms / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                   "unit": "TFLOP/s", "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 x 2.07 GHz"}
        elif st == "fd" and args.precision in ("tf32", "bf16") and args.workload == "sipg3x3":
            bf16, src = bf16_peak_tflops()
            ratio = 0.5 if args.precision == "tf32" else 1.0  # nominal dense TF32 / BF16 = 1.1 / 2.25
            rec = {"bound": "tensor", "achieved": fl / (t_ms / 1e3) / 1e12, "peak": bf16 * ratio,
                   "unit": "TFLOP/s", "peak_source": src + (" (bf16 x nominal tf32/bf16 ratio 0.5)"
                                                         if ratio != 1.0 else "")}
        elif st == "fd":
            rec = {"bound": "alu", "achieved": fl / (t_ms / 1e3) / 1e12, "peak": FP32_PEAK_TFLOPS,
                   "unit": "TFLOP/s", "peak_source": "derived: 152 SMs x 128 FFMA/clk x 2 x 2.07 GHz"}
        else:
            rec = {"bound": "hbm", "achieved": by / (t_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                   "peak_source": hbm_src}
        rec["frac"] = rec["achieved"] / rec["peak"]
        rec["ms_per_application"] = t_ms / len(solvers)
        rec["algorithmic_bytes_per_application"] = by / len(solvers)
        rec["share_weight_ms"] = count * t_ms
        rec["kernel"] = names[st]
        rec["traffic"] = dram_traffic(st, degrees, args, f32)
        stages[st] = rec
    progress("stage rooflines done")
    mf = None
    if args.matrix_free and args.precision != "fp64" and rank == 0:
        mf = matfree_leg(args, mgiga, W, torch, degrees, solvers)
        progress("matrix-free residual done")
    dom = max(stages, key=lambda k: stages[k]["share_weight_ms"])
    roof = dict(stages[dom])
    roof["stages"] = {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv) for kk, vv in v.items()}
                      for k, v in stages.items()}

    # error of both arms against the FP64 oracle, on the oracle-sized sample of the layout
    oracle_err = None
    if legs is not None:
        progress("waiting for the oracle's 2D solutions")
        sols = legs.solutions()
        progress("oracle's 2D solutions in")
        per = {}
        for p in degrees:
            ref = sols[p]
            prob, opts = W.sipg_3x3(p, scale=1, smoother=args.smoother)
            rec = {"unknowns": ref["ndof"], "oracle_iterations": ref["iterations"]}
            for pr in precisions:
                s = mgiga.Solver(prob, levels=opts["levels"], smoother=opts["smoother"], tau=opts["tau"],
                                 delta=opts["delta"], precision=pr)
                u, it, rel, _ = s.solve(ref["f"], tol=1e-8)
                r_true = ref["f"] - s.apply("matvec", -1, u)
                s.close()
                rec[pr] = {"rel_error_vs_oracle": float(np.linalg.norm(u - ref["u"]) / np.linalg.norm(ref["u"])),
                           "iterations": it, "true_relres": float(np.linalg.norm(r_true) / np.linalg.norm(ref["f"]))}
            per[str(p)] = rec
        oracle_err = {"sample": f"the same layout at 64/96 intervals (the oracle's size), p = {degrees}, the "
                                f"oracle's load vector; ||u - u_oracle|| / ||u_oracle||, both stopped at 1e-8",
                      "per_degree": per}
        cpu = legs.baseline()

    line = {"metric": METRIC_OF[args.workload], "value": value, "unit": "DoF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {"fp32": "f32+f64", "tf32": "tf32+f32+f64", "bf16": "bf16+f32+f64"}.get(args.precision, "f64"),
            "data": "synthetic",
            "config": {"workload": workload_name(args),
                       "degrees": degrees, "unknowns": ndofs, "smoother": args.smoother, "outer": args.outer,
                       "cycle": {"mu": args.mu, "nu": args.nu}, "autotune": bool(args.autotune),
                       "precision": {"fp32": "fp32 smoothers, fp64 CG/coarse",
                                     "tf32": "tf32 contractions on large levels, fp32 smoothers, fp64 CG/coarse",
                                     "bf16": "bf16 contractions on large levels, fp32 smoothers, fp64 CG/coarse"
                                     }.get(args.precision, "fp64"),
                       "tol": 1e-8, "iterations": iters, "final_relres": rels,
                       "step_ms_p50": float(np.percentile(step_ms, 50)),
                       "step_ms_p99": float(np.percentile(step_ms, 99)),
                       "solve_ms": {str(p): {"p50": round(float(np.percentile(v, 50)), 3),
                                             "p99": round(float(np.percentile(v, 99)), 3)}
                                    for p, v in solve_ms.items()},
                       "l2": f"inputs larger than L2 ({dev_bytes / 1e9:.1f} GB of device data per step)",
                       "parallelism": f"replicas x{world}", "setup_s": round(t_setup, 1),
                       "solves": ("concurrent: one CUDA stream and host thread per degree"
                                  + (", stream priority by degree" if args.priority == "degree" else "")
                                  if concurrent else "sequential"),
                       "gs_cluster": None if args.sequential else cs},
            "e2e": e2e, "gpu_launches": launches, "roofline": roof, "plain_fp64": plain,
            "mixed_sequential": mixed_seq, "oracle_error": oracle_err, "matrix_free": mf,
            "clocks": clk.summary()}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    for hs in handles.values():
        for s in hs:
            s.close()
    handles = {}
    if args.cube and args.workload == "sipg3x3" and rank == 0 and world == 1:
        progress("waiting for the oracle's cube solutions")
        csol = legs.cube_solutions() if legs is not None else None
        progress("cube configurations")
        line["cube"] = cube_leg(args, mgiga, W, torch, csol)
    if args.lshape and args.workload == "sipg3x3" and rank == 0 and world == 1:
        progress("L-shape, one degree per patch")
        line["lshape_nonmatching"] = lshape_leg(args, mgiga, W, torch)
    if legs is not None:
        progress("all-core oracle leg")
        line["cpu_all_cores"] = legs.all_cores()
    progress("done")
    if rank == 0:
        print(json.dumps(line), flush=True)
    for hs in handles.values():
        for s in hs:
            s.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
