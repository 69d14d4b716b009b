"""A request loop for Poisson solves: continuous batching over resident operators.

Requests (a problem, solver options, a right-hand side) arrive at any time and are
served by `workers` host threads; every operator gets its own handle, hence its own
CUDA stream, so solves of different requests overlap on the device.  Handles stay
resident in a cache keyed by the request's operator key: a request that reuses an
operator skips the set-up.  Admission is by an HBM budget: a new handle is assembled
with `hbm_budget` = what the budget leaves (the library refuses with MGIGA_ENOMEM
when its footprint would exceed it); on refusal idle handles are evicted (least
recently used first) and the set-up retried; when nothing is idle the worker waits
for a running solve to finish; a request larger than the whole budget is rejected.
One handle is used by one thread at a time.

    srv = Server(workers=4, hbm_budget=120 << 30)
    srv.start()
    fut = srv.submit(key, problem, options, rhs)   # rhs: array, or an int seed
    u, iterations, relres, latency_s = fut.result()
    srv.stop(); srv.stats()  # solves, solves/s, rejected, p50/p99 latency, set-ups,
                             # evictions, resident bytes, queue length (now / largest)

An int rhs is a seed: the worker draws i.i.d. N(0, 1) load coefficients of the
operator's size once the handle exists.  `python -m paper_1902_01818_gb300.serve`
serves the seeded serving stream with Poisson arrivals and prints the statistics
as one JSON line.
"""
import collections
import concurrent.futures as cf
import threading
import time

import numpy as np


class Rejected(RuntimeError):
    """The request's operator does not fit the HBM budget even alone."""


class _Entry:
    def __init__(self, solver, nbytes):
        self.solver = solver
        self.nbytes = nbytes
        self.lock = threading.Lock()
        self.busy = 0


class Server:
    def __init__(self, workers=4, hbm_budget=120 << 30, precision="tf32", tol=1e-8, solver_factory=None,
                 enomem_status=None):
        self.workers = workers
        self.budget = int(hbm_budget)
        self.precision = precision
        self.tol = tol
        if solver_factory is None:
            from . import mgiga  # loads libmgiga.so (CUDA)
            solver_factory = self._mgiga_factory(mgiga)
            enomem_status = mgiga.ENOMEM
        self.factory = solver_factory
        self.enomem = enomem_status
        self.cache = collections.OrderedDict()  # key -> _Entry, least recently used first
        self.used = 0
        self.cv = threading.Condition()
        self.queue = collections.deque()
        self.threads = []
        self.running = False
        self.latencies, self.rejected, self.setups, self.evictions = [], 0, 0, 0
        self.t_first, self.t_last, self.max_queue = None, None, 0

    @staticmethod
    def _mgiga_factory(mgiga):
        def make(problem, options, precision, budget):
            o = dict(options)
            return mgiga.Solver(problem, levels=o.get("levels", 0), smoother=o.get("smoother", "hybrid"),
                                tau=o.get("tau", 0.25), delta=o.get("delta", 0.1), nu=o.get("nu", 1),
                                precision=precision, hbm_budget=budget, gs_cluster=o.get("gs_cluster", 8))
        return make

    # -- lifecycle -----------------------------------------------------------
    def start(self):
        self.running = True
        for _ in range(self.workers):
            t = threading.Thread(target=self._work, daemon=True)
            t.start()
            self.threads.append(t)

    def stop(self):
        with self.cv:
            self.running = False
            self.cv.notify_all()
        for t in self.threads:
            t.join()
        self.threads = []
        for e in self.cache.values():
            e.solver.close()
        self.cache.clear()
        self.used = 0

    def submit(self, key, problem, options, rhs):
        fut = cf.Future()
        rhs = rhs if isinstance(rhs, (int, np.integer)) else np.asarray(rhs, dtype=np.float64)
        with self.cv:
            now = time.perf_counter()
            if self.t_first is None:
                self.t_first = now
            self.queue.append((key, problem, options, rhs, now, fut))
            self.max_queue = max(self.max_queue, len(self.queue))
            self.cv.notify()
        return fut

    def stats(self):
        with self.cv:
            lat = np.array(self.latencies) if self.latencies else np.zeros(1)
            span = (self.t_last - self.t_first) if self.t_last is not None else 0.0
            return {"solves": len(self.latencies), "rejected": self.rejected, "setups": self.setups,
                    "evictions": self.evictions, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                    "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                    "solves_per_s": len(self.latencies) / span if span > 0 else 0.0,
                    "resident_bytes": self.used, "queue": len(self.queue), "max_queue": self.max_queue}

    # -- admission -----------------------------------------------------------
    def _evict_one_idle(self):
        """Drop the least recently used idle handle (cv held); False if none is idle."""
        for k, e in self.cache.items():
            if e.busy == 0:
                del self.cache[k]
                self.used -= e.nbytes
                e.solver.close()
                self.evictions += 1
                return True
        return False

    def _acquire(self, key, problem, options):
        """The resident entry for `key`, set up within the budget (cv not held on entry)."""
        with self.cv:
            e = self.cache.get(key)
            if e is not None:
                e.busy += 1
                self.cache.move_to_end(key)
                return e
        while True:
            with self.cv:
                left = self.budget - self.used
            try:
                s = self.factory(problem, options, self.precision, max(left, 1))
            except Exception as exc:  # noqa: BLE001 -- only the budget refusal is retried
                if getattr(exc, "status", None) != self.enomem:
                    raise
                with self.cv:
                    if self._evict_one_idle():
                        continue
                    if self.used == 0:
                        raise Rejected(f"operator {key!r} exceeds the HBM budget alone") from exc
                    self.cv.wait(timeout=0.05)  # a running solve will release its handle
                continue
            with self.cv:
                e = self.cache.get(key)
                if e is not None:  # another worker set it up meanwhile
                    s.close()
                else:
                    e = _Entry(s, s.device_bytes())
                    self.cache[key] = e
                    self.used += e.nbytes
                    self.setups += 1
                e.busy += 1
                self.cache.move_to_end(key)
                return e

    def _release(self, e):
        with self.cv:
            e.busy -= 1
            self.cv.notify_all()

    # -- workers -------------------------------------------------------------
    def _work(self):
        while True:
            with self.cv:
                while self.running and not self.queue:
                    self.cv.wait()
                if not self.queue:
                    return
                key, problem, options, rhs, t0, fut = self.queue.popleft()
            try:
                e = self._acquire(key, problem, options)
            except Rejected as exc:
                with self.cv:
                    self.rejected += 1
                fut.set_exception(exc)
                continue
            except Exception as exc:  # noqa: BLE001 -- reported to the caller
                fut.set_exception(exc)
                continue
            try:
                with e.lock:
                    if isinstance(rhs, (int, np.integer)):
                        from .workloads import random_vector
                        rhs = random_vector(e.solver.ndof(), int(rhs), kind="normal")
                    u, it, rel, _st = e.solver.solve(rhs, tol=self.tol)
                done = time.perf_counter()
                with self.cv:
                    self.latencies.append(done - t0)
                    self.t_last = done if self.t_last is None else max(self.t_last, done)
                fut.set_result((u, it, rel, done - t0))
            except Exception as exc:  # noqa: BLE001 -- reported to the caller
                fut.set_exception(exc)
            finally:
                self._release(e)


def main(argv=None):
    """Serve the seeded serving stream with Poisson arrivals; print the statistics."""
    import argparse
    import json

    from . import workloads as W
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--workers", type=int, default=4)
    ap.add_argument("--budget-gb", type=float, default=120.0, help="HBM budget of the resident operators")
    ap.add_argument("--rate", type=float, default=0.0,
                    help="mean arrivals per second; 0: calibrated -- the stream is first served with every "
                         "request submitted at once (capacity X solves/s, set-ups included), then replayed "
                         "on a fresh server with Poisson arrivals at 0.8 X")
    ap.add_argument("--max-patch-dof", type=float, default=1e5, help="upper end of the per-patch DoF range")
    ap.add_argument("--precision", default="tf32", choices=["fp64", "fp32", "tf32", "bf16"])
    ap.add_argument("--seed", type=int, default=501)
    args = ap.parse_args(argv)
    stream = list(W.serving_stream(args.requests, seed=args.seed, max_patch_dof=args.max_patch_dof))

    def serve(rate):
        srv = Server(workers=args.workers, hbm_budget=int(args.budget_gb * (1 << 30)), precision=args.precision)
        arrivals = np.random.default_rng(args.seed + 7)
        srv.start()
        futs = []
        t = time.perf_counter()
        for key, prob, opts, rhs_seed in stream:
            if rate > 0:
                t += arrivals.exponential(1.0 / rate)
                wait = t - time.perf_counter()
                if wait > 0:
                    time.sleep(wait)
            futs.append(srv.submit(key, prob, opts, int(rhs_seed)))
        failed, iters = 0, []
        for f in futs:
            try:
                iters.append(f.result()[1])
            except Rejected:
                pass
            except Exception:  # noqa: BLE001 -- counted and reported
                failed += 1
        st = srv.stats()
        srv.stop()
        st.update(failed=failed, mean_iterations=float(np.mean(iters)) if iters else None)
        return st

    rate, calib = args.rate, None
    if rate <= 0:
        calib = serve(0.0)
        rate = 0.8 * calib["solves_per_s"]
    st = serve(rate)
    st.update(requests=args.requests, workers=args.workers, budget_gb=args.budget_gb, rate_per_s=rate,
              precision=args.precision, max_patch_dof=args.max_patch_dof,
              calibration=None if calib is None else {"capacity_solves_per_s": calib["solves_per_s"],
                                                       "p50_ms": calib["p50_ms"], "p99_ms": calib["p99_ms"]})
    print(json.dumps(st), flush=True)


if __name__ == "__main__":
    main()
