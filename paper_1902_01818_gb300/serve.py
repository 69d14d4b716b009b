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
    fut = srv.submit(key, problem, options, rhs)
    u, iterations, relres, latency_s = fut.result()
    srv.stop(); srv.stats()  # solves, rejected, p50/p99 latency, set-ups, evictions
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
        with self.cv:
            self.queue.append((key, problem, options, np.asarray(rhs, dtype=np.float64), time.perf_counter(), fut))
            self.cv.notify()
        return fut

    def stats(self):
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        return {"solves": len(self.latencies), "rejected": self.rejected, "setups": self.setups,
                "evictions": self.evictions, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)), "resident_bytes": self.used}

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
                    u, it, rel, _st = e.solver.solve(rhs, tol=self.tol)
                lat = time.perf_counter() - t0
                with self.cv:
                    self.latencies.append(lat)
                fut.set_result((u, it, rel, lat))
            except Exception as exc:  # noqa: BLE001 -- reported to the caller
                fut.set_exception(exc)
            finally:
                self._release(e)
