"""Continuous-batching request loop for state / state+adjoint solves.

Requests arrive over time (each: grid edge n, buoyancy factor alpha, design, adjoint flag). A pool
of worker slots runs them concurrently, each slot on its own problem and CUDA stream, so the work of
different requests overlaps on the device (the ctypes calls release the GIL). Problems, and with
them their multigrid hierarchies, stay resident in a per-grid pool and are reused across requests
with nc_set_params (a new alpha) and nc_set_design. A request is admitted when a slot is free and
either an idle problem for its grid exists or creating one keeps the pool within the HBM budget
(nc_footprint_bytes); otherwise it waits, and idle problems of other grids may be evicted to make
room. Latency is measured from arrival to completion.
"""

import collections
import threading
import time

import numpy as np

from . import _abi
from .problem import Problem


class Request:
    """One request: a state solve (or a state solve, its adjoint and the sensitivities) of `design` on
    an n^3 grid at buoyancy factor alpha. The design may be a host array or a device tensor that is
    ready (its producing work complete) when the request arrives."""
    __slots__ = ("rid", "t_arrival", "n", "alpha", "adjoint", "design", "t_start", "t_done", "f", "grad",
                 "fields", "state_stats", "error")

    def __init__(self, rid, t_arrival, n, alpha, adjoint, design):
        self.rid, self.t_arrival, self.n, self.alpha, self.adjoint, self.design = rid, t_arrival, n, alpha, adjoint, design
        self.t_start = self.t_done = None
        self.f = self.grad = self.fields = self.state_stats = self.error = None


class Server:
    def __init__(self, slots=6, hbm_budget_bytes=64 << 30, keep_gradients=False, keep_fields=False, device="cuda",
                 **params):
        self.slots = slots
        self.budget = hbm_budget_bytes
        self.keep_gradients = keep_gradients
        self.keep_fields = keep_fields   # keep (P, T, u) of every request (device tensors)
        self.device = device
        self.params = params
        self.pool = collections.defaultdict(list)    # n -> idle Problems
        self.pool_bytes = 0
        self.footprints = {}
        self.lock = threading.Condition()
        self.queue = collections.deque()
        self.done = []
        self.peak_bytes = 0

    def _footprint(self, n):
        if n not in self.footprints:
            p = _abi.default_params(**self.params)
            self.footprints[n] = _abi.footprint_bytes(_abi.Grid(n, n, n, 1.0 / n), p)
        return self.footprints[n]

    def _acquire(self, n):
        """An idle problem for grid n, or None if the budget does not allow one now (lock held)."""
        if self.pool[n]:
            return self.pool[n].pop()
        need = self._footprint(n)
        if self.pool_bytes + need > self.budget:
            # evict idle problems of other grids, largest first
            for m in sorted(self.pool, key=lambda k: -self._footprint(k)):
                while self.pool[m] and self.pool_bytes + need > self.budget:
                    self.pool[m].pop().close()
                    self.pool_bytes -= self._footprint(m)
            if self.pool_bytes + need > self.budget:
                return None
        self.pool_bytes += need
        self.peak_bytes = max(self.peak_bytes, self.pool_bytes)
        return "new"

    def _run(self, req, pb):
        if pb == "new":
            pb = Problem(req.n, req.n, req.n, 1.0 / req.n, device=self.device, alpha=req.alpha, **self.params)
        else:
            pb.set_params(alpha=req.alpha)
        pb.set_design(req.design)
        req.state_stats = pb.solve_state()
        if self.keep_fields:
            req.fields = pb.get_fields()
        if req.adjoint:
            req.f, _ = pb.solve_adjoint()
            g = pb.sensitivities()
            req.grad = g if self.keep_gradients else None
        else:
            req.f = pb.objective()
        return pb

    def _worker(self):
        while True:
            with self.lock:
                while True:
                    if self.stop and not self.queue:
                        return
                    pick = None
                    for i, req in enumerate(self.queue):
                        pb = self._acquire(req.n)
                        if pb is not None:
                            pick = (i, req, pb)
                            break
                    if pick:
                        del self.queue[pick[0]]
                        break
                    self.lock.wait(0.01)
            _, req, pb = pick
            req.t_start = time.perf_counter()
            try:
                pb = self._run(req, pb)
            except Exception as e:  # the request fails, the server keeps going
                req.error = repr(e)
            req.t_done = time.perf_counter()
            with self.lock:
                if isinstance(pb, Problem):
                    self.pool[req.n].append(pb)
                else:
                    self.pool_bytes -= self._footprint(req.n)
                self.done.append(req)
                self.lock.notify_all()

    def run(self, requests):
        """Serve requests (objects with t_arrival relative to the start); returns them completed."""
        self.stop = False
        workers = [threading.Thread(target=self._worker, daemon=True) for _ in range(self.slots)]
        for w in workers:
            w.start()
        t0 = time.perf_counter()
        for req in sorted(requests, key=lambda r: r.t_arrival):
            delay = t0 + req.t_arrival - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            req.t_arrival = t0 + req.t_arrival
            with self.lock:
                self.queue.append(req)
                self.lock.notify_all()
        with self.lock:
            self.stop = True
            self.lock.notify_all()
        for w in workers:
            w.join()
        self.t_total = time.perf_counter() - t0
        return self.done

    def close(self):
        for n in list(self.pool):
            for pb in self.pool[n]:
                pb.close()
            self.pool[n] = []
        self.pool_bytes = 0


def summarize(done, wall):
    """Latency percentiles (arrival to completion) and rates over the wall time of the stream:
    requests_per_s counts each completed request once (a state solve, or a state solve with its adjoint
    and sensitivities, the unit of the one-problem benchmark's whole path); state_solves_per_s and
    adjoint_solves_per_s count the solves of each kind."""
    ok = [r for r in done if r.error is None]
    lat = np.array([r.t_done - r.t_arrival for r in ok])
    return {"requests": len(done), "errors": len(done) - len(ok),
            "p50_ms": float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99) * 1e3) if len(lat) else None,
            "mean_ms": float(lat.mean() * 1e3) if len(lat) else None,
            "requests_per_s": len(ok) / wall, "state_solves_per_s": len(ok) / wall,
            "adjoint_solves_per_s": sum(1 for r in ok if r.adjoint) / wall, "wall_s": wall}
