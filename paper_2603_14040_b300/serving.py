"""Continuous-batching Stokes solve server.

Requests (grid, material fields, tolerance) arrive at arbitrary times. The server keeps up to
`max_slots` solves in flight, each on its own CUDA stream and host worker thread; a request is
admitted as soon as a slot is free AND the device memory it needs fits the HBM budget. Solver
handles are pooled per grid shape: a handle keeps its multigrid hierarchy, Krylov bases and the
captured CUDA graph of its FGMRES iteration resident, so later requests of that shape reuse them
(no allocation, no re-capture). Idle handles are evicted least-recently-used when a new shape
needs the memory. Every solve is deterministic (fixed-order reductions, no atomics in any value
the result depends on), so a request's result is the same alone and in the mix.

The scheduling logic is backend-agnostic: `backend` provides footprint(shape) -> bytes,
create(shape) -> handle, solve(handle, request, stream) -> (outputs, stats) and
destroy(handle). `PyroBackend` is the libpyro one; tests drive the same server with a fake one.
"""
import heapq
import itertools
import threading
import time
from collections import OrderedDict
from dataclasses import dataclass, field
from typing import Any, Optional

import numpy as np


@dataclass
class Request:
    rid: int
    nx: int
    ny: int
    Lx: float
    Ly: float
    eta_n: Any
    eta_c: Any
    rho: Any
    g: tuple = (0.0, 1.0)
    tol: float = 1e-8
    arrival: float = 0.0          # seconds on the server clock (set by submit if 0)
    # filled by the server
    admitted: float = 0.0
    done: float = 0.0
    status: int = 0
    iters: int = 0
    result: Any = None
    error: Optional[str] = None

    @property
    def shape(self):
        return (self.nx, self.ny, self.Lx, self.Ly)

    @property
    def latency(self):
        return self.done - self.arrival


@dataclass(order=True)
class _Pending:
    arrival: float
    seq: int
    req: Request = field(compare=False)


class HandlePool:
    """Per-shape pool of solver handles with byte accounting and LRU eviction of idle handles."""

    def __init__(self, backend, budget_bytes):
        self.backend = backend
        self.budget = int(budget_bytes)
        self.idle = OrderedDict()     # shape -> list of idle handles (LRU order of shapes)
        self.bytes_in_use = 0         # bytes of every live handle (idle or busy)
        self.live = 0

    def acquire(self, shape):
        """Return a handle for `shape` (reused if one is idle), creating one if the budget allows
        after evicting idle handles of other shapes; None if it cannot fit now."""
        lst = self.idle.get(shape)
        if lst:
            h = lst.pop()
            if not lst:
                del self.idle[shape]
            else:
                self.idle.move_to_end(shape)
            return h
        need = self.backend.footprint(shape)
        if need <= 0 or need > self.budget:
            raise ValueError(f"request shape {shape} cannot be served (footprint {need} B, budget {self.budget} B)")
        while self.bytes_in_use + need > self.budget and self.idle:
            old_shape, old_list = next(iter(self.idle.items()))
            h = old_list.pop()
            if not old_list:
                del self.idle[old_shape]
            self.backend.destroy(h)
            self.bytes_in_use -= self.backend.footprint(old_shape)
            self.live -= 1
        if self.bytes_in_use + need > self.budget:
            return None
        h = self.backend.create(shape)
        self.bytes_in_use += need
        self.live += 1
        return h

    def release(self, shape, h):
        self.idle.setdefault(shape, []).append(h)
        self.idle.move_to_end(shape)

    def close(self):
        for shape, lst in self.idle.items():
            for h in lst:
                self.backend.destroy(h)
                self.bytes_in_use -= self.backend.footprint(shape)
                self.live -= 1
        self.idle.clear()


class SolveServer:
    def __init__(self, backend, max_slots=4, budget_bytes=None, clock=time.perf_counter):
        self.backend = backend
        self.max_slots = int(max_slots)
        self.clock = clock
        budget = budget_bytes if budget_bytes is not None else backend.default_budget()
        self.pool = HandlePool(backend, budget)
        self._lock = threading.Condition()
        self._pending = []            # heap by arrival time (FIFO among equal arrivals)
        self._seq = itertools.count()
        self._running = 0
        self._done = []
        self._stop = False
        self._workers = []
        self._streams = [backend.make_stream() for _ in range(self.max_slots)]
        self._free_streams = list(range(self.max_slots))
        self.t0 = clock()
        self.max_concurrent = 0
        self._dispatcher = threading.Thread(target=self._dispatch, daemon=True)
        self._dispatcher.start()

    def now(self):
        return self.clock() - self.t0

    def submit(self, req):
        with self._lock:
            if req.arrival == 0.0:
                req.arrival = self.now()
            heapq.heappush(self._pending, _Pending(req.arrival, next(self._seq), req))
            self._lock.notify_all()

    def _dispatch(self):
        while True:
            with self._lock:
                while not self._stop and (not self._pending or self._running >= self.max_slots):
                    self._lock.wait(0.05)
                if self._stop and not self._pending:
                    return
                if self._running >= self.max_slots or not self._pending:
                    continue
                item = self._pending[0]
                try:
                    h = self.pool.acquire(item.req.shape)
                except Exception as e:              # unservable shape or a failed handle creation
                    heapq.heappop(self._pending)
                    item.req.error = str(e)
                    item.req.status = -1
                    item.req.done = self.now()
                    self._done.append(item.req)
                    self._lock.notify_all()
                    continue
                if h is None:                       # memory busy: wait for a running solve to end
                    self._lock.wait(0.01)
                    continue
                heapq.heappop(self._pending)
                req = item.req
                req.admitted = self.now()
                sidx = self._free_streams.pop()
                self._running += 1
                self.max_concurrent = max(self.max_concurrent, self._running)
            t = threading.Thread(target=self._run_one, args=(req, h, sidx), daemon=True)
            t.start()
            self._workers.append(t)

    def _run_one(self, req, h, sidx):
        try:
            out, stats = self.backend.solve(h, req, self._streams[sidx])
            req.result = out
            req.status = int(stats.get("status", 0))
            req.iters = int(stats.get("iters", 0))
        except Exception as e:  # a failing request must not take the server down
            req.error = repr(e)
            req.status = -3
        finally:
            with self._lock:
                req.done = self.now()
                self.pool.release(req.shape, h)
                self._free_streams.append(sidx)
                self._running -= 1
                self._done.append(req)
                self._lock.notify_all()

    def drain(self, timeout=None):
        """Block until every submitted request has finished; returns them in completion order."""
        t_end = None if timeout is None else time.perf_counter() + timeout
        with self._lock:
            while self._pending or self._running:
                if t_end is not None and time.perf_counter() > t_end:
                    raise TimeoutError("server did not drain in time")
                self._lock.wait(0.05)
            return list(self._done)

    def close(self):
        with self._lock:
            self._stop = True
            self._lock.notify_all()
        self._dispatcher.join(timeout=5)
        for t in self._workers:
            t.join(timeout=5)
        self.pool.close()


def latency_stats(reqs):
    lat = np.array([r.latency for r in reqs if r.error is None])
    if len(lat) == 0:
        return {"n": 0}
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    return {"n": int(len(lat)), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "throughput_solves_per_s": float(len(lat) / span) if span > 0 else None}


def poisson_arrivals(n, rate, seed):
    """Arrival times (s) of n requests of a Poisson process with the given rate (1/s)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


class PyroBackend:
    """libpyro backend: handles are pyro.Stokes objects; inputs/outputs are CUDA tensors.

    With restart_choices (descending FGMRES restart lengths), each shape gets the longest restart
    whose handle fits in per_handle_bytes (default: the budget shared by four slots), so large
    grids still admit several concurrent solves while small ones keep long Krylov cycles (the
    high-contrast requests need them)."""

    # V(8, 8) cycles unless the caller says otherwise: on sharp high-contrast inclusions (the
    # serving workload) eight sweeps per level about halve the total solve time of V(2, 2)
    DEFAULT_OPTS = {"nu1": 8, "nu2": 8}

    def __init__(self, opts_kw=None, device=0, restart_choices=None, per_handle_bytes=None):
        import torch
        from . import pyro as P
        self.P = P
        self.torch = torch
        self.device = device
        self.opts_kw = dict(self.DEFAULT_OPTS)
        self.opts_kw.update(opts_kw or {})
        self.restart_choices = tuple(restart_choices) if restart_choices else None
        self.per_handle_bytes = per_handle_bytes
        self._fp = {}

    def default_budget(self):
        free, total = self.torch.cuda.mem_get_info(self.device)
        return int(0.8 * free)

    def make_stream(self):
        return self.torch.cuda.Stream(device=self.device)

    def opts_for(self, shape):
        """Options of the handle for `shape` (the restart length chosen for it)."""
        if shape not in self._fp:
            kw = dict(self.opts_kw)
            if self.restart_choices:
                cap = self.per_handle_bytes if self.per_handle_bytes is not None else self.default_budget() // 4
                for m in self.restart_choices:
                    kw["restart_m"] = m
                    if self.P.footprint(shape[0], shape[1], self.P.default_opts(**kw)) <= cap:
                        break
            self._fp[shape] = (kw, self.P.footprint(shape[0], shape[1], self.P.default_opts(**kw)))
        return self._fp[shape][0]

    def footprint(self, shape):
        self.opts_for(shape)
        return self._fp[shape][1]

    def create(self, shape):
        nx, ny, Lx, Ly = shape
        return self.P.Stokes(nx, ny, Lx, Ly, **self.opts_for(shape))

    def destroy(self, h):
        h.close()

    def solve(self, h, req, stream):
        torch = self.torch
        with torch.cuda.stream(stream):
            outs = [torch.zeros((req.ny + 2, req.nx + 2), dtype=torch.float64, device="cuda") for _ in range(3)]
            st = h.solve(req.eta_n, req.eta_c, req.rho, req.g, req.tol, *outs, stream=stream)
        return outs, st.as_dict()
