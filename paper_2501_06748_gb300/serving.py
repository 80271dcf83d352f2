"""Request serving around the library with continuous batching (a harness; the method's
arithmetic all runs in the CUDA library).

A request asks, for one point source on one model (mesh, radial points, density, time
step), for the receiver traces of K steps and optionally, given observed traces, for the
misfit and its density gradient (the paper's adjoint, Sections 2 and 4).  Requests that
share a model and receivers run as the shot columns ("slots") of library sessions
(``sbfwi.Session``): a forward session for the forward solves and an adjoint session for
the gradients.  A worker thread drives the GPU: it advances every session with work by
one window of steps, collects the requests that finished, and between windows admits
waiting requests into free slots, so a request that arrives while others are in flight
joins them at the next window instead of waiting for them to end.  A gradient request
moves through three stages: its forward solve (the nodal velocities of every step are
kept in a device array of its own), the misfit and residual, and its adjoint.

Admission is bounded by device memory: a request is admitted only while the free device
memory (``torch.cuda.mem_get_info``) minus ``mem_reserve`` covers what it keeps resident
(its forward field for a gradient request; the session state is allocated once per
session), and with ``mem_budget`` also while the resident bytes of all requests in flight
stay within that budget.  Set-up models are cached (LRU).  Latency runs from a request's
arrival to the end of the window that finished its last stage.
"""

from __future__ import annotations

import queue
import threading
import time
from collections import OrderedDict
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    model_key: tuple            # identifies mesh + density + time step (the cache key)
    src_node: int
    wavelet: np.ndarray         # (K,)
    rec_nodes: np.ndarray       # (R,)
    arrival: float              # seconds on the engine's clock
    observed: np.ndarray = None  # (R, K): with it, the misfit and gradient are computed too
    done: float = -1.0
    traces: np.ndarray = field(default=None, repr=False)
    misfit: float = None
    gradient: np.ndarray = field(default=None, repr=False)
    # when the request entered its first slot: (session window count, requests then in flight)
    admitted_at: tuple = None

    @property
    def K(self) -> int:
        return int(self.wavelet.shape[0])

    @property
    def wants_gradient(self) -> bool:
        return self.observed is not None


class ModelCache:
    """Set-up models by key, least recently used first out."""

    def __init__(self, build, capacity=8):
        self.build, self.capacity = build, capacity
        self.models = OrderedDict()
        self.setups = 0

    def get(self, key):
        if key in self.models:
            self.models.move_to_end(key)
            return self.models[key]
        m = self.build(key)
        self.setups += 1
        self.models[key] = m
        if len(self.models) > self.capacity:
            self.models.popitem(last=False)
        return m


def request_bytes(stride: int, r: Request) -> int:
    """Device memory a request keeps resident while in flight: its wavelet or residual and
    traces, and for a gradient request its forward velocity field (K x field stride)."""
    b = 8 * r.K * (1 + 2 * r.rec_nodes.size)
    if r.wants_gradient:
        b += 8 * r.K * stride
    return b


class _Group:
    """The sessions of one (model, receivers) pair."""

    def __init__(self, model, rec, slots, window):
        from . import sbfwi
        self.model, self.rec = model, rec
        self.fwd = sbfwi.Session(model, sbfwi.SESSION_FORWARD, slots, rec, window)
        self.adj = None
        self.slots, self.window = slots, window
        self.fwd_slot = {}          # slot -> request
        self.adj_slot = {}
        self.ready_adj = []         # (request, residual, field) waiting for an adjoint slot

    def adjoint(self):
        from . import sbfwi
        if self.adj is None:
            self.adj = sbfwi.Session(self.model, sbfwi.SESSION_ADJOINT, self.slots, self.rec, self.window)
        return self.adj

    def busy(self):
        return bool(self.fwd_slot or self.adj_slot)


class Engine:
    def __init__(self, build_model, max_batch=8, window=32, cache_capacity=8, mem_budget=None, mem_reserve=2 << 30):
        self.cache = ModelCache(build_model, cache_capacity)
        self.slots, self.window = max_batch, window
        self.mem_budget, self.mem_reserve = mem_budget, mem_reserve
        self.groups = {}
        self.windows = 0                    # windows run (all sessions)
        self.in_flight = {}                 # rid -> resident bytes
        self.max_in_flight = 0
        self.batches = []                   # slots busy in each forward window run
        self._q = queue.Queue()
        self._err = None

    # -- worker side ------------------------------------------------------------------
    def _group(self, r):
        key = (r.model_key, tuple(int(x) for x in r.rec_nodes))
        g = self.groups.get(key)
        if g is None:
            g = self.groups[key] = _Group(self.cache.get(r.model_key), np.asarray(r.rec_nodes, dtype=np.int64),
                                          self.slots, self.window)
        return g

    def _fits(self, need):
        import torch
        if self.mem_budget is not None and self.in_flight and sum(self.in_flight.values()) + need > self.mem_budget:
            return False
        free, _ = torch.cuda.mem_get_info()
        return free - self.mem_reserve >= need

    def _admit(self, waiting):
        import torch
        left = []
        for r in waiting:
            g = self._group(r)
            free = [s for s in range(self.slots) if s not in g.fwd_slot]
            need = request_bytes(g.fwd.field_stride, r)
            if not free or not self._fits(need):
                left.append(r)
                continue
            fld = None
            if r.wants_gradient:
                fld = torch.empty((r.K, g.fwd.field_stride), dtype=torch.float64, device=g.fwd.device)
            wav = torch.as_tensor(np.ascontiguousarray(r.wavelet, dtype=np.float64), device=g.fwd.device)
            g.fwd.admit(free[0], wav, src_node=r.src_node, field=fld)
            g.fwd_slot[free[0]] = (r, fld)
            self.in_flight[r.rid] = need
            self.max_in_flight = max(self.max_in_flight, len(self.in_flight))
            r.admitted_at = (self.windows, len(self.in_flight) - 1)
        return left

    def _admit_adjoints(self, g):
        adj = g.adjoint()
        while g.ready_adj:
            free = [s for s in range(self.slots) if s not in g.adj_slot]
            if not free:
                return
            r, res, fld = g.ready_adj.pop(0)
            adj.admit(free[0], res, field=fld)
            g.adj_slot[free[0]] = (r, fld)

    def _run_window(self, g, now):
        from . import sbfwi
        if g.fwd_slot:
            self.batches.append(len(g.fwd_slot))
            for s in g.fwd.step():
                r, fld = g.fwd_slot.pop(s)
                tr = g.fwd.collect(s)
                r.traces = tr.cpu().numpy()
                if r.wants_gradient:
                    obs = np.ascontiguousarray(r.observed, dtype=np.float64)[None]
                    E, res = sbfwi.misfit(tr[None].contiguous(), _on_device(obs, tr), g.model.dt)
                    r.misfit = E
                    g.ready_adj.append((r, res[0].contiguous(), fld))
                else:
                    r.done = now()
                    self.in_flight.pop(r.rid, None)
            self.windows += 1
        if g.ready_adj:
            self._admit_adjoints(g)
        if g.adj_slot:
            for s in g.adj.step():
                r, _ = g.adj_slot.pop(s)
                r.gradient = g.adj.collect(s).cpu().numpy()
                r.done = now()
                self.in_flight.pop(r.rid, None)
            self.windows += 1

    def _worker(self, total, now, stop):
        try:
            import torch
            torch.cuda.set_device(torch.cuda.current_device())
            waiting, finished = [], 0
            while finished < total and not stop.is_set():
                # arrivals
                block = not waiting and not any(g.busy() or g.ready_adj for g in self.groups.values())
                try:
                    while True:
                        r = self._q.get(timeout=0.01) if block else self._q.get_nowait()
                        waiting.append(r)
                        block = False
                except queue.Empty:
                    pass
                waiting = self._admit(waiting)
                for g in list(self.groups.values()):
                    if g.busy() or g.ready_adj:
                        self._run_window(g, now)
                finished = sum(1 for r in self._all if r.done >= 0)
        except BaseException as e:      # reported by run()
            self._err = e

    # -- caller side -------------------------------------------------------------------
    def run(self, requests, clock=time.perf_counter):
        """Serve ``requests`` (arrival times relative to the start, in seconds): they are
        handed to the worker thread at their arrival times while it runs; returns them with
        ``done`` and the results filled in."""
        pending = sorted(requests, key=lambda r: r.arrival)
        self._all = pending
        t0 = clock()
        now = lambda: clock() - t0
        stop = threading.Event()
        w = threading.Thread(target=self._worker, args=(len(pending), now, stop), daemon=True)
        w.start()
        try:
            for r in pending:
                dt = r.arrival - now()
                if dt > 0:
                    time.sleep(dt)
                self._q.put(r)
            while w.is_alive():
                w.join(timeout=0.1)
                if self._err is not None:
                    break
        finally:
            stop.set()
            w.join()
        if self._err is not None:
            raise self._err
        return requests


def _on_device(a, like):
    import torch
    return torch.as_tensor(a, device=like.device)


def latency_stats(requests):
    lat = np.array([r.done - r.arrival for r in requests])
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max())}
