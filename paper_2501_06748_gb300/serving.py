"""Request serving around the library: forward-modelling requests with continuous
batching (a harness; the method's arithmetic all runs in the CUDA library).

A request asks for the receiver traces of one point source on one model (mesh,
radial points, density, time step, number of steps).  The engine keeps a cache of
set-up models (the set-up is paid once per model), queues requests as they arrive
and, whenever the device is free, launches the oldest waiting request together
with up to ``max_batch - 1`` other waiting requests that share its model, step
count and receivers: they run as one batch of shots through ``sbfwi.forward``
(every operator read once for all of them).  Admission is also bounded by device
memory: with ``mem_budget`` set, a batch takes requests only while the device memory
their shots need (the stepper's per-shot state and the traces, ``request_bytes``) fits
the budget; a request that does not fit waits for the next batch.  Latency is measured
from a request's arrival to the end of the batch that served it.
"""

from __future__ import annotations

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
    done: float = -1.0
    traces: np.ndarray = field(default=None, repr=False)

    @property
    def K(self) -> int:
        return int(self.wavelet.shape[0])


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


def request_bytes(model, r: Request) -> int:
    """Device memory one shot of a forward pass needs: the interior state of every
    element at the padded n_b (predictor, z, q and their neighbours: 5 arrays), the
    boundary state and solution (6 arrays), the effective sources and the traces."""
    mesh = model.mesh
    interior = mesh.n_elem * (mesh.n_r - 1) * mesh.n_b
    return 8 * (5 * interior + 6 * (mesh.n_nodes + 1) + mesh.n_elem * mesh.n_b + r.rec_nodes.size * r.K)


class Engine:
    def __init__(self, build_model, max_batch=8, cache_capacity=8, mem_budget=None):
        self.cache = ModelCache(build_model, cache_capacity)
        self.max_batch = max_batch
        self.mem_budget = mem_budget
        self.batches = []

    def _pick(self, waiting, model):
        head = waiting[0]
        same = [r for r in waiting if r.model_key == head.model_key and r.K == head.K
                and np.array_equal(r.rec_nodes, head.rec_nodes)]
        batch, used = [], 0
        for r in same[:self.max_batch]:
            need = request_bytes(model, r)
            if batch and self.mem_budget is not None and used + need > self.mem_budget:
                break
            batch.append(r)
            used += need
        return batch

    def run(self, requests, clock=time.perf_counter):
        """Serve ``requests`` (sorted by arrival, arrival times relative to the start);
        returns them with ``done`` and ``traces`` filled in."""
        from . import sbfwi
        pending = sorted(requests, key=lambda r: r.arrival)
        waiting = []
        t0 = clock()
        now = lambda: clock() - t0
        i = 0
        while i < len(pending) or waiting:
            while i < len(pending) and pending[i].arrival <= now():
                waiting.append(pending[i])
                i += 1
            if not waiting:
                time.sleep(max(0.0, min(pending[i].arrival - now(), 0.01)))
                continue
            model = self.cache.get(waiting[0].model_key)
            batch = self._pick(waiting, model)
            src = np.array([r.src_node for r in batch], dtype=np.int64)
            wav = np.stack([r.wavelet for r in batch])
            tr, _ = sbfwi.forward(model, src, wav, batch[0].rec_nodes, keep=False)
            t = now()
            for k, r in enumerate(batch):
                r.traces = tr[k]
                r.done = t
                waiting.remove(r)
            self.batches.append(len(batch))
        return requests


def latency_stats(requests):
    lat = np.array([r.done - r.arrival for r in requests])
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max())}
