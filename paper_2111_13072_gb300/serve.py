"""Continuous-batching service for spectrum requests.

A request asks for the admittance spectrum (Sec. 4) of one plasma/probe
configuration: N super-particles, T_e, n_e, l_max, a drive and a number of
steps. The server

* admits waiting requests (first come, first served) as soon as a slot and
  enough device memory are free -- the footprint of each request comes from the
  library (imrp_footprint), checked against an HBM budget;
* keeps every admitted request's particle state resident on the device;
* advances all admitted requests together, chunk by chunk, with one captured
  CUDA graph per step pair over all of them (imrp_batch_*), so requests that
  arrive while others run join at the next chunk and their work overlaps on the
  GPU;
* finishes a request when its steps are done: the spectrum is computed on the
  GPU (imrp_spectrum), the context is freed and its memory returns to the pool;
* evicts a request whose context reports an error (a non-finite state, a
  particle outside the domain): its result carries the error, its memory
  returns to the pool, and the others keep running.

A request's result does not depend on what else is in the mix: batched steps
compute bit for bit what the request's steps compute alone.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass

import numpy as np

from . import imrp
from .inputs import Workload, workload_state


@dataclass
class SpectrumRequest:
    rid: int
    workload: Workload
    steps: int
    arrival: float = 0.0          # seconds after the server starts
    n_freq: int = 1000
    w_max: float = 2.0


@dataclass
class SpectrumResult:
    rid: int
    w_res: float
    dw: float
    fit: np.ndarray
    omega: np.ndarray
    reY: np.ndarray
    qdiff: np.ndarray
    arrival: float
    admitted: float
    finished: float
    error: str | None = None      # set when the request was evicted

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class _Slot:
    req: SpectrumRequest
    sim: imrp.Sim
    remaining: int
    footprint: int
    admitted: float


class SpectrumServer:
    def __init__(self, hbm_budget: int | None = None, chunk: int = 200, max_slots: int = 64,
                 autotune: bool = False, backend=None, state_fn=None):
        """backend: the module with Sim, Batch, footprint, params_from_workload
        and IMRPError (the library binding by default; tests pass a fake);
        state_fn: workload -> (x, v) initial state."""
        self.lib = imrp if backend is None else backend
        self.state_fn = workload_state if state_fn is None else state_fn
        if hbm_budget is None:
            import torch
            free, _ = torch.cuda.mem_get_info()
            hbm_budget = int(0.8 * free)
        self.budget = hbm_budget
        self.chunk = chunk
        self.max_slots = max_slots
        self.autotune = autotune
        self.stats = {"chunks": 0, "max_active": 0, "peak_bytes": 0, "evicted": 0}

    def _admit(self, req: SpectrumRequest, now: float) -> _Slot:
        p = self.lib.params_from_workload(req.workload)
        sim = self.lib.Sim(p)
        x, v = self.state_fn(req.workload)
        sim.load(x, v)
        if self.autotune:
            sim.autotune()
        return _Slot(req, sim, req.steps, self.lib.footprint(p, req.steps), now)

    def _failed_slots(self, batch, ids, err) -> list[tuple[int, str]]:
        """The requests whose contexts failed in the last chunk: the one the
        batch reported (its flags are cleared by the report) and any other
        whose own check still fails."""
        k = batch.failed_index()
        if k < 0:
            raise err  # an error of the batch itself: not one request's
        out = [(ids[k], str(err))]
        for i, rid in enumerate(ids):
            if i == k:
                continue
            try:
                self._active[rid].sim.sync()
            except self.lib.IMRPError as e:
                out.append((rid, str(e)))
        return out

    def serve(self, requests: list[SpectrumRequest], realtime: bool = True) -> list[SpectrumResult]:
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        waiting: collections.deque[SpectrumRequest] = collections.deque()
        active: dict[int, _Slot] = {}
        self._active = active
        results: list[SpectrumResult] = []
        used = 0
        batch, batch_ids = None, None
        t0 = time.perf_counter()
        clock = (lambda: time.perf_counter() - t0) if realtime else None
        vtime = 0.0
        while pending or waiting or active:
            now = clock() if realtime else vtime
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            # admission: FIFO, as long as a slot and the memory budget allow
            while waiting and len(active) < self.max_slots:
                req = waiting[0]
                need = self.lib.footprint(self.lib.params_from_workload(req.workload), req.steps)
                if used + need > self.budget and active:
                    break
                waiting.popleft()
                slot = self._admit(req, now)
                active[req.rid] = slot
                used += slot.footprint
            self.stats["max_active"] = max(self.stats["max_active"], len(active))
            self.stats["peak_bytes"] = max(self.stats["peak_bytes"], used)
            if not active:
                nxt = pending[0].arrival if pending else now
                if realtime:
                    time.sleep(max(0.0, nxt - now))
                else:
                    vtime = max(vtime, nxt)
                continue
            ids = tuple(sorted(active))
            if ids != batch_ids:
                if batch is not None:
                    batch.close()
                batch = self.lib.Batch([active[i].sim for i in ids])
                batch_ids = ids
            n = min(self.chunk, min(s.remaining for s in active.values()))
            tc = time.perf_counter()
            batch.step(n)  # a launch error is not one request's: it propagates
            try:
                batch.sync()
                failed = []
            except self.lib.IMRPError as e:
                failed = self._failed_slots(batch, ids, e)
            self.stats["chunks"] += 1
            if not realtime:
                vtime += time.perf_counter() - tc
            now = clock() if realtime else vtime
            for rid, msg in failed:
                s = active.pop(rid)
                nan = float("nan")
                results.append(SpectrumResult(rid, nan, nan, np.full(4, nan), np.zeros(0), np.zeros(0),
                                              np.zeros(0), s.req.arrival, s.admitted, now, error=msg))
                s.sim.close()
                used -= s.footprint
                self.stats["evicted"] += 1
            for rid in [r for r in ids if r in active]:
                s = active[rid]
                s.remaining -= n
                if s.remaining == 0:
                    sp = s.sim.spectrum(s.req.n_freq, s.req.w_max)
                    q, _ = s.sim.qdiff()
                    done = clock() if realtime else vtime
                    results.append(SpectrumResult(rid, sp["w_res"], sp["dw"], sp["fit"], sp["omega"],
                                                  sp["reY"], q, s.req.arrival, s.admitted, done))
                    s.sim.close()
                    used -= s.footprint
                    del active[rid]
        if batch is not None:
            batch.close()
        return sorted(results, key=lambda r: r.rid)


def serving_requests(n_requests: int, rate: float = 20.0, steps: int = 5000, seed: int = 5,
                     l_choices=(8, 16), n_range=(1e5, 4e6), precision: int = 1) -> list[SpectrumRequest]:
    """Poisson arrivals of spectrum requests with N log-uniform in n_range,
    T_e uniform in [0.5, 5] eV, n_e log-uniform in [1e14, 1e17] m^-3 and
    l_max drawn from l_choices (seeded)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate)
        N = int(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1]))))
        T = float(rng.uniform(0.5, 5.0))
        n = float(math.exp(rng.uniform(math.log(1e14), math.log(1e17))))
        L = int(rng.choice(l_choices))
        w = Workload(f"req{i}", N=N, l_max=L, T_e_eV=T, n_e_m3=n, steps=steps, precision=precision,
                     seed=seed * 1000 + i)
        out.append(SpectrumRequest(i, w, steps, arrival=t))
    return out


def ensemble_workloads(n_instances: int = 64, seed: int = 3, n_range=(1e4, 1e6), l_choices=(8, 12, 16),
                       precision: int = 1) -> list[Workload]:
    """Batched ensemble: N log-uniform in n_range, T_e uniform in [0.5, 5] eV,
    n_e log-uniform in [1e14, 1e17] m^-3, l_max from l_choices (seeded)."""
    rng = np.random.default_rng(seed)
    ws = []
    for i in range(n_instances):
        N = int(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1]))))
        T = float(rng.uniform(0.5, 5.0))
        n = float(math.exp(rng.uniform(math.log(1e14), math.log(1e17))))
        L = int(rng.choice(l_choices))
        ws.append(Workload(f"ens{i}", N=N, l_max=L, T_e_eV=T, n_e_m3=n, precision=precision,
                           seed=seed * 1000 + i))
    return ws
