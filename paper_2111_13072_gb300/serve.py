"""Continuous-batching service for spectrum requests.

A request asks for the admittance spectrum (Sec. 4) of one plasma/probe
configuration: N super-particles, T_e, n_e, l_max, a drive and a number of
steps. The server

* admits waiting requests (first come, first served) as soon as a slot and
  enough device memory are free -- the footprint of each request comes from the
  library (imrp_footprint), checked against an HBM budget;
* prepares an admitted request off the loop's critical path: a worker thread
  draws its initial state, creates its context and loads the particles, while
  the loop keeps the running requests going;
* keeps every admitted request's particle state resident on the device and
  advances each in chunks of steps on its own stream, replaying the context's
  own captured step graphs (a fixed graph per slot, captured once: admissions
  and completions never re-capture anything), so that the steps of all
  admitted requests overlap on the GPU and a request that arrives while
  others run starts as soon as it is prepared;
* polls the contexts without blocking (imrp_ready) and starts the next chunk
  of whichever request is done with its last one;
* finishes a request when its steps are done on another worker thread: the
  spectrum is computed (imrp_spectrum: the transform on the GPU, the fit on
  the host), the context is freed and its memory returns to the pool;
* evicts a request whose context reports an error (a non-finite state, a
  particle outside the domain): its result carries the error, its memory
  returns to the pool, and the others keep running.

A request's result does not depend on what else is in the mix: its context
computes bit for bit what it computes alone.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
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
    sim: object
    remaining: int
    footprint: int
    admitted: float
    inflight: int = 0


def _failed(req, admitted, now, msg):
    nan = float("nan")
    return SpectrumResult(req.rid, nan, nan, np.full(4, nan), np.zeros(0), np.zeros(0), np.zeros(0),
                          req.arrival, admitted, now, error=msg)


class SpectrumServer:
    def __init__(self, hbm_budget: int | None = None, chunk: int = 200, max_slots: int = 64,
                 autotune: bool = False, backend=None, state_fn=None, prep_workers: int = 2,
                 poll_s: float = 2e-4):
        """backend: the module with Sim, footprint, params_from_workload and
        IMRPError (the library binding by default; tests pass a fake);
        state_fn: workload -> (x, v) initial state; prep_workers: threads that
        draw initial states and create and load contexts."""
        self.lib = imrp if backend is None else backend
        self.state_fn = workload_state if state_fn is None else state_fn
        self.device = None
        if backend is None:
            import torch
            self.device = torch.cuda.current_device()
            if hbm_budget is None:
                free, _ = torch.cuda.mem_get_info()
                hbm_budget = int(0.8 * free)
        self.budget = hbm_budget
        self.chunk = chunk
        self.max_slots = max_slots
        self.autotune = autotune
        self.prep_workers = prep_workers
        self.poll_s = poll_s
        self.stats = {"chunks": 0, "max_active": 0, "peak_bytes": 0, "evicted": 0}

    def _on_device(self):
        if self.device is not None:
            import torch
            torch.cuda.set_device(self.device)

    def _prepare(self, req: SpectrumRequest):
        """Worker thread: initial state, context, load (and autotuning)."""
        self._on_device()
        x, v = self.state_fn(req.workload)
        sim = self.lib.Sim(self.lib.params_from_workload(req.workload))
        try:
            sim.load(x, v)
            if self.autotune:
                sim.autotune()
        except Exception:
            sim.close()
            raise
        return sim

    def _finish(self, slot: _Slot, clock):
        """Worker thread: spectrum, Q_diff read-back, free the context."""
        self._on_device()
        try:
            sp = slot.sim.spectrum(slot.req.n_freq, slot.req.w_max)
            q, _ = slot.sim.qdiff()
        except self.lib.IMRPError as e:
            slot.sim.close()
            return _failed(slot.req, slot.admitted, clock(), str(e))
        slot.sim.close()
        return SpectrumResult(slot.req.rid, sp["w_res"], sp["dw"], sp["fit"], sp["omega"], sp["reY"], q,
                              slot.req.arrival, slot.admitted, clock())

    def _launch(self, slot: _Slot):
        n = min(self.chunk, slot.remaining)
        slot.sim.step_async(n)  # a launch error is not one request's: it propagates
        slot.inflight = n
        self.stats["chunks"] += 1

    def serve(self, requests: list[SpectrumRequest], realtime: bool = True) -> list[SpectrumResult]:
        """realtime: requests arrive at their arrival times (else all at once,
        in arrival order). Latencies are measured from the arrival."""
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        waiting: collections.deque[SpectrumRequest] = collections.deque()
        preparing: dict[int, tuple] = {}
        active: dict[int, _Slot] = {}
        finishing: dict[int, tuple] = {}
        results: list[SpectrumResult] = []
        used = 0
        t0 = time.perf_counter()

        def clock():
            return time.perf_counter() - t0

        prep = cf.ThreadPoolExecutor(max_workers=self.prep_workers)
        fin = cf.ThreadPoolExecutor(max_workers=1)
        try:
            while pending or waiting or preparing or active or finishing:
                now = clock()
                while pending and (pending[0].arrival <= now or not realtime):
                    waiting.append(pending.popleft())
                # admission: FIFO, as long as a slot and the memory budget allow
                while waiting and len(active) + len(preparing) < self.max_slots:
                    req = waiting[0]
                    need = self.lib.footprint(self.lib.params_from_workload(req.workload), req.steps)
                    if used + need > self.budget and (active or preparing or finishing):
                        break
                    waiting.popleft()
                    used += need
                    preparing[req.rid] = (prep.submit(self._prepare, req), req, need, now)
                self.stats["peak_bytes"] = max(self.stats["peak_bytes"], used)
                progressed = False
                for rid, (fut, req, need, adm) in list(preparing.items()):
                    if not fut.done():
                        continue
                    del preparing[rid]
                    progressed = True
                    try:
                        sim = fut.result()
                    except self.lib.IMRPError as e:
                        results.append(_failed(req, adm, clock(), str(e)))
                        used -= need
                        self.stats["evicted"] += 1
                        continue
                    slot = _Slot(req, sim, req.steps, need, adm)
                    active[rid] = slot
                    self._launch(slot)
                self.stats["max_active"] = max(self.stats["max_active"], len(active))
                for rid, slot in list(active.items()):
                    if not slot.sim.ready():
                        continue
                    progressed = True
                    try:
                        slot.sim.sync()  # this context's device error flags
                    except self.lib.IMRPError as e:
                        del active[rid]
                        results.append(_failed(slot.req, slot.admitted, clock(), str(e)))
                        slot.sim.close()
                        used -= slot.footprint
                        self.stats["evicted"] += 1
                        continue
                    slot.remaining -= slot.inflight
                    slot.inflight = 0
                    if slot.remaining > 0:
                        self._launch(slot)
                    else:
                        del active[rid]
                        finishing[rid] = (fin.submit(self._finish, slot, clock), slot.footprint)
                for rid, (fut, fp) in list(finishing.items()):
                    if fut.done():
                        del finishing[rid]
                        used -= fp
                        results.append(fut.result())
                        progressed = True
                if not progressed:
                    if not (active or preparing or finishing) and pending and realtime:
                        time.sleep(max(0.0, min(pending[0].arrival - clock(), 0.05)))
                    else:
                        time.sleep(self.poll_s)
        finally:
            prep.shutdown(wait=True)
            fin.shutdown(wait=True)
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
