"""Continuous-batching server for stability-sweep runs.

Requests (a channel size, the groups T, C, M, Fe, Lambda, an Eq. 29
perturbation and a step budget) arrive over time.  The server keeps every
admitted run's populations resident on the GPU, admits a waiting request as
soon as a batch slot is free and its device footprint (``ehd_footprint``)
fits the HBM budget -- the batch itself keeps that account behind the C ABI
(``ehd_batch_create`` takes the budget, ``ehd_batch_admits`` answers before a
run is allocated, ``ehd_batch_add`` refuses with EHD_EBUSY) -- and advances all admitted runs together, tick by tick,
through one :class:`~paper_1812_05711_gb300.Batch`.  A run leaves at the end
of the tick in which its budget is used up; its result (the final
diagnostics and, optionally, fields) is recorded with its latency
(completion minus arrival).  Requests that arrive while others run join the
next tick: their work overlaps on the device with the runs already in flight.

Each run's result is the one it gets alone (the batch kernels apply the
single-run arithmetic per run), which ``tests/test_gpu_serve.py`` checks.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import STORAGE, Batch, Run, ehd_footprint

OK, EINVAL, EBUSY = 0, -1, -6  # ehd_status values of the batch's admission query


@dataclass
class Request:
    rid: int
    Nx: int
    Ny: int
    T: float
    C: float
    M: float
    Fe: float
    Lambda: float
    steps: int
    amp: list = field(default_factory=list)
    phase: list = field(default_factory=list)
    arrival: float = 0.0  # seconds after the start of the stream
    # the last `window` steps of the budget are a measurement window: the
    # collected charge over them (FP64 wall fluxes) is reported per step
    window: int = 0
    # start from the final populations of request `after` (which must keep
    # its state); the request waits until that one has finished
    after: int | None = None
    keep_state: bool = False  # report the final populations (f, g)
    u_ion: float | None = None  # lattice ion drift speed (None: the server's)
    # 1: the FP32 perturbation form (charge populations as the departure from
    # an FP64 x-uniform base state: growth rates of small rolls as in FP64)
    perturbation: int = 0


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    done: float
    steps: int
    diagnostics: dict
    fields: dict | None = None
    current: float | None = None  # collected charge per step over the window
    state: tuple | None = None    # (f, g) when keep_state

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class Server:
    """Continuous batching over one GPU.

    hbm_budget: bytes of device memory the resident runs may hold.
    tick_steps: even number of steps every admitted run advances per tick.
    """

    def __init__(self, hbm_budget: int, max_runs: int = 256, tick_steps: int = 200, max_nx: int = 1024,
                 max_ny: int = 840, u_ion: float = 2e-3, keep_fields=(), clock=time.perf_counter):
        if tick_steps < 2 or tick_steps % 2:
            raise ValueError("tick_steps must be even and >= 2")
        self.batch = Batch(max_runs, max_nx=max_nx, max_ny=max_ny, hbm_budget=int(hbm_budget))
        self.max_runs, self.max_nx, self.max_ny = max_runs, max_nx, max_ny
        self.hbm_budget, self.tick_steps, self.u_ion = int(hbm_budget), int(tick_steps), u_ion
        self.keep_fields = tuple(keep_fields)
        self.clock = clock
        self.waiting = collections.deque()
        self.active = {}   # run handle -> (request, run, admitted time)
        self.windows = {}  # run handle -> q_out at the start of its measurement window
        self.states = {}   # rid -> final (f, g) of finished requests that others continue from
        self.done_ids = set()
        self.results = []
        self.t0 = None
        self.ticks = 0

    # ------------------------------------------------------------ intake
    def footprint(self, req: Request) -> int:
        return ehd_footprint(req.Nx, req.Ny, STORAGE["f32"])

    @property
    def used(self) -> int:
        """Bytes the admitted runs hold, as the batch accounts them."""
        return self.batch.memory()[0]

    def submit(self, req: Request):
        if req.Nx > self.max_nx or req.Ny > self.max_ny or req.Nx < 64:
            raise ValueError(f"request {req.rid}: grid {req.Nx}x{req.Ny} outside the server limits")
        if self.batch.admits(req.Nx, req.Ny) == EINVAL:
            raise ValueError(f"request {req.rid}: footprint exceeds the whole HBM budget")
        if not 0 <= req.window <= req.steps:
            raise ValueError(f"request {req.rid}: window outside the step budget")
        if req.after is not None:
            pred = next((q for q in self.waiting if q.rid == req.after), None)
            if pred is None and req.after not in self.done_ids:
                raise ValueError(f"request {req.rid}: continues from unknown request {req.after}")
            if pred is not None:
                if (pred.Nx, pred.Ny) != (req.Nx, req.Ny):
                    raise ValueError(f"request {req.rid}: grid differs from request {req.after}")
                pred.keep_state = True
        self.waiting.append(req)

    def _now(self) -> float:
        return self.clock() - self.t0

    def _ready(self, req: Request, now: float) -> bool:
        return req.arrival <= now and (req.after is None or req.after in self.done_ids)

    def _admit(self, now: float):
        # first come, first served among the requests that may start (arrived,
        # and the request they continue from has finished): the first of those
        # that does not fit makes the rest wait for a slot or memory
        for req in list(self.waiting):
            if len(self.active) >= self.max_runs:
                break
            if not self._ready(req, now):
                if req.arrival > now:
                    break
                continue  # waits for its predecessor; later requests may go ahead
            if self.batch.admits(req.Nx, req.Ny) != OK:
                break
            self.waiting.remove(req)
            u_ion = self.u_ion if req.u_ion is None else req.u_ion
            cont = req.after is not None
            run = Run(req.Nx, req.Ny, req.T, req.C, req.M, req.Fe, req.Lambda, storage="f32",
                      u_ion=u_ion, amp=[] if cont else req.amp, phase=[] if cont else req.phase,
                      perturbation=req.perturbation)
            if cont:
                run.load(*self.states.pop(req.after))
            first = req.steps - req.window if req.window else req.steps
            self.batch.add(run, first)  # the batch accounts the run's footprint
            self.active[run.handle] = (req, run, now)
            if req.window and first == 0:
                self.windows[run.handle] = run.diagnostics()["q_out"]
                self.batch.remove(run)
                self.batch.add(run, req.window)

    def _retire(self, now: float):
        for h in [h for h, (req, run, _) in self.active.items() if self.batch.remaining(run) == 0]:
            req, run, t_adm = self.active[h]
            if req.window and h not in self.windows:
                # the budget before the measurement window is used up: note the
                # collected charge so far and give the run its window (it stays
                # resident in its slot)
                self.windows[h] = run.diagnostics()["q_out"]
                self.batch.remove(run)
                self.batch.add(run, req.window)
                continue
            del self.active[h]
            self.batch.remove(run)
            diag = run.diagnostics()
            flds = run.fields(self.keep_fields) if self.keep_fields else None
            cur = (diag["q_out"] - self.windows.pop(h)) / req.window if req.window else None
            st = run.save() if req.keep_state else None
            if st is not None:
                self.states[req.rid] = st
            self.results.append(Result(req.rid, req.arrival, t_adm, now, req.steps, diag, flds, cur, st))
            self.done_ids.add(req.rid)
            run.close()

    # --------------------------------------------------------------- loop
    def step(self) -> bool:
        """One scheduling round: admit, tick, retire.  False when idle."""
        now = self._now()
        self._admit(now)
        if not self.active:
            return False
        self.batch.tick(self.tick_steps)
        self.batch.sync()
        self.ticks += 1
        self._retire(self._now())
        return True

    def serve(self, requests, realtime: bool = True):
        """Run a whole arrival stream (requests sorted by arrival time);
        returns the results in completion order."""
        for r in sorted(requests, key=lambda q: q.arrival):
            self.submit(r)
        self.t0 = self.clock()
        if not realtime:  # every request has arrived at time 0
            for r in self.waiting:
                r.arrival = 0.0
        while self.waiting or self.active:
            if not self.step() and self.waiting:
                nxt = self.waiting[0].arrival
                wait = nxt - self._now()
                if wait > 0:
                    time.sleep(min(wait, 0.05))
        return self.results

    def close(self):
        for req, run, _ in list(self.active.values()):
            self.batch.remove(run)
            run.close()
        self.active.clear()
        self.batch.close()


def summarize(results, cells_of=None) -> dict:
    lat = np.array([r.latency for r in results])
    makespan = max(r.done for r in results) - min(r.arrival for r in results)
    out = {"runs": len(results), "makespan_s": makespan, "runs_per_s": len(results) / makespan,
           "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
           "mean_s": float(lat.mean())}
    if cells_of is not None:
        out["glups"] = sum(cells_of(r) * r.steps for r in results) / makespan / 1e9
    return out


def serve_plain_fp64(requests, realtime: bool = True, clock=time.perf_counter):
    """The comparison path: each request alone, in arrival order, on the plain
    double-precision path (FP64 storage and compute, one run at a time)."""
    t0 = clock()
    results = []
    for req in sorted(requests, key=lambda q: q.arrival):
        if realtime:
            wait = req.arrival - (clock() - t0)
            if wait > 0:
                time.sleep(wait)
        t_adm = clock() - t0
        run = Run(req.Nx, req.Ny, req.T, req.C, req.M, req.Fe, req.Lambda, storage="f64", amp=req.amp,
                  phase=req.phase)
        run.step(req.steps)
        diag = run.diagnostics()
        run.close()
        results.append(Result(req.rid, req.arrival if realtime else 0.0, t_adm, clock() - t0, req.steps, diag))
    return results
