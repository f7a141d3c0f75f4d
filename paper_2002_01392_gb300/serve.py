"""Request loop over resident simulations (continuous batching on CUDA streams).

Requests (ns_rhs, fc_poisson_project, rk_step) arrive at given times for
simulations that stay resident on the device with their FC tables.  New
simulations are admitted while their workspace (``ns_workspace_bytes``) fits
in the HBM budget.  Each request runs on one of ``slots`` CUDA streams as soon
as a stream is free and no earlier request for the same simulation is still
in flight (requests of one simulation keep their arrival order; different
simulations overlap on the device).  Completion is observed with CUDA events,
so latencies are arrival-to-completion on the host clock.

This module only orchestrates calls of the C ABI (through ``api``); every
step of the work runs in the library's kernels.
"""
from __future__ import annotations

import collections
import dataclasses
import time

from . import api


@dataclasses.dataclass
class Request:
    kind: str                 # "rhs" | "project" | "step"
    sim: int                  # resident simulation id
    arrival: float = 0.0      # seconds from the start of the run
    dt: float = 1e-3
    inp: object = None        # device tensor for rhs / project (physical fields)
    out: object = None        # filled for rhs / project
    t_start: float = -1.0
    t_done: float = -1.0


class Server:
    def __init__(self, hbm_budget_bytes: int, slots: int = 8):
        import torch
        self.torch = torch
        self.budget = int(hbm_budget_bytes)
        self.used = 0
        self.sims: dict[int, api.Sim] = {}
        self.points: dict[int, int] = {}
        self.rejected = 0
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.busy: list[tuple[Request, object] | None] = [None] * slots
        self.inflight_sims: set[int] = set()

    # -- admission -------------------------------------------------------
    def admit(self, params, fields=None) -> int | None:
        """Create a resident simulation if its workspace fits; returns its id
        or None (counted as a rejection)."""
        need = api.ns_workspace_bytes(params)
        if self.used + need > self.budget:
            self.rejected += 1
            return None
        sim = api.Sim(params)
        sid = len(self.sims)
        self.sims[sid] = sim
        self.used += need
        self.points[sid] = params.Nx * params.Ny * params.Nz
        if fields is not None:
            sim.set_fields(fields)
        return sid

    def release(self, sid: int):
        sim = self.sims.pop(sid)
        self.used -= api.ns_workspace_bytes(sim.p)
        sim.close()

    # -- execution -------------------------------------------------------
    def _launch(self, r: Request, slot: int, t0: float):
        torch = self.torch
        s = self.streams[slot]
        sim = self.sims[r.sim]
        h = torch.cuda.current_stream()
        s.wait_stream(h)                    # inputs written on the caller's stream
        with torch.cuda.stream(s):
            if r.kind == "step":
                sim.step(r.dt, stream=s)
            elif r.kind == "project":
                r.out = sim.project(r.inp, r.dt, stream=s)
            elif r.kind == "rhs":
                r.out = sim.rhs(r.inp, stream=s)
            else:
                raise ValueError(r.kind)
            ev = torch.cuda.Event()
            ev.record(s)
        r.t_start = time.perf_counter() - t0
        self.busy[slot] = (r, ev)
        self.inflight_sims.add(r.sim)

    def _reap(self, t0: float, done: list):
        for k, b in enumerate(self.busy):
            if b is not None and b[1].query():
                r = b[0]
                r.t_done = time.perf_counter() - t0
                done.append(r)
                self.inflight_sims.discard(r.sim)
                self.busy[k] = None

    def run(self, requests: list[Request]) -> dict:
        """Serve the requests (sorted by arrival time) in real time; returns
        latency and throughput statistics."""
        torch = self.torch
        reqs = sorted(requests, key=lambda r: r.arrival)
        pending: collections.deque[Request] = collections.deque()
        done: list[Request] = []
        i = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while len(done) < len(reqs):
            now = time.perf_counter() - t0
            while i < len(reqs) and reqs[i].arrival <= now:
                pending.append(reqs[i])
                i += 1
            self._reap(t0, done)
            # dispatch in arrival order; a request waits while its simulation is in flight
            blocked: set[int] = set()
            for _ in range(len(pending)):
                r = pending.popleft()
                if r.sim in self.inflight_sims or r.sim in blocked:
                    blocked.add(r.sim)
                    pending.append(r)
                    continue
                free = next((k for k, b in enumerate(self.busy) if b is None), None)
                if free is None:
                    pending.appendleft(r)
                    break
                self._launch(r, free, t0)
        wall = time.perf_counter() - t0
        lat = sorted(r.t_done - r.arrival for r in done)
        pts = sum(self.points[r.sim] * (3 if r.kind == "step" else 1) for r in done)
        pick = lambda q: lat[min(len(lat) - 1, int(q * len(lat)))]
        return {"requests": len(done), "wall_s": wall, "p50_latency_ms": pick(0.5) * 1e3,
                "p99_latency_ms": pick(0.99) * 1e3, "grid_points_per_s": pts / wall,
                "requests_per_s": len(done) / wall, "rejected_admissions": self.rejected,
                "resident": len(self.sims), "hbm_used_GB": self.used / 1e9}

    def close(self):
        for sid in list(self.sims):
            self.release(sid)


def poisson_requests(rate: float, duration: float, sims: list[int], rng, kinds=("project", "step"),
                     dt: float = 1e-3) -> list[Request]:
    """Poisson arrivals of mean ``rate`` per second over ``duration`` seconds,
    kind and target simulation drawn uniformly."""
    out, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            return out
        out.append(Request(kind=kinds[int(rng.integers(len(kinds)))], sim=int(sims[int(rng.integers(len(sims)))]),
                           arrival=t, dt=dt))
