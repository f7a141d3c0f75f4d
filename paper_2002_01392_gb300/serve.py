"""Request loop over resident simulations (continuous batching on CUDA streams).

Requests (ns_rhs, fc_poisson_project, rk_step) arrive at given times for
simulations that stay resident on the device with their FC tables.  New
simulations are admitted while their workspace (``ns_workspace_bytes``) fits
in the HBM budget (and get the kernel variants the autotuner of ``ns_tune``
picks for their size).  Each request runs on one of ``slots`` CUDA streams as soon
as a stream is free and no earlier request for the same simulation is still
in flight (requests of one simulation keep their arrival order; different
simulations overlap on the device).  Completion is observed with CUDA events,
so latencies are arrival-to-completion on the host clock.

Simulations can also arrive and leave while the loop runs: an "admit"
request (params, initial fields, and a name in ``sim``) creates the
simulation as soon as its workspace fits in what the resident simulations
leave of the HBM budget, waiting for releases if it does not fit yet; a
"release" request frees a simulation once its earlier requests are done.
Later requests may name a simulation admitted mid-run by the name of its
admission; they wait for it.  An admission that can never fit (nothing left
to release) fails with FC_ERR_NOMEM.

Errors: a request whose call fails with FC_ERR_CUDA, FC_ERR_NOMEM or
FC_ERR_TIMEOUT is requeued at the head of the queue, up to ``max_retries``
times (a failing call enqueues nothing that changes the simulation's state:
an RK step only replaces the state when all its stages were enqueued).  Other
errors complete the request with ``error`` set.  With ``check_every`` > 0 the
resident simulations check their state for non-finite values after every
``check_every``-th step (``ns_set_finite_check``); a simulation whose check
failed is quarantined: its later requests complete at once with
``error = "FC_ERR_NONFINITE"``.

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
    kind: str                 # "rhs" | "project" | "step" | "admit" | "release"
    sim: object               # resident simulation id, or the name given at its mid-run admission
    arrival: float = 0.0      # seconds from the start of the run
    dt: float = 1e-3
    inp: object = None        # device tensor for rhs / project (physical fields)
    out: object = None        # filled for rhs / project
    t_start: float = -1.0
    t_done: float = -1.0
    attempts: int = 0         # retries taken
    error: str | None = None  # status name when the request failed
    params: object = None     # "admit": the simulation's ns_params (inp: its initial fields or None)
    points: int = 0           # grid points of the simulation it ran on (set at launch)
    sid: int | None = None    # the simulation id it ran on (set at launch)


RETRYABLE = ("FC_ERR_CUDA", "FC_ERR_NOMEM", "FC_ERR_TIMEOUT")


class Server:
    def __init__(self, hbm_budget_bytes: int, slots: int = 8, max_retries: int = 2, check_every: int = 0,
                 tune: bool = True, cuda=None, lib=None):
        """cuda: the stream / event provider (torch.cuda unless given); lib: the
        binding module (``api`` unless given) -- both replaceable so that the
        host logic can be exercised without a GPU."""
        if cuda is None:
            import torch
            cuda = torch.cuda
        self.cuda = cuda
        self.lib = lib if lib is not None else api
        self.tune = tune
        self.budget = int(hbm_budget_bytes)
        self.max_retries = int(max_retries)
        self.check_every = int(check_every)
        self.retried = 0
        self.failed = 0
        self.quarantined: set[int] = set()
        self.used = 0
        self.sims: dict = {}
        self._next_id = 0
        self.points: dict[int, int] = {}
        self.rejected = 0
        self.streams = [cuda.Stream() for _ in range(slots)]
        self.busy: list[tuple[Request, object] | None] = [None] * slots
        self.inflight_sims: set[int] = set()
        self.names: dict = {}          # name of a mid-run admission -> simulation id
        self.admitted_midrun = 0
        self.released_midrun = 0

    # -- admission -------------------------------------------------------
    def admit(self, params, fields=None) -> int | None:
        """Create a resident simulation if its workspace fits; returns its id
        or None (counted as a rejection)."""
        need = self.lib.ns_workspace_bytes(params)
        if self.used + need > self.budget:
            self.rejected += 1
            return None
        sim = self.lib.Sim(params)
        if self.tune:
            sim.tune(1)     # kernel variants timed once per grid size (cached)
        sid = self._next_id  # ids are never reused (a released id may still name old requests)
        self._next_id += 1
        self.sims[sid] = sim
        self.used += need
        self.points[sid] = params.Nx * params.Ny * params.Nz
        if fields is not None:
            sim.set_fields(fields)
        if self.check_every > 0:
            sim.set_finite_check(self.check_every)
        return sid

    def release(self, sid: int):
        sim = self.sims.pop(sid)
        self.used -= self.lib.ns_workspace_bytes(sim.p)
        sim.close()

    # -- execution -------------------------------------------------------
    def _launch(self, r: Request, slot: int, t0: float, sid: int):
        """Enqueue r on stream ``slot``; returns the library error of the call
        (nothing is marked busy then) or None."""
        cuda = self.cuda
        s = self.streams[slot]
        sim = self.sims[sid]
        r.points = self.points[sid]
        h = cuda.current_stream()
        s.wait_stream(h)                    # inputs written on the caller's stream
        try:
            with cuda.stream(s):
                if r.kind == "step":
                    sim.step(r.dt, stream=s)
                elif r.kind == "project":
                    r.out = sim.project(r.inp, r.dt, stream=s)
                elif r.kind == "rhs":
                    r.out = sim.rhs(r.inp, stream=s)
                else:
                    raise ValueError(r.kind)
                ev = cuda.Event()
                ev.record(s)
        except self.lib.FcError as e:
            return e
        r.t_start = time.perf_counter() - t0
        self.busy[slot] = (r, ev)
        self.inflight_sims.add(sid)
        r.sid = sid
        return None

    def _fail(self, r: Request, name: str, t0: float, done: list):
        r.error = name
        r.t_done = time.perf_counter() - t0
        self.failed += 1
        if name == "FC_ERR_NONFINITE":
            sid = self._resolve(r)
            if sid is not None:
                self.quarantined.add(sid)
        done.append(r)

    def _reap(self, t0: float, done: list):
        for k, b in enumerate(self.busy):
            if b is not None and b[1].query():
                r = b[0]
                r.t_done = time.perf_counter() - t0
                done.append(r)
                self.inflight_sims.discard(r.sid)
                self.busy[k] = None

    def _resolve(self, r: Request):
        """The simulation id a request refers to (None: named, not admitted yet)."""
        if r.kind == "admit":
            return None
        if isinstance(r.sim, int) and r.sim in self.sims:
            return r.sim
        return self.names.get(r.sim)

    def _admit_or_release(self, r: Request, sid, t0: float, done: list) -> bool:
        """Handle an "admit" / "release" request now if it can run; returns
        False if it must wait (admission: not enough budget yet)."""
        if r.kind == "admit":
            if self.used + self.lib.ns_workspace_bytes(r.params) > self.budget:
                return False
            new = self.admit(r.params, r.inp)
            self.names[r.sim] = new
            self.admitted_midrun += 1
        else:
            self.release(sid)
            self.released_midrun += 1
        r.t_start = r.t_done = time.perf_counter() - t0
        done.append(r)
        return True

    def run(self, requests: list[Request], max_wall_s: float | None = None) -> dict:
        """Serve the requests (sorted by arrival time) in real time; returns
        latency and throughput statistics.  With ``max_wall_s``, requests not
        yet launched when that much time has passed complete at once with
        ``error = "FC_ERR_TIMEOUT"`` (those in flight still finish)."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        pending: collections.deque[Request] = collections.deque()
        done: list[Request] = []
        i = 0
        self.cuda.synchronize()
        t0 = time.perf_counter()
        while len(done) < len(reqs):
            now = time.perf_counter() - t0
            if max_wall_s is not None and now > max_wall_s:
                while i < len(reqs):
                    pending.append(reqs[i])
                    i += 1
                while pending:
                    self._fail(pending.popleft(), "FC_ERR_TIMEOUT", t0, done)
                self._reap(t0, done)
                if len(done) < len(reqs):
                    time.sleep(1e-4)
                continue
            while i < len(reqs) and reqs[i].arrival <= now:
                pending.append(reqs[i])
                i += 1
            self._reap(t0, done)
            # dispatch in arrival order; a request waits while its simulation is in
            # flight, or (named) not admitted yet, or behind an earlier request for it
            blocked: set = set()
            progress = False
            for _ in range(len(pending)):
                r = pending.popleft()
                key = r.sim
                sid = self._resolve(r)
                if sid is None and r.kind != "admit" and isinstance(key, int):
                    self._fail(r, "FC_ERR_STATE", t0, done)     # no such resident simulation
                    progress = True
                    continue
                if key in blocked or (sid is not None and sid in self.inflight_sims) or \
                        (sid is None and r.kind != "admit"):
                    blocked.add(key)
                    pending.append(r)
                    continue
                if r.kind in ("admit", "release"):
                    if self._admit_or_release(r, sid, t0, done):
                        progress = True
                    else:
                        blocked.add(key)
                        pending.append(r)
                    continue
                if sid in self.quarantined:
                    self._fail(r, "FC_ERR_NONFINITE", t0, done)
                    continue
                free = next((k for k, b in enumerate(self.busy) if b is None), None)
                if free is None:
                    pending.appendleft(r)
                    break
                err = self._launch(r, free, t0, sid)
                progress = True
                if err is None:
                    continue
                if err.name in RETRYABLE and r.attempts < self.max_retries:
                    r.attempts += 1
                    self.retried += 1
                    pending.appendleft(r)
                else:
                    self._fail(r, err.name, t0, done)
            # nothing in flight, nothing still to arrive and nothing dispatched in
            # this pass: what is left waits for an admission that cannot fit
            # (FC_ERR_NOMEM) or names a simulation never admitted (FC_ERR_STATE)
            if pending and not progress and i == len(reqs) and all(b is None for b in self.busy):
                for r in list(pending):
                    pending.remove(r)
                    self._fail(r, "FC_ERR_NOMEM" if r.kind == "admit" else "FC_ERR_STATE", t0, done)
        wall = time.perf_counter() - t0
        ok = [r for r in done if r.error is None and r.kind not in ("admit", "release")]
        lat = sorted(r.t_done - r.arrival for r in ok) or [0.0]
        pts = sum(r.points * (3 if r.kind == "step" else 1) for r in ok)
        pick = lambda q: lat[min(len(lat) - 1, int(q * len(lat)))]
        return {"requests": len(done), "wall_s": wall, "p50_latency_ms": pick(0.5) * 1e3,
                "p99_latency_ms": pick(0.99) * 1e3, "grid_points_per_s": pts / wall,
                "requests_per_s": len(ok) / wall, "rejected_admissions": self.rejected,
                "failed": self.failed, "retried": self.retried, "quarantined": len(self.quarantined),
                "resident": len(self.sims), "hbm_used_GB": self.used / 1e9,
                "admitted_midrun": self.admitted_midrun, "released_midrun": self.released_midrun}

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
