"""Host logic of the serving loop without a GPU: admission by footprint,
per-simulation arrival order, retries of transient failures, quarantine after a
non-finite check, immediate failure of other errors.  The CUDA streams / events
and the simulations are stand-ins that run each request when it is launched."""
import contextlib

import pytest


class FakeCuda:
    class Stream:
        def wait_stream(self, other):
            pass

    class Event:
        def record(self, stream=None):
            pass

        def query(self):
            return True

    @staticmethod
    def current_stream():
        return None

    @staticmethod
    def stream(s):
        return contextlib.nullcontext()

    @staticmethod
    def synchronize():
        pass


class FakeError(RuntimeError):
    def __init__(self, name):
        super().__init__(name)
        self.name = name


class FakeParams:
    def __init__(self, nbytes, Nx=8, Ny=8, Nz=9, failures=None):
        self.nbytes, self.Nx, self.Ny, self.Nz = nbytes, Nx, Ny, Nz
        self.failures = list(failures or [])    # status names raised by the next calls, in order


class FakeLib:
    FcError = FakeError
    log = []

    @staticmethod
    def ns_workspace_bytes(p):
        return p.nbytes

    class Sim:
        count = 0

        def __init__(self, p):
            self.p = p
            self.id = FakeLib.Sim.count
            FakeLib.Sim.count += 1
            self.checks = 0

        def _run(self, what):
            if self.p.failures:
                st = self.p.failures.pop(0)
                if st:
                    raise FakeError(st)
            FakeLib.log.append((self.id, what))

        def step(self, dt, stream=None):
            self._run(("step", dt))

        def project(self, inp, dt, stream=None):
            self._run(("project", dt))
            return "projected"

        def rhs(self, inp, stream=None):
            self._run(("rhs", None))
            return "rhs"

        def tune(self, mode):
            return [0] * 5

        def set_finite_check(self, every):
            self.checks = every

        def set_fields(self, f):
            pass

        def close(self):
            pass


@pytest.fixture()
def serve():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2002_01392_gb300 import serve as s
    FakeLib.log = []
    FakeLib.Sim.count = 0
    return s


def _server(serve, budget=100, **kw):
    return serve.Server(budget, slots=3, cuda=FakeCuda, lib=FakeLib, **kw)


def test_admission_by_footprint(serve):
    srv = _server(serve, budget=100)
    assert srv.admit(FakeParams(40)) == 0 and srv.admit(FakeParams(40)) == 1
    assert srv.admit(FakeParams(40)) is None and srv.rejected == 1
    srv.release(0)
    assert srv.admit(FakeParams(60)) is not None and srv.used == 100
    srv.close()
    assert srv.used == 0


def test_arrival_order_per_simulation(serve):
    srv = _server(serve, budget=10 ** 9, check_every=1)
    a, b = srv.admit(FakeParams(1)), srv.admit(FakeParams(1))
    assert all(s.checks == 1 for s in srv.sims.values())
    reqs = [serve.Request(kind=k, sim=(a if i % 3 else b), arrival=0.0, dt=1e-3 * (i + 1))
            for i, k in enumerate(["step", "project", "rhs", "step", "project", "step", "rhs", "step"])]
    stats = srv.run(reqs)
    assert stats["requests"] == len(reqs) and stats["failed"] == 0 and stats["retried"] == 0
    for sid in (a, b):
        mine = [r for r in reqs if r.sim == sid]
        got = [w for (s, w) in FakeLib.log if s == sid]
        assert got == [(r.kind, None if r.kind == "rhs" else r.dt) for r in mine]
    assert [r.out for r in reqs if r.kind == "project"] == ["projected"] * 2


def test_transient_failures_are_retried(serve):
    srv = _server(serve, budget=10 ** 9, max_retries=2)
    s0 = srv.admit(FakeParams(1, failures=["FC_ERR_CUDA", "FC_ERR_TIMEOUT"]))
    s1 = srv.admit(FakeParams(1, failures=["FC_ERR_NOMEM", "FC_ERR_NOMEM", "FC_ERR_NOMEM"]))
    reqs = [serve.Request(kind="step", sim=s0, arrival=0.0), serve.Request(kind="step", sim=s1, arrival=0.0),
            serve.Request(kind="step", sim=s1, arrival=0.0)]
    stats = srv.run(reqs)
    assert reqs[0].error is None and reqs[0].attempts == 2          # two retries, then done
    assert reqs[1].error == "FC_ERR_NOMEM" and reqs[1].attempts == 2  # third failure: given up
    assert reqs[2].error is None                                     # the simulation serves on
    assert stats["retried"] == 4 and stats["failed"] == 1 and stats["quarantined"] == 0


def test_nonfinite_quarantines_and_other_errors_fail_at_once(serve):
    srv = _server(serve, budget=10 ** 9)
    bad = srv.admit(FakeParams(1, failures=[None, "FC_ERR_NONFINITE"]))
    odd = srv.admit(FakeParams(1, failures=["FC_ERR_ARG"]))
    good = srv.admit(FakeParams(1))
    reqs = [serve.Request(kind="step", sim=bad, arrival=0.0) for _ in range(4)]
    reqs += [serve.Request(kind="step", sim=odd, arrival=0.0), serve.Request(kind="step", sim=good, arrival=0.0)]
    stats = srv.run(reqs)
    assert [r.error for r in reqs[:4]] == [None, "FC_ERR_NONFINITE", "FC_ERR_NONFINITE", "FC_ERR_NONFINITE"]
    assert [s for (s, _) in FakeLib.log].count(bad) == 1              # quarantined requests never ran
    assert reqs[4].error == "FC_ERR_ARG" and reqs[4].attempts == 0
    assert reqs[5].error is None
    assert stats["quarantined"] == 1 and stats["failed"] == 4 and stats["retried"] == 0


def test_admission_and_release_while_running(serve):
    """A simulation that arrives while the loop runs is admitted once a release
    frees enough of the budget; requests naming it wait for it; a release waits
    for the simulation's earlier requests; an admission that can never fit
    fails with FC_ERR_NOMEM and requests naming it with FC_ERR_STATE, as do
    requests for a simulation already released."""
    srv = _server(serve, budget=100)
    a = srv.admit(FakeParams(60))
    reqs = [serve.Request(kind="step", sim=a, arrival=0.0, dt=1.0),
            serve.Request(kind="admit", sim="B", arrival=0.0, params=FakeParams(60)),
            serve.Request(kind="step", sim="B", arrival=0.0, dt=2.0),
            serve.Request(kind="release", sim=a, arrival=0.0),
            serve.Request(kind="step", sim="B", arrival=0.0, dt=3.0),
            serve.Request(kind="admit", sim="C", arrival=0.0, params=FakeParams(200)),
            serve.Request(kind="step", sim="C", arrival=0.0),
            serve.Request(kind="step", sim=a, arrival=0.001)]
    stats = srv.run(reqs)
    assert [r.error for r in reqs[:5]] == [None] * 5
    b = srv.names["B"]
    assert [w for (s, w) in FakeLib.log if s == a] == [("step", 1.0)]
    assert [w for (s, w) in FakeLib.log if s == b] == [("step", 2.0), ("step", 3.0)]
    assert reqs[5].error == "FC_ERR_NOMEM" and reqs[6].error == "FC_ERR_STATE"
    assert reqs[7].error == "FC_ERR_STATE"
    assert stats["admitted_midrun"] == 1 and stats["released_midrun"] == 1
    assert srv.used == 60 and list(srv.sims) == [b]
    srv.close()


def test_wall_limit_times_out_unlaunched_requests(serve):
    """With max_wall_s = 0 every request not yet launched completes at once
    with FC_ERR_TIMEOUT (nothing is launched)."""
    srv = _server(serve, budget=10 ** 9)
    sid = srv.admit(FakeParams(1))
    reqs = [serve.Request(kind="step", sim=sid, arrival=0.0) for _ in range(5)]
    st = srv.run(reqs, max_wall_s=0.0)
    assert st["requests"] == 5 and st["failed"] == 5
    assert all(r.error == "FC_ERR_TIMEOUT" for r in reqs)
    assert not [w for (s, w) in FakeLib.log if s == sid]
