"""Serving loop: requests on resident simulations of different sizes overlap on
the device (several CUDA streams, continuous admission); every result equals
the one the same request sequence gives when run alone, and admission stops at
the HBM budget."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRIDS = ((64, 64, 65), (128, 128, 129), (32, 32, 33))


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2002_01392_gb300 import api as a
    assert torch.cuda.is_available()
    return a


def _params(api, g, nu):
    return api.ns_params(Nx=g[0], Ny=g[1], Nz=g[2], nu=nu, forcing_x=10 * nu, prec="f32")


def _fields(g, seed):
    v = synth.channel_velocity(g[0], g[1], g[2], nu=5e-3, seed_offset=seed)
    return torch.from_numpy(v.astype(np.float32)).cuda()


def _setup(api, serve, budget):
    srv = serve.Server(budget, slots=6)
    sims, grids = [], []
    for i in range(6):
        g = GRIDS[i % len(GRIDS)]
        sid = srv.admit(_params(api, g, 5e-3), _fields(g, 50 + i))
        sims.append(sid)
        grids.append(g)
    return srv, sims, grids


def test_mix_equals_alone(api):
    from paper_2002_01392_gb300 import serve
    srv, sims, grids = _setup(api, serve, 1 << 40)
    rng = np.random.default_rng(7)
    reqs = serve.poisson_requests(4000.0, 0.02, sims, rng, kinds=("project", "step", "rhs"), dt=5e-4)
    assert len(reqs) > 40
    # inputs of rhs / project requests: seeded fields of the target's grid
    for k, r in enumerate(reqs):
        if r.kind != "step":
            g = grids[r.sim]
            f = _fields(g, 500 + k)
            r.inp = f if r.kind == "rhs" else f[:3].contiguous()
    stats = srv.run(reqs)
    assert stats["requests"] == len(reqs) and stats["p99_latency_ms"] >= stats["p50_latency_ms"] > 0
    mixed_final = [srv.sims[s].get_fields() for s in sims]
    # alone: a fresh server replays each simulation's requests in order, one at a time
    alone, sims2, _ = _setup(api, serve, 1 << 40)
    for sid in sims2:
        sim = alone.sims[sid]
        for r in (r for r in reqs if r.sim == sid):
            if r.kind == "step":
                sim.step(r.dt)
            elif r.kind == "project":
                out = sim.project(r.inp, r.dt)
                assert torch.equal(out, r.out)
            else:
                assert torch.equal(sim.rhs(r.inp), r.out)
        assert torch.equal(sim.get_fields(), mixed_final[sid])
    srv.close()
    alone.close()


def test_admission_by_hbm_footprint(api):
    from paper_2002_01392_gb300 import serve
    one = api.ns_workspace_bytes(_params(api, GRIDS[1], 5e-3))
    srv = serve.Server(int(2.5 * one), slots=2)
    ids = [srv.admit(_params(api, GRIDS[1], 5e-3)) for _ in range(3)]
    assert ids[:2] == [0, 1] and ids[2] is None and srv.rejected == 1
    srv.release(0)
    assert srv.admit(_params(api, GRIDS[1], 5e-3)) is not None
    srv.close()
