"""Batched ensemble (independent channel instances of uneven sizes advanced by
one CUDA graph launch per step) on the GPU: bitwise equal to stepping each
member alone, and a float64 member against the oracle."""
import numpy as np
import pytest

from oracle import ns
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2002_01392_gb300 import api as a
    assert torch.cuda.is_available()
    return a


def _make(api, spec, prec):
    p = api.ns_params(Nx=spec["Nx"], Ny=spec["Ny"], Nz=spec["Nz"], nu=spec["nu"],
                      forcing_x=10 * spec["nu"], prec=prec)
    sim = api.Sim(p)
    v = synth.channel_velocity(spec["Nx"], spec["Ny"], spec["Nz"], nu=spec["nu"], seed_offset=spec["seed_offset"])
    sim.set_fields(torch.from_numpy(v).to("cuda", sim.dtype))
    return sim, v


def test_batch_equals_members_alone(api):
    specs = synth.ensemble_specs(8)
    assert len({(s["Nx"], s["Nz"]) for s in specs}) >= 3          # uneven sizes
    alone = [_make(api, s, "f32")[0] for s in specs]
    batched = [_make(api, s, "f32")[0] for s in specs]
    dts = [2e-4 * (1 + i % 3) for i in range(len(specs))]
    b = api.Batch(batched)      # autotunes every member (tiles and radix schedules)
    for a_ in alone:            # the same choices (cached per size) for the members run alone
        a_.tune(1)
    for _ in range(4):
        for sim, dt in zip(alone, dts):
            sim.step(dt)
        b.step(dts)
    torch.cuda.synchronize()
    for a_, b_ in zip(alone, batched):
        assert torch.equal(a_.get_fields(), b_.get_fields())
        assert torch.equal(a_.wall_gradp(), b_.wall_gradp())
    info = b.info()
    assert info["members"] == len(specs) and info["graphs_cached"] <= 3 and info["graph_nodes"] >= 7 * len(specs)
    b.close()
    for s in alone + batched:
        s.close()


def test_batch_float64_member_matches_oracle(api):
    spec = dict(Nx=64, Ny=64, Nz=65, nu=3e-3, seed_offset=1001)
    other = dict(Nx=96, Ny=96, Nz=97, nu=5e-3, seed_offset=1002)
    sim, v = _make(api, spec, "f64")
    sim2, _ = _make(api, other, "f32")
    b = api.Batch([sim, sim2])
    for _ in range(2):
        b.step([1e-3, 5e-4])
    P = ns.Params(64, 64, 65, nu=3e-3, forcing_x=3e-2)
    st = ns.to_spectral(v, P)
    gp = np.zeros((2, 2, 64, P.Kx), complex)
    for _ in range(2):
        st, gp = ns.rk_step(st, gp, P, 1e-3)
    ref = np.stack([ns.to_physical(c, P) for c in st])
    out = sim.get_fields().cpu().numpy()
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 1e-11
    b.close()
    sim.close()
    sim2.close()


def test_batch_argument_checks(api):
    sim, _ = _make(api, dict(Nx=32, Ny=32, Nz=33, nu=1e-2, seed_offset=0), "f64")
    with pytest.raises(api.FcError):
        api.Batch([sim, sim])
    b = api.Batch([sim])
    with pytest.raises(api.FcError):
        b.step([-1.0])
    b.close()
    sim.close()
