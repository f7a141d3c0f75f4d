"""Failure detection on the GPU without a GPU fault: non-finite values are
counted by kernels (fc_count_nonfinite, ns_check_finite, the per-step check of
ns_set_finite_check); failures are injected on the host (fc_inject_failure),
and the serving loop retries them or quarantines a simulation that blew up.
No test makes a kernel fault, trap or wait."""
import math

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2002_01392_gb300 import api as a
    assert torch.cuda.is_available()
    a.clear_injected()
    yield a
    a.clear_injected()


def _sim(api, N=64, Nz=65, prec="f32", seed=0):
    p = api.ns_params(Nx=N, Ny=N, Nz=Nz, nu=5e-3, forcing_x=5e-2, prec=prec)
    s = api.Sim(p)
    v = synth.channel_velocity(N, N, Nz, nu=5e-3, seed_offset=seed)
    t = torch.from_numpy(v.astype(np.float32 if prec == "f32" else np.float64)).cuda()
    s.set_fields(t)
    return s, t


def _plant_nan(sim, f=1, z=7, ky=3, kx=2):
    """NaN into the real part of state value (field f, continued row z, ky, kx)."""
    p = sim.p
    Kxp, Np, TL = (p.Nx // 2 + 1 + 15) // 16 * 16, p.Nz + p.C, 16
    line = ky * Kxp + kx
    ntiles = p.Ny * Kxp // TL
    st = sim.get_state()
    st[((f * ntiles + line // TL) * Np + z) * TL + line % TL] = complex(math.nan, 0.0)
    sim.put_state(st)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_count_nonfinite_exact(api, dtype):
    n = 1_000_003                      # not a multiple of the per-CTA chunk
    x = torch.randn(n, dtype=dtype, device="cuda")
    assert api.count_nonfinite(x) == 0
    x[0], x[n // 2], x[-1] = math.nan, math.inf, -math.inf
    x[7] = torch.finfo(dtype).max      # finite
    assert api.count_nonfinite(x) == 3
    assert api.count_nonfinite(torch.empty(0, dtype=dtype, device="cuda")) == 0


def test_deriv_outputs_are_finite(api):
    plan = api.Plan(5, 25, 129)
    f = torch.from_numpy(synth.SeparableField(64, 48, 129).field(0).astype(np.float32)).cuda()
    d1, d2 = torch.empty_like(f), torch.empty_like(f)
    api.fc_deriv_z(plan, f, d1, d2)
    assert api.count_nonfinite(d1) == 0 and api.count_nonfinite(d2) == 0


def test_check_finite_counts_physical_state(api):
    s, _ = _sim(api)
    assert s.check_finite() == 0
    _plant_nan(s)
    assert s.check_finite() == 1
    s.close()


def test_step_check_flags_blow_up_and_recovers(api):
    s, v = _sim(api, seed=3)
    s.set_finite_check(1)
    s.step(5e-4)
    torch.cuda.synchronize()
    s.step(5e-4)                       # clean state: the checks pass
    _plant_nan(s)
    s.step(5e-4)                       # the NaN spreads; the check after this step sees it
    torch.cuda.synchronize()
    with pytest.raises(api.FcError) as e:
        s.step(5e-4)
    assert e.value.name == "FC_ERR_NONFINITE"
    s.set_fields(v)                    # new state: the flag stays until a clean check
    with pytest.raises(api.FcError):
        s.step(5e-4)
    assert s.check_finite() == 0
    s.step(5e-4)
    torch.cuda.synchronize()
    assert s.check_finite() == 0
    s.close()


def test_batch_member_check(api):
    a, _ = _sim(api, seed=4)
    b, vb = _sim(api, N=32, Nz=33, seed=5)
    b.set_finite_check(1)
    batch = api.Batch([a, b])
    batch.step(5e-4)
    torch.cuda.synchronize()
    _plant_nan(b, f=0, z=40, ky=5, kx=9)
    batch.step(5e-4)
    torch.cuda.synchronize()
    with pytest.raises(api.FcError) as e:
        batch.step(5e-4)
    assert e.value.name == "FC_ERR_NONFINITE" and "member 1" in str(e.value)
    b.set_fields(vb)
    assert b.check_finite() == 0
    batch.step(5e-4)
    torch.cuda.synchronize()
    assert a.check_finite() == 0 and b.check_finite() == 0
    batch.close()
    a.close()
    b.close()


def test_injected_step_failure_then_retry_is_exact(api):
    ref, _ = _sim(api, seed=6)
    s, _ = _sim(api, seed=6)
    for _ in range(4):
        ref.step(5e-4)
    api.inject_failure("rk_step", "FC_ERR_CUDA", skip=2, count=1)
    fails = 0
    done = 0
    while done < 4:
        try:
            s.step(5e-4)
            done += 1
        except api.FcError as e:
            assert e.name == "FC_ERR_CUDA"
            fails += 1
    assert fails == 1
    assert torch.equal(s.get_fields(), ref.get_fields())
    s.close()
    ref.close()


def test_serving_retries_and_quarantine(api):
    from paper_2002_01392_gb300 import serve
    srv = serve.Server(1 << 40, slots=4, max_retries=2, check_every=1)
    alone = serve.Server(1 << 40, slots=1)
    ids, ids2 = [], []
    for i, g in enumerate(((64, 64, 65), (32, 32, 33), (64, 64, 65))):
        p = api.ns_params(Nx=g[0], Ny=g[1], Nz=g[2], nu=5e-3, forcing_x=5e-2, prec="f32")
        v = torch.from_numpy(synth.channel_velocity(*g, nu=5e-3, seed_offset=60 + i).astype(np.float32)).cuda()
        ids.append(srv.admit(p, v))
        ids2.append(alone.admit(p, v))
    _plant_nan(srv.sims[ids[2]], f=2, z=20, ky=1, kx=1)   # simulation 2 blows up on its first step
    reqs = [serve.Request(kind="step", sim=ids[k % 3], arrival=0.0005 * k, dt=5e-4) for k in range(24)]
    api.inject_failure("rk_step", "FC_ERR_CUDA", skip=3, count=2)
    stats = srv.run(reqs)
    api.clear_injected()
    assert stats["requests"] == 24 and stats["retried"] == 2 and stats["quarantined"] == 1
    bad = [r for r in reqs if r.sim == ids[2]]
    assert all(r.error == "FC_ERR_NONFINITE" for r in bad[1:]) and bad[0].error is None
    assert stats["failed"] == len(bad) - 1
    for k in (0, 1):                                 # the others equal the same steps run alone
        sim = alone.sims[ids2[k]]
        for r in reqs:
            if r.sim == ids[k]:
                assert r.error is None
                sim.step(r.dt)
        assert torch.equal(sim.get_fields(), srv.sims[ids[k]].get_fields())
    srv.close()
    alone.close()
