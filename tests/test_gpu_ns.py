"""Navier-Stokes / Boussinesq path on the GPU vs the FP64 oracle (through the C ABI)."""
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


def _rel(a, b):
    a = np.asarray(a)
    a = a.astype(np.complex128 if np.iscomplexobj(a) else np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _wall_err(out, ref):
    """Largest error on the wall rows z = 0 and z = Lz (where the continuation
    and the boundary-condition injection act), per field relative to that
    field's largest value, maximised over the fields: an error confined to the
    walls can hide inside a relative L2 norm over every point."""
    out = np.asarray(out, dtype=np.float64)
    worst = 0.0
    for f in range(ref.shape[0]):
        scale = max(np.abs(ref[f]).max(), 1e-300)
        for s in (0, ref.shape[1] - 1):
            worst = max(worst, float(np.abs(out[f, s] - ref[f, s]).max() / scale))
    return worst


def _cuda(x, dt=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dt)


def _oracle_steps(v, P, dt, n):
    st = ns.to_spectral(v, P)
    gp = np.zeros((2, 2, P.Ny, P.Kx), complex)
    for _ in range(n):
        st, gp = ns.rk_step(st, gp, P, dt)
    return np.stack([ns.to_physical(c, P) for c in st]), gp, st


# ---------------------------------------------------------------------------
# the plain FP64 channel workload: 32 x 32 x 33, d = 5, C = 25, nu = 1e-2
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def cfg0(api):
    N, Nz, nu = 32, 33, 1e-2
    p = api.ns_params(Nx=N, Ny=N, Nz=Nz, nu=nu, forcing_x=10 * nu, prec="f64")
    sim = api.Sim(p)
    P = ns.Params(N, N, Nz, nu=nu, forcing_x=10 * nu)
    v = synth.channel_velocity(N, N, Nz, nu=nu)
    yield sim, P, v
    sim.close()


def test_cfg0_fields_roundtrip(cfg0):
    sim, P, v = cfg0
    sim.set_fields(_cuda(v))
    out = sim.get_fields().cpu().numpy()
    assert np.abs(out - v).max() < 1e-14


def test_cfg0_rhs(cfg0):
    sim, P, v = cfg0
    out = sim.rhs(_cuda(v)).cpu().numpy()
    ref = ns.ns_rhs(v, P)
    assert _rel(out, ref) < 1e-11
    assert _wall_err(out, ref) < 1e-11


def test_cfg0_projection(cfg0):
    sim, P, v = cfg0
    g = np.random.default_rng(2)
    z = synth.z_grid(P.Nz)
    vs = v + 0.2 * (z * (1 - z))[None, :, None, None] * g.standard_normal((3, 1, P.Ny, P.Nx))
    sim.set_fields(_cuda(v))
    gp = torch.zeros((2, 2, P.Ny, P.Kx), dtype=torch.complex128, device="cuda")
    out = sim.project(_cuda(vs), 1e-3, gradp_out=gp).cpu().numpy()
    ref, gref = ns.poisson_project(vs, P, 1e-3)
    assert _rel(out, ref) < 1e-11
    assert _wall_err(out, ref) < 1e-11
    assert _rel(gp.cpu().numpy(), gref) < 1e-11
    # wall-normal velocity after projection is zero to round-off (Sec. 6)
    assert np.abs(out[2][[0, -1]]).max() < 1e-13


def test_cfg0_rk3_steps(cfg0):
    sim, P, v = cfg0
    sim.set_fields(_cuda(v))
    for _ in range(3):
        sim.step(1e-3)
    out = sim.get_fields().cpu().numpy()
    ref, gref, _ = _oracle_steps(v, P, 1e-3, 3)
    assert _rel(out, ref) < 1e-11
    assert _wall_err(out, ref) < 1e-11
    # grad p = grad phi / dt_j carries 1/dt_j (down to 3/dt): its rounding is a
    # velocity-scale rounding divided by dt_j, so it is measured on that scale
    dgp = sim.wall_gradp().cpu().numpy() - gref
    rms = lambda a: float(np.sqrt(np.mean(np.abs(a) ** 2)))
    assert rms(dgp) * (1e-3 / 3) < 1e-11 * rms(ref)


def test_poiseuille_fixed_point(api):
    N, Nz, nu = 32, 33, 1e-2
    sim = api.Sim(api.ns_params(Nx=N, Ny=N, Nz=Nz, nu=nu, forcing_x=10 * nu, prec="f64"))
    v = synth.poiseuille(N, N, Nz, F=10 * nu, nu=nu)
    sim.set_fields(_cuda(v))
    sim.step(1e-3)
    assert np.abs(sim.get_fields().cpu().numpy() - v).max() < 1e-10 * 1.25
    sim.close()


def test_checkpoint_restore_bitwise(cfg0):
    sim, P, v = cfg0
    sim.set_fields(_cuda(v))
    sim.step(1e-3)
    st = sim.get_state().clone()
    gp = sim.wall_gradp().clone()
    sim.step(1e-3)
    a = sim.get_fields().clone()
    sim.put_state(st)
    sim.put_wall_gradp(gp)
    sim.step(1e-3)
    b = sim.get_fields()
    assert torch.equal(a, b)


def test_caller_workspace_and_determinism(api):
    N, Nz = 32, 33
    p = api.ns_params(Nx=N, Ny=N, Nz=Nz, prec="f64")
    nb = api.ns_workspace_bytes(p)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    s1 = api.Sim(p, workspace=ws)
    s2 = api.Sim(p)
    v = _cuda(synth.channel_velocity(N, N, Nz))
    for s in (s1, s2):
        s.set_fields(v)
        s.step(1e-3)
    assert torch.equal(s1.get_fields(), s2.get_fields())
    s1.close()
    s2.close()


@pytest.mark.parametrize("N,Nz", [(32, 33), (64, 65)])
def test_channel_float32(api, N, Nz):
    nu = 1e-2
    sim = api.Sim(api.ns_params(Nx=N, Ny=N, Nz=Nz, nu=nu, forcing_x=10 * nu, prec="f32"))
    P = ns.Params(N, N, Nz, nu=nu, forcing_x=10 * nu)
    v = synth.channel_velocity(N, N, Nz, nu=nu).astype(np.float32).astype(np.float64)
    sim.set_fields(_cuda(v, torch.float32))
    for _ in range(2):
        sim.step(1e-3)
    out = sim.get_fields().cpu().numpy()
    ref, _, _ = _oracle_steps(v, P, 1e-3, 2)
    assert _rel(out, ref) < 1e-5
    assert _wall_err(out, ref) < 1e-5
    sim.close()


@pytest.mark.parametrize("N,Nz", [(32, 65), (128, 129)])
def test_boussinesq_float32(api, N, Nz):
    kw = dict(nu=3.162e-3, kappa=3.162e-3, gamma=1.0)
    sim = api.Sim(api.ns_params(Nx=N, Ny=N, Nz=Nz, nfields=4, prec="f32", **kw))
    P = ns.Params(N, N, Nz, nfields=4, **kw)
    f = synth.boussinesq_fields(N, N, Nz, amp=1e-1).astype(np.float32).astype(np.float64)
    sim.set_fields(_cuda(f, torch.float32))
    sim.step(2e-3)
    out = sim.get_fields().cpu().numpy()
    ref, _, _ = _oracle_steps(f, P, 2e-3, 1)
    for c in range(4):
        assert _rel(out[c], ref[c]) < 5e-5, c
    assert _wall_err(out, ref) < 5e-5
    sim.close()


@pytest.mark.parametrize("N,Nz", [(32, 39), (32, 103), (16, 231)])
def test_direct_length_channel_matches_oracle(api, N, Nz):
    """N' = Nz + 25 = 64, 128, 256: compiled transform lengths, so the z
    derivatives and filter are length-N' spectral multipliers and the
    projection uses plain length-N' DFTs (the paper's smooth N')."""
    nu = 1e-2
    p = api.ns_params(Nx=N, Ny=N, Nz=Nz, nu=nu, forcing_x=10 * nu, prec="f64")
    sim = api.Sim(p)
    P = ns.Params(N, N, Nz, nu=nu, forcing_x=10 * nu)
    v = synth.channel_velocity(N, N, Nz, nu=nu)
    vc = _cuda(v)
    assert _rel(sim.rhs(vc).cpu().numpy(), ns.ns_rhs(v, P)) < 1e-11
    sim.set_fields(vc)
    for _ in range(3):
        sim.step(1e-3)
    ref, gref, _ = _oracle_steps(v, P, 1e-3, 3)
    out = sim.get_fields().cpu().numpy()
    assert _rel(out, ref) < 1e-11
    assert _wall_err(out, ref) < 1e-11
    assert _rel(sim.wall_gradp().cpu().numpy(), gref) < 1e-9
    sim.close()


def test_d7_channel_float32_at_nz513(api, Mr_7_33):
    """d = 7, C = 33 at Nz = 513 (N' = 546): the padded length must reach
    2 N' - 1 = 1091, so the step runs on the 1152 = 32 x 36 transforms; one
    float32 RK3 step of the channel workload against the oracle with the
    same tables (float32 bound of the float32 channel tests)."""
    N, Nz, nu, dt = 16, 513, 3.162e-4, 1e-5
    sim = api.Sim(api.ns_params(Nx=N, Ny=N, Nz=Nz, d=7, C=33, nu=nu, forcing_x=10 * nu, prec="f32"))
    P = ns.Params(N, N, Nz, d=7, C=33, nu=nu, forcing_x=10 * nu, Mr=Mr_7_33)
    v = synth.channel_velocity(N, N, Nz, nu=nu).astype(np.float32).astype(np.float64)
    sim.set_fields(_cuda(v, torch.float32))
    sim.step(dt)
    out = sim.get_fields().cpu().numpy()
    ref, _, _ = _oracle_steps(v, P, dt, 1)
    assert _rel(out, ref) < 3e-5
    assert _wall_err(out, ref) < 3e-5
    sim.close()


def test_direct_length_1536_float32(api):
    """N' = Nz + 25 = 1536 (Nz = 1511), the largest smooth N' of the paper's
    runs: direct length-1536 = 32 x 48 z transforms; one float32 RK3 step of
    the channel workload against the oracle (dt nu k_max^2 = 7e-3 keeps the
    explicit viscous term stable at this resolution)."""
    N, Nz, nu, dt = 16, 1511, 3.162e-4, 1e-6
    sim = api.Sim(api.ns_params(Nx=N, Ny=N, Nz=Nz, nu=nu, forcing_x=10 * nu, prec="f32"))
    P = ns.Params(N, N, Nz, nu=nu, forcing_x=10 * nu)
    v = synth.channel_velocity(N, N, Nz, nu=nu).astype(np.float32).astype(np.float64)
    sim.set_fields(_cuda(v, torch.float32))
    sim.step(dt)
    out = sim.get_fields().cpu().numpy()
    ref, _, _ = _oracle_steps(v, P, dt, 1)
    assert _rel(out, ref) < 3e-5
    assert _wall_err(out, ref) < 3e-5
    sim.close()


def test_d7_channel_matches_oracle(api, Mr_7_33):
    """d = 7, C = 33 (N' = 66) on the 32 x 32 x 33 channel: right-hand side and
    three RK3 steps vs the oracle with the same tables; float64 floor scaled by
    the continuation's amplification (cancellation in M_r f)."""
    from numerics import fc_amplification
    N, Nz, nu = 32, 33, 1e-2
    sim = api.Sim(api.ns_params(Nx=N, Ny=N, Nz=Nz, d=7, C=33, nu=nu, forcing_x=10 * nu, prec="f64"))
    P = ns.Params(N, N, Nz, d=7, C=33, nu=nu, forcing_x=10 * nu, Mr=Mr_7_33)
    v = synth.channel_velocity(N, N, Nz, nu=nu)
    tol = 1e-11 * fc_amplification(Mr_7_33)
    assert _rel(sim.rhs(_cuda(v)).cpu().numpy(), ns.ns_rhs(v, P)) < tol
    sim.set_fields(_cuda(v))
    for _ in range(3):
        sim.step(1e-3)
    ref, _, _ = _oracle_steps(v, P, 1e-3, 3)
    assert _rel(sim.get_fields().cpu().numpy(), ref) < tol
    sim.close()


def test_full_size_smooth_boussinesq_float32(api):
    """1024 x 1024 x 487 (N' = 512, direct), 4 fields, FP32: the conduction
    state (all zero) is an exact fixed point, and one RK3 step of the seeded
    fields stays finite with w = 0 and theta = 0 at the walls."""
    N, Nz = 1024, 487
    kw = dict(nu=3.162e-4, kappa=3.162e-4, gamma=1.0)
    sim = api.Sim(api.ns_params(Nx=N, Ny=N, Nz=Nz, nfields=4, prec="f32", **kw))
    z = torch.zeros((4, Nz, N, N), dtype=torch.float32, device="cuda")
    sim.set_fields(z)
    sim.step(1e-3)
    assert torch.count_nonzero(sim.get_fields()) == 0
    del z
    f = torch.from_numpy(synth.boussinesq_fields(N, N, Nz, dtype=np.float32)).cuda()
    sim.set_fields(f)
    del f
    sim.step(1e-3)
    out = sim.get_fields()
    assert torch.isfinite(out).all()
    scale = out[:3].abs().max().item()
    assert out[2, [0, -1]].abs().max().item() < 1e-5 * scale
    assert out[3, [0, -1]].abs().max().item() < 1e-5 * out[3].abs().max().item()
    sim.close()


def test_full_size_boussinesq_properties(api):
    """1024 x 1024 x 513, 4 fields, FP32, as bench.py runs it: one RK3 step stays
    finite, keeps w = 0 at the walls and theta = 0 at the walls, and the
    conduction state (all zero) is an exact fixed point."""
    N, Nz = 1024, 513
    kw = dict(nu=3.162e-4, kappa=3.162e-4, gamma=1.0)
    sim = api.Sim(api.ns_params(Nx=N, Ny=N, Nz=Nz, nfields=4, prec="f32", **kw))
    z = torch.zeros((4, Nz, N, N), dtype=torch.float32, device="cuda")
    sim.set_fields(z)
    sim.step(1e-3)
    assert torch.count_nonzero(sim.get_fields()) == 0
    f = torch.from_numpy(synth.boussinesq_fields(N, N, Nz, dtype=np.float32)).cuda()
    sim.set_fields(f)
    del f
    sim.step(1e-3)
    out = sim.get_fields()
    assert torch.isfinite(out).all()
    scale = out[:3].abs().max().item()
    assert out[2, [0, -1]].abs().max().item() < 1e-5 * scale
    assert out[3, [0, -1]].abs().max().item() < 1e-5 * out[3].abs().max().item()
    sim.close()


def _band_limited(Nx, Nz, kmax, seed, xp, dtype):
    """Four fields sum_{|kx|,|ky| <= kmax} A(z) cos(kx x + ky y) + B(z) sin(...),
    A, B seeded polynomials times z(1 - z), on an Nx x Nx grid (x = 2 pi i / Nx);
    xp = numpy or torch (on the GPU)."""
    g = np.random.default_rng(seed)
    z = np.linspace(0.0, 1.0, Nz)
    modes = [(kx, ky) for kx in range(0, kmax + 1) for ky in range(-kmax, kmax + 1) if kx > 0 or ky >= 0]
    coef = g.uniform(-1, 1, size=(4, len(modes), 2, 3))
    x = 2 * np.pi * np.arange(Nx) / Nx
    out = []
    for f in range(4):
        acc = None
        for m, (kx, ky) in enumerate(modes):
            ph = kx * x[None, :] + ky * x[:, None]                     # [y][x]
            for part, fn in ((0, np.cos), (1, np.sin)):
                if kx == 0 and ky == 0 and part == 1:
                    continue
                c = coef[f, m, part]
                prof = 0.1 * z * (1 - z) * (1 + c[0] + c[1] * z + c[2] * z * z) / (1 + kx * kx + ky * ky)
                if xp is np:
                    term = prof[:, None, None] * fn(ph)[None]
                else:
                    term = (xp.from_numpy(prof).to("cuda", dtype)[:, None, None]
                            * xp.from_numpy(fn(ph)).to("cuda", dtype)[None])
                acc = term if acc is None else acc + term
        out.append(acc)
    return np.stack(out) if xp is np else xp.stack(out)


@pytest.mark.parametrize("Nz", [513, 487])
def test_full_size_boussinesq_matches_oracle_on_band_limited_fields(api, Nz):
    """1024 x 1024 x Nz, 4 fields, FP32, autotuned variants as bench.py runs
    it, one RK3 step, against the FP64 oracle: for fields band-limited to
    |kx|, |ky| <= 2 the step raises the horizontal bandwidth to 16 at most
    (each stage's product doubles it), which the 2/3 rule keeps and a
    64 x 64 grid represents without aliasing, so the exact result on the
    1024^2 grid restricted to every 16th point is the exact result on the 64^2
    grid; the oracle computes the latter (Nz = 513: padded N' = 538; 487:
    direct N' = 512)."""
    N, Nc, dt = 1024, 64, 1e-3
    kw = dict(nu=3.162e-4, kappa=3.162e-4, gamma=1.0)
    sim = api.Sim(api.ns_params(Nx=N, Ny=N, Nz=Nz, nfields=4, prec="f32", **kw))
    sim.tune(1)
    f = _band_limited(N, Nz, 2, 77 + Nz, torch, torch.float32)
    sim.set_fields(f)
    del f
    sim.step(dt)
    out = sim.get_fields()[:, :, ::N // Nc, ::N // Nc].cpu().numpy()
    sim.close()
    torch.cuda.empty_cache()
    P = ns.Params(Nc, Nc, Nz, nfields=4, **kw)
    fc_ = _band_limited(Nc, Nz, 2, 77 + Nz, np, None)
    st, _ = ns.rk_step(ns.to_spectral(fc_, P), np.zeros((2, 2, Nc, P.Kx), complex), P, dt)
    ref = np.stack([ns.to_physical(c, P) for c in st])
    for fi in range(4):
        assert _rel(out[fi], ref[fi]) < 5e-5, (fi, _rel(out[fi], ref[fi]))
    assert _wall_err(out, ref) < 5e-5


def test_diagnostics_boussinesq(api):
    """ns_diagnostics on the GPU vs the oracle's diagnostics after one RK3 step."""
    N, Nz = 32, 33
    kw = dict(nu=3.162e-3, kappa=3.162e-3, gamma=1.0)
    sim = api.Sim(api.ns_params(Nx=N, Ny=N, Nz=Nz, nfields=4, prec="f64", **kw))
    P = ns.Params(N, N, Nz, nfields=4, **kw)
    f = synth.boussinesq_fields(N, N, Nz, amp=1e-1)
    f[0] += 0.3 * (synth.z_grid(Nz) * (1 - synth.z_grid(Nz)))[:, None, None]
    sim.set_fields(_cuda(f))
    sim.step(2e-3)
    _, _, st = _oracle_steps(f, P, 2e-3, 1)
    d = sim.diagnostics()
    div = (ns.divergence_phys(st, P) ** 2).mean()
    wu, wv, ww = ns.wall_mean_squares(st, P)
    nb, nt = ns.nusselt(st, P)
    assert abs(d["div_ms"] - div) <= 1e-6 * div
    assert abs(d["wall_u_ms"] - wu) <= 1e-10 * wu
    assert d["wall_w_ms"] <= 1e-25
    assert abs(d["flow_rate"] - ns.flow_rate(st, P)) <= 1e-12
    assert abs(d["nusselt"] - 0.5 * (nb + nt)) <= 1e-10
    sim.close()


@pytest.mark.parametrize("kind,N,Nz", [("rb", 32, 33), ("rb", 128, 129), ("channel", 64, 65)])
def test_diagnostics_float32_errors(api, kind, N, Nz):
    """Error of every float32 diagnostic against the FP64 oracle after one RK3
    step (Sec. 6 and 7 diagnostics), on the scale where it is meaningful.
    Flow rate and Nusselt number come from the (kx, ky) = (0, 0) line, which
    the float32 path carries in float64: relative error <= 1e-7 (flow rate;
    the nonlinear term that feeds the mean line is float32) and absolute
    <= 1e-9 (Nu ~ 1).  Horizontal-mean, r.m.s. and shell-spectrum profiles:
    <= 1e-6 of their largest value (float32 products over the grid).  The
    divergence and the wall mean squares of u and w are quadratic in
    quantities that vanish in the exact solution, so in float32 they sit at
    the rounding floor: each is within (eps32 v_max k_z,max)^2 (divergence) or
    (eps32 v_max)^2 (wall values) of the oracle, plus 1e-3 relative for the
    wall slip of the Boussinesq runs, which is above that floor (measured:
    flow rate 1.3e-8 - 3.1e-8, Nu 2e-12 - 1.3e-11, profiles <= 2e-7, wall slip
    0.12 - 0.28 %)."""
    eps = float(np.finfo(np.float32).eps)
    if kind == "rb":
        kw = dict(nu=3.162e-3, kappa=3.162e-3, gamma=1.0, nfields=4)
        f = synth.boussinesq_fields(N, N, Nz, amp=1e-1)
        f[0] += 0.3 * (synth.z_grid(Nz) * (1 - synth.z_grid(Nz)))[:, None, None]
        dt = 2e-3
    else:
        kw = dict(nu=1e-2, forcing_x=0.1)
        f = synth.channel_velocity(N, N, Nz, nu=1e-2)
        dt = 1e-3
    f = f.astype(np.float32).astype(np.float64)
    P = ns.Params(N, N, Nz, **kw)
    sim = api.Sim(api.ns_params(Nx=N, Ny=N, Nz=Nz, prec="f32", **kw))
    sim.set_fields(_cuda(f, torch.float32))
    sim.step(dt)
    d = sim.diagnostics()
    pr = sim.profiles()
    sim.close()
    _, _, st = _oracle_steps(f, P, dt, 1)
    vmax = float(np.abs(f[:3]).max())
    kz_max = np.pi * (Nz - 1)
    div = (ns.divergence_phys(st, P) ** 2).mean()
    wu, _, ww = ns.wall_mean_squares(st, P)
    assert abs(d["flow_rate"] - ns.flow_rate(st, P)) <= 1e-7 * abs(ns.flow_rate(st, P))
    if kind == "rb":
        nb, nt = ns.nusselt(st, P)
        assert abs(d["nusselt"] - 0.5 * (nb + nt)) <= 1e-9
        assert abs(d["wall_u_ms"] - wu) <= 1e-3 * wu + (eps * vmax) ** 2
    else:
        assert abs(d["wall_u_ms"] - wu) <= (eps * vmax) ** 2
    assert abs(d["wall_w_ms"] - ww) <= (eps * vmax) ** 2
    assert abs(d["div_ms"] - div) <= (eps * vmax * kz_max) ** 2
    mean, rms = ns.profiles(st, P)
    E, _ = ns.shell_spectrum(st, P)
    assert np.abs(pr["mean"] - mean).max() <= 1e-6 * np.abs(mean).max()
    assert np.abs(pr["rms"] - rms).max() <= 1e-6 * rms.max()
    assert np.abs(pr["spectrum"] - E).max() <= 1e-6 * E.max()


def test_float32_mean_flow_island_long_run(api):
    """2000 float32 RK3 steps of a decaying mean profile u = 0.5 sin(pi z) with
    weak fluctuations: the mean-flow line, accumulated in float64, stays within
    float32 output rounding of the float64 run (float32 accumulation of that
    line would random-walk by ~1e-6)."""
    N, Nz = 32, 33
    z = synth.z_grid(Nz)
    f = synth.channel_velocity(N, N, Nz, mean_flow=False, fluct=0.01)
    f[0] += 0.5 * np.sin(np.pi * z)[:, None, None]
    f = f.astype(np.float32).astype(np.float64)
    means = []
    for prec, dt in (("f32", torch.float32), ("f64", torch.float64)):
        sim = api.Sim(api.ns_params(Nx=N, Ny=N, Nz=Nz, nu=1e-2, prec=prec))
        sim.set_fields(_cuda(f, dt))
        for _ in range(2000):
            sim.step(1e-3)
        means.append(sim.get_fields()[0].double().mean(dim=(1, 2)).cpu().numpy())
        sim.close()
    rel = np.abs(means[0] - means[1]).max() / np.abs(means[1]).max()
    assert rel < 2.4e-7, rel


@pytest.mark.parametrize("o", [1, 2, 3])
def test_wall_slip_dt_study(api, o):
    """Slip study (Sec. 6) on the GPU: <u^2|wall> from ns_diagnostics matches the
    oracle run by run, falls like dt^4 above the resolution floor for o <= 2, and
    <w^2|wall> stays at round-off for every dt."""
    N, Nz, T = 32, 33, 0.032
    v0 = synth.channel_velocity(N, N, Nz, nu=1e-2, fluct=1.0)
    P = ns.Params(N, N, Nz, nu=1e-2, forcing_x=0.1, rk_order=o)
    slips = []
    for dt in (8e-3, 4e-3):
        sim = api.Sim(api.ns_params(Nx=N, Ny=N, Nz=Nz, nu=1e-2, forcing_x=0.1, rk_order=o, prec="f64"))
        sim.set_fields(_cuda(v0))
        for _ in range(int(round(T / dt))):
            sim.step(dt)
        d = sim.diagnostics()
        sim.close()
        st = ns.to_spectral(v0, P)
        gp = np.zeros((2, 2, N, N // 2 + 1), complex)
        for _ in range(int(round(T / dt))):
            st, gp = ns.rk_step(st, gp, P, dt)
        wu, _, ww = ns.wall_mean_squares(st, P)
        assert abs(d["wall_u_ms"] - wu) <= 1e-6 * wu
        assert d["wall_w_ms"] < 1e-28
        slips.append(d["wall_u_ms"])
    if o <= 2:
        assert np.log2(slips[0] / slips[1]) > 3.5


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_restart_interpolation(api, prec, tol):
    """ns_interpolate (Sec. 6 restarts): 64^2 x 65 after one RK3 step onto
    128^2 x 129, against the oracle's spectral interpolation."""
    nu = 1e-2
    src = api.Sim(api.ns_params(Nx=64, Ny=64, Nz=65, nu=nu, forcing_x=10 * nu, prec=prec))
    dst = api.Sim(api.ns_params(Nx=128, Ny=128, Nz=129, nu=nu, forcing_x=10 * nu, prec=prec))
    v = synth.channel_velocity(64, 64, 65, nu=nu)
    src.set_fields(_cuda(v, src.dtype))
    src.step(1e-3)
    dst.interpolate_from(src)
    P1, P2 = ns.Params(64, 64, 65, nu=nu, forcing_x=10 * nu), ns.Params(128, 128, 129, nu=nu, forcing_x=10 * nu)
    st = ns.to_spectral(v, P1)
    st, _ = ns.rk_step(st, np.zeros((2, 2, 64, P1.Kx), complex), P1, 1e-3)
    ref = ns.to_physical(ns.spectral_interpolate(st, P1, P2), P2)
    assert _rel(dst.get_fields().cpu().numpy(), ref) < tol
    assert torch.count_nonzero(dst.wall_gradp()) == 0
    dst.step(5e-4)                                    # the restarted run advances
    assert torch.isfinite(dst.get_fields()).all()
    src.close()
    dst.close()



def test_profiles_and_spectrum(api):
    """ns_profiles on the GPU vs the oracle after one RK3 step (float64)."""
    N, Nz, nu = 64, 65, 1e-2
    sim = api.Sim(api.ns_params(Nx=N, Ny=N, Nz=Nz, nu=nu, forcing_x=10 * nu, prec="f64"))
    P = ns.Params(N, N, Nz, nu=nu, forcing_x=10 * nu)
    v = synth.channel_velocity(N, N, Nz, nu=nu)
    sim.set_fields(_cuda(v))
    sim.step(1e-3)
    _, _, st = _oracle_steps(v, P, 1e-3, 1)
    mean, rms = ns.profiles(st, P)
    E, dk = ns.shell_spectrum(st, P)
    d = sim.profiles()
    assert d["dk"] == dk and d["spectrum"].shape == E.shape
    assert np.abs(d["mean"] - mean).max() < 1e-12 * np.abs(mean).max()
    assert np.abs(d["rms"] - rms).max() < 1e-11 * rms.max()
    assert np.abs(d["spectrum"] - E).max() < 1e-11 * E.max()
    sim.close()



def test_tiles_do_not_change_results(api):
    """ns_tune: the alternative tiles give bitwise the same step as the
    defaults; the alternative radix schedules of the z kinds (288 = 18 x 16
    here) agree with the oracle to float32 rounding; the autotuned choice is
    bitwise the same as that choice set by hand (float32 Boussinesq,
    64^2 x 65)."""
    N, Nz = 64, 65
    kw = dict(nu=3.162e-3, kappa=3.162e-3, gamma=1.0)
    v = synth.boussinesq_fields(N, N, Nz, amp=1e-1)
    f = torch.from_numpy(v.astype(np.float32)).cuda()

    def run(mode, tiles):
        sim = api.Sim(api.ns_params(Nx=N, Ny=N, Nz=Nz, nfields=4, prec="f32", **kw))
        choice = sim.tune(mode, tiles)
        sim.set_fields(f)
        for _ in range(2):
            sim.step(1e-3)
        out = sim.get_fields()
        sim.close()
        return choice, out

    c0, o0 = run(0, None)
    c1, o1 = run(2, [1, 1, 1, 1, 1])
    c2, o2 = run(2, [3, 3, 3, 3, 3])
    ct, ot = run(1, None)
    assert c0 == [0] * 5 and c1 == [1] * 5 and c2 == [3, 3, 3, 1, 1]
    assert all(0 <= c <= 3 for c in ct[:3]) and all(c in (0, 1) for c in ct[3:])
    assert torch.equal(o0, o1)
    _, oh = run(2, ct)
    assert torch.equal(ot, oh)
    P = ns.Params(N, N, Nz, nfields=4, **kw)
    st = ns.to_spectral(v, P)
    gp = np.zeros((2, 2, N, P.Kx), complex)
    for _ in range(2):
        st, gp = ns.rk_step(st, gp, P, 1e-3)
    ref = np.stack([ns.to_physical(c, P) for c in st])
    for o in (o0, o2, ot):
        for fi in range(4):
            r = ref[fi]
            assert np.linalg.norm(o[fi].cpu().numpy() - r) / np.linalg.norm(r) < 5e-5, fi


@pytest.mark.parametrize("Nz,prec,tol", [(10, "f64", 1e-11), (129, "f64", 1e-11), (257, "f64", 1e-11),
                                         (257, "f32", 3e-5), (743, "f32", 3e-5), (999, "f32", 3e-5)])
def test_every_z_length_one_step(api, Nz, prec, tol):
    """One RK3 step on a 16 x 16 horizontal grid for the remaining compiled z
    lengths: the smallest grid (Nz = 2d = 10, padded 160), padded 320
    (N' = 154) and 576 (N' = 282), direct 768 and 1024."""
    N, nu = 16, 1e-2
    sim = api.Sim(api.ns_params(Nx=N, Ny=N, Nz=Nz, nu=nu, forcing_x=10 * nu, prec=prec))
    P = ns.Params(N, N, Nz, nu=nu, forcing_x=10 * nu)
    v = synth.channel_velocity(N, N, Nz, nu=nu)
    sim.set_fields(_cuda(v, sim.dtype))
    sim.step(1e-4)
    ref, _, _ = _oracle_steps(v, P, 1e-4, 1)
    out = sim.get_fields().cpu().numpy()
    assert _rel(out, ref) < tol
    assert _wall_err(out, ref) < tol
    sim.close()


def test_general_parameters_match_oracle(api):
    """Exponential filter in x, y, z (mode 0), a 4 x 3 x 2 box with Nx != Ny,
    kappa != nu, gamma = 2.5, fourth-order time splitting, float64."""
    kw = dict(nfields=4, nu=1e-3, kappa=2e-3, gamma=2.5, rk_order=4, filter=0, Lx=4.0, Ly=3.0, Lz=2.0)
    Nx, Ny, Nz = 64, 32, 65
    sim = api.Sim(api.ns_params(Nx=Nx, Ny=Ny, Nz=Nz, prec="f64", **kw))
    P = ns.Params(Nx, Ny, Nz, **kw)
    f = synth.boussinesq_fields(Nx, Ny, Nz, Lz=2.0, amp=1e-1)
    assert _rel(sim.rhs(_cuda(f)).cpu().numpy(), ns.ns_rhs(f, P)) < 1e-11
    sim.set_fields(_cuda(f))
    for _ in range(2):
        sim.step(2e-3)
    ref, gref, _ = _oracle_steps(f, P, 2e-3, 2)
    out = sim.get_fields().cpu().numpy()
    assert _rel(out, ref) < 1e-11
    assert _wall_err(out, ref) < 1e-11
    assert _rel(sim.wall_gradp().cpu().numpy(), gref) < 1e-9
    sim.close()


def test_diag_series_equals_synchronous_diagnostics(api):
    """ns_set_diag_series / ns_get_diag_series: the device-recorded diagnostics
    after every 2nd step are the values ns_diagnostics returns for the same
    states (Boussinesq, float32, Nu and flow rate included), up to the order of
    the reduction's float64 atomic additions."""
    import synth
    p = api.ns_params(Nx=32, Ny=32, Nz=33, nfields=4, prec="f32", nu=1e-2, kappa=1e-2, gamma=1.0)
    v = synth.boussinesq_fields(32, 32, 33, seed_offset=5).astype(np.float32)
    a, b = api.Sim(p), api.Sim(p)
    for s_ in (a, b):
        s_.set_fields(torch.from_numpy(v).cuda())
    a.set_diag_series(2)
    ref = []
    for k in range(1, 8):
        a.step(1e-3)
        b.step(1e-3)
        if k % 2 == 0:
            ref.append(b.diagnostics())
    ser = a.diag_series()
    assert list(ser["step"]) == [2, 4, 6]
    for i, r in enumerate(ref):
        for key, val in r.items():
            assert abs(ser[key][i] - val) <= 1e-12 * abs(val) + 1e-300, (i, key)
    a.set_diag_series(0)
    a.step(1e-3)
    assert len(a.diag_series()["step"]) == 0
    with pytest.raises(api.FcError):
        a.set_diag_series(-1)
    a.close()
    b.close()
