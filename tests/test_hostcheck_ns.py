"""The NS kernel sequence executed on the CPU (host-check library) vs the oracle.

Checks every kernel's index arithmetic and the orchestration (buffer roles,
stage steps, wall planes) without a GPU."""
import numpy as np
import pytest

from hostcheck_ns import HostSim
from oracle import ns
import synth


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def chan():
    N, Nz = 32, 33
    hs = HostSim(Nx=N, Ny=N, Nz=Nz, nu=1e-2, forcing_x=0.1, prec="f64")
    P = ns.Params(N, N, Nz, nu=1e-2, forcing_x=0.1)
    v = synth.channel_velocity(N, N, Nz)
    yield hs, P, v
    hs.close()


def test_fields_roundtrip(chan):
    hs, P, v = chan
    hs.set_fields(v)
    assert np.abs(hs.get_fields() - v).max() < 1e-14


def test_rhs_matches_oracle(chan):
    hs, P, v = chan
    assert _rel(hs.rhs(v), ns.ns_rhs(v, P)) < 1e-12


def test_projection_matches_oracle(chan):
    hs, P, v = chan
    g = np.random.default_rng(2)
    z = synth.z_grid(P.Nz)
    vs = v + 0.2 * (z * (1 - z))[None, :, None, None] * g.standard_normal((3, 1, P.Ny, P.Nx))
    hs.set_fields(v)                                   # wall planes reset to zero
    out, gp = hs.project(vs, 1e-3)
    ref, gref = ns.poisson_project(vs, P, 1e-3)
    assert _rel(out, ref) < 1e-13
    assert _rel(gp, gref) < 1e-12


def test_rk3_steps_match_oracle(chan):
    hs, P, v = chan
    hs.set_fields(v)
    st = ns.to_spectral(v, P)
    gp = np.zeros((2, 2, P.Ny, P.Kx), complex)
    for _ in range(3):
        hs.step(1e-3)
        st, gp = ns.rk_step(st, gp, P, 1e-3)
    ref = np.stack([ns.to_physical(c, P) for c in st])
    assert _rel(hs.get_fields(), ref) < 1e-13


@pytest.mark.parametrize("Nz,nu,dt,prec,tol,tol_rhs", [(39, 1e-2, 1e-3, "f64", 1e-12, 1e-12),
                                                       (39, 1e-2, 1e-3, "f32", 2e-5, 5e-4),
                                                       (487, 3.162e-4, 1e-4, "f64", 1e-12, 1e-11),
                                                       (487, 3.162e-4, 1e-4, "f32", 2e-5, 5e-3)])
def test_direct_length_steps_match_oracle(Nz, nu, dt, prec, tol, tol_rhs):
    """N' = Nz + C = 64 or 512 (the paper-shaped smooth companion) is itself a
    compiled transform length: z derivatives and the filter become spectral
    multipliers of length N' and the projection's DFTs plain length-N'
    transforms (no padding, no Bluestein).  The right-hand side carries
    nu d2/dz2, whose rounding floor is eps (k_max/k)^2: ~1e-4 in float32 at
    N' = 64, ~1e-3 at N' = 512.  The explicit step needs dt nu k_max^2 = O(1)
    at most (k_max = pi (Nz - 1)): at Nz = 487 with nu = 1e-2 and dt = 1e-3
    the top z modes grow from rounding by orders of magnitude per step, so the
    larger grid runs at the Rayleigh-Benard viscosity with dt = 1e-4."""
    N = 16
    hs = HostSim(Nx=N, Ny=N, Nz=Nz, nu=nu, forcing_x=10 * nu, prec=prec)
    P = ns.Params(N, N, Nz, nu=nu, forcing_x=10 * nu)
    v = synth.channel_velocity(N, N, Nz, nu=nu)
    assert _rel(hs.rhs(v), ns.ns_rhs(v, P)) < tol_rhs
    g = np.random.default_rng(3)
    z = synth.z_grid(Nz)
    vs = v + 0.2 * (z * (1 - z))[None, :, None, None] * g.standard_normal((3, 1, N, N))
    hs.set_fields(v)
    out, gp = hs.project(vs, dt)
    ref, gref = ns.poisson_project(vs, P, dt)
    assert _rel(out, ref) < tol
    assert _rel(gp, gref) < 10 * tol
    hs.set_fields(v)
    st = ns.to_spectral(v, P)
    gp = np.zeros((2, 2, N, P.Kx), complex)
    for _ in range(2):
        hs.step(dt)
        st, gp = ns.rk_step(st, gp, P, dt)
    ref = np.stack([ns.to_physical(c, P) for c in st])
    assert _rel(hs.get_fields(), ref) < tol
    hs.close()


def test_d7_tables_channel_matches_oracle(Mr_7_33):
    """d = 7, C = 33 (N' = 58 + 8 = 66): the library's double-binary128 tables
    through the whole kernel sequence, float64, tolerance scaled by the
    continuation's amplification."""
    from numerics import fc_amplification
    N, Nz = 16, 33
    hs = HostSim(Nx=N, Ny=N, Nz=Nz, d=7, C=33, nu=1e-2, forcing_x=0.1, prec="f64")
    P = ns.Params(N, N, Nz, d=7, C=33, nu=1e-2, forcing_x=0.1, Mr=Mr_7_33)
    v = synth.channel_velocity(N, N, Nz)
    tol = 1e-12 * fc_amplification(Mr_7_33)
    assert _rel(hs.rhs(v), ns.ns_rhs(v, P)) < tol
    hs.set_fields(v)
    st = ns.to_spectral(v, P)
    gp = np.zeros((2, 2, N, P.Kx), complex)
    hs.step(1e-3)
    st, gp = ns.rk_step(st, gp, P, 1e-3)
    ref = np.stack([ns.to_physical(c, P) for c in st])
    assert _rel(hs.get_fields(), ref) < tol
    hs.close()


def test_boussinesq_float32_steps():
    N, Nz = 16, 65
    kw = dict(Nx=N, Ny=N, Nz=Nz, nfields=4, nu=3.162e-3, kappa=3.162e-3, gamma=1.0, prec="f32")
    hs = HostSim(**kw)
    P = ns.Params(N, N, Nz, nfields=4, nu=3.162e-3, kappa=3.162e-3, gamma=1.0)
    f = synth.boussinesq_fields(N, N, Nz, amp=1e-1)
    hs.set_fields(f)
    st = ns.to_spectral(f.astype(np.float32).astype(np.float64), P)
    gp = np.zeros((2, 2, P.Ny, P.Kx), complex)
    for _ in range(2):
        hs.step(2e-3)
        st, gp = ns.rk_step(st, gp, P, 2e-3)
    ref = np.stack([ns.to_physical(c, P) for c in st])
    out = hs.get_fields().astype(np.float64)
    for c in range(4):
        assert _rel(out[c], ref[c]) < 2e-5, c
    hs.close()


def _diag_from_raw(acc, p):
    n2 = float(p.Nx * p.Ny) ** 2
    nu_b = 1 - acc[4] / (p.Nx * p.Ny) / p.gamma if p.nfields == 4 else 0.0
    nu_t = 1 - acc[5] / (p.Nx * p.Ny) / p.gamma if p.nfields == 4 else 0.0
    return dict(div=acc[0] / n2 / p.Nz, wu=acc[1] / n2 / 2, ww=acc[2] / n2 / 2,
                flow=acc[3] / (p.Nx * p.Ny) / p.Nz, nu=0.5 * (nu_b + nu_t))


def test_diagnostics_match_oracle():
    import ctypes
    N, Nz = 16, 33
    kw = dict(nu=3.162e-3, kappa=3.162e-3, gamma=1.0)
    hs = HostSim(Nx=N, Ny=N, Nz=Nz, nfields=4, prec="f64", **kw)
    P = ns.Params(N, N, Nz, nfields=4, **kw)
    f = synth.boussinesq_fields(N, N, Nz, amp=1e-1)
    f[0] += 0.3 * (synth.z_grid(Nz) * (1 - synth.z_grid(Nz)))[:, None, None]
    hs.set_fields(f)
    hs.step(2e-3)
    st = ns.to_spectral(f, P)
    st, _ = ns.rk_step(st, np.zeros((2, 2, N, N // 2 + 1), complex), P, 2e-3)
    acc = np.zeros(6)
    assert hs.lib.fchc_ns_diag_raw(ctypes.c_void_p(hs.h), acc.ctypes.data_as(ctypes.c_void_p)) == 0
    d = _diag_from_raw(acc, hs.p)
    div = (ns.divergence_phys(st, P) ** 2).mean()
    wu, wv, ww = ns.wall_mean_squares(st, P)
    nb, nt = ns.nusselt(st, P)
    # div v ~ 4e-8 here is a difference of O(1) derivatives: its rounding floor
    # (~1e-15 absolute) limits the relative agreement of its mean square to ~1e-7
    assert abs(d["div"] - div) <= 1e-6 * div
    assert abs(d["wu"] - wu) <= 1e-10 * wu
    assert abs(d["ww"] - ww) <= 1e-12 * max(wu, 1e-30)
    assert abs(d["flow"] - ns.flow_rate(st, P)) <= 1e-12
    assert abs(d["nu"] - 0.5 * (nb + nt)) <= 1e-10
    hs.close()


def test_float32_mean_flow_accumulates_in_float64():
    """Float64 island of the float32 path: the mean-flow line of a decaying
    profile u = 0.5 sin(pi z) (plus weak solenoidal fluctuations) follows the
    float64 run over 100 steps to the float32 rounding of the output fields
    (2 ulps); the GPU test runs 2000 steps, where float32 accumulation of the
    line would drift by ~1e-6."""
    N, Nz = 16, 33
    z = synth.z_grid(Nz)
    f = synth.channel_velocity(N, N, Nz, mean_flow=False, fluct=0.01)
    f[0] += 0.5 * np.sin(np.pi * z)[:, None, None]
    f = f.astype(np.float32).astype(np.float64)
    means = []
    for prec in ("f32", "f64"):
        hs = HostSim(Nx=N, Ny=N, Nz=Nz, nu=1e-2, prec=prec)
        hs.set_fields(f)
        for _ in range(100):
            hs.step(1e-3)
        means.append(hs.get_fields()[0].astype(np.float64).mean(axis=(1, 2)))
        hs.close()
    rel = np.abs(means[0] - means[1]).max() / np.abs(means[1]).max()
    assert rel < 2.4e-7, rel


@pytest.mark.parametrize("src,dst", [((16, 16, 33), (32, 32, 65)), ((16, 16, 33), (16, 16, 49)),
                                     ((32, 32, 33), (32, 32, 33))])
def test_interpolation_matches_oracle(src, dst):
    """Restart on another grid (Sec. 6): KInterp + re-continuation vs the
    oracle's zero padding / series evaluation (float64)."""
    hs1 = HostSim(Nx=src[0], Ny=src[1], Nz=src[2], nu=1e-2, prec="f64")
    hs2 = HostSim(Nx=dst[0], Ny=dst[1], Nz=dst[2], nu=1e-2, prec="f64")
    P1, P2 = ns.Params(*src), ns.Params(*dst)
    v = synth.channel_velocity(*src)
    hs1.set_fields(v)
    hs1.step(1e-3)                     # a state that is not a plain continuation
    st = ns.to_spectral(v, P1)
    st, _ = ns.rk_step(st, np.zeros((2, 2, src[1], P1.Kx), complex), P1, 1e-3)
    assert hs2.interpolate_from(hs1) == 0
    ref = ns.to_physical(ns.spectral_interpolate(st, P1, P2), P2)
    assert _rel(hs2.get_fields(), ref) < 1e-12
    hs1.close()
    hs2.close()



def test_profiles_kernel_matches_oracle():
    """KProf sums (Parseval from the state rows) vs the oracle's physical-space
    statistics: means, r.m.s. profiles and the z-averaged shell spectrum."""
    N, Nz = 32, 33
    hs = HostSim(Nx=N, Ny=N, Nz=Nz, nu=1e-2, prec="f64")
    P = ns.Params(N, N, Nz)
    v = synth.channel_velocity(N, N, Nz)
    hs.set_fields(v)
    st = ns.to_spectral(v, P)
    mean, rms = ns.profiles(st, P)
    E, dk = ns.shell_spectrum(st, P)
    raw = hs.profiles_raw(E.shape[1])
    n2 = float(N * N) ** 2
    np.testing.assert_allclose(raw[..., 1] / (N * N), mean, atol=1e-13 * np.abs(mean).max())
    np.testing.assert_allclose(np.sqrt(raw[..., 0] / n2), rms, rtol=1e-12, atol=1e-15)
    wz = np.full(Nz, 1.0 / (Nz - 1))
    wz[[0, -1]] *= 0.5
    spec = np.einsum("fzj,z->fj", raw[..., 2:], wz) / n2
    np.testing.assert_allclose(spec, E, rtol=1e-12, atol=1e-14 * E.max())
    hs.close()



@pytest.mark.parametrize("Nz", [33, 39])
def test_alternative_tiles_match_oracle(Nz):
    """Every kernel kind of the step with its alternative (autotuner) tile size:
    padded (Nz = 33) and direct (Nz = 39, N' = 64) z lengths."""
    N = 16 if Nz == 39 else 32
    hs = HostSim(Nx=N, Ny=N, Nz=Nz, nu=1e-2, forcing_x=0.1, prec="f64")
    hs.set_tiles([1, 1, 1, 1, 1])
    P = ns.Params(N, N, Nz, nu=1e-2, forcing_x=0.1)
    v = synth.channel_velocity(N, N, Nz)
    hs.set_fields(v)
    st = ns.to_spectral(v, P)
    gp = np.zeros((2, 2, N, P.Kx), complex)
    for _ in range(2):
        hs.step(1e-3)
        st, gp = ns.rk_step(st, gp, P, 1e-3)
    ref = np.stack([ns.to_physical(c, P) for c in st])
    assert _rel(hs.get_fields(), ref) < 1e-12
    hs.close()


@pytest.mark.parametrize("Nz,N", [(33, 32), (65, 16)])
@pytest.mark.parametrize("tiles", [[2, 2, 2, 0, 0], [3, 3, 3, 1, 1]])
def test_alternative_radix_schedules_match_oracle(Nz, N, tiles):
    """float32 z kernels with the second radix schedule of their padded length
    (160 = 16 x 10, 288 = 18 x 16), with both tiles, against the oracle; the
    first-pass length and the engine twiddles change, the result only by
    float32 rounding."""
    kw = dict(nfields=4, nu=3e-3, kappa=3e-3, gamma=1.0)
    hs = HostSim(Nx=N, Ny=N, Nz=Nz, prec="f32", **kw)
    hs.set_tiles(tiles)
    P = ns.Params(N, N, Nz, **kw)
    v = synth.boussinesq_fields(N, N, Nz, amp=1e-1)
    hs.set_fields(v)
    st = ns.to_spectral(v, P)
    gp = np.zeros((2, 2, N, P.Kx), complex)
    for _ in range(2):
        hs.step(1e-3)
        st, gp = ns.rk_step(st, gp, P, 1e-3)
    ref = np.stack([ns.to_physical(c, P) for c in st])
    out = hs.get_fields()
    for f in range(4):
        assert _rel(out[f], ref[f]) < 5e-5, f
    hs.close()


def test_wide_y_tiles_bitwise_and_match_oracle():
    """Ny = 128 (float32): the wide alternative y tiles (16 lines; the y
    inverse with one exchange buffer and its dy input read again from global
    memory) give bitwise the defaults' step, which matches the oracle."""
    Nx, Ny, Nz = 16, 128, 33
    kw = dict(nu=1e-2, forcing_x=0.1)
    v = synth.channel_velocity(Nx, Ny, Nz)
    outs = []
    for tiles in ([0, 0, 0, 0, 0], [0, 0, 0, 1, 1]):
        hs = HostSim(Nx=Nx, Ny=Ny, Nz=Nz, prec="f32", **kw)
        hs.set_tiles(tiles)
        hs.set_fields(v)
        hs.step(1e-3)
        outs.append(hs.get_fields())
        hs.close()
    assert np.array_equal(outs[0], outs[1])
    P = ns.Params(Nx, Ny, Nz, **kw)
    st, _ = ns.rk_step(ns.to_spectral(v, P), np.zeros((2, 2, Ny, P.Kx), complex), P, 1e-3)
    ref = np.stack([ns.to_physical(c, P) for c in st])
    assert _rel(outs[1], ref) < 1e-5


@pytest.mark.parametrize("tiles", [[0, 0, 0, 0, 0], [1, 1, 1, 1, 1]])
def test_padded_1080_boussinesq_matches_oracle(tiles):
    """The z kernels at the benchmark's transform length (Nz = 513, N' = 538,
    L = 1080 = 30 x 36: 4-line z derivatives, 8-line stage combine and
    projection, and their alternative tiles), float32 Boussinesq, two RK3
    steps on a 16 x 16 horizontal grid against the oracle."""
    N, Nz = 16, 513
    kw = dict(nu=3.162e-4, kappa=3.162e-4, gamma=1.0)
    hs = HostSim(Nx=N, Ny=N, Nz=Nz, nfields=4, prec="f32", **kw)
    hs.set_tiles(tiles)
    P = ns.Params(N, N, Nz, nfields=4, **kw)
    v = synth.boussinesq_fields(N, N, Nz, amp=1e-1)
    hs.set_fields(v)
    st = ns.to_spectral(v, P)
    gp = np.zeros((2, 2, N, P.Kx), complex)
    for _ in range(2):
        hs.step(1e-3)
        st, gp = ns.rk_step(st, gp, P, 1e-3)
    ref = np.stack([ns.to_physical(c, P) for c in st])
    out = hs.get_fields()
    for f in range(4):
        assert _rel(out[f], ref[f]) < 5e-5, (f, _rel(out[f], ref[f]))
    hs.close()


def test_autotuner_keeps_state_and_caches():
    """ns_tune mode 1 run on the CPU emulation (variants timed by host wall
    clock): the choice stays within each kind's variants (tile bit; radix bit
    only for the z kinds of float32 padded lengths with a second schedule),
    the state and the wall planes are left as they were (the step afterwards
    equals the step of an untuned twin run with the same variants), and a
    second simulation of the same size gets the cached choice."""
    N, Nz = 16, 33
    kw = dict(nu=1e-2, forcing_x=0.1)
    v = synth.channel_velocity(N, N, Nz)
    hs = HostSim(Nx=N, Ny=N, Nz=Nz, prec="f32", **kw)
    hs.set_fields(v)
    hs.step(1e-3)                       # non-zero wall planes before tuning
    st0 = hs.get_state()
    choice = hs.autotune()
    assert all(0 <= c <= 3 for c in choice[:3]) and all(c in (0, 1) for c in choice[3:])
    assert np.array_equal(hs.get_state(), st0)
    hs.step(1e-3)
    twin = HostSim(Nx=N, Ny=N, Nz=Nz, prec="f32", **kw)
    twin.set_fields(v)
    twin.step(1e-3)                     # defaults, as hs before tuning
    twin.set_tiles(choice)
    twin.step(1e-3)
    assert np.array_equal(hs.get_fields(), twin.get_fields())
    assert twin.autotune() == choice    # cached per size
    hs.close()
    twin.close()


def test_general_parameters_match_oracle():
    """Everything away from the defaults at once: exponential filter in x, y
    and z (mode 0), a 4 x 3 x 2 box with Nx != Ny, kappa != nu, gamma = 2.5,
    fourth-order time splitting, float64."""
    kw = dict(nfields=4, nu=1e-3, kappa=2e-3, gamma=2.5, rk_order=4, filter=0, Lx=4.0, Ly=3.0, Lz=2.0)
    Nx, Ny, Nz = 32, 16, 33
    hs = HostSim(Nx=Nx, Ny=Ny, Nz=Nz, prec="f64", **kw)
    P = ns.Params(Nx, Ny, Nz, **kw)
    f = synth.boussinesq_fields(Nx, Ny, Nz, Lz=2.0, amp=1e-1)
    assert _rel(hs.rhs(f), ns.ns_rhs(f, P)) < 1e-12
    hs.set_fields(f)
    st = ns.to_spectral(f, P)
    gp = np.zeros((2, 2, Ny, P.Kx), complex)
    for _ in range(2):
        hs.step(2e-3)
        st, gp = ns.rk_step(st, gp, P, 2e-3)
    ref = np.stack([ns.to_physical(c, P) for c in st])
    assert _rel(hs.get_fields(), ref) < 1e-12
    hs.close()
