"""Pins of the Navier-Stokes / Boussinesq oracle (CPU)."""
import math

import numpy as np
import pytest

from oracle import ns
import synth


def _zeros_gp(p):
    return np.zeros((2, 2, p.Ny, p.Kx), dtype=complex)


def test_poiseuille_is_a_fixed_point(Mr_5_25):
    """Sec. 6 laminar solution with F/nu = 10 (runs L1-L3): max U = 1.25 and one
    RK3 step leaves it unchanged up to the FC second-derivative floor."""
    nu = 1e-2
    p = ns.Params(32, 32, 33, nu=nu, forcing_x=10 * nu, Mr=Mr_5_25)
    v = synth.poiseuille(32, 32, 33, F=10 * nu, nu=nu)
    assert abs(v[0].max() - 1.25) < 1e-12
    st = ns.to_spectral(v, p)
    st2, gp = ns.rk_step(st, _zeros_gp(p), p, 1e-3)
    v2 = np.stack([ns.to_physical(c, p) for c in st2])
    assert np.abs(v2 - v).max() < 1e-10 * 1.25
    rhs = ns.ns_rhs(v, p)
    assert np.abs(rhs).max() < 1e-8


def test_rhs_closed_form(Mr_5_25):
    """-(v.grad)v + nu lap v for v = (z sin y, z cos x, 0): polynomial z-dependence
    of degree < d is differentiated exactly, so the RHS has a closed form."""
    N, Nz, nu = 16, 33, 0.3
    p = ns.Params(N, N, Nz, nu=nu, Mr=Mr_5_25)
    x = np.arange(N) * 2 * np.pi / N
    z = synth.z_grid(Nz)
    Z, Y, X = np.meshgrid(z, x, x, indexing="ij")
    v = np.stack([Z * np.sin(Y), Z * np.cos(X), 0 * Z])
    rhs = ns.ns_rhs(v, p)
    ex_u = -(Z * np.cos(X) * Z * np.cos(Y)) - nu * Z * np.sin(Y)
    ex_v = -(Z * np.sin(Y) * (-Z * np.sin(X))) - nu * Z * np.cos(X)
    assert np.abs(rhs[0] - ex_u).max() < 1e-8
    assert np.abs(rhs[1] - ex_v).max() < 1e-8
    assert np.abs(rhs[2]).max() < 1e-8


def test_boussinesq_buoyancy_sign_and_theta_source(Mr_5_25):
    """Sec. 7 with reading B1: dw/dt gets +gamma theta; dtheta/dt gets +gamma w."""
    N, Nz = 8, 33
    p = ns.Params(N, N, Nz, nfields=4, nu=1e-3, kappa=0.5, gamma=2.0, Mr=Mr_5_25)
    z = synth.z_grid(Nz)
    f = np.zeros((4, Nz, N, N))
    f[3] = (z * (1 - z))[:, None, None]
    rhs = ns.ns_rhs(f, p)
    assert np.abs(rhs[2] - 2.0 * f[3]).max() < 1e-9
    assert np.abs(rhs[3] - 0.5 * (-2.0)).max() < 1e-8
    g = np.zeros((4, Nz, N, N))
    g[2] = 0.25
    rhs = ns.ns_rhs(g, p)
    assert np.abs(rhs[3] - 2.0 * 0.25).max() < 1e-9


def test_conduction_state_is_exactly_fixed(Mr_5_25):
    p = ns.Params(16, 16, 33, nfields=4, nu=3.162e-4, kappa=3.162e-4, gamma=1.0, Mr=Mr_5_25)
    st = np.zeros((4, p.Np, p.Ny, p.Kx), dtype=complex)
    st2, gp = ns.rk_step(st, _zeros_gp(p), p, 1e-3)
    assert np.abs(st2).max() == 0.0 and np.abs(gp).max() == 0.0
    assert ns.nusselt(st2 + 0.0, p) == (1.0, 1.0)


@pytest.mark.parametrize("Lz", [1.0, 2.0])
def test_nusselt_closed_form(Mr_5_25, Lz):
    """Sec. 7 Nusselt number with reading B2, Nu = 1 - <d_z theta>/gamma at each
    wall.  theta = a z (Lz - z) + c z^2 (Lz - z) + (zero horizontal mean part)
    is a polynomial of degree 3 < d in z, differentiated exactly by FC-Gram, so
    <d_z theta> = a Lz at z = 0 and -a Lz - c Lz^2 at z = Lz, and
    Nu = (1 - a Lz / gamma, 1 + (a Lz + c Lz^2) / gamma).  The cubic term makes
    the two walls differ, gamma != 1 exposes a misplaced 1/gamma, the
    x, y-varying part exposes a sum in place of a mean, and a w with wall
    gradients of its own exposes a wrong field."""
    N, Nz, gamma, a, c = 16, 33, 2.5, 0.8, -0.3
    p = ns.Params(N, N, Nz, nfields=4, nu=1e-3, kappa=1e-3, gamma=gamma, Lz=Lz, Mr=Mr_5_25)
    z = synth.z_grid(Nz, Lz)
    x = np.arange(N) * 2 * np.pi / N
    Z, Y, X = np.meshgrid(z, x, x, indexing="ij")
    f = np.zeros((4, Nz, N, N))
    f[2] = 0.7 * Z * (Lz - Z)
    f[3] = a * Z * (Lz - Z) + c * Z ** 2 * (Lz - Z) + 0.4 * np.cos(2 * X + Y) * Z ** 2 * (Lz - Z)
    nu0, nu1 = ns.nusselt(ns.to_spectral(f, p), p)
    assert abs(nu0 - (1 - a * Lz / gamma)) < 1e-9
    assert abs(nu1 - (1 + (a * Lz + c * Lz ** 2) / gamma)) < 1e-9


def test_flow_rate_is_the_grid_point_mean_of_u(Mr_5_25):
    """Sec. 6 channel diagnostic: the flow rate reported is the mean of u over
    the Nx Ny Nz physical grid points (both walls included), not a quadrature of
    the continuous profile.  For the laminar profile U = F z (1 - z)/(2 nu) on
    z_s = s/(Nz - 1) that mean is F/(2 nu) (Nz - 2)/(6 (Nz - 1)) in closed form
    (sum of s/M - s^2/M^2 over s = 0..M, M = Nz - 1, divided by Nz), which tends
    to the continuous flow rate F/(12 nu) as Nz grows.  A zero-mean x, y
    fluctuation of u and nonzero v, w must not change it."""
    nu, F = 1e-2, 0.1
    for Nz in (17, 33, 65):
        p = ns.Params(16, 8, Nz, nu=nu, forcing_x=F, Mr=Mr_5_25)
        v = synth.poiseuille(16, 8, Nz, F=F, nu=nu)
        z = synth.z_grid(Nz)
        x = np.arange(16) * 2 * np.pi / 16
        v[0] += 0.3 * np.cos(x)[None, None, :] * (z * (1 - z))[:, None, None]
        v[1] += 0.2
        v[2] += (z ** 2)[:, None, None]
        q = ns.flow_rate(ns.to_spectral(v, p), p)
        exact = F / (2 * nu) * (Nz - 2) / (6 * (Nz - 1))
        assert abs(q - exact) < 1e-12 * exact, (Nz, q, exact)
        assert abs(exact - F / (12 * nu)) < F / (12 * nu) * 2.0 / (Nz - 1)


def test_projection_wall_normal_velocity_is_roundoff(Mr_5_25):
    """After projection w = 0 at the walls to round-off (Sec. 6: <w^2|wall> ~ 1e-35)."""
    p = ns.Params(32, 32, 33, nu=1e-2, Mr=Mr_5_25)
    v = _divergent_field(32, 33)
    vp, gp = ns.poisson_project(v, p, 1e-3)
    assert np.abs(vp[2][[0, -1]]).max() < 1e-14
    st = ns.to_spectral(v, p)
    st2, _ = ns.rk_step(st, _zeros_gp(p), p, 1e-3)
    assert ns.wall_mean_squares(st2, p)[2] < 1e-28


def _divergent_field(N, Nz):
    """Solenoidal channel field plus a seeded non-solenoidal, wall-vanishing part."""
    v = synth.channel_velocity(N, N, Nz)
    g = np.random.default_rng(5)
    z = synth.z_grid(Nz)
    for c in range(3):
        X = synth.xy_modes_field(g, N, N)
        v[c] += 0.2 * (z * (1 - z))[:, None, None] * X[None]
    return v


def test_projection_reduces_divergence(Mr_5_25):
    p = ns.Params(32, 32, 33, nu=1e-2, forcing_x=0.1, Mr=Mr_5_25)
    v = _divergent_field(32, 33)
    st = ns.to_spectral(v, p)
    before = (ns.divergence_phys(st, p) ** 2).mean()
    st2, _ = ns.rk_step(st, _zeros_gp(p), p, 1e-3)
    after = (ns.divergence_phys(st2, p) ** 2).mean()
    assert after < 1e-5 * before


def _manufactured(N, Nz, Mr, with_u=True):
    p = ns.Params(N, N, Nz, Mr=Mr)
    x = np.arange(N) * 2 * np.pi / N
    z = synth.z_grid(Nz)
    Z, Y, X = np.meshgrid(z, x, x, indexing="ij")
    h = Z ** 2 * (1 - Z) ** 2
    sx = np.cos(X) * np.cos(2 * Y)
    sy = -2 * np.sin(X) * np.sin(2 * Y)
    u = np.stack([sy * h, -sx * h, 0 * h]) * (1.0 if with_u else 0.0)
    gpsi = np.stack([-np.sin(X) * np.cos(2 * Y) * np.cosh(Z),
                     -2 * np.cos(X) * np.sin(2 * Y) * np.cosh(Z),
                     np.cos(X) * np.cos(2 * Y) * np.sinh(Z) + 3 * Z ** 2])
    vs = u + gpsi
    dt = 1e-3
    m = ns.xy_forward(vs)
    gpp = np.zeros((2, 2, p.Ny, p.Kx), complex)
    gpp[0, 0], gpp[0, 1] = m[0, 0] / dt, m[1, 0] / dt
    gpp[1, 0], gpp[1, 1] = m[0, -1] / dt, m[1, -1] / dt
    v, _ = ns.poisson_project(vs, p, dt, gradp_prev=gpp)
    return np.abs(v - u).max()


def test_manufactured_poisson_converges(Mr_5_25):
    """v* = u + grad psi with u solenoidal and u.z = 0 at the walls: the projection
    returns u, with errors shrinking fast as Nz grows."""
    e = [_manufactured(16, Nz, Mr_5_25) for Nz in (17, 33, 65)]
    assert e[0] < 1e-7 and e[1] < 1e-9 and e[2] < 1e-10
    assert e[2] < e[1] < e[0]
    # a pure gradient is annihilated
    assert _manufactured(16, 65, Mr_5_25, with_u=False) < 1e-10


def test_projection_idempotent_with_consistent_injection(Mr_5_25):
    p = ns.Params(32, 32, 33, Mr=Mr_5_25)
    v = _divergent_field(32, 33)
    vp, g = ns.poisson_project(v, p, 1e-3)
    vp2, _ = ns.poisson_project(vp, p, 1e-3, gradp_prev=-g)
    assert np.abs(vp2 - vp).max() < 1e-6 * np.abs(vp).max()


def test_stage_steps_give_taylor_amplification():
    """Reading R1: the low-storage stages reproduce exp(z) to order o for y' = lam y."""
    for o in (1, 2, 3, 4):
        for zval in (-0.3, 0.2 + 0.5j):
            y0 = 1.0
            y = y0
            for j in range(1, o + 1):
                y = y0 + ns.stage_dt(1.0, o, j) * zval * y
            want = sum(zval ** k / math.factorial(k) for k in range(o + 1))
            assert abs(y - want) < 1e-15


def test_rk3_time_convergence_on_diffusion(Mr_5_25):
    """Third-order global convergence of the full step on theta diffusion."""
    p = ns.Params(8, 8, 33, nfields=4, nu=1e-3, kappa=2e-3, gamma=0.0, Mr=Mr_5_25)
    z = synth.z_grid(33)
    x = np.arange(8) * 2 * np.pi / 8
    f = np.zeros((4, 33, 8, 8))
    f[3] = np.sin(np.pi * z)[:, None, None] * (1 + 0.5 * np.cos(x))[None, None, :]
    st0 = ns.to_spectral(f, p)

    def run(dt, n):
        st, gp = st0, _zeros_gp(p)
        for _ in range(n):
            st, gp = ns.rk_step(st, gp, p, dt)
        return st[3]

    a, b, c = run(0.04, 5), run(0.02, 10), run(0.01, 20)
    r = np.abs(a - b).max() / np.abs(b - c).max()
    assert r > 6.0          # ~8 for third order; ~2 for the printed j dt/o stage steps


def test_filter_factor_values():
    """Sec. 4.3: the Nyquist mode is attenuated by e^{-beta} = 1e-16; the 2/3 mask
    keeps |n| <= N/3 in x and y."""
    p = ns.Params(12, 12, 33)
    F = ns.filter_factor(p)
    nyq = p.Np // 2
    assert abs(F[nyq, 0, 0] - 1e-16) < 1e-28
    assert abs(F[1, 0, 0] - 1.0) < 1e-15
    assert F[0, 0, 4] == 1.0 and F[0, 0, 5] == 0.0
    assert F[0, 4, 0] == 1.0 and F[0, 5, 0] == 0.0 and F[0, -4, 0] == 1.0 and F[0, -5, 0] == 0.0
    p0 = ns.Params(12, 12, 33, filter=0)
    F0 = ns.filter_factor(p0)
    assert abs(F0[0, 0, 6] - 1e-16) < 1e-28


def test_channel_ic_is_solenoidal_no_slip():
    v = synth.channel_velocity(32, 32, 33)
    p = ns.Params(32, 32, 33)
    st = ns.to_spectral(v, p)
    assert np.abs(v[:, [0, -1]]).max() < 1e-15
    assert (ns.divergence_phys(st, p) ** 2).mean() < 1e-10


@pytest.mark.parametrize("o", [2, 3])
def test_multistep_stability_at_nyquist_modes(Mr_5_25, o):
    """Reading K1: with gamma = |k_perp| of the Nyquist-zeroed wavenumbers the
    projection is divergence-consistent at every (kx, ky); several RK steps stay
    bounded (with the true Nyquist wavenumber in gamma the x/y Nyquist modes grow
    by ~1e10 per step from round-off)."""
    p = ns.Params(32, 32, 33, nu=1e-2, forcing_x=0.1, rk_order=o, Mr=Mr_5_25)
    v = synth.channel_velocity(32, 32, 33)
    st = ns.to_spectral(v, p)
    gp = _zeros_gp(p)
    for _ in range(5):
        st, gp = ns.rk_step(st, gp, p, 1e-3)
    v5 = np.stack([ns.to_physical(c, p) for c in st])
    assert np.abs(v5).max() < 1.01 * np.abs(v).max()
    m = ns.z_inverse(st, p)
    assert np.abs(m[:, :, :, p.Nx // 2]).max() < 1e-12
    assert np.abs(m[:, :, p.Ny // 2, :]).max() < 1e-12


def _slip_run(P, v0, dt, T):
    st = ns.to_spectral(v0, P)
    gp = _zeros_gp(P)
    for _ in range(int(round(T / dt))):
        st, gp = ns.rk_step(st, gp, P, dt)
    return ns.wall_mean_squares(st, P)


@pytest.mark.parametrize("o", [1, 2])
def test_wall_slip_converges_with_dt(Mr_5_25, o):
    """Sec. 6 / Sec. 4.4: the tangential slip <u^2|wall> falls like dt^4 (dt^2 in
    r.m.s.) for o = 1 and o = 2 above the resolution floor, while <w^2|wall> stays
    at round-off (the paper reports O(1e-35)) independently of dt."""
    N, Nz = 16, 33
    v0 = synth.channel_velocity(N, N, Nz, nu=1e-2, fluct=1.0)
    P = ns.Params(N, N, Nz, nu=1e-2, forcing_x=0.1, rk_order=o, Mr=Mr_5_25)
    res = [_slip_run(P, v0, dt, 0.032) for dt in (8e-3, 4e-3)]
    order = math.log2(res[0][0] / res[1][0])
    assert order > 3.5, order
    assert max(r[2] for r in res) < 1e-28



def _bandlimited(Nx, Ny, Nz):
    """Band-limited in x, y (including both Nyquist cosines of a 16-point grid),
    smooth in z."""
    x = np.arange(Nx) * 2 * np.pi / Nx
    y = np.arange(Ny) * 2 * np.pi / Ny
    z = synth.z_grid(Nz)
    X, Y = np.meshgrid(x, y)
    a = (np.cos(2 * X + Y)[None] * np.sin(2 * z)[:, None, None]
         + np.cos(3 * X - 2 * Y)[None] * (z ** 2)[:, None, None]
         + np.cos(8 * X)[None] * np.exp(z)[:, None, None] + np.cos(8 * Y)[None] * np.cos(z)[:, None, None])
    return np.stack([a, 0.5 * a, -a])


def test_interpolation_identity():
    """Interpolating onto the same grid returns the same fields."""
    P = ns.Params(16, 16, 33)
    v = synth.channel_velocity(16, 16, 33)
    out = ns.to_physical(ns.spectral_interpolate(ns.to_spectral(v, P), P, P), P)
    assert np.abs(out - v).max() < 1e-13 * np.abs(v).max()


def test_interpolation_horizontal_refinement_is_exact():
    """Same Nz, finer x, y: a band-limited field (Nyquist cosines included) is
    reproduced to round-off on the finer grid."""
    P1, P2 = ns.Params(16, 16, 33), ns.Params(32, 48, 33, Ly=2 * np.pi)
    f1, f2 = _bandlimited(16, 16, 33), _bandlimited(32, 48, 33)
    out = ns.to_physical(ns.spectral_interpolate(ns.to_spectral(f1, P1), P1, P2), P2)
    assert np.abs(out - f2).max() < 1e-12


def test_interpolation_vertical_refinement_converges():
    """Finer Nz: the continued series is evaluated between the old points; the
    error is the FC error of the source grid and falls with its Nz."""
    errs = []
    for nz1, nz2 in ((33, 65), (65, 129)):
        P1, P2 = ns.Params(16, 16, nz1), ns.Params(32, 32, nz2)
        out = ns.to_physical(ns.spectral_interpolate(ns.to_spectral(_bandlimited(16, 16, nz1), P1), P1, P2), P2)
        errs.append(np.abs(out - _bandlimited(32, 32, nz2)).max())
    assert errs[0] < 1e-7 and errs[1] < 3e-9 and errs[1] < errs[0] / 10



def test_profiles_and_spectrum_closed_forms():
    """cos(3x + 4y) g(z) + U(z): mean U, rms |g|/sqrt(2), and all its power in
    shell 5 (|k| = 5) with the trapezoid mean of g^2/2; Parseval sum rule."""
    P = ns.Params(32, 32, 33)
    z = synth.z_grid(33)
    x = np.arange(32) * 2 * np.pi / 32
    X, Y = np.meshgrid(x, x)
    g = np.sin(np.pi * z) * (1 + z)
    U = z * (1 - z)
    f = np.cos(3 * X + 4 * Y)[None] * g[:, None, None] + U[:, None, None]
    phys = np.stack([f, 2 * f, 0 * f])
    st = ns.to_spectral(phys, P)
    mean, rms = ns.profiles(st, P)
    np.testing.assert_allclose(mean[0], U, atol=1e-13)
    np.testing.assert_allclose(rms[1], 2 * np.abs(g) / np.sqrt(2), atol=1e-13)
    E, dk = ns.shell_spectrum(st, P)
    wz = np.full(33, 1 / 32.0)
    wz[[0, -1]] *= 0.5
    assert dk == 1.0 and abs(E[0, 5] - (wz * g ** 2 / 2).sum()) < 1e-14
    assert abs(E[0].sum() - E[0, 5]) < 1e-14
    # sum rule on a general field
    v = synth.channel_velocity(32, 32, 33)
    st = ns.to_spectral(v, P)
    E, _ = ns.shell_spectrum(st, P)
    _, rms = ns.profiles(st, P)
    np.testing.assert_allclose(E.sum(axis=1), (wz * rms ** 2).sum(axis=1), rtol=1e-12)
