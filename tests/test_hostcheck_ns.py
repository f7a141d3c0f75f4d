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
