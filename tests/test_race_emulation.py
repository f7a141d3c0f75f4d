"""Race and initialisation checks of the kernels on the CPU (no GPU involved).

The host-check library runs each kernel's phase functions thread by thread,
with a block barrier between phases.  Rerunning with the threads of every
phase in descending order and with shared memory filled with NaN bytes at the
start of every block changes the result of any kernel in which a thread reads
shared memory that another thread writes in the same phase (a missing
__syncthreads) or that the block never wrote.  Every kernel sequence below
must give bitwise the same outputs under both settings."""
import ctypes
import os

import numpy as np
import pytest

from conftest import ROOT
from hostcheck_ns import HostSim
import synth

HC = os.path.join(ROOT, "paper_2002_01392_gb300", "libfcns_hostcheck.so")


@pytest.fixture(scope="module")
def hc():
    import __graft_entry__
    __graft_entry__.build()
    lib = ctypes.CDLL(HC)
    lib.fchc_set_emulation.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.fchc_set_emulation.restype = None
    yield lib
    lib.fchc_set_emulation(0, 0)


def _vp(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _both(hc, run):
    hc.fchc_set_emulation(0, 0)
    ref = run()
    hc.fchc_set_emulation(1, 1)
    try:
        chk = run()
    finally:
        hc.fchc_set_emulation(0, 0)
    for a, b in zip(ref, chk):
        assert np.all(np.isfinite(a))
        assert np.array_equal(a.view(np.uint8), b.view(np.uint8))


@pytest.mark.parametrize("Nz,L,Nx,Ny", [(33, 160, 5, 3), (39, 64, 4, 3), (129, 288, 3, 1), (513, 1080, 3, 1)])
@pytest.mark.parametrize("dtype", [0, 1])
def test_deriv_kernel_race_free(hc, Mr_5_25, Nz, L, Nx, Ny, dtype):
    sf = synth.SeparableField(Nx, Ny, Nz, rank=2, seed_offset=Nz + 3)
    f = np.ascontiguousarray(sf.field(0)[None].astype(np.float32 if dtype == 0 else np.float64))

    def run():
        d1, d2 = np.zeros_like(f), np.zeros_like(f)
        assert hc.fchc_deriv_z(dtype, L, _vp(Mr_5_25), 5, 25, Nz, 1, Nx, Ny, ctypes.c_double(1.0),
                               _vp(f), _vp(d1), _vp(d2)) == 0
        return d1, d2

    _both(hc, run)


@pytest.mark.parametrize("N,Nz,nf,prec,tiles", [(32, 33, 3, "f64", None), (16, 33, 4, "f32", None),
                                                 (16, 39, 3, "f32", None), (16, 33, 4, "f32", [3, 3, 3, 1, 1]),
                                                 ((16, 128), 33, 3, "f32", [0, 0, 0, 1, 1]),
                                                 (16, 513, 4, "f32", None), (16, 513, 4, "f32", [1, 1, 1, 1, 1]),
                                                 (16, 487, 4, "f32", None)])
def test_ns_kernels_race_free(hc, N, Nz, nf, prec, tiles):
    """RK3 step (every z / y / x kernel of a stage, the mean line, the
    projection), the right-hand side, the projection call and get_fields; the
    Nz = 39 case runs the direct length-64 z transforms; then the alternative
    tiles and radix schedules, the wide y tiles (Ny = 128), the benchmark's
    z length 1080 (Nz = 513) with both tiles, and the direct length 512
    (Nz = 487)."""
    Nx, Ny = (N, N) if isinstance(N, int) else N
    kw = dict(nu=3e-3, kappa=3e-3, gamma=1.0) if nf == 4 else dict(nu=1e-2, forcing_x=0.1)
    v = synth.boussinesq_fields(Nx, Ny, Nz, amp=1e-1) if nf == 4 else synth.channel_velocity(Nx, Ny, Nz)
    g = np.random.default_rng(5)
    vs = v[:3] + 1e-2 * g.standard_normal(v[:3].shape)

    def run():
        hs = HostSim(Nx=Nx, Ny=Ny, Nz=Nz, nfields=nf, prec=prec, **kw)
        try:
            if tiles:
                hs.set_tiles(tiles)
            hs.set_fields(v)
            r = hs.rhs(v)
            pv, gp = hs.project(vs, 1e-3)
            hs.step(1e-3)
            return r, pv, gp, hs.get_fields(), hs.get_state()
        finally:
            hs.close()

    _both(hc, run)


def test_nonfinite_count_on_host():
    """KFinite on the CPU: counts Inf / NaN in physical lines only (padding
    lines kx >= Kx are not part of the state)."""
    N, Nz = 16, 33
    hs = HostSim(Nx=N, Ny=N, Nz=Nz, nu=1e-2, prec="f64")
    try:
        hs.set_fields(synth.channel_velocity(N, N, Nz))
        assert hs.count_nonfinite() == 0
        st = hs.get_state()
        Kx, Kxp, Np, TL = N // 2 + 1, 16, Nz + 25, 16
        ntiles = N * Kxp // TL

        def idx(f, z, ky, kx):
            line = ky * Kxp + kx
            return ((f * ntiles + line // TL) * Np + z) * TL + line % TL

        bad = st.copy()
        bad[idx(0, 0, 0, 0)] = complex(np.nan, 0.0)          # 1
        bad[idx(2, Np - 1, N - 1, Kx - 1)] = complex(np.inf, -np.inf)  # 2
        bad[idx(1, 7, 3, Kx)] = complex(np.nan, np.nan)      # padding line: not counted
        hs.put_state(bad)
        assert hs.count_nonfinite() == 3
        hs.put_state(st)
        assert hs.count_nonfinite() == 0
    finally:
        hs.close()
