"""Runs the kernel sequences of the host-check library built with
AddressSanitizer (guard bands between the workspace arrays poisoned): every
derivative shape in both precisions and every simulation call on a few small
grids.  Started in a subprocess that preloads libasan by
test_memory_safety.py; exits 0 when no access strayed (the sanitizer aborts
the process on the first bad access)."""
import ctypes
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

from oracle.fc_tables import fc_matrix  # noqa: E402  (precomputed tables, as the CPU tests use)
import synth  # noqa: E402


def _vp(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def main(path):
    lib = ctypes.CDLL(path)
    lib.fchc_ns_create.restype = ctypes.c_void_p
    lib.fchc_ns_create.argtypes = [ctypes.c_void_p]
    for n in ("fchc_ns_set_fields", "fchc_ns_get_fields", "fchc_ns_rhs", "fchc_ns_step", "fchc_ns_project",
              "fchc_ns_destroy", "fchc_ns_get_state", "fchc_ns_put_state", "fchc_ns_diag_raw",
              "fchc_ns_interpolate", "fchc_ns_profiles_raw", "fchc_ns_count_nonfinite", "fchc_ns_set_tiles"):
        getattr(lib, n).argtypes = None
    Mr = fc_matrix(5, 25, table_dir=os.path.join(HERE, "golden"))
    for Nz, L in ((33, 96), (33, 160), (39, 64), (129, 288), (513, 1080)):
        for dtype, npdt in ((0, np.float32), (1, np.float64)):
            f = np.ascontiguousarray(synth.SeparableField(3, 2, Nz).field(0)[None].astype(npdt))
            d1, d2 = np.empty_like(f), np.empty_like(f)
            assert lib.fchc_deriv_z(dtype, L, _vp(Mr), 5, 25, Nz, 1, 3, 2, ctypes.c_double(1.0),
                                    _vp(f), _vp(d1), _vp(d2)) == 0
            assert np.isfinite(d1).all() and np.isfinite(d2).all()

    from paper_2002_01392_gb300.api import ns_params
    cases = [dict(Nx=32, Ny=32, Nz=33, prec="f64", nu=1e-2, forcing_x=0.1),
             dict(Nx=32, Ny=16, Nz=33, nfields=4, prec="f32", nu=3e-3, kappa=2e-3, gamma=1.0),
             dict(Nx=16, Ny=16, Nz=39, prec="f32", nu=1e-2),
             dict(Nx=16, Ny=128, Nz=33, prec="f32", nu=1e-2),
             dict(Nx=16, Ny=16, Nz=513, nfields=4, prec="f32", nu=3.162e-4, kappa=3.162e-4, gamma=1.0),
             dict(Nx=16, Ny=16, Nz=487, prec="f64", nu=3.162e-4),
             dict(Nx=16, Ny=16, Nz=1511, prec="f32", nu=3.162e-4)]     # N' = 1536, the longest line
    for kw in cases:
        p = ns_params(**kw)
        nf = p.nfields
        npdt = np.float32 if p.prec == 0 else np.float64
        h = ctypes.c_void_p(lib.fchc_ns_create(ctypes.addressof(p)))
        assert h.value
        if nf == 4:
            v = synth.boussinesq_fields(p.Nx, p.Ny, p.Nz, amp=1e-1)
        else:
            v = synth.channel_velocity(p.Nx, p.Ny, p.Nz)
        v = np.ascontiguousarray(v.astype(npdt))
        out = np.empty_like(v)
        gp = np.empty((2, 2, p.Ny, p.Nx // 2 + 1), complex)
        assert lib.fchc_ns_set_fields(h, _vp(v)) == 0
        assert lib.fchc_ns_rhs(h, _vp(v), _vp(out)) == 0
        vs = np.ascontiguousarray(v[:3])
        po = np.empty_like(vs)
        assert lib.fchc_ns_project(h, ctypes.c_double(1e-3), _vp(vs), _vp(po), _vp(gp)) == 0
        for tiles in ([0] * 5, [1] * 5, [3] * 5):
            t = np.array(tiles, np.int32)
            assert lib.fchc_ns_set_tiles(h, _vp(t)) == 0
            assert lib.fchc_ns_step(h, ctypes.c_double(1e-3)) == 0
        assert lib.fchc_ns_get_fields(h, _vp(out)) == 0
        Kxp = (p.Nx // 2 + 1 + 15) // 16 * 16
        st = np.empty(nf * (p.Nz + p.C) * p.Ny * Kxp, np.complex64 if p.prec == 0 else np.complex128)
        assert lib.fchc_ns_get_state(h, _vp(st)) == 0
        assert lib.fchc_ns_put_state(h, _vp(st)) == 0
        cnt = ctypes.c_longlong()
        assert lib.fchc_ns_count_nonfinite(h, ctypes.byref(cnt)) == 0 and cnt.value == 0
        acc = np.empty(6)
        assert lib.fchc_ns_diag_raw(h, _vp(acc)) == 0
        kxm, kym = math.pi * p.Nx / p.Lx, math.pi * p.Ny / p.Ly
        ns = int(math.floor(math.hypot(kxm, kym) / min(2 * math.pi / p.Lx, 2 * math.pi / p.Ly) + 0.5)) + 1
        prof = np.empty((nf, p.Nz, 2 + ns))
        assert lib.fchc_ns_profiles_raw(h, _vp(prof)) == 0
        if p.Nx == p.Ny == 16 and p.Nz < 100:  # restart on a grid twice as fine in x and y
            p2 = ns_params(**dict(kw, Nx=32, Ny=32))
            h2 = ctypes.c_void_p(lib.fchc_ns_create(ctypes.addressof(p2)))
            assert h2.value
            assert lib.fchc_ns_interpolate(h2, h) == 0
            assert lib.fchc_ns_step(h2, ctypes.c_double(1e-3)) == 0
            lib.fchc_ns_destroy(h2)
        lib.fchc_ns_destroy(h)
    print("asan driver: all sequences ran")


if __name__ == "__main__":
    main(sys.argv[1])
