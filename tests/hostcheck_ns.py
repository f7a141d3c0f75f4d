"""ctypes access to the CPU execution of the NS kernel sequence (host-check library)."""
import ctypes
import os

import numpy as np

from conftest import ROOT

HC = os.path.join(ROOT, "paper_2002_01392_gb300", "libfcns_hostcheck.so")


class HostSim:
    def __init__(self, **kw):
        import __graft_entry__
        __graft_entry__.build()
        from paper_2002_01392_gb300.api import ns_params
        self.lib = ctypes.CDLL(HC)
        self.lib.fchc_ns_create.restype = ctypes.c_void_p
        self.lib.fchc_ns_create.argtypes = [ctypes.c_void_p]
        for n in ("fchc_ns_set_fields", "fchc_ns_get_fields", "fchc_ns_rhs", "fchc_ns_step", "fchc_ns_project",
                  "fchc_ns_destroy", "fchc_ns_get_state", "fchc_ns_diag_raw", "fchc_ns_interpolate",
                  "fchc_ns_profiles_raw", "fchc_ns_set_tiles", "fchc_ns_put_state", "fchc_ns_count_nonfinite", "fchc_ns_autotune"):
            getattr(self.lib, n).argtypes = None
        self.p = ns_params(**kw)
        self.h = self.lib.fchc_ns_create(ctypes.addressof(self.p))
        assert self.h, "host-check create failed"
        self.dt = np.float32 if self.p.prec == 0 else np.float64
        self.shape = (self.p.nfields, self.p.Nz, self.p.Ny, self.p.Nx)

    @staticmethod
    def _vp(a):
        return a.ctypes.data_as(ctypes.c_void_p)

    def set_fields(self, v):
        a = np.ascontiguousarray(v, dtype=self.dt)
        assert self.lib.fchc_ns_set_fields(ctypes.c_void_p(self.h), self._vp(a)) == 0

    def get_fields(self):
        out = np.zeros(self.shape, dtype=self.dt)
        assert self.lib.fchc_ns_get_fields(ctypes.c_void_p(self.h), self._vp(out)) == 0
        return out

    def rhs(self, v):
        a = np.ascontiguousarray(v, dtype=self.dt)
        out = np.zeros_like(a)
        assert self.lib.fchc_ns_rhs(ctypes.c_void_p(self.h), self._vp(a), self._vp(out)) == 0
        return out

    def project(self, v, dt):
        a = np.ascontiguousarray(v, dtype=self.dt)
        out = np.zeros_like(a)
        gp = np.zeros((2, 2, self.p.Ny, self.p.Nx // 2 + 1), dtype=complex)
        assert self.lib.fchc_ns_project(ctypes.c_void_p(self.h), ctypes.c_double(dt), self._vp(a), self._vp(out),
                                        self._vp(gp)) == 0
        return out, gp

    def set_tiles(self, tiles):
        arr = np.ascontiguousarray(tiles, dtype=np.int32)
        assert self.lib.fchc_ns_set_tiles(ctypes.c_void_p(self.h), self._vp(arr)) == 0

    def profiles_raw(self, nshell):
        out = np.zeros((self.p.nfields, self.p.Nz, 2 + nshell))
        assert self.lib.fchc_ns_profiles_raw(ctypes.c_void_p(self.h), self._vp(out)) == 0
        return out

    def interpolate_from(self, src):
        return self.lib.fchc_ns_interpolate(ctypes.c_void_p(self.h), ctypes.c_void_p(src.h))

    def get_state(self):
        Kxp = (self.p.Nx // 2 + 1 + 15) // 16 * 16
        n = self.p.nfields * (self.p.Nz + self.p.C) * self.p.Ny * Kxp
        out = np.zeros(n, dtype=np.complex64 if self.p.prec == 0 else np.complex128)
        assert self.lib.fchc_ns_get_state(ctypes.c_void_p(self.h), self._vp(out)) == 0
        return out

    def put_state(self, st):
        a = np.ascontiguousarray(st)
        assert self.lib.fchc_ns_put_state(ctypes.c_void_p(self.h), self._vp(a)) == 0

    def autotune(self):
        out = np.zeros(5, dtype=np.int32)
        assert self.lib.fchc_ns_autotune(ctypes.c_void_p(self.h), self._vp(out)) == 0
        return [int(x) for x in out]

    def count_nonfinite(self):
        n = ctypes.c_longlong()
        assert self.lib.fchc_ns_count_nonfinite(ctypes.c_void_p(self.h), ctypes.byref(n)) == 0
        return n.value

    def step(self, dt):
        assert self.lib.fchc_ns_step(ctypes.c_void_p(self.h), ctypes.c_double(dt)) == 0

    def close(self):
        if self.h:
            self.lib.fchc_ns_destroy(ctypes.c_void_p(self.h))
            self.h = None
