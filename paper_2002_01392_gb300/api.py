"""Thin Python binding of the libfcns C ABI (argument marshalling only).

Every numerical step runs in the CUDA kernels of ``libfcns.so``; this module
checks tensor dtypes / shapes / devices, passes raw device pointers and the
current CUDA stream, and turns status codes into exceptions.  If the library
is missing the import fails: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfcns.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libfcns.so not built ({LIB_PATH}); run __graft_entry__.build()")

_lib = ctypes.CDLL(LIB_PATH)

FC_F32, FC_F64 = 0, 1

_c_int, _c_double, _vp = ctypes.c_int, ctypes.c_double, ctypes.c_void_p


class FcError(RuntimeError):
    def __init__(self, status: int, where: str):
        name = _lib.fc_status_str(status).decode()
        detail = _lib.fc_last_error().decode()
        super().__init__(f"{where}: {name} ({detail})")
        self.status = status
        self.name = name


class NsParams(ctypes.Structure):
    _fields_ = [("Nx", _c_int), ("Ny", _c_int), ("Nz", _c_int), ("d", _c_int), ("C", _c_int),
                ("nfields", _c_int), ("rk_order", _c_int),
                ("Lx", _c_double), ("Ly", _c_double), ("Lz", _c_double),
                ("nu", _c_double), ("kappa", _c_double), ("gamma", _c_double), ("forcing_x", _c_double),
                ("filter", _c_int), ("filter_beta", _c_double), ("filter_2p", _c_double),
                ("prec", _c_int)]


class NoiseParams(ctypes.Structure):
    _fields_ = [("Lx", _c_double), ("Ly", _c_double), ("Lz", _c_double),
                ("kperp2_min", _c_double), ("kperp2_max", _c_double), ("m_min", _c_int), ("m_max", _c_int),
                ("slope_phi", _c_double), ("slope_psi", _c_double), ("amplitude", _c_double)]


def _sig(name, args, res=_c_int):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res
    return f


_lib.fc_status_str.argtypes = [_c_int]
_lib.fc_status_str.restype = ctypes.c_char_p
_lib.fc_last_error.argtypes = []
_lib.fc_last_error.restype = ctypes.c_char_p
_sig("fc_setup", [_c_int, _c_int, _c_int, ctypes.POINTER(_vp)])
_sig("fc_setup_ex", [_c_int, _c_int, _c_int, _c_int, _c_int, ctypes.POINTER(_vp)])
_sig("fc_plan_matrix", [_vp, ctypes.POINTER(_c_double)])
_sig("fc_plan_info", [_vp] + [ctypes.POINTER(_c_int)] * 5 + [ctypes.POINTER(_c_double)])
_sig("fc_destroy", [_vp])
_sig("ns_interpolate", [_vp, _vp, _vp])
_sig("ns_tune", [_vp, _c_int, ctypes.POINTER(_c_int), _vp])
_sig("ns_profiles", [_vp] + [ctypes.POINTER(_c_double)] * 3 + [_vp])
_sig("ns_spectrum_shells", [_vp, ctypes.POINTER(_c_int), ctypes.POINTER(_c_double)])
_sig("ns_batch_create", [ctypes.POINTER(_vp), _c_int, ctypes.POINTER(_vp)])
_sig("ns_batch_step", [_vp, ctypes.POINTER(_c_double), _vp])
_sig("ns_batch_info", [_vp, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)])
_sig("ns_batch_destroy", [_vp])
_sig("fc_deriv_z", [_vp, _c_int, _c_int, _c_int, _c_int, _c_double, _vp, _vp, _vp, _vp])
_sig("fc_deriv_z_noalloc", [_vp, _c_int, _c_int, _c_int, _c_int, _c_double, _vp, _vp, _vp, _vp])
_sig("fc_deriv_z_host", [_vp, _c_int, _c_int, _c_int, _c_int, _c_double, _vp, _vp, _vp, _vp])
_sig("fc_deriv_z_host_ex", [_vp, _c_int, _c_int, _c_int, _c_int, _c_double, _vp, _vp, _vp, ctypes.c_size_t, _vp])
_sig("fc_count_nonfinite", [_c_int, _vp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong), _vp])
_sig("ns_check_finite", [_vp, ctypes.POINTER(ctypes.c_longlong), _vp])
_sig("ns_set_finite_check", [_vp, _c_int])
_sig("fc_inject_failure", [ctypes.c_char_p, _c_int, ctypes.c_longlong, ctypes.c_longlong])
_sig("fc_alu_probe", [_c_int, _c_int, _vp, ctypes.POINTER(_c_double), _vp])
_sig("ns_set_diag_series", [_vp, _c_int])
_sig("ns_get_diag_series", [_vp, _c_int, ctypes.POINTER(_c_double), ctypes.POINTER(ctypes.c_longlong),
                            ctypes.POINTER(_c_int), _vp])
_sig("fc_noise_params_default", [ctypes.POINTER(NoiseParams)])
_sig("fc_noise_modes", [ctypes.POINTER(NoiseParams), ctypes.POINTER(_c_int)])
_sig("fc_noise", [ctypes.POINTER(NoiseParams), _c_int, _c_int, _c_int, _c_int, ctypes.POINTER(_c_double), _c_int,
                  _vp, _vp])

EXPORTED = ["fc_status_str", "fc_last_error", "fc_setup", "fc_setup_ex", "fc_plan_matrix", "fc_plan_info",
            "fc_destroy", "fc_deriv_z", "fc_deriv_z_noalloc", "ns_params_default", "ns_workspace_bytes", "ns_create", "ns_destroy",
            "ns_set_fields", "ns_get_fields", "ns_get_state", "ns_put_state", "ns_get_wall_gradp",
            "ns_put_wall_gradp", "ns_rhs", "fc_poisson_project", "rk_step", "ns_diagnostics",
            "ns_batch_create", "ns_batch_step", "ns_batch_info", "ns_batch_destroy", "ns_interpolate",
            "ns_profiles", "ns_spectrum_shells", "ns_tune", "fc_count_nonfinite", "ns_check_finite",
            "ns_set_finite_check", "fc_inject_failure", "fc_deriv_z_host", "fc_deriv_z_host_ex", "fc_alu_probe",
            "fc_noise_params_default", "fc_noise_modes", "fc_noise", "ns_set_diag_series", "ns_get_diag_series"]


def _check(status: int, where: str):
    if status != 0:
        raise FcError(status, where)


STATUS = {"FC_OK": 0, "FC_ERR_ARG": 1, "FC_ERR_UNSUPPORTED": 2, "FC_ERR_CUDA": 3, "FC_ERR_NOMEM": 4,
          "FC_ERR_TIMEOUT": 5, "FC_ERR_NONFINITE": 6, "FC_ERR_STATE": 7}


def inject_failure(entry: str, status="FC_ERR_CUDA", skip: int = 0, count: int = 1):
    """fc_inject_failure: after ``skip`` calls of ``entry`` the next ``count``
    calls (all later ones if negative) return ``status`` without doing anything."""
    code = STATUS[status] if isinstance(status, str) else int(status)
    _check(_lib.fc_inject_failure(entry.encode(), code, int(skip), int(count)), "fc_inject_failure")


def clear_injected():
    _check(_lib.fc_inject_failure(None, 0, 0, 0), "fc_inject_failure")


def count_nonfinite(t, stream=None) -> int:
    """fc_count_nonfinite: number of Inf / NaN values of a float32 / float64
    CUDA tensor (synchronous; no exception for a positive count)."""
    if not t.is_cuda:
        raise ValueError("t must be a CUDA tensor")
    n = ctypes.c_longlong()
    st = _lib.fc_count_nonfinite(_dtype_code(t), _ptr(t), t.numel(), ctypes.byref(n), _stream(stream))
    if st not in (0, STATUS["FC_ERR_NONFINITE"]):
        _check(st, "fc_count_nonfinite")
    return n.value


ALU_KINDS = {"ffma": 0, "fadd": 1, "ffma2": 2, "fadd2": 3, "dfma": 4}


def noise_params(**kw) -> NoiseParams:
    """fc_noise_params with the App. A defaults, fields overridden by keyword."""
    p = NoiseParams()
    _check(_lib.fc_noise_params_default(ctypes.byref(p)), "fc_noise_params_default")
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def noise_modes(p: NoiseParams) -> int:
    """Number of (n, l, m) modes (two draws each) of the App. A perturbation."""
    n = _c_int(0)
    _check(_lib.fc_noise_modes(ctypes.byref(p), ctypes.byref(n)), "fc_noise_modes")
    return n.value


def fc_noise(p: NoiseParams, draws, out, stream=None):
    """Write the App. A perturbation built from ``draws`` (2 per mode, host,
    float64 in [0, 1)) into the device tensor ``out`` of shape [3][Nz][Ny][Nx]
    (float32 or float64)."""
    import numpy as np
    d = np.ascontiguousarray(np.asarray(draws, dtype=np.float64))
    if out.dim() != 4 or out.shape[0] != 3 or not out.is_contiguous():
        raise ValueError("out must be a contiguous [3][Nz][Ny][Nx] tensor")
    _, Nz, Ny, Nx = out.shape
    _check(_lib.fc_noise(ctypes.byref(p), _dtype_code(out), Nx, Ny, Nz,
                         d.ctypes.data_as(ctypes.POINTER(_c_double)), int(d.size), _ptr(out), _stream(stream)),
           "fc_noise")
    return out


def alu_probe(kind: str, iters: int, sink, stream=None) -> float:
    """Enqueue the arithmetic-pipe probe kernel (fc_alu_probe); returns the lane
    operations it performs (the caller times it with CUDA events)."""
    ops = _c_double(0.0)
    _check(_lib.fc_alu_probe(ALU_KINDS[kind], int(iters), _ptr(sink), ctypes.byref(ops), _stream(stream)),
           "fc_alu_probe")
    return ops.value


def _stream(stream=None) -> int:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float32:
        return FC_F32
    if t.dtype == torch.float64:
        return FC_F64
    raise TypeError(f"unsupported dtype {t.dtype}")


def _ptr(t):
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


class Plan:
    """FC-Gram continuation plan (``fc_setup``)."""

    def __init__(self, d: int, C: int, Nz: int, M: int | None = None, n_os: int | None = None):
        h = _vp()
        if M is None and n_os is None:
            _check(_lib.fc_setup(d, C, Nz, ctypes.byref(h)), "fc_setup")
        else:
            M = (2 * (d + C)) // 3 if M is None else M
            n_os = 20 if n_os is None else n_os
            _check(_lib.fc_setup_ex(d, C, Nz, M, n_os, ctypes.byref(h)), "fc_setup_ex")
        self.handle = h
        self.d, self.C, self.Nz = d, C, Nz

    def matrix(self):
        import numpy as np
        out = np.empty((self.C, self.d), dtype=np.float64)
        _check(_lib.fc_plan_matrix(self.handle, out.ctypes.data_as(ctypes.POINTER(_c_double))), "fc_plan_matrix")
        return out

    def info(self):
        vals = [_c_int() for _ in range(5)]
        res = _c_double()
        _check(_lib.fc_plan_info(self.handle, *[ctypes.byref(v) for v in vals], ctypes.byref(res)), "fc_plan_info")
        d, C, Nz, M, n_os = (v.value for v in vals)
        return dict(d=d, C=C, Nz=Nz, M=M, n_os=n_os, ls_residual=res.value)

    def close(self):
        if self.handle:
            _lib.fc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fc_setup(d: int, C: int, Nz: int) -> Plan:
    return Plan(d, C, Nz)


def fc_deriv_z(plan: Plan, f, df=None, d2f=None, Lz: float = 1.0, stream=None):
    """z-derivatives of f [batch][Nz][Ny][Nx] (or [Nz][Ny][Nx]) on the GPU."""
    if f.dim() == 3:
        f = f.unsqueeze(0)
        df = df.unsqueeze(0) if df is not None else None
        d2f = d2f.unsqueeze(0) if d2f is not None else None
    if f.dim() != 4 or f.shape[1] != plan.Nz:
        raise ValueError("f must be [batch][Nz][Ny][Nx] with Nz = plan.Nz")
    if not f.is_cuda:
        raise ValueError("f must be a CUDA tensor")
    for o in (df, d2f):
        if o is not None and (o.shape != f.shape or o.dtype != f.dtype or o.device != f.device):
            raise ValueError("outputs must match f in shape, dtype and device")
    B, _, Ny, Nx = f.shape
    _check(_lib.fc_deriv_z(plan.handle, _dtype_code(f), B, Nx, Ny, float(Lz), _ptr(f), _ptr(df), _ptr(d2f),
                           _stream(stream)), "fc_deriv_z")
    return df, d2f

def fc_deriv_z_host(plan: Plan, f, df=None, d2f=None, Lz: float = 1.0, slab_bytes: int | None = None, stream=None):
    """fc_deriv_z on CPU tensors [batch][Nz][Ny][Nx] (page-locked for overlapped
    copies): the library moves them through the GPU in slabs (synchronous)."""
    if f.dim() == 3:
        f = f.unsqueeze(0)
        df = df.unsqueeze(0) if df is not None else None
        d2f = d2f.unsqueeze(0) if d2f is not None else None
    if f.dim() != 4 or f.shape[1] != plan.Nz or f.is_cuda:
        raise ValueError("f must be a CPU tensor [batch][Nz][Ny][Nx] with Nz = plan.Nz")
    for o in (df, d2f):
        if o is not None and (o.shape != f.shape or o.dtype != f.dtype or o.is_cuda):
            raise ValueError("outputs must be CPU tensors matching f in shape and dtype")
    B, _, Ny, Nx = f.shape
    args = (plan.handle, _dtype_code(f), B, Nx, Ny, float(Lz), _ptr(f), _ptr(df), _ptr(d2f))
    if slab_bytes is None:
        _check(_lib.fc_deriv_z_host(*args, _stream(stream)), "fc_deriv_z_host")
    else:
        _check(_lib.fc_deriv_z_host_ex(*args, int(slab_bytes), _stream(stream)), "fc_deriv_z_host_ex")
    return df, d2f

_sig("ns_params_default", [ctypes.POINTER(NsParams)])
_sig("ns_workspace_bytes", [ctypes.POINTER(NsParams), ctypes.POINTER(ctypes.c_size_t)])
_sig("ns_create", [ctypes.POINTER(NsParams), _vp, ctypes.c_size_t, ctypes.POINTER(_vp)])
_sig("ns_destroy", [_vp])
_sig("ns_set_fields", [_vp, _vp, _vp])
_sig("ns_get_fields", [_vp, _vp, _vp])
_sig("ns_get_state", [_vp, _vp, _vp])
_sig("ns_put_state", [_vp, _vp, _vp])
_sig("ns_get_wall_gradp", [_vp, _vp, _vp])
_sig("ns_put_wall_gradp", [_vp, _vp, _vp])
_sig("ns_rhs", [_vp, _vp, _vp, _vp])
_sig("fc_poisson_project", [_vp, _c_double, _vp, _vp, _vp, _vp])
_sig("rk_step", [_vp, _c_double, _vp])
_sig("ns_diagnostics", [_vp] + [ctypes.POINTER(_c_double)] * 5 + [_vp])


def ns_params(**kw) -> NsParams:
    """ns_params with the library defaults, overridden by keyword arguments
    (prec may be given as 'f32' / 'f64')."""
    p = NsParams()
    _check(_lib.ns_params_default(ctypes.byref(p)), "ns_params_default")
    for k, v in kw.items():
        if k == "prec" and isinstance(v, str):
            v = FC_F32 if v == "f32" else FC_F64
        setattr(p, k, v)
    return p


def ns_workspace_bytes(p: NsParams) -> int:
    n = ctypes.c_size_t()
    _check(_lib.ns_workspace_bytes(ctypes.byref(p), ctypes.byref(n)), "ns_workspace_bytes")
    return n.value


class Sim:
    """Navier-Stokes / Boussinesq simulation object (ns_create ... ns_destroy).

    ``workspace``: optional caller-owned uint8 CUDA tensor of at least
    ``ns_workspace_bytes(p)`` bytes; otherwise the library allocates."""

    def __init__(self, p: NsParams, workspace=None):
        import torch
        self.p = p
        self.dtype = torch.float32 if p.prec == FC_F32 else torch.float64
        self.cdtype = torch.complex64 if p.prec == FC_F32 else torch.complex128
        self.shape = (p.nfields, p.Nz, p.Ny, p.Nx)
        self.Kx = p.Nx // 2 + 1
        self._ws = workspace
        h = _vp()
        wptr = workspace.data_ptr() if workspace is not None else None
        wbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
        _check(_lib.ns_create(ctypes.byref(p), wptr, wbytes, ctypes.byref(h)), "ns_create")
        self.handle = h

    def _chk(self, t, shape, dtype=None):
        if t.shape != shape or t.dtype != (dtype or self.dtype) or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"expected contiguous CUDA tensor {shape} {dtype or self.dtype}, got {tuple(t.shape)} {t.dtype}")

    def set_fields(self, phys, stream=None):
        self._chk(phys, self.shape)
        _check(_lib.ns_set_fields(self.handle, phys.data_ptr(), _stream(stream)), "ns_set_fields")

    def get_fields(self, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.shape, dtype=self.dtype, device="cuda")
        self._chk(out, self.shape)
        _check(_lib.ns_get_fields(self.handle, out.data_ptr(), _stream(stream)), "ns_get_fields")
        return out

    def state_shape(self):
        plines = self.p.Ny * ((self.Kx + 15) // 16 * 16)
        return (self.p.nfields * (self.p.Nz + self.p.C) * plines,)

    def get_state(self, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.state_shape(), dtype=self.cdtype, device="cuda")
        self._chk(out, self.state_shape(), self.cdtype)
        _check(_lib.ns_get_state(self.handle, out.data_ptr(), _stream(stream)), "ns_get_state")
        return out

    def put_state(self, st, stream=None):
        self._chk(st, self.state_shape(), self.cdtype)
        _check(_lib.ns_put_state(self.handle, st.data_ptr(), _stream(stream)), "ns_put_state")

    def wall_gradp(self, stream=None):
        import torch
        out = torch.empty((2, 2, self.p.Ny, self.Kx), dtype=torch.complex128, device="cuda")
        _check(_lib.ns_get_wall_gradp(self.handle, out.data_ptr(), _stream(stream)), "ns_get_wall_gradp")
        return out

    def put_wall_gradp(self, gp, stream=None):
        import torch
        self._chk(gp, (2, 2, self.p.Ny, self.Kx), torch.complex128)
        _check(_lib.ns_put_wall_gradp(self.handle, gp.data_ptr(), _stream(stream)), "ns_put_wall_gradp")

    def rhs(self, phys, out=None, stream=None):
        import torch
        self._chk(phys, self.shape)
        if out is None:
            out = torch.empty(self.shape, dtype=self.dtype, device="cuda")
        self._chk(out, self.shape)
        _check(_lib.ns_rhs(self.handle, phys.data_ptr(), out.data_ptr(), _stream(stream)), "ns_rhs")
        return out

    def project(self, vstar, dt_stage: float, out=None, gradp_out=None, stream=None):
        import torch
        vs = (3, self.p.Nz, self.p.Ny, self.p.Nx)
        self._chk(vstar, vs)
        if out is None:
            out = torch.empty(vs, dtype=self.dtype, device="cuda")
        self._chk(out, vs)
        gptr = None
        if gradp_out is not None:
            self._chk(gradp_out, (2, 2, self.p.Ny, self.Kx), torch.complex128)
            gptr = gradp_out.data_ptr()
        _check(_lib.fc_poisson_project(self.handle, float(dt_stage), vstar.data_ptr(), out.data_ptr(), gptr,
                                       _stream(stream)), "fc_poisson_project")
        return out

    def step(self, dt: float, stream=None):
        _check(_lib.rk_step(self.handle, float(dt), _stream(stream)), "rk_step")

    def check_finite(self, stream=None) -> int:
        """ns_check_finite: number of non-finite state values (synchronous;
        no exception for a positive count)."""
        n = ctypes.c_longlong()
        st = _lib.ns_check_finite(self.handle, ctypes.byref(n), _stream(stream))
        if st not in (0, STATUS["FC_ERR_NONFINITE"]):
            _check(st, "ns_check_finite")
        return n.value

    def set_finite_check(self, every: int):
        """ns_set_finite_check: check the state after every ``every``-th step (0: off)."""
        _check(_lib.ns_set_finite_check(self.handle, int(every)), "ns_set_finite_check")

    def profiles(self, stream=None):
        """ns_profiles: dict of numpy arrays mean [nf][Nz], rms [nf][Nz],
        spectrum [nf][nshell] and the shell width dk (synchronous)."""
        import numpy as np
        ns_, dk = _c_int(), _c_double()
        _check(_lib.ns_spectrum_shells(self.handle, ctypes.byref(ns_), ctypes.byref(dk)), "ns_spectrum_shells")
        nf, Nz = self.p.nfields, self.p.Nz
        mean, rms = np.empty((nf, Nz)), np.empty((nf, Nz))
        spec = np.empty((nf, ns_.value))
        P = ctypes.POINTER(_c_double)
        _check(_lib.ns_profiles(self.handle, mean.ctypes.data_as(P), rms.ctypes.data_as(P), spec.ctypes.data_as(P),
                                _stream(stream)), "ns_profiles")
        return dict(mean=mean, rms=rms, spectrum=spec, dk=dk.value)

    def tune(self, mode: int = 1, tiles=None, stream=None):
        """ns_tune: 0 defaults, 1 autotune, 2 set ``tiles`` (5 ints: bit 0 tile,
        bit 1 radix schedule of the z kinds); returns the choice."""
        arr = (_c_int * 5)(*(tiles or [0] * 5))
        _check(_lib.ns_tune(self.handle, int(mode), arr, _stream(stream)), "ns_tune")
        return list(arr)

    def interpolate_from(self, src: "Sim", stream=None):
        """ns_interpolate: this state := spectral interpolation of src's state."""
        _check(_lib.ns_interpolate(self.handle, src.handle, _stream(stream)), "ns_interpolate")

    def diagnostics(self, stream=None):
        """ns_diagnostics: div_ms, wall_u_ms, wall_w_ms, flow_rate, nusselt (synchronous)."""
        vals = [_c_double() for _ in range(5)]
        _check(_lib.ns_diagnostics(self.handle, *[ctypes.byref(v) for v in vals], _stream(stream)), "ns_diagnostics")
        return dict(zip(["div_ms", "wall_u_ms", "wall_w_ms", "flow_rate", "nusselt"], (v.value for v in vals)))

    def set_diag_series(self, every: int):
        """ns_set_diag_series: record the diagnostics on the device after every
        ``every``-th step (0: off); clears the series."""
        _check(_lib.ns_set_diag_series(self.handle, int(every)), "ns_set_diag_series")

    def diag_series(self, stream=None):
        """ns_get_diag_series: dict of step numbers and the five diagnostics per
        recorded step (numpy arrays; synchronous)."""
        import numpy as np
        n = _c_int(0)
        _check(_lib.ns_get_diag_series(self.handle, 0, None, None, ctypes.byref(n), _stream(stream)),
               "ns_get_diag_series")
        vals = np.zeros((max(n.value, 1), 5))
        steps = np.zeros(max(n.value, 1), dtype=np.int64)
        _check(_lib.ns_get_diag_series(self.handle, n.value, vals.ctypes.data_as(ctypes.POINTER(_c_double)),
                                       steps.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), ctypes.byref(n),
                                       _stream(stream)), "ns_get_diag_series")
        vals, steps = vals[:n.value], steps[:n.value]
        out = {"step": steps}
        for i, k in enumerate(["div_ms", "wall_u_ms", "wall_w_ms", "flow_rate", "nusselt"]):
            out[k] = vals[:, i]
        return out

    def close(self):
        if getattr(self, "handle", None):
            _lib.ns_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """ns_batch: independent simulations advanced together, one CUDA graph
    launch per step (the members stay owned by the caller)."""

    def __init__(self, sims):
        self.sims = list(sims)
        arr = (_vp * len(self.sims))(*[x.handle for x in self.sims])
        h = _vp()
        _check(_lib.ns_batch_create(arr, len(self.sims), ctypes.byref(h)), "ns_batch_create")
        self.handle = h

    def step(self, dt, stream=None):
        """dt: one step size for all members or a sequence of per-member sizes."""
        n = len(self.sims)
        vals = [float(dt)] * n if not hasattr(dt, "__len__") else [float(x) for x in dt]
        if len(vals) != n:
            raise ValueError("one dt per member")
        _check(_lib.ns_batch_step(self.handle, (_c_double * n)(*vals), _stream(stream)), "ns_batch_step")

    def info(self):
        m, g, c = _c_int(), _c_int(), _c_int()
        _check(_lib.ns_batch_info(self.handle, ctypes.byref(m), ctypes.byref(g), ctypes.byref(c)), "ns_batch_info")
        return dict(members=m.value, graph_nodes=g.value, graphs_cached=c.value)

    def close(self):
        if getattr(self, "handle", None):
            _lib.ns_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
