"""C ABI: the library loads, exports every declared symbol, host-only calls work (CPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "fcns.h")


@pytest.fixture(scope="session")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2002_01392_gb300 import api as a
    return a


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(?:fc_status|const char\*)\s+(\w+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(api):
    names = declared_functions()
    assert len(names) >= 20
    lib = ctypes.CDLL(api.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(api.EXPORTED) == names


def test_status_strings(api):
    for code, name in enumerate(["FC_OK", "FC_ERR_ARG", "FC_ERR_UNSUPPORTED", "FC_ERR_CUDA", "FC_ERR_NOMEM",
                                 "FC_ERR_TIMEOUT", "FC_ERR_NONFINITE", "FC_ERR_STATE"]):
        assert api._lib.fc_status_str(code).decode() == name


def test_fc_setup_tables_match_oracle(api, Mr_5_25):
    """Library Gram/QR tables (double-binary128, ~67 digits) vs oracle Lagrange
    tables (mpmath, 60 digits, another basis): both are the correctly rounded
    doubles of the same matrix, so they are equal bit for bit."""
    plan = api.Plan(5, 25, 33)
    Mr = plan.matrix()
    assert np.array_equal(Mr, Mr_5_25)
    info = plan.info()
    assert info["M"] == 20 and info["n_os"] == 20 and info["ls_residual"] < 1e-15


def test_fc_setup_d7_tables_match_oracle(api, Mr_7_33):
    """(d, C) = (7, 33), M = 26: the fits need more than binary128, so the
    library builds them in double-binary128 arithmetic; the oracle's are mpmath
    at 60 digits in another basis."""
    plan = api.Plan(7, 33, 65)
    Mr = plan.matrix()
    assert np.array_equal(Mr, Mr_7_33)
    info = plan.info()
    assert info["M"] == 26 and info["ls_residual"] < 1e-17


def test_fc_setup_demo_tables(api, golden_dir):
    from oracle import fc_tables
    ref = fc_tables.fc_matrix(5, 15, table_dir=golden_dir)
    Mr = api.Plan(5, 15, 49).matrix()
    assert np.abs(Mr - ref).max() / np.abs(ref).max() < 1e-13


@pytest.mark.parametrize("args", [(1, 25, 33), (5, 4, 33), (5, 25, 9), (11, 25, 33), (5, 65, 200)])
def test_fc_setup_rejects_bad_sizes(api, args):
    with pytest.raises(api.FcError) as e:
        api.Plan(*args)
    assert e.value.name == "FC_ERR_ARG"


def test_fc_deriv_z_argument_checks_need_no_gpu(api):
    plan = api.Plan(5, 25, 33)
    st = api._lib.fc_deriv_z(plan.handle, 0, 1, 4, 4, 1.0, None, None, None, None)
    assert api._lib.fc_status_str(st).decode() == "FC_ERR_ARG"
    st = api._lib.fc_deriv_z(plan.handle, 7, 1, 4, 4, 1.0, 16, 32, None, None)
    assert api._lib.fc_status_str(st).decode() == "FC_ERR_ARG"
    st = api._lib.fc_deriv_z(plan.handle, 0, 1, 4, 4, -1.0, 16, 32, None, None)
    assert api._lib.fc_status_str(st).decode() == "FC_ERR_ARG"
    # overlapping input and output
    st = api._lib.fc_deriv_z(plan.handle, 0, 1, 4, 4, 1.0, 4096, 4100, None, None)
    assert api._lib.fc_status_str(st).decode() == "FC_ERR_ARG"
    # empty batches / grids are argument errors (nothing is launched or written)
    for b, nx, ny in ((0, 4, 4), (1, 0, 4), (1, 4, 0), (-1, 4, 4)):
        st = api._lib.fc_deriv_z(plan.handle, 0, b, nx, ny, 1.0, 16, 1 << 40, None, None)
        assert api._lib.fc_status_str(st).decode() == "FC_ERR_ARG", (b, nx, ny)


def test_fc_deriv_z_host_argument_checks_need_no_gpu(api):
    plan = api.Plan(5, 25, 33)
    for fn in ("fc_deriv_z_host", "fc_deriv_z_noalloc"):
        st = getattr(api._lib, fn)(plan.handle, 0, 1, 4, 4, 1.0, None, None, None, None)
        assert api._lib.fc_status_str(st).decode() == "FC_ERR_ARG"
    st = api._lib.fc_deriv_z_host_ex(plan.handle, 0, 1, 4, 4, 1.0, 4096, 4100, None, 1 << 20, None)
    assert api._lib.fc_status_str(st).decode() == "FC_ERR_ARG"


def test_unsupported_length(api):
    plan = api.Plan(5, 25, 800)          # N' + Nz - 1 = 1624 > 1536, N' = 825 not a compiled length
    st = api._lib.fc_deriv_z(plan.handle, 0, 1, 4, 4, 1.0, 16, 1 << 40, None, None)
    assert api._lib.fc_status_str(st).decode() == "FC_ERR_UNSUPPORTED"


def test_size_limits_need_no_gpu(api):
    """Largest sizes: every array is indexed with 32-bit element offsets, so
    fc_deriv_z refuses batch * Nx * Ny >= 2^31 lines and ns_create /
    ns_workspace_bytes refuse states of >= 2^31 complex values (the
    1024^2 x 999 Boussinesq state, 4 x 1024 x 1024 x 528 > 2^31); lengths
    outside the compiled shapes are FC_ERR_UNSUPPORTED, bad parameters
    FC_ERR_ARG; the benchmark's 1024^2 x 513 Boussinesq case fits."""
    plan = api.Plan(5, 25, 33)
    st = api._lib.fc_deriv_z(plan.handle, 0, 3, 1 << 15, 1 << 15, 1.0, 16, 1 << 44, None, None)
    assert api._lib.fc_status_str(st).decode() == "FC_ERR_UNSUPPORTED"
    ok = api.ns_workspace_bytes(api.ns_params(Nx=1024, Ny=1024, Nz=513, nfields=4, prec="f32"))
    assert 60e9 < ok < 90e9

    def status(**kw):
        import ctypes
        p = api.ns_params(**kw)
        n = ctypes.c_size_t()
        return api._lib.fc_status_str(api._lib.ns_workspace_bytes(ctypes.byref(p), ctypes.byref(n))).decode()

    assert status(Nx=1024, Ny=1024, Nz=999, nfields=4, prec="f32") == "FC_ERR_UNSUPPORTED"   # 2^31 elements
    assert status(Nx=1024, Ny=1024, Nz=999, nfields=3, prec="f32") == "FC_OK"
    assert status(Nx=100, Ny=64, Nz=33) == "FC_ERR_UNSUPPORTED"                            # x length not compiled
    assert status(Nx=64, Ny=64, Nz=743, prec="f64") == "FC_ERR_UNSUPPORTED"                # f64 z length > 576
    assert status(Nx=64, Ny=64, Nz=1200) == "FC_ERR_UNSUPPORTED"                           # 2 N' - 1 > 1152, N' = 1225
    assert status(Nx=64, Ny=64, Nz=9) == "FC_ERR_ARG"                                      # Nz < 2d
    assert status(Nx=64, Ny=64, Nz=33, nfields=5) == "FC_ERR_ARG"
    assert status(Nx=64, Ny=64, Nz=33, nu=-1.0) == "FC_ERR_ARG"
    assert status(Nx=64, Ny=64, Nz=33, rk_order=5) == "FC_ERR_ARG"
    assert status(Nx=64, Ny=64, Nz=10) == "FC_OK"                                          # Nz = 2d


def test_host_array_binding_checks_need_no_gpu(api):
    """fc_deriv_z_host through the binding: shapes and dtypes are checked
    before the library is called."""
    import torch
    plan = api.Plan(5, 25, 33)
    f = torch.zeros(2, 33, 4, 6)
    with pytest.raises(ValueError):
        api.fc_deriv_z_host(plan, torch.zeros(2, 32, 4, 6), torch.zeros(2, 32, 4, 6))   # Nz != plan.Nz
    with pytest.raises(ValueError):
        api.fc_deriv_z_host(plan, f, torch.zeros(2, 33, 4, 5))                          # output shape
    with pytest.raises(ValueError):
        api.fc_deriv_z_host(plan, f, torch.zeros(2, 33, 4, 6, dtype=torch.float64))    # output dtype
    with pytest.raises(TypeError):
        api.fc_deriv_z_host(plan, f.to(torch.int32), None, torch.zeros(2, 33, 4, 6, dtype=torch.int32))



def test_noise_mode_count_and_argument_checks_need_no_gpu(api):
    """fc_noise_modes enumerates the same (n, l, m) modes as the oracle (App. A
    defaults and other boxes); fc_noise rejects bad arguments before any
    device work."""
    import math
    from oracle import noise
    for kw, ref in (({}, noise.modes(2 * math.pi, 2 * math.pi)),
                    ({"Lx": 4 * math.pi}, noise.modes(4 * math.pi, 2 * math.pi)),
                    ({"Ly": 3.0, "kperp2_min": 1.0, "kperp2_max": 9.0, "m_min": 1, "m_max": 3},
                     noise.modes(2 * math.pi, 3.0, (1.0, 9.0), (1, 3)))):
        assert api.noise_modes(api.noise_params(**kw)) == len(ref), kw
    p = api.noise_params()
    cnt = api.noise_modes(p)
    draws = (ctypes.c_double * (2 * cnt))()
    lib = api._lib

    def st(pp, dtype=0, Nx=16, Ny=16, Nz=17, nd=2 * cnt, out=1 << 40):
        return lib.fc_status_str(lib.fc_noise(ctypes.byref(pp), dtype, Nx, Ny, Nz, draws, nd, out, None)).decode()

    assert st(p, nd=2 * cnt - 1) == "FC_ERR_ARG"          # wrong draw count
    assert st(p, Nx=10) == "FC_ERR_ARG"                   # the mode n = 5 is not resolved
    assert st(p, Ny=9) == "FC_ERR_ARG"                    # l = 5
    assert st(p, Nz=1) == "FC_ERR_ARG"
    assert st(p, dtype=7) == "FC_ERR_ARG"
    assert st(p, out=None) == "FC_ERR_ARG"
    for bad in ({"Lz": 0.0}, {"kperp2_min": 30.0}, {"m_min": 0}, {"m_max": 65}, {"amplitude": float("nan")}):
        assert st(api.noise_params(**bad)) == "FC_ERR_ARG", bad
    assert st(api.noise_params(kperp2_min=0.1, kperp2_max=0.2)) == "FC_ERR_ARG"   # empty annulus
    # max |n| = 600 > 511: refused before any device work (grid and draws sized to pass the other checks)
    big = api.noise_params(kperp2_min=599.5 ** 2, kperp2_max=600.0 ** 2, m_min=2, m_max=2)
    nb = api.noise_modes(big)
    big_draws = (ctypes.c_double * (2 * nb))()
    assert lib.fc_status_str(lib.fc_noise(ctypes.byref(big), 0, 1300, 1300, 17, big_draws, 2 * nb, 1 << 40,
                                          None)).decode() == "FC_ERR_UNSUPPORTED"
