"""Kernel index arithmetic checked on the CPU: the host-check library runs the
same phase functions as the CUDA kernels, block by block, and is compared with
the oracle (no GPU involved)."""
import ctypes
import os

import numpy as np
import pytest

from conftest import ROOT
from oracle import fc
from numerics import fc_amplification, norm_bound, rel_bound_f64
import synth

HC = os.path.join(ROOT, "paper_2002_01392_gb300", "libfcns_hostcheck.so")


@pytest.fixture(scope="session")
def hc():
    import __graft_entry__
    __graft_entry__.build()
    return ctypes.CDLL(HC)


def _vp(a):
    return a.ctypes.data_as(ctypes.c_void_p)


@pytest.mark.parametrize("Nz,L,Nx,Ny,B", [(33, 160, 6, 5, 2), (513, 1080, 9, 2, 1)])
def test_deriv_kernel_d7_matches_oracle(hc, Mr_7_33, Nz, L, Nx, Ny, B):
    """d = 7, C = 33 tables (entries up to 4.5e5) through the same kernel, float64."""
    sf = synth.SeparableField(Nx, Ny, Nz, rank=3, seed_offset=Nz + 7)
    f = np.ascontiguousarray(np.stack([sf.field(0)] * B))
    d1, d2 = np.zeros_like(f), np.zeros_like(f)
    assert hc.fchc_deriv_z(1, L, _vp(Mr_7_33), 7, 33, Nz, B, Nx, Ny, ctypes.c_double(1.0),
                           _vp(f), _vp(d1), _vp(d2)) == 0
    Np = Nz + 33
    amp = fc_amplification(Mr_7_33)
    for order, out in ((1, d1), (2, d2)):
        ref = fc.fc_deriv_z(f, 1.0, Mr_7_33, order, axis=1)
        rel = np.linalg.norm(out - ref) / np.linalg.norm(ref)
        assert rel < amp * rel_bound_f64(order, Np), (order, rel)


@pytest.mark.parametrize("Nz,L,Nx,Ny,B", [(33, 96, 5, 7, 2), (10, 96, 33, 1, 1), (65, 160, 40, 3, 1),
                                           (39, 64, 9, 3, 2),
                                           (129, 288, 33, 1, 1), (513, 1080, 17, 2, 1), (513, 1080, 8, 2, 2),
                                           # the smallest Nz that L = 1080 serves with C = 25 (need 1025)
                                           (501, 1080, 8, 2, 1),
                                           # an odd line count: element loads of the last pair
                                           (513, 1080, 9, 3, 1)])
@pytest.mark.parametrize("dtype", [0, 1])
def test_deriv_kernel_phases_match_oracle(hc, Mr_5_25, Nz, L, Nx, Ny, B, dtype):
    sf = synth.SeparableField(Nx, Ny, Nz, rank=3, seed_offset=Nz)
    f = np.stack([sf.field(0)] * B) * np.arange(1, B + 1)[:, None, None, None]
    npdt = np.float32 if dtype == 0 else np.float64
    fin = np.ascontiguousarray(f.astype(npdt))
    d1, d2 = np.zeros_like(fin), np.zeros_like(fin)
    rc = hc.fchc_deriv_z(dtype, L, _vp(Mr_5_25), 5, 25, Nz, B, Nx, Ny, ctypes.c_double(1.0),
                         _vp(fin), _vp(d1), _vp(d2))
    assert rc == 0
    Np = Nz + 25
    kmax = np.pi * (Nz - 1)
    # scale of the transformed data: the continued lines
    xnorm = np.linalg.norm(fc.extend(fin.astype(np.float64), Mr_5_25, axis=1))
    for order, out in ((1, d1), (2, d2)):
        ref = fc.fc_deriv_z(fin.astype(np.float64), 1.0, Mr_5_25, order, axis=1)
        en = np.linalg.norm(out - ref) / (xnorm * kmax ** order)
        assert en < norm_bound(npdt, Nz), (order, en)
        if dtype == 1:
            rel = np.linalg.norm(out - ref) / np.linalg.norm(ref)
            assert rel < rel_bound_f64(order, Np), (order, rel)


def test_deriv_kernel_converges_to_exact_derivative(hc, Mr_5_25):
    """Against the exact z-derivatives of the separable workload field (its z
    profiles are degree-16 Chebyshev series): the float64 kernel has the
    oracle's discretisation error (to the float64 parity bound), and it falls at
    least like h^(d-1) = h^4 for d/dz (boundary order of the d = 5 FC-Gram
    continuation) and h^3 for d2/dz2 from Nz = 129 to 513."""
    errs = {}
    for Nz, L in ((129, 288), (513, 1080)):
        sf = synth.SeparableField(6, 3, Nz, seed_offset=4)
        f = np.ascontiguousarray(sf.field(0)[None])
        d1, d2 = np.zeros_like(f), np.zeros_like(f)
        assert hc.fchc_deriv_z(1, L, _vp(Mr_5_25), 5, 25, Nz, 1, 6, 3, ctypes.c_double(1.0),
                               _vp(f), _vp(d1), _vp(d2)) == 0
        for order, out in ((1, d1), (2, d2)):
            ex = sf.field(order)[None]
            ke = np.linalg.norm(out - ex) / np.linalg.norm(ex)
            oe = np.linalg.norm(fc.fc_deriv_z(f, 1.0, Mr_5_25, order, axis=1) - ex) / np.linalg.norm(ex)
            # the two differ by at most the kernel's float64 parity bound
            assert abs(ke - oe) <= rel_bound_f64(order, Nz + 25), (Nz, order, ke, oe)
            errs[(Nz, order)] = ke
    h_ratio = 512 / 128
    assert errs[(129, 1)] / errs[(513, 1)] >= h_ratio ** 4 * 0.8
    assert errs[(129, 2)] / errs[(513, 2)] >= h_ratio ** 3 * 0.8



@pytest.mark.parametrize("batch,Ny,rows_per_slab", [(3, 512, 242), (2, 23, 6), (1, 23, 6), (1, 7, 100), (2, 9, 2),
                                                    (4, 1024, 7), (1, 2, 2), (3, 513, 64)])
def test_host_array_slab_plan(hc, batch, Ny, rows_per_slab):
    """fc_deriv_z_host's slabs cover every y row of every field exactly once,
    in order; every slab but a field's last has an even row count and starts
    on an even row (the kernel pairs the same lines as on the whole field); no
    slab exceeds the staging rows, which stay within the requested bytes
    (rounded to an even count, at least 2); the first slab of the call is at
    most about a quarter of the staging rows."""
    yrow = 513 * 37 * 4
    out = (ctypes.c_longlong * 30000)()
    n = ctypes.c_int()
    hc.fchc_slab_plan.restype = ctypes.c_longlong
    hc.fchc_slab_plan.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.c_size_t, ctypes.c_size_t,
                                  ctypes.POINTER(ctypes.c_longlong), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    Yc = hc.fchc_slab_plan(batch, Ny, yrow, rows_per_slab * yrow, out, 10000, ctypes.byref(n))
    slabs = [tuple(out[3 * i:3 * i + 3]) for i in range(n.value)]
    assert 0 < Yc <= max(2, rows_per_slab + rows_per_slab % 2) or Yc == Ny
    for b in range(batch):
        mine = [(y0, yc) for (bb, y0, yc) in slabs if bb == b]
        assert [y0 for y0, _ in mine] == [sum(yc for _, yc in mine[:k]) for k in range(len(mine))]
        assert sum(yc for _, yc in mine) == Ny
        for k, (y0, yc) in enumerate(mine):
            assert 0 < yc <= Yc and y0 % 2 == 0
            if k < len(mine) - 1:
                assert yc % 2 == 0
    if Yc < Ny:
        assert slabs[0][2] <= max(2, Yc // 4)
    assert [bb for bb, _, _ in slabs] == sorted(bb for bb, _, _ in slabs)
