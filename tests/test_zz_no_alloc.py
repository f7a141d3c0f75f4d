"""fc_deriv_z_noalloc: the allocation-free variant of fc_deriv_z.

Some callers cannot let a library call cudaMalloc (graph capture in
progress, device memory owned by a host framework, latency-critical loops).
For them fc_deriv_z_noalloc keeps the plan's tables in a fixed static device
array instead of library-allocated device memory.  This file checks, through
the C ABI, that it returns what fc_deriv_z returns, on two calls in a row
with different plans (so the second call must have replaced the first call's
tables).  It is named to run after every other test file.
"""
import ctypes

import numpy as np
import pytest

import synth
from numerics import norm_bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2002_01392_gb300 import api as a
    assert torch.cuda.is_available()
    return a


def _call(api, name, plan, f, d1, d2):
    fn = getattr(api._lib, name)
    B, Nz, Ny, Nx = f.shape
    dt = api.FC_F32 if f.dtype == torch.float32 else api.FC_F64
    st = fn(plan.handle, dt, B, Nx, Ny, ctypes.c_double(1.0), f.data_ptr(), d1.data_ptr(), d2.data_ptr(),
            torch.cuda.current_stream().cuda_stream)
    assert st == 0, api._lib.fc_last_error().decode()


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_noalloc_matches_fc_deriv_z_on_two_calls(api, dtype):
    cases = [(129, 40, 6, 2), (513, 33, 8, 1)]          # two plans: different tables
    outs = []
    inputs = []
    for Nz, Nx, Ny, B in cases:
        sf = synth.SeparableField(Nx, Ny, Nz, seed_offset=Nz)
        z = synth.z_grid(Nz)
        base = sf.field(0) + np.sin(3 * z + 1)[:, None, None]
        f = torch.from_numpy(np.stack([base * (b + 1) for b in range(B)])).to("cuda", dtype)
        inputs.append((api.Plan(5, 25, Nz), f))
    # two no-alloc calls in a row, then the reference entry point
    for plan, f in inputs:
        d1, d2 = torch.empty_like(f), torch.empty_like(f)
        _call(api, "fc_deriv_z_noalloc", plan, f, d1, d2)
        outs.append((d1, d2))
    torch.cuda.synchronize()
    for (plan, f), (n1, n2) in zip(inputs, outs):
        r1, r2 = torch.empty_like(f), torch.empty_like(f)
        _call(api, "fc_deriv_z", plan, f, r1, r2)
        torch.cuda.synchronize()
        Nz = f.shape[1]
        kmax = np.pi * (Nz - 1)
        fnorm = float(f.double().norm())
        for o, (a, b) in enumerate(((n1, r1), (n2, r2)), start=1):
            err = float((a.double() - b.double()).norm()) / (fnorm * kmax ** o)
            assert err <= norm_bound(np.float32 if dtype == torch.float32 else np.float64, Nz), (o, err)
