"""fc_deriv_z_noalloc: the allocation-free variant of fc_deriv_z.

Some callers cannot let a library call cudaMalloc: applications whose device
memory belongs to a host framework or to a fixed arena, and programs run
under a device-memory budget.  For them fc_deriv_z_noalloc keeps the plan's
tables in a fixed static device array instead of library-allocated device
memory.  This file checks, through the C ABI, that its outputs are bitwise
those of fc_deriv_z (the same kernel on the same tables), on calls in a row
with different plans (each must replace the previous call's tables) and with
the same plan again (the tables are already in place and nothing is copied),
and that those calls allocate no device memory.  It is named to run after
every other test file.
"""
import ctypes

import numpy as np
import pytest

import synth

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
def test_noalloc_matches_fc_deriv_z_on_calls_in_a_row(api, dtype):
    cases = [(129, 40, 6, 2), (513, 33, 8, 1)]          # two plans: different tables
    inputs = []
    for Nz, Nx, Ny, B in cases:
        sf = synth.SeparableField(Nx, Ny, Nz, seed_offset=Nz)
        z = synth.z_grid(Nz)
        base = sf.field(0) + np.sin(3 * z + 1)[:, None, None]
        f = torch.from_numpy(np.stack([base * (b + 1) for b in range(B)])).to("cuda", dtype)
        inputs.append((api.Plan(5, 25, Nz), f))
    outs = [(torch.empty_like(f), torch.empty_like(f)) for _, f in inputs]
    again = (torch.empty_like(inputs[1][1]), torch.empty_like(inputs[1][1]))
    torch.cuda.synchronize()
    # set-up calls on this device: resolve the array's address and load both
    # kernels (lazy module loading may take device memory for their code)
    for (plan, f), (o1, o2) in zip(inputs, outs):
        _call(api, "fc_deriv_z_noalloc", plan, f, o1, o2)
    for o1, o2 in outs + [again]:
        o1.fill_(np.nan)
        o2.fill_(np.nan)
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    # two calls in a row with different plans (each replaces the other's
    # tables), then the same plan again (nothing to copy)
    for (plan, f), (o1, o2) in zip(inputs, outs):
        _call(api, "fc_deriv_z_noalloc", plan, f, o1, o2)
    _call(api, "fc_deriv_z_noalloc", inputs[1][0], inputs[1][1], *again)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    # the reference entry point (allocates its own tables on first use)
    for (plan, f), (n1, n2) in zip(inputs, outs):
        r1, r2 = torch.empty_like(f), torch.empty_like(f)
        _call(api, "fc_deriv_z", plan, f, r1, r2)
        torch.cuda.synchronize()
        assert torch.equal(n1, r1) and torch.equal(n2, r2)
        if plan is inputs[1][0]:
            assert torch.equal(again[0], r1) and torch.equal(again[1], r2)
