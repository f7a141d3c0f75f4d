"""fc_deriv_z on the GPU vs the FP64 oracle (parity tests, through the C ABI)."""
import numpy as np
import pytest

from oracle import fc
import synth
from numerics import fc_amplification, normalized_error, norm_bound, rel_bound_f64, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2002_01392_gb300 import api as a
    assert torch.cuda.is_available()
    return a


def _wall_rows_error(out, ref, xext, kmax, order, axis):
    """Largest error on the wall rows (z index 0 and Nz - 1, where the
    continuation acts) in the pointwise form of the rounding model: relative to
    max |x_ext| k_max^p."""
    o = np.moveaxis(np.asarray(out, dtype=np.float64), axis, 0)
    r = np.moveaxis(ref, axis, 0)
    worst = max(np.abs(o[0] - r[0]).max(), np.abs(o[-1] - r[-1]).max())
    return float(worst / (np.abs(xext).max() * kmax ** order))


def _check(out, f64, Mr, Nz, order, dtype):
    ref = fc.fc_deriv_z(f64, 1.0, Mr, order, axis=-3)
    xext = fc.extend(f64, Mr, axis=-3)
    xnorm = np.linalg.norm(xext)
    kmax = np.pi * (Nz - 1)
    amp = fc_amplification(Mr)
    en = normalized_error(out, ref, xnorm, kmax, order)
    assert en < amp * norm_bound(dtype, Nz), (order, en)
    ew = _wall_rows_error(out, ref, xext, kmax, order, axis=-3)
    assert ew < amp * norm_bound(dtype, Nz), (order, ew)
    if dtype == np.float64:
        rel = rel_l2(out, ref)
        assert rel < amp * rel_bound_f64(order, Nz + Mr.shape[0]), (order, rel)


@pytest.mark.parametrize("Nz,Nx,Ny,B", [(10, 33, 1, 1), (33, 20, 6, 3), (33, 1, 1, 1), (65, 40, 3, 1),
                                         (129, 33, 5, 2), (257, 24, 2, 1), (513, 17, 2, 1), (513, 64, 16, 2),
                                         # smooth N' = Nz + 25 (64, 512, 1024, 1536): transform length N' itself
                                         (39, 21, 4, 2), (487, 33, 3, 1), (999, 16, 3, 1), (1511, 8, 2, 1),
                                         # padded length 1152 (N' + Nz - 1 = 1124)
                                         (550, 16, 2, 1)])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_deriv_parity_small(api, Mr_5_25, Nz, Nx, Ny, B, dtype):
    plan = api.Plan(5, 25, Nz)
    sf = synth.SeparableField(Nx, Ny, Nz, seed_offset=Nz + B)
    z = synth.z_grid(Nz)
    base = sf.field(0) + np.sin(3 * z + 1)[:, None, None]      # nonzero even on a 1 x 1 grid
    f = np.stack([base * (b + 1) for b in range(B)]).astype(dtype)
    ft = torch.from_numpy(f).cuda()
    d1, d2 = torch.empty_like(ft), torch.empty_like(ft)
    api.fc_deriv_z(plan, ft, d1, d2, Lz=1.0)
    torch.cuda.synchronize()
    f64 = f.astype(np.float64)
    _check(d1.cpu().numpy(), f64, Mr_5_25, Nz, 1, dtype)
    _check(d2.cpu().numpy(), f64, Mr_5_25, Nz, 2, dtype)


def test_single_outputs_and_lz_scaling(api, Mr_5_25):
    Nz = 65
    plan = api.Plan(5, 25, Nz)
    f = synth.SeparableField(8, 8, Nz).field(0)
    ft = torch.from_numpy(f).cuda()
    d1 = torch.empty_like(ft)
    api.fc_deriv_z(plan, ft, d1, None, Lz=2.0)
    d2 = torch.empty_like(ft)
    api.fc_deriv_z(plan, ft, None, d2, Lz=2.0)
    torch.cuda.synchronize()
    np.testing.assert_allclose(d1.cpu().numpy(), fc.fc_deriv_z(f, 2.0, Mr_5_25, 1), rtol=0, atol=1e-11 * np.abs(f).max() * 64)
    np.testing.assert_allclose(d2.cpu().numpy(), fc.fc_deriv_z(f, 2.0, Mr_5_25, 2), rtol=0, atol=1e-9 * np.abs(f).max() * 64 ** 2)


def test_exact_derivatives_of_polynomials_and_sines(api):
    """Closed forms on the GPU path: z^p (p < d) exact, sin(az) at the boundary order."""
    Nz = 129
    plan = api.Plan(5, 25, Nz)
    z = synth.z_grid(Nz)
    cols = [z ** p for p in range(5)] + [np.sin(a * z) for a in (1.0, 5.0, 15.0)]
    f = np.stack(cols, axis=1)[:, None, :]               # [Nz][1][8]
    ft = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    d1 = torch.empty_like(ft)
    api.fc_deriv_z(plan, ft, d1, None)
    torch.cuda.synchronize()
    out = d1.cpu().numpy()[:, 0, :]
    for p in range(5):
        ex = p * z ** max(p - 1, 0) if p else 0 * z
        assert np.abs(out[:, p] - ex).max() < 2e-9
    for i, a in enumerate((1.0, 5.0, 15.0)):
        assert np.abs(out[:, 5 + i] - a * np.cos(a * z)).max() / a < 5e-5


def test_deterministic_and_stream(api):
    Nz = 129
    plan = api.Plan(5, 25, Nz)
    ft = torch.from_numpy(synth.SeparableField(50, 7, Nz).field(0).astype(np.float32)).cuda()
    a1, a2 = torch.empty_like(ft), torch.empty_like(ft)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        api.fc_deriv_z(plan, ft, a1, a2)
    s.synchronize()
    b1, b2 = torch.empty_like(ft), torch.empty_like(ft)
    api.fc_deriv_z(plan, ft, b1, b2)
    torch.cuda.synchronize()
    assert torch.equal(a1, b1) and torch.equal(a2, b2)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_full_size_sampled_lines(api, Mr_5_25, dtype):
    """3 x 512 x 512 x 513 (the fc_deriv_z throughput workload, launched as bench.py
    launches it); 256 sampled z-lines compared with the oracle, all outputs finite."""
    Nx = Ny = 512
    Nz, B = 513, 3
    plan = api.Plan(5, 25, Nz)
    fields = [synth.SeparableField(Nx, Ny, Nz, seed_offset=b) for b in range(B)]
    f = torch.empty((B, Nz, Ny, Nx), dtype=torch.float32 if dtype == np.float32 else torch.float64, device="cuda")
    for b, sf in enumerate(fields):
        f[b] = torch.from_numpy(sf.field(0).astype(dtype)).cuda()
    d1, d2 = torch.empty_like(f), torch.empty_like(f)
    api.fc_deriv_z(plan, f, d1, d2)
    torch.cuda.synchronize()
    assert torch.isfinite(d1).all() and torch.isfinite(d2).all()
    g = np.random.default_rng(7)
    bs, ys, xs = g.integers(0, B, 256), g.integers(0, Ny, 256), g.integers(0, Nx, 256)
    lines = f[bs, :, ys, xs].cpu().numpy().astype(np.float64).T          # [Nz][256]
    o1 = d1[bs, :, ys, xs].cpu().numpy().T
    o2 = d2[bs, :, ys, xs].cpu().numpy().T
    for order, out in ((1, o1), (2, o2)):
        ref = fc.fc_deriv_z(lines, 1.0, Mr_5_25, order, axis=0)
        xnorm = np.linalg.norm(fc.extend(lines, Mr_5_25, axis=0))
        en = normalized_error(out, ref, xnorm, np.pi * (Nz - 1), order)
        assert en < norm_bound(dtype, Nz), (order, en)
        xext = fc.extend(lines, Mr_5_25, axis=0)
        ew = _wall_rows_error(out, ref, xext, np.pi * (Nz - 1), order, axis=0)
        assert ew < norm_bound(dtype, Nz), (order, ew)
        if dtype == np.float64:
            assert rel_l2(out, ref) < rel_bound_f64(order, Nz + 25)


@pytest.mark.parametrize("Nz,Nx,Ny,B", [(33, 20, 6, 3), (513, 64, 16, 2)])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_deriv_parity_d7(api, Mr_7_33, Nz, Nx, Ny, B, dtype):
    """(d, C) = (7, 33) tables (built by the library in double-binary128)."""
    plan = api.Plan(7, 33, Nz)
    assert np.abs(plan.matrix() - Mr_7_33).max() <= 1e-15 * np.abs(Mr_7_33).max()
    f64 = np.stack([synth.SeparableField(Nx, Ny, Nz, seed_offset=Nz + 7 * b).field(0) for b in range(B)])
    f = torch.from_numpy(f64.astype(dtype)).cuda()
    d1, d2 = torch.empty_like(f), torch.empty_like(f)
    api.fc_deriv_z(plan, f, d1, d2)
    fin = f.cpu().numpy().astype(np.float64)
    _check(d1.cpu().numpy(), fin, Mr_7_33, Nz, 1, dtype)
    _check(d2.cpu().numpy(), fin, Mr_7_33, Nz, 2, dtype)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffers_bitwise_device_path(api, dtype, pinned):
    """fc_deriv_z_host (host arrays moved through the GPU in slabs of y rows on
    three streams) gives bitwise the device fc_deriv_z result: several slabs
    per field with a ragged last one, an odd x length (the slab keeps an even
    number of rows, so the same lines are paired), two fields, page-locked and
    pageable host arrays, and one output omitted."""
    Nz, Nx, Ny, B = 129, 37, 23, 2
    plan = api.Plan(5, 25, Nz)
    sf = synth.SeparableField(Nx, Ny, Nz, rank=3, seed_offset=11)
    f = torch.from_numpy(np.stack([sf.field(0), -0.5 * sf.field(0)]).astype(dtype))
    if pinned:
        f = f.pin_memory()
    d1, d2 = torch.empty_like(f.cuda()), torch.empty_like(f.cuda())
    api.fc_deriv_z(plan, f.cuda(), d1, d2)
    mk = (lambda: torch.empty_like(f).pin_memory()) if pinned else (lambda: torch.empty_like(f))
    h1, h2 = mk(), mk()
    row = Nz * Nx * f.element_size()
    api.fc_deriv_z_host(plan, f, h1, h2, slab_bytes=6 * row)     # slabs: 2, 6, 6, 6, 3 rows, then 6, 6, 6, 5
    torch.cuda.synchronize()
    assert torch.equal(h1, d1.cpu()) and torch.equal(h2, d2.cpu())
    h3 = mk()
    api.fc_deriv_z_host(plan, f, None, h3)                         # one slab per field, d/dz omitted
    assert torch.equal(h3, d2.cpu())
    plan.close()



def test_length_1080_paths_agree_bitwise(api, Mr_5_25):
    """At L = 1080 (Nz = 513) the float32 launcher picks among three forms of
    the same kernel: whole tiles of aligned pair vectors (line count a
    multiple of 8), bounds-checked pairs (other even line counts), and
    element loads (arrays not 8-byte aligned).  All compute the same
    arithmetic, so lines they share agree bitwise."""
    Nz = 513
    plan = api.Plan(5, 25, Nz)
    sf = synth.SeparableField(16, 8, Nz, seed_offset=3)
    f = torch.from_numpy(sf.field(0).astype(np.float32)).cuda()          # 128 lines: whole tiles
    d1, d2 = torch.empty_like(f), torch.empty_like(f)
    api.fc_deriv_z(plan, f, d1, d2)
    # the first 6 lines of every z row: 6 lines, not a multiple of 8
    g = f[:, 0, :6].contiguous().reshape(Nz, 1, 6)
    e1, e2 = torch.empty_like(g), torch.empty_like(g)
    api.fc_deriv_z(plan, g, e1, e2)
    # the same 128 lines in buffers offset by one float (4-byte aligned only)
    buf = torch.empty(Nz * 128 + 1, device="cuda")
    h = buf[1:].view(Nz, 8, 16)
    h.copy_(f)
    ob1, ob2 = torch.empty(Nz * 128 + 1, device="cuda"), torch.empty(Nz * 128 + 1, device="cuda")
    o1, o2 = ob1[1:].view(Nz, 8, 16), ob2[1:].view(Nz, 8, 16)
    api.fc_deriv_z(plan, h, o1, o2)
    torch.cuda.synchronize()
    assert torch.equal(o1, d1) and torch.equal(o2, d2)
    assert torch.equal(e1.reshape(Nz, 6), d1[:, 0, :6]) and torch.equal(e2.reshape(Nz, 6), d2[:, 0, :6])
    f64 = sf.field(0)[None].astype(np.float32).astype(np.float64)
    _check(d1[None].cpu().numpy(), f64, Mr_5_25, Nz, 1, np.float32)
    _check(d2[None].cpu().numpy(), f64, Mr_5_25, Nz, 2, np.float32)
