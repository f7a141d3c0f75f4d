"""The plain float64 cuFFT comparison path of bench.py (PlainCufftNS: torch.fft
and separate torch kernels) against the oracle, on the CPU (torch.fft runs
there too): the comparison arm must compute the method it is compared with."""
import numpy as np
import pytest

from oracle import ns
import synth

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bench():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2002_01392_gb300 import api
    import bench as b
    return b, api


@pytest.mark.parametrize("kind", ["channel", "rb"])
def test_plain_cufft_step_matches_oracle(bench, kind):
    b, api = bench
    N, Nz = 16, 33
    if kind == "channel":
        kw = dict(nu=1e-2, forcing_x=0.1)
        f = synth.channel_velocity(N, N, Nz, nu=1e-2)
    else:
        kw = dict(nu=3.162e-3, kappa=3.162e-3, gamma=1.0, nfields=4)
        f = synth.boussinesq_fields(N, N, Nz, amp=1e-1)
    P = ns.Params(N, N, Nz, **kw)
    pl = b.PlainCufftNS(api, torch, N, N, Nz, device="cpu", **kw)
    st = pl.to_spectral(torch.from_numpy(f))
    gp = torch.zeros((2, 2, N, N // 2 + 1), dtype=torch.complex128)
    so = ns.to_spectral(f, P)
    go = np.zeros((2, 2, N, N // 2 + 1), complex)
    for _ in range(2):
        st, gp = pl.step(st, gp, 1e-3)
        so, go = ns.rk_step(so, go, P, 1e-3)
    out = pl.to_physical(st).numpy()
    ref = np.stack([ns.to_physical(c, P) for c in so])
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 1e-11
    assert np.linalg.norm(gp.numpy() - go) / np.linalg.norm(go) < 1e-9
