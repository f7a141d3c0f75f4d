"""fc_noise (App. A perturbation) on the GPU vs the FP64 oracle, through the C ABI."""
import math

import numpy as np
import pytest

from oracle import noise
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


def _run(api, Nx, Ny, Nz, dtype, seed, **kw):
    p = api.noise_params(**kw)
    cnt = api.noise_modes(p)
    draws = synth.noise_draws(cnt, seed)
    out = torch.full((3, Nz, Ny, Nx), float("nan"), dtype=dtype, device="cuda")
    api.fc_noise(p, draws, out)
    torch.cuda.synchronize()
    return out.cpu().double().numpy(), draws


def _oracle(Nx, Ny, Nz, draws, **kw):
    d = noise.DEFAULTS
    return noise.noise_field(Nx, Ny, Nz, draws, kw.get("Lx", d["Lx"]), kw.get("Ly", d["Ly"]), kw.get("Lz", 1.0),
                             (kw.get("kperp2_min", 4.0), kw.get("kperp2_max", 25.0)),
                             (kw.get("m_min", 2), kw.get("m_max", 5)), (kw.get("slope_phi", -4.0),
                                                                        kw.get("slope_psi", -3.0)),
                             kw.get("amplitude", 1.0))


@pytest.mark.parametrize("Nx,Ny,Nz,kw", [
    (16, 16, 33, {}),
    (13, 11, 20, {}),                                                    # odd sizes, smallest resolving grid
    (24, 14, 21, {"Lx": 4 * math.pi, "Lz": 2.0, "amplitude": 0.3}),
    (18, 20, 40, {"Ly": 3.0, "kperp2_min": 1.0, "kperp2_max": 9.0, "m_min": 1, "m_max": 3,
                  "slope_phi": -2.0, "slope_psi": -1.5}),
])
def test_noise_float64_matches_oracle(api, Nx, Ny, Nz, kw):
    out, draws = _run(api, Nx, Ny, Nz, torch.float64, 11, **kw)
    ref = _oracle(Nx, Ny, Nz, draws, **kw)
    amp = kw.get("amplitude", 1.0)
    assert np.abs(out - ref).max() < 1e-13 * amp
    assert np.abs(out[:, [0, -1]]).max() < 1e-14 * amp        # no slip at both walls
    assert abs(np.abs(out).max() - amp) < 1e-15 * amp


def test_noise_float32_matches_oracle(api):
    out, draws = _run(api, 32, 32, 65, torch.float32, 12)
    ref = _oracle(32, 32, 65, draws)
    # two float32 roundings of values <= 1 (synthesis, scaling) and the float32 maximum
    assert np.abs(out - ref).max() < 3e-7
    assert np.abs(out[:, [0, -1]]).max() < 1e-7


def test_noise_full_size_sampled(api):
    """1024^2 x 513 float32 (the Boussinesq grid of the RK-step workload):
    every 64th x and y column against the oracle on the 16 x 16 x 513 grid
    that holds exactly those points, up to the one global scale (the maximum
    is taken over different point sets), which the largest magnitude fixes."""
    Nx = Ny = 1024
    Nz = 513
    p = api.noise_params()
    draws = synth.noise_draws(api.noise_modes(p), 13)
    out = torch.empty((3, Nz, Ny, Nx), dtype=torch.float32, device="cuda")
    api.fc_noise(p, draws, out)
    torch.cuda.synchronize()
    assert abs(out.abs().max().item() - 1.0) < 1.2e-7
    assert out[:, [0, -1]].abs().max().item() < 1e-7
    assert torch.isfinite(out).all().item()
    sample = out[:, :, ::64, ::64].cpu().double().numpy()
    ref = _oracle(16, 16, Nz, draws)
    c = float((sample * ref).sum() / (ref * ref).sum())
    assert 0.5 < c <= 1.0 + 1e-6
    assert np.abs(sample - c * ref).max() < 3e-7
    del out
    torch.cuda.empty_cache()
