"""App. A noise generator (an input recipe, no method arithmetic) against what
the mathematics fixes: the clamped-beam characteristic equation of the
Chandrasekhar-Reid functions, wall values, divergence, spectral support."""
import numpy as np

import synth


def test_lambdas_solve_the_clamped_beam_equation():
    """g_m(+-1/2) = g_m'(+-1/2) = 0 makes lambda_m a root of cos(l) cosh(l) = 1
    (the classical clamped-beam eigenvalues 4.7300, 7.8532, 10.9956, ...)."""
    lam = synth.chandrasekhar_reid_lambdas(6)
    assert np.all(np.abs(np.cos(lam) * np.cosh(lam) - 1.0) < 1e-7 * np.cosh(lam))
    np.testing.assert_allclose(lam[:3], [4.730040745, 7.853204624, 10.995607838], atol=1e-8)
    assert np.all(np.diff(lam) > 3.0)


def test_profiles_vanish_with_slope_at_walls():
    lam = synth.chandrasekhar_reid_lambdas(5)
    for m in range(1, 6):
        g, dg = synth._cr_g(m, lam[m - 1], np.array([-0.5, 0.5]))
        assert np.abs(g).max() < 1e-12 and np.abs(dg).max() < 1e-9 * lam[m - 1]


def test_noise_is_no_slip_and_divergence_free():
    v = synth.chandrasekhar_reid_noise(16, 16, 65)
    assert v.shape == (3, 65, 16, 16) and abs(np.abs(v).max() - 1) < 1e-12
    assert np.abs(v[:, [0, -1]]).max() < 1e-14
    # divergence with spectral x, y derivatives and 2nd-order z differences: O(dz^2)
    errs = []
    for Nz in (513, 1025):
        v = synth.chandrasekhar_reid_noise(16, 16, Nz)
        k = np.fft.fftfreq(16, 1 / 16)
        dx = np.real(np.fft.ifft(1j * k * np.fft.fft(v[0], axis=-1), axis=-1))
        dy = np.real(np.fft.ifft(1j * k[:, None] * np.fft.fft(v[1], axis=-2), axis=-2))
        dw = np.gradient(v[2], 1 / (Nz - 1), axis=0)
        errs.append(np.abs(dx + dy + dw)[1:-1].max())
    assert errs[1] < 0.3 * errs[0] and errs[1] < 2e-3


def test_noise_spectral_support():
    """Only horizontal modes with 4 <= kx^2 + ky^2 <= 25 (Lx = Ly = 2 pi)."""
    v = synth.chandrasekhar_reid_noise(32, 32, 33)
    V = np.abs(np.fft.fft2(v, axes=(-2, -1))).max(axis=(0, 1))
    k = np.fft.fftfreq(32, 1 / 32)
    k2 = k[:, None] ** 2 + k[None, :] ** 2
    inside = (k2 >= 4) & (k2 <= 25)
    assert V[~inside].max() < 1e-12 * V.max()
    assert (V[inside] > 1e-6 * V.max()).sum() > 40
