"""Oracle App. A perturbation against what the mathematics fixes: the
clamped-beam characteristic equation and its textbook roots, wall values,
the curl of the potentials taken by numerical differentiation (complex step
in z, exact trigonometric differentiation in x, y), divergence and spectral
support."""
import math

import numpy as np
import pytest

import synth
from oracle import noise


def test_lambdas_are_the_clamped_beam_roots():
    """g_m(+-1/2) = g_m'(+-1/2) = 0 makes lambda_m a root of cos(l) cosh(l) = 1;
    its positive roots are the clamped-clamped beam eigenvalues 4.730040745,
    7.853204624, 10.995607838, 14.137165491, 17.278759657 (ascending, one per
    m, so that m odd gives the even function)."""
    lam = noise.cr_lambdas(6)
    assert np.all(np.abs(np.cos(lam) * np.cosh(lam) - 1.0) < 1e-12 * np.cosh(lam))
    np.testing.assert_allclose(lam[:5], [4.730040745, 7.853204624, 10.995607838, 14.137165491, 17.278759657],
                               atol=2e-9)
    # large-m asymptote (2m + 1) pi / 2
    assert abs(lam[5] - 13 * math.pi / 2) < 1e-4


def test_profiles_vanish_with_slope_at_walls_and_have_parity():
    lam = noise.cr_lambdas(5)
    zp = np.linspace(-0.5, 0.5, 41)
    for m in range(1, 6):
        g, dg = noise.cr_g(m, lam[m - 1], np.array([-0.5, 0.5]))
        assert np.abs(g).max() < 1e-13 and np.abs(dg).max() < 1e-12 * lam[m - 1] ** 2
        gz, _ = noise.cr_g(m, lam[m - 1], zp)
        sign = 1 if m % 2 == 1 else -1
        np.testing.assert_allclose(gz[::-1], sign * gz, atol=1e-14)
        # interior zeros: g_m has m - 1 sign changes inside (-1/2, 1/2)
        inner = gz[1:-1]
        assert np.count_nonzero(np.diff(np.sign(inner[np.abs(inner) > 1e-12])) != 0) == m - 1


def test_mode_enumeration():
    """Half-plane annulus 4 <= n^2 + l^2 <= 25 for Lx = Ly = 2 pi, times m = 2..5."""
    ms = noise.modes(2 * math.pi, 2 * math.pi)
    hor = sorted({(n, l) for n, l, _ in ms})
    brute = sorted((n, l) for n in range(-6, 7) for l in range(0, 7)
                   if 4 <= n * n + l * l <= 25 and (l > 0 or n > 0))
    assert hor == brute and len(ms) == 4 * len(brute)
    assert [m for _, _, m in ms[:4]] == [2, 3, 4, 5]
    # longer boxes hold more modes (kx = 2 pi n / Lx)
    assert len(noise.modes(4 * math.pi, 2 * math.pi)) > len(ms)


def _curl_of_potentials(Nx, Ny, Nz, draws, Lx, Ly, Lz, kperp2, mrange):
    """q = curl curl(Phi z) + curl(Psi z) with Phi = Re phi, Psi = Re psi
    built from their definitions (App. A) and differentiated numerically:
    complex step in z (g_m and sin are real analytic), exact discrete
    Fourier differentiation in x and y (Nx > 2 max |n|, Ny > 2 max |l|)."""
    ms = noise.modes(Lx, Ly, kperp2, mrange)
    lam = noise.cr_lambdas(mrange[1])
    x = np.arange(Nx) * Lx / Nx
    y = np.arange(Ny) * Ly / Ny
    z = np.arange(Nz) * Lz / (Nz - 1)
    h = 1e-30
    zc = z + 1j * h
    Phi = np.zeros((Nz, Ny, Nx))
    Psi = np.zeros((Nz, Ny, Nx))
    dPhi = np.zeros((Nz, Ny, Nx))
    for j, (n, l, m) in enumerate(ms):
        kx, ky = 2 * math.pi * n / Lx, 2 * math.pi * l / Ly
        k = math.sqrt(kx * kx + ky * ky + lam[m - 1] ** 2)
        a = k ** -4 * np.exp(2j * math.pi * draws[2 * j])
        b = k ** -3 * np.exp(2j * math.pi * draws[2 * j + 1])
        E = np.exp(1j * (kx * x[None, :] + ky * y[:, None]))
        ca, cb = np.real(a * E), np.real(b * E)          # real coefficient fields of g_m(z') and sin(.)
        L = lam[m - 1]
        zp = zc / Lz - 0.5
        if m % 2 == 1:
            g = np.cosh(L * zp) / np.cosh(L / 2) - np.cos(L * zp) / np.cos(L / 2)
        else:
            g = np.sinh(L * zp) / np.sinh(L / 2) - np.sin(L * zp) / np.sin(L / 2)
        s = np.sin(m * math.pi * (zp + 0.5))
        Phi += g.real[:, None, None] * ca
        dPhi += (g.imag / h)[:, None, None] * ca
        Psi += s.real[:, None, None] * cb
    kxv = 2 * math.pi / Lx * np.fft.fftfreq(Nx, 1.0 / Nx)
    kyv = 2 * math.pi / Ly * np.fft.fftfreq(Ny, 1.0 / Ny)
    dx = lambda F: np.real(np.fft.ifft(1j * kxv * np.fft.fft(F, axis=-1), axis=-1))
    dy = lambda F: np.real(np.fft.ifft(1j * kyv[:, None] * np.fft.fft(F, axis=-2), axis=-2))
    u = dx(dPhi) + dy(Psi)
    v = dy(dPhi) - dx(Psi)
    w = -(dx(dx(Phi)) + dy(dy(Phi)))
    return np.stack([u, v, w])


@pytest.mark.parametrize("Nx,Ny,Nz,Lx,Ly,Lz", [(16, 16, 33, 2 * math.pi, 2 * math.pi, 1.0),
                                               (24, 14, 21, 4 * math.pi, 2 * math.pi, 2.0)])
def test_field_is_the_curl_of_the_potentials(Nx, Ny, Nz, Lx, Ly, Lz):
    kperp2, mrange = (4.0, 25.0), (2, 5)
    cnt = len(noise.modes(Lx, Ly, kperp2, mrange))
    draws = synth.noise_draws(cnt, 7)
    q = noise.noise_field(Nx, Ny, Nz, draws, Lx, Ly, Lz, kperp2, mrange, amplitude=1.0)
    ref = _curl_of_potentials(Nx, Ny, Nz, draws, Lx, Ly, Lz, kperp2, mrange)
    ref = ref / np.abs(ref).max()
    assert np.abs(q - ref).max() < 1e-13
    assert abs(np.abs(q).max() - 1.0) < 1e-15


def test_amplitude_and_draw_count():
    cnt = len(noise.modes(2 * math.pi, 2 * math.pi))
    d = synth.noise_draws(cnt)
    q = noise.noise_field(16, 16, 17, d, amplitude=0.25)
    assert abs(np.abs(q).max() - 0.25) < 1e-16
    with pytest.raises(ValueError):
        noise.noise_field(16, 16, 17, d[:-1])


def test_noise_is_no_slip_and_divergence_free():
    cnt = len(noise.modes(2 * math.pi, 2 * math.pi))
    d = synth.noise_draws(cnt, 1)
    v = noise.noise_field(16, 16, 65, d)
    assert v.shape == (3, 65, 16, 16)
    assert np.abs(v[:, [0, -1]]).max() < 1e-14
    # divergence with spectral x, y derivatives and 2nd-order z differences: O(dz^2)
    errs = []
    for Nz in (513, 1025):
        v = noise.noise_field(16, 16, Nz, d)
        k = np.fft.fftfreq(16, 1 / 16)
        dx = np.real(np.fft.ifft(1j * k * np.fft.fft(v[0], axis=-1), axis=-1))
        dy = np.real(np.fft.ifft(1j * k[:, None] * np.fft.fft(v[1], axis=-2), axis=-2))
        dw = np.gradient(v[2], 1 / (Nz - 1), axis=0)
        errs.append(np.abs(dx + dy + dw)[1:-1].max())
    assert errs[1] < 0.3 * errs[0] and errs[1] < 2e-3


def test_noise_spectral_support():
    """Only horizontal modes with 4 <= kx^2 + ky^2 <= 25 (Lx = Ly = 2 pi)."""
    cnt = len(noise.modes(2 * math.pi, 2 * math.pi))
    v = noise.noise_field(32, 32, 33, synth.noise_draws(cnt, 2))
    V = np.abs(np.fft.fft2(v, axes=(-2, -1))).max(axis=(0, 1))
    k = np.fft.fftfreq(32, 1 / 32)
    k2 = k[:, None] ** 2 + k[None, :] ** 2
    inside = (k2 >= 4) & (k2 <= 25)
    assert V[~inside].max() < 1e-12 * V.max()
    assert (V[inside] > 1e-6 * V.max()).sum() > 40
