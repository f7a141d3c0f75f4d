"""App. A: random solenoidal no-slip perturbations built from curl
eigenfunctions, plain float64.  TEST INFRASTRUCTURE ONLY (see the package
header).

The velocity is the toroidal-poloidal sum
    q = curl curl(phi z_hat) + curl(psi z_hat)
      = (d_x d_z phi + d_y psi,  d_y d_z phi - d_x psi,  -(d_xx + d_yy) phi)
of the potentials
    phi = sum a_nlm exp(i(kx x + ky y)) g_m(z'),
    psi = sum b_nlm exp(i(kx x + ky y)) sin(m pi (z' + 1/2)),    z' = z/Lz - 1/2,
with the Chandrasekhar-Reid functions
    g_m(z') = cosh(l z')/cosh(l/2) - cos(l z')/cos(l/2)   (m odd),
              sinh(l z')/sinh(l/2) - sin(l z')/sin(l/2)   (m even),   l = lambda_m,
lambda_m fixed by g_m'(-1/2) = g_m'(1/2) = 0; random phases; amplitudes
|a| = k^-4, |b| = k^-3 with k^2 = kx^2 + ky^2 + lambda_m^2; modes with
kperp2_min <= kx^2 + ky^2 <= kperp2_max and m_min <= m <= m_max (App. A:
4 <= kx^2 + ky^2 <= 25, 2 <= m <= 5).

Readings (App. A is silent on these):
  A1  the field is real: the sums run over the half plane of horizontal
      modes (ky > 0, or ky = 0 and kx > 0) and the real part is taken, which
      supplies the conjugate modes.
  A2  kx = 2 pi n / Lx, ky = 2 pi l / Ly with integer n, l; the annulus
      bounds apply to kx^2 + ky^2 (integers n^2 + l^2 for Lx = Ly = 2 pi)
      and are inclusive: a mode counts as inside when it is within a
      relative 1e-12 of a bound (so that rounding of 2 pi n / Lx never drops
      a mode that lies on the bound, such as n^2 + l^2 = 25).
  A3  the random numbers are two per (n, l, m) mode, u_a and u_b in [0, 1):
      a = k^-4 e^{2 pi i u_a}, b = k^-3 e^{2 pi i u_b}; modes are enumerated
      with n ascending, then l ascending, then m ascending, and draw (u_a,
      u_b) in that order.  The draws are an input of the function.
  A4  the result is scaled so that its largest component magnitude on the
      grid equals ``amplitude`` (the perturbation amplitude is a run
      parameter of the paper's simulations).
"""
from __future__ import annotations

import math

import numpy as np

DEFAULTS = dict(Lx=2 * math.pi, Ly=2 * math.pi, Lz=1.0, kperp2=(4.0, 25.0), mrange=(2, 5),
                slopes=(-4.0, -3.0), amplitude=1.0)


def cr_lambdas(count: int) -> np.ndarray:
    """lambda_1 .. lambda_count (App. A).  g_m'(+-1/2) = 0 with g_m as above
    means, for t = lambda/2: tanh t + tan t = 0 (m odd, even g_m) and
    tanh t - tan t = 0 (m even, odd g_m).  The m-th positive root of the pair
    of equations, taken alternately: odd m in (j pi - pi/2, j pi),
    j = (m + 1)/2; even m in (j pi, j pi + pi/2), j = m/2."""
    from scipy.optimize import brentq
    out = np.empty(count)
    for m in range(1, count + 1):
        if m % 2 == 1:
            j = (m + 1) // 2
            lo, hi = j * math.pi - math.pi / 2, j * math.pi
            f = lambda t: math.tanh(t) + math.tan(t)
        else:
            j = m // 2
            lo, hi = j * math.pi, j * math.pi + math.pi / 2
            f = lambda t: math.tanh(t) - math.tan(t)
        eps = 1e-9
        out[m - 1] = 2.0 * brentq(f, lo + eps, hi - eps, xtol=1e-16, rtol=8.9e-16, maxiter=500)
    return out


def cr_g(m: int, lam: float, zp: np.ndarray):
    """g_m(z') and dg_m/dz' (App. A)."""
    if m % 2 == 1:
        g = np.cosh(lam * zp) / math.cosh(lam / 2) - np.cos(lam * zp) / math.cos(lam / 2)
        dg = lam * (np.sinh(lam * zp) / math.cosh(lam / 2) + np.sin(lam * zp) / math.cos(lam / 2))
    else:
        g = np.sinh(lam * zp) / math.sinh(lam / 2) - np.sin(lam * zp) / math.sin(lam / 2)
        dg = lam * (np.cosh(lam * zp) / math.sinh(lam / 2) - np.cos(lam * zp) / math.sin(lam / 2))
    return g, dg


def modes(Lx: float, Ly: float, kperp2=(4.0, 25.0), mrange=(2, 5)) -> list[tuple[int, int, int]]:
    """The (n, l, m) modes in the order of reading A3."""
    nmax = int(math.floor(math.sqrt(kperp2[1]) * Lx / (2 * math.pi))) + 1
    lmax = int(math.floor(math.sqrt(kperp2[1]) * Ly / (2 * math.pi))) + 1
    out = []
    for n in range(-nmax, nmax + 1):
        for l in range(0, lmax + 1):
            if l == 0 and n <= 0:
                continue
            kx, ky = 2 * math.pi * n / Lx, 2 * math.pi * l / Ly
            kp2 = kx * kx + ky * ky
            if not (kperp2[0] * (1 - 1e-12) <= kp2 <= kperp2[1] * (1 + 1e-12)):
                continue
            for m in range(mrange[0], mrange[1] + 1):
                out.append((n, l, m))
    return out


def noise_field(Nx: int, Ny: int, Nz: int, draws: np.ndarray, Lx: float = DEFAULTS["Lx"],
                Ly: float = DEFAULTS["Ly"], Lz: float = 1.0, kperp2=(4.0, 25.0), mrange=(2, 5),
                slopes=(-4.0, -3.0), amplitude: float = 1.0) -> np.ndarray:
    """q on the grid x_i = i Lx/Nx, y_j = j Ly/Ny, z_s = s Lz/(Nz - 1), shape
    [3][Nz][Ny][Nx] float64; ``draws`` holds the 2 * len(modes(...)) uniform
    numbers of reading A3."""
    ms = modes(Lx, Ly, kperp2, mrange)
    draws = np.asarray(draws, dtype=np.float64)
    if draws.shape != (2 * len(ms),):
        raise ValueError(f"need {2 * len(ms)} draws, got {draws.shape}")
    lams = cr_lambdas(max(mrange[1], 1))
    x = np.arange(Nx) * Lx / Nx
    y = np.arange(Ny) * Ly / Ny
    z = np.arange(Nz) * Lz / (Nz - 1)
    zp = z / Lz - 0.5
    q = np.zeros((3, Nz, Ny, Nx), dtype=np.complex128)
    for j, (n, l, m) in enumerate(ms):
        kx, ky = 2 * math.pi * n / Lx, 2 * math.pi * l / Ly
        lam = lams[m - 1]
        k = math.sqrt(kx * kx + ky * ky + lam * lam)
        a = k ** slopes[0] * np.exp(2j * math.pi * draws[2 * j])
        b = k ** slopes[1] * np.exp(2j * math.pi * draws[2 * j + 1])
        E = np.exp(1j * (kx * x[None, :] + ky * y[:, None]))            # [Ny][Nx]
        g, dg = cr_g(m, lam, zp)
        dgdz = dg / Lz                                                     # d/dz = (1/Lz) d/dz'
        s = np.sin(m * math.pi * (zp + 0.5))
        # poloidal part curl curl(phi z_hat) = (d_x d_z phi, d_y d_z phi, -(d_xx + d_yy) phi)
        q[0] += (1j * kx * a * dgdz)[:, None, None] * E
        q[1] += (1j * ky * a * dgdz)[:, None, None] * E
        q[2] += ((kx * kx + ky * ky) * a * g)[:, None, None] * E
        # toroidal part curl(psi z_hat) = (d_y psi, -d_x psi, 0)
        q[0] += (1j * ky * b * s)[:, None, None] * E
        q[1] += (-1j * kx * b * s)[:, None, None] * E
    v = q.real
    return v * (amplitude / np.abs(v).max())
