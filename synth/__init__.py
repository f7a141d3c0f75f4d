"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA path.

This module only draws random numbers and evaluates closed-form test
functions (Fourier modes, Chebyshev and polynomial profiles).  It holds none
of the FC-Gram method's arithmetic: no continuation, no spectral
differentiation, no projection.  Both sides receive the same float64 arrays
(cast to float32 for reduced-precision runs).

Seeds: ``numpy.random.Generator(PCG64(BASE_SEED + workload + instance))``.

Workload recipes (shapes follow the channel and Rayleigh-Benard runs of the
paper, Sec. 6 table of channel runs and Sec. 7 table of convection runs):

* channel velocity: a solenoidal no-slip fluctuation built from a toroidal
  and a poloidal potential (the construction of App. A, with polynomial
  instead of Chandrasekhar-Reid profiles),
      v' = curl(psi z_hat) + curl curl(chi z_hat),
      psi = X1(x,y) z(Lz - z)(1 + a1 z + a2 z^2),
      chi = X2(x,y) z^2 (Lz - z)^2 (1 + b1 z),
  X1, X2 sums of horizontal Fourier modes with 0 < |k_perp| <= 8, random
  phases and amplitudes |k_perp|^-3 and |k_perp|^-4 (velocity spectrum
  ~ |k_perp|^-2), scaled to 0.1 max U, plus the laminar profile
  U = F z (Lz - z) / (2 nu) in x (Sec. 6, laminar solution; F/nu = 10 as in
  runs L1-L3).  v' vanishes at both walls and is divergence-free.
* derivative field: f = sum_p X_p(x, y) Z_p(z), X_p a random 2D field with
  |a_k| ~ k^-4/3 up to the 2/3 cutoff, Z_p a Chebyshev series with
  coefficients N(0,1) 2^(-n/2), n <= 16 (exact z-derivatives in closed form).
* Boussinesq: theta = 1e-3 eta(x,y) sin(pi z / Lz), velocity = 1e-3 times a
  channel-type solenoidal fluctuation (no mean flow).
* App. A noise: only the uniform phase draws (``noise_draws``); the
  curl-eigenfunction field built from them is method arithmetic (the library's
  ``fc_noise`` and the oracle's ``noise_field``).
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import chebyshev as _cheb

BASE_SEED = 2002013920


def rng(workload: int, instance: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(BASE_SEED + workload + instance))


def z_grid(Nz: int, Lz: float = 1.0) -> np.ndarray:
    """Uniform grid including both walls: z_s = s Lz/(Nz-1)."""
    return np.arange(Nz, dtype=np.float64) * (Lz / (Nz - 1))


def xy_modes_field(g: np.random.Generator, Nx: int, Ny: int, kmax: float = 8.0,
                   slope: float = -2.0, Lx: float = 2 * np.pi, Ly: float = 2 * np.pi,
                   shell_cut: bool = True) -> np.ndarray:
    """Real field X[y, x] = sum over modes 0 < |k| <= kmax of |k|^slope cos(k.x + phi).

    Returned with max |X| = 1.  Wavenumbers are integers times 2 pi / L.
    """
    kx = np.fft.rfftfreq(Nx, d=1.0 / Nx) * (2 * np.pi / Lx)
    ky = np.fft.fftfreq(Ny, d=1.0 / Ny) * (2 * np.pi / Ly)
    KX, KY = np.meshgrid(kx, ky)
    K = np.sqrt(KX ** 2 + KY ** 2)
    amp = np.zeros_like(K)
    sel = (K > 0) & (K <= kmax)
    amp[sel] = K[sel] ** slope
    phase = g.uniform(0.0, 2 * np.pi, size=K.shape)
    spec = amp * np.exp(1j * phase)
    # Nyquist rows/columns are excluded by kmax for every grid used here.
    X = np.fft.irfft2(spec, s=(Ny, Nx)) * (Nx * Ny)
    m = np.abs(X).max()
    return X / m if m > 0 else X


def kolmogorov_xy_field(g: np.random.Generator, Nx: int, Ny: int,
                        Lx: float = 2 * np.pi, Ly: float = 2 * np.pi) -> np.ndarray:
    """Random 2D field with |a_k| ~ k^-4/3 (shell spectrum ~ k^-5/3), zero above 2/3 k_Nyq."""
    kx = np.fft.rfftfreq(Nx, d=1.0 / Nx)
    ky = np.fft.fftfreq(Ny, d=1.0 / Ny)
    KX, KY = np.meshgrid(kx, ky)
    keep = (3 * np.abs(KX) <= Nx) & (3 * np.abs(KY) <= Ny)
    K = np.sqrt((KX * 2 * np.pi / Lx) ** 2 + (KY * 2 * np.pi / Ly) ** 2)
    amp = np.zeros_like(K)
    sel = keep & (K > 0)
    amp[sel] = K[sel] ** (-4.0 / 3.0)
    phase = g.uniform(0.0, 2 * np.pi, size=K.shape)
    X = np.fft.irfft2(amp * np.exp(1j * phase), s=(Ny, Nx)) * (Nx * Ny)
    m = np.abs(X).max()
    return X / m if m > 0 else X


# ----------------------------------------------------------------------------
# channel flow (incompressible Navier-Stokes, walls at z = 0, Lz)
# ----------------------------------------------------------------------------

def _xy_derivs(X: np.ndarray, Lx: float, Ly: float):
    """Exact x, y derivatives of a trigonometric polynomial sampled on the grid."""
    Ny, Nx = X.shape
    Xh = np.fft.fft2(X)
    kx = 2 * np.pi * np.fft.fftfreq(Nx, d=Lx / Nx)
    ky = 2 * np.pi * np.fft.fftfreq(Ny, d=Ly / Ny)
    KY, KX = np.meshgrid(ky, kx, indexing="ij")
    dx = np.real(np.fft.ifft2(1j * KX * Xh))
    dy = np.real(np.fft.ifft2(1j * KY * Xh))
    lap = np.real(np.fft.ifft2(-(KX ** 2 + KY ** 2) * Xh))
    return dx, dy, lap


def solenoidal_fluctuation(g: np.random.Generator, Nx: int, Ny: int, Nz: int, Lz: float = 1.0,
                           Lx: float = 2 * np.pi, Ly: float = 2 * np.pi, dtype=np.float64) -> np.ndarray:
    """curl(psi z) + curl curl(chi z) with wall-vanishing polynomial profiles,
    shape [3][Nz][Ny][Nx], scaled to max |v| = 1."""
    z = z_grid(Nz, Lz)
    X1 = xy_modes_field(g, Nx, Ny, slope=-3.0, Lx=Lx, Ly=Ly)
    X2 = xy_modes_field(g, Nx, Ny, slope=-4.0, Lx=Lx, Ly=Ly)
    a1, a2, b1 = g.uniform(-1.0, 1.0, size=3)
    poly = np.polynomial.Polynomial
    P = poly([0.0, Lz, -1.0]) * poly([1.0, a1, a2])          # z (Lz - z)(1 + a1 z + a2 z^2)
    Q = poly([0.0, Lz, -1.0]) ** 2 * poly([1.0, b1])         # z^2 (Lz - z)^2 (1 + b1 z)
    Pv, Qv, dQv = P(z), Q(z), Q.deriv()(z)
    X1x, X1y, _ = _xy_derivs(X1, Lx, Ly)
    X2x, X2y, X2lap = _xy_derivs(X2, Lx, Ly)
    # curl(psi z) = (d_y psi, -d_x psi, 0); curl curl(chi z) = (d_x d_z chi, d_y d_z chi, -lap_h chi)
    terms = [((X1y, Pv), (X2x, dQv)), ((-X1x, Pv), (X2y, dQv)), ((-X2lap, Qv), None)]
    # scale: max over the grid of each component, evaluated on the profiles' extrema per xy point
    out = np.empty((3, Nz, Ny, Nx), dtype=dtype)
    tmp = np.empty((Nz, Ny, Nx), dtype=dtype)
    for c, (t1, t2) in enumerate(terms):
        np.multiply(t1[1].astype(dtype)[:, None, None], t1[0].astype(dtype)[None], out=out[c])
        if t2 is not None:
            np.multiply(t2[1].astype(dtype)[:, None, None], t2[0].astype(dtype)[None], out=tmp)
            out[c] += tmp
    del tmp
    out *= dtype(1.0) / np.abs(out).max() if dtype is not np.float64 else 1.0 / np.abs(out).max()
    return out


def channel_velocity(Nx: int, Ny: int, Nz: int, nu: float = 1e-2, F_over_nu: float = 10.0,
                     Lz: float = 1.0, seed_offset: int = 0, fluct: float = 0.1,
                     mean_flow: bool = True) -> np.ndarray:
    """Seeded channel-flow velocity, shape [3][Nz][Ny][Nx] float64."""
    g = rng(0, seed_offset)
    z = z_grid(Nz, Lz)
    F = F_over_nu * nu
    U = F * z * (Lz - z) / (2 * nu)
    Umax = F * Lz * Lz / (8 * nu)
    out = (fluct * Umax) * solenoidal_fluctuation(g, Nx, Ny, Nz, Lz)
    if mean_flow:
        out[0] += U[:, None, None]
    return out


def poiseuille(Nx: int, Ny: int, Nz: int, F: float, nu: float, Lz: float = 1.0) -> np.ndarray:
    """Laminar plane Poiseuille profile U = F z (Lz - z)/(2 nu) (Sec. 6, laminar solution)."""
    z = z_grid(Nz, Lz)
    out = np.zeros((3, Nz, Ny, Nx))
    out[0] = (F * z * (Lz - z) / (2 * nu))[:, None, None]
    return out


# ----------------------------------------------------------------------------
# App. A: the random draws of the curl-eigenfunction perturbation
# ----------------------------------------------------------------------------

def noise_draws(count: int, seed_offset: int = 0) -> np.ndarray:
    """The 2 * count uniform numbers in [0, 1) of an App. A perturbation with
    count (n, l, m) modes (two phases per mode, in mode order); the field
    itself is built by the library (``fc_noise``) and by the oracle from
    these draws."""
    return rng(3, seed_offset).uniform(size=2 * count)


# ----------------------------------------------------------------------------
# ensembles of independent channel instances of uneven sizes
# ----------------------------------------------------------------------------

ENSEMBLE_GRIDS = ((64, 64, 65), (96, 96, 97), (128, 128, 129), (192, 192, 129))


def ensemble_specs(n: int = 64, seed_offset: int = 0, grids=ENSEMBLE_GRIDS, nu_range=(1e-3, 1e-2)):
    """n channel instances: grid drawn uniformly from ``grids``, viscosity
    log-uniform in ``nu_range`` (the batched-ensemble workload).  Returns a list
    of dicts (Nx, Ny, Nz, nu, seed_offset); each instance's fields come from
    ``channel_velocity(..., seed_offset=...)``."""
    g = rng(4, seed_offset)
    out = []
    for i in range(n):
        Nx, Ny, Nz = grids[int(g.integers(0, len(grids)))]
        nu = float(np.exp(g.uniform(np.log(nu_range[0]), np.log(nu_range[1]))))
        out.append(dict(Nx=Nx, Ny=Ny, Nz=Nz, nu=nu, seed_offset=1000 + i))
    return out


# ----------------------------------------------------------------------------
# Rayleigh-Benard (Boussinesq): fields u, v, w, theta
# ----------------------------------------------------------------------------

def boussinesq_fields(Nx: int, Ny: int, Nz: int, Lz: float = 1.0, seed_offset: int = 0,
                      amp: float = 1e-3, dtype=np.float64) -> np.ndarray:
    """Seeded Boussinesq fields, shape [4][Nz][Ny][Nx]; theta is the deviation
    from the linear conduction profile (Sec. 7)."""
    g = rng(2, seed_offset)
    z = z_grid(Nz, Lz)
    out = np.empty((4, Nz, Ny, Nx), dtype=dtype)
    out[:3] = solenoidal_fluctuation(g, Nx, Ny, Nz, Lz, dtype=dtype)
    out[:3] *= dtype(amp * 0.1 * 1.25)
    eta = xy_modes_field(g, Nx, Ny).astype(dtype)
    prof = (amp * np.sin(np.pi * z / Lz)).astype(dtype)
    np.multiply(prof[:, None, None], eta[None, :, :], out=out[3])
    return out


# ----------------------------------------------------------------------------
# fc_deriv_z test field: separable rank-8, exact derivatives in closed form
# ----------------------------------------------------------------------------

class SeparableField:
    """f(x,y,z) = sum_p X_p(x,y) Z_p(z) with Chebyshev Z_p on [0, Lz]."""

    def __init__(self, Nx: int, Ny: int, Nz: int, rank: int = 8, nmax: int = 16,
                 Lz: float = 1.0, seed_offset: int = 0):
        g = rng(1, seed_offset)
        self.Nx, self.Ny, self.Nz, self.Lz = Nx, Ny, Nz, Lz
        self.X = np.stack([kolmogorov_xy_field(g, Nx, Ny) for _ in range(rank)])
        n = np.arange(nmax + 1)
        self.coef = g.standard_normal((rank, nmax + 1)) * 2.0 ** (-n / 2.0)

    def _z(self, order: int) -> np.ndarray:
        z = z_grid(self.Nz, self.Lz)
        t = 2 * z / self.Lz - 1
        rows = []
        for c in self.coef:
            cc = c
            for _ in range(order):
                cc = _cheb.chebder(cc) * (2.0 / self.Lz)
            rows.append(_cheb.chebval(t, cc))
        return np.stack(rows)  # [rank][Nz]

    def field(self, order: int = 0, dtype=np.float64) -> np.ndarray:
        """Values (order 0) or exact z-derivatives, shape [Nz][Ny][Nx]."""
        Z = self._z(order)
        out = np.tensordot(Z.astype(dtype), self.X.astype(dtype), axes=(0, 0))
        return out

    def z_profiles(self, order: int = 0) -> np.ndarray:
        return self._z(order)


def fc_demo_function(Nz: int = 49) -> tuple[np.ndarray, np.ndarray]:
    """The Sec. 3 demonstration function f(z) = sin(15z) sin(5.5z) exp(0.3z) on [0,1]
    and its exact derivative."""
    z = z_grid(Nz, 1.0)
    f = np.sin(15 * z) * np.sin(5.5 * z) * np.exp(0.3 * z)
    df = (15 * np.cos(15 * z) * np.sin(5.5 * z) + 5.5 * np.sin(15 * z) * np.cos(5.5 * z)
          + 0.3 * np.sin(15 * z) * np.sin(5.5 * z)) * np.exp(0.3 * z)
    return f, df
