"""Time-splitting FC-Gram Navier-Stokes / Boussinesq step, plain float64.

Follows Sec. 4 (time splitting, boundary conditions bound-v / bound-p,
pressure split into an inhomogeneous part solved in 3D Fourier space and an
analytic homogeneous part per (kx, ky), Eqs. pressure-analy, A, B, D and
nablap-homogeneous), Sec. 4.3 (exponential filter on the nonlinear term),
Sec. 4.4 (low-storage o-th order Runge-Kutta loop, steps 1-5), Sec. 6
(constant mean-pressure forcing of the channel) and Sec. 7 (Boussinesq
buoyancy and temperature equation).

Array layouts (same as the CUDA library):
  physical  [nf][Nz][Ny][Nx]  real
  mixed     [nf][Nz][Ny][Kx]  complex, Kx = Nx/2 + 1   (x: rfft, y: fft)
  spectral  [nf][N'][Ny][Kx]  complex, N' = Nz + C      (z: FC extension + fft)
Forward transforms are unnormalised, inverse ones carry 1/N (numpy.fft).

Readings of the paper taken here (the paper is silent, garbled or
inconsistent at these points):
  N1  nonlinear term is -(v.grad)v in advective form (the printed momentum
      update of Sec. 4.1/4.4 carries a + sign that contradicts the governing
      equation of Sec. 2).
  N2  inverse transforms are truncated to the Nz physical points; products,
      forcing and buoyancy are formed there; the result is FC-continued and
      transformed forward.
  N3  exponential filter argument is |k|/k_Nyq per direction (the printed
      normalisation gives 2^{2p} at the Nyquist wavenumber, contradicting the
      stated e^{-beta} attenuation there); beta = 16 ln 10, 2p = 100; applied
      to the nonlinear term only.
  N4  filter mode 1 (used by every workload here): sharp 2/3 mask in kx, ky
      (keep 3|n| <= N) and the exponential filter in kz.  Mode 0: exponential
      filter in all three directions as printed in Sec. 4.3.
  R1  stage step dt_j = dt / (o + 1 - j)  (the printed j dt / o is only
      first-order accurate for o = 3; both agree for the o = 2 the paper ran).
  R2  the state is the continued spectral field; the wall pressure-gradient
      planes start at zero.
  R3  channel forcing +F x_hat is added in physical space before the forward
      transform (sign fixed by the laminar profile of Sec. 6).
  P1  phi = dt_j p is used throughout: grad phi^I = k (k.v*)/k^2,
      b, t = w*(wall) - d_z phi^I(wall); p = phi / dt_j.
  P2  mean mode (kx, ky) = (0, 0): phi^H = D z with D = (b + t)/2.
  P3  only tangential velocity (and theta = 0) is injected; the line is
      re-continued from its Nz physical values.
  P4  A = (t - b E)/(gamma (1 - E^2)), B = -(b - t E)/(gamma (1 - E^2)),
      E = exp(-gamma Lz)  (Eqs. A, B).
  K1  odd-order factors (i k, and the k k^T / k^2 projector) use k with the
      Nyquist entries zeroed; the k^2 of the viscous term keeps them.  The
      homogeneous solution uses gamma = |k_perp| of the same Nyquist-zeroed
      wavenumbers as its gradient (i kx Phi, i ky Phi, Phi'), so that
      grad phi^H is divergence-free at every (kx, ky); where that gamma is 0
      (the mean mode and the Nyquist-only modes) phi^H = D z with
      D = (b + t)/2.  With the true Nyquist wavenumber in gamma the x / y
      Nyquist modes grow by ~1e10 per RK2/RK3 step from round-off.
  B1  buoyancy enters the vertical momentum equation as +gamma theta (with the
      +gamma w source in the theta equation this is the convecting sign).
  B2  Nusselt number Nu = 1 - (1/gamma) <d_z theta> at a wall.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .fc import extend, kz_wavenumbers, periodic_wavenumbers
from .fc_tables import fc_matrix


@dataclass
class Params:
    Nx: int
    Ny: int
    Nz: int
    d: int = 5
    C: int = 25
    nfields: int = 3            # 3: Navier-Stokes, 4: Boussinesq (u, v, w, theta)
    rk_order: int = 3
    Lx: float = 2 * math.pi
    Ly: float = 2 * math.pi
    Lz: float = 1.0
    nu: float = 1e-2
    kappa: float = 0.0
    gamma: float = 0.0
    forcing_x: float = 0.0
    filter: int = 1
    filter_beta: float = 16 * math.log(10.0)
    filter_2p: float = 100.0
    Mr: np.ndarray | None = field(default=None, repr=False)

    def __post_init__(self):
        if self.Mr is None:
            self.Mr = fc_matrix(self.d, self.C)

    @property
    def Np(self):
        return self.Nz + self.C

    @property
    def Kx(self):
        return self.Nx // 2 + 1


# ----------------------------------------------------------------------------
# wavenumbers (Eq. (k), FFT ordering) and factors
# ----------------------------------------------------------------------------

def _zero_nyq(k: np.ndarray, N: int, half: bool = False) -> np.ndarray:
    k = k.copy()
    if N % 2 == 0:
        k[N // 2] = 0.0
    return k


def wavenumbers(p: Params):
    kx = 2 * np.pi * np.arange(p.Kx) / p.Lx                  # rfft ordering
    ky = periodic_wavenumbers(p.Ny, p.Ly)
    kz = kz_wavenumbers(p.Nz, p.C, p.Lz)
    return kx, ky, kz


def odd_wavenumbers(p: Params):
    kx, ky, kz = wavenumbers(p)
    kxo = kx.copy()
    if p.Nx % 2 == 0:
        kxo[p.Nx // 2] = 0.0
    return kxo, _zero_nyq(ky, p.Ny), _zero_nyq(kz, p.Np)


def _bcast(kx, ky, kz):
    return kz[:, None, None], ky[None, :, None], kx[None, None, :]


def filter_factor(p: Params) -> np.ndarray:
    """Per-mode filter applied to the nonlinear term, shape [N'][Ny][Kx] (Sec. 4.3, N3, N4)."""
    nx = np.arange(p.Kx)
    ny = np.fft.fftfreq(p.Ny, d=1.0 / p.Ny)
    nz = np.fft.fftfreq(p.Np, d=1.0 / p.Np)
    two_p = p.filter_2p
    fz = np.exp(-p.filter_beta * (np.abs(nz) / (p.Np / 2)) ** two_p)
    if p.filter == 0:
        fx = np.exp(-p.filter_beta * (np.abs(nx) / (p.Nx / 2)) ** two_p)
        fy = np.exp(-p.filter_beta * (np.abs(ny) / (p.Ny / 2)) ** two_p)
        # exp(-b(a+b+c)) = product of the three per-direction factors
        return fz[:, None, None] * fy[None, :, None] * fx[None, None, :]
    mx = (3 * np.abs(nx) <= p.Nx).astype(float)
    my = (3 * np.abs(ny) <= p.Ny).astype(float)
    return fz[:, None, None] * my[None, :, None] * mx[None, None, :]


# ----------------------------------------------------------------------------
# transforms between the three spaces
# ----------------------------------------------------------------------------

def xy_forward(phys: np.ndarray) -> np.ndarray:
    """[.., Nz, Ny, Nx] real -> [.., Nz, Ny, Kx] complex (rfft in x, fft in y)."""
    return np.fft.fft(np.fft.rfft(phys, axis=-1), axis=-2)


def xy_inverse(mixed: np.ndarray, Nx: int) -> np.ndarray:
    return np.fft.irfft(np.fft.ifft(mixed, axis=-2), n=Nx, axis=-1)


def z_forward(mixed: np.ndarray, p: Params) -> np.ndarray:
    """FC-continue each z-line, then DFT of length N' (Sec. 3, mixed-space ordering)."""
    return np.fft.fft(extend(mixed, p.Mr, axis=-3), axis=-3)


def z_inverse(spec: np.ndarray, p: Params) -> np.ndarray:
    """Inverse DFT along z, truncated to the Nz physical points."""
    return np.fft.ifft(spec, axis=-3)[..., :p.Nz, :, :]


def to_spectral(phys: np.ndarray, p: Params) -> np.ndarray:
    return z_forward(xy_forward(phys), p)


def to_physical(spec: np.ndarray, p: Params) -> np.ndarray:
    return xy_inverse(z_inverse(spec, p), p.Nx)


# ----------------------------------------------------------------------------
# right-hand side (Sec. 4.2, Sec. 4.4 step 1, Sec. 6, Sec. 7)
# ----------------------------------------------------------------------------

def nonlinear_hat(state: np.ndarray, p: Params) -> np.ndarray:
    """Filtered spectral nonlinear term (advection, forcing, buoyancy)."""
    kxo, kyo, kzo = odd_wavenumbers(p)
    KZ, KY, KX = _bcast(kxo, kyo, kzo)
    nf = state.shape[0]
    val = np.empty((nf, p.Nz, p.Ny, p.Nx))
    grad = np.empty((nf, 3, p.Nz, p.Ny, p.Nx))
    for c in range(nf):
        m = z_inverse(state[c], p)
        val[c] = xy_inverse(m, p.Nx)
        grad[c, 0] = xy_inverse(1j * KX * m, p.Nx)
        grad[c, 1] = xy_inverse(1j * KY * m, p.Nx)
        grad[c, 2] = xy_inverse(z_inverse(1j * KZ * state[c], p), p.Nx)
    u = val[:3]
    N = np.empty((nf, p.Nz, p.Ny, p.Nx))
    for c in range(nf):
        N[c] = -(u[0] * grad[c, 0] + u[1] * grad[c, 1] + u[2] * grad[c, 2])
    N[0] += p.forcing_x
    if nf == 4:
        N[2] += p.gamma * val[3]
        N[3] += p.gamma * val[2]
    return to_spectral(N, p) * filter_factor(p)[None]


def diffusivities(p: Params, nf: int) -> list:
    return [p.nu, p.nu, p.nu, p.kappa][:nf]


def ksq(p: Params) -> np.ndarray:
    kx, ky, kz = wavenumbers(p)
    KZ, KY, KX = _bcast(kx, ky, kz)
    return KX ** 2 + KY ** 2 + KZ ** 2


def rhs_hat(state: np.ndarray, p: Params) -> np.ndarray:
    """N_hat - nu k^2 v_hat (the bracket of Sec. 4.4 step 1)."""
    Nh = nonlinear_hat(state, p)
    K2 = ksq(p)
    out = np.empty_like(Nh)
    for c, dif in enumerate(diffusivities(p, state.shape[0])):
        out[c] = Nh[c] - dif * K2 * state[c]
    return out


def ns_rhs(phys: np.ndarray, p: Params) -> np.ndarray:
    """Physical-space RHS for fields ``phys``: state = FC continuation of phys."""
    st = to_spectral(phys, p)
    return np.stack([to_physical(r, p) for r in rhs_hat(st, p)])


# ----------------------------------------------------------------------------
# pressure: inhomogeneous (Fourier) + homogeneous (analytic) parts, projection
# ----------------------------------------------------------------------------

def inject(mixed: np.ndarray, p: Params, dt_stage: float, gradp_prev: np.ndarray) -> np.ndarray:
    """Strong imposition at z = 0, Lz (Sec. 4.1 bound-v, Sec. 4.4 step 2, P3).

    mixed: [nf][Nz][Ny][Kx]; gradp_prev: [2 walls][2 comps][Ny][Kx].
    """
    m = mixed.copy()
    for wall, s in ((0, 0), (1, p.Nz - 1)):
        m[0, s] = dt_stage * gradp_prev[wall, 0]
        m[1, s] = dt_stage * gradp_prev[wall, 1]
        if m.shape[0] == 4:
            m[3, s] = 0.0
    return m


def homogeneous_coefficients(b: np.ndarray, t: np.ndarray, p: Params):
    """A, B (and D where gamma = 0) of Eqs. A, B, D with the P1/P2/P4/K1 readings.

    Returns gamma [Ny][Kx], A, B [Ny][Kx] and D [Ny][Kx] (nonzero only where
    gamma = 0)."""
    kxo, kyo, _ = odd_wavenumbers(p)
    gam = np.sqrt(kxo[None, :] ** 2 + kyo[:, None] ** 2)         # [Ny][Kx]
    E = np.exp(-gam * p.Lz)
    flat = gam == 0
    with np.errstate(divide="ignore", invalid="ignore"):
        den = gam * (1 - E * E)
        A = np.where(flat, 0.0, (t - b * E) / den)
        B = np.where(flat, 0.0, -(b - t * E) / den)
    D = np.where(flat, 0.5 * (b + t), 0.0)
    return gam, A, B, D


def project_core(vs: np.ndarray, p: Params, dt_stage: float):
    """Project continued spectral v*c (3 comps) -> v; returns (v_hat, gradp_walls, |b00 - t00|).

    Sec. 4.4 steps 3-5: inhomogeneous part in (kx, ky, kz), b and t from the
    mixed-space values of w* - d_z phi^I at the walls, analytic homogeneous
    gradient sampled at the Nz points, FC-continued and transformed.
    """
    kxo, kyo, kzo = odd_wavenumbers(p)
    KZ, KY, KX = _bcast(kxo, kyo, kzo)
    kk = KX ** 2 + KY ** 2 + KZ ** 2
    div = KX * vs[0] + KY * vs[1] + KZ * vs[2]
    with np.errstate(divide="ignore", invalid="ignore"):
        s = np.where(kk > 0, div / kk, 0.0)
    gI = np.stack([KX * s, KY * s, KZ * s])
    wz = z_inverse(vs[2] - gI[2], p)                              # [Nz][Ny][Kx]
    b, t = wz[0], wz[p.Nz - 1]
    gam, A, B, D = homogeneous_coefficients(b, t, p)
    z = np.arange(p.Nz) * (p.Lz / (p.Nz - 1))
    ep = np.exp(gam[None] * (z[:, None, None] - p.Lz))            # e^{gamma (z - Lz)}
    em = np.exp(-gam[None] * z[:, None, None])                    # e^{-gamma z}
    Phi = A[None] * ep + B[None] * em
    dPhi = gam[None] * (A[None] * ep - B[None] * em) + D[None]
    kx1 = kxo[None, None, :]
    ky1 = kyo[None, :, None]
    gH_mixed = np.stack([1j * kx1 * Phi, 1j * ky1 * Phi, dPhi])
    gH = z_forward(gH_mixed, p)
    v = vs - gI - gH
    # wall pressure gradient (tangential), p = phi / dt_j
    gIw = z_inverse(gI[:2], p)                                    # [2][Nz][Ny][Kx]
    gp = np.empty((2, 2, p.Ny, p.Kx), dtype=complex)
    for wall, s_ in ((0, 0), (1, p.Nz - 1)):
        gp[wall, 0] = (gIw[0, s_] + gH_mixed[0, s_]) / dt_stage
        gp[wall, 1] = (gIw[1, s_] + gH_mixed[1, s_]) / dt_stage
    return v, gp, abs(b[0, 0] - t[0, 0])


def poisson_project(vstar_phys: np.ndarray, p: Params, dt_stage: float,
                    gradp_prev: np.ndarray | None = None):
    """Physical v* (3 comps) -> projected physical v and the new wall grad p."""
    if gradp_prev is None:
        gradp_prev = np.zeros((2, 2, p.Ny, p.Kx), dtype=complex)
    m = inject(xy_forward(vstar_phys), p, dt_stage, gradp_prev)
    vs = z_forward(m, p)
    v, gp, _ = project_core(vs, p, dt_stage)
    return np.stack([to_physical(c, p) for c in v]), gp


# ----------------------------------------------------------------------------
# low-storage time-splitting Runge-Kutta (Sec. 4.4)
# ----------------------------------------------------------------------------

def stage_dt(dt: float, o: int, j: int) -> float:
    """Stage step of stage j = 1..o (reading R1)."""
    return dt / (o + 1 - j)


def rk_step(state: np.ndarray, gradp: np.ndarray, p: Params, dt: float):
    """One time step; returns (new state, new wall grad p planes)."""
    o = p.rk_order
    nf = state.shape[0]
    v0 = state
    vj = state
    K2 = ksq(p)
    difs = diffusivities(p, nf)
    for j in range(1, o + 1):
        dtj = stage_dt(dt, o, j)
        Nh = nonlinear_hat(vj, p)
        vstar = np.empty_like(v0)
        for c in range(nf):
            vstar[c] = v0[c] + dtj * (Nh[c] - difs[c] * K2 * vj[c])
        m = inject(z_inverse(vstar, p), p, dtj, gradp)
        vsc = z_forward(m, p)
        vnew = np.empty_like(vsc)
        vnew[:3], gradp, _ = project_core(vsc[:3], p, dtj)
        if nf == 4:
            vnew[3] = vsc[3]
        vj = vnew
    return vj, gradp


# ----------------------------------------------------------------------------
# diagnostics (Sec. 6 wall slip / divergence, Sec. 7 Nusselt)
# ----------------------------------------------------------------------------

def divergence_phys(state: np.ndarray, p: Params) -> np.ndarray:
    kxo, kyo, kzo = odd_wavenumbers(p)
    KZ, KY, KX = _bcast(kxo, kyo, kzo)
    return to_physical(1j * (KX * state[0] + KY * state[1] + KZ * state[2]), p)


def wall_mean_squares(state: np.ndarray, p: Params):
    v = np.stack([to_physical(c, p) for c in state[:3]])
    walls = v[:, [0, p.Nz - 1]]
    return (walls[0] ** 2).mean(), (walls[1] ** 2).mean(), (walls[2] ** 2).mean()


def nusselt(state: np.ndarray, p: Params):
    """(Nu at z=0, Nu at z=Lz) from the mean of d_z theta at each wall (B2)."""
    _, _, kzo = odd_wavenumbers(p)
    dth = to_physical(1j * kzo[:, None, None] * state[3], p)
    return (1 - dth[0].mean() / p.gamma, 1 - dth[-1].mean() / p.gamma)


def flow_rate(state: np.ndarray, p: Params) -> float:
    return to_physical(state[0], p).mean()


# ----------------------------------------------------------------------------
# restarts on another grid (Sec. 6: spectral interpolation by zero padding)
# ----------------------------------------------------------------------------

def spectral_interpolate(state: np.ndarray, p1: Params, p2: Params) -> np.ndarray:
    """State of grid p1 -> state of grid p2 (Nx2 >= Nx1, Ny2 >= Ny1, same box,
    fields and (d, C)), following the restart procedure of Sec. 6.

    x, y: the transformed field is zero-padded in the wavenumber domain; the
    coefficients scale with (Nx2 Ny2)/(Nx1 Ny1) (unnormalised forward
    transforms) and a Nyquist coefficient of the coarse grid, which stands for
    a cosine, is split in half between +N/2 and -N/2 (reading I1).
    z: the continued field is N'1-periodic with period L'1 = N'1 dz1; its
    Fourier series (the Nyquist term as a cosine, reading I2) is evaluated at
    the Nz2 physical points of the new grid, and those values are FC-continued
    on the new grid (the continuation period changes with the grid, so the z
    coefficients cannot be zero-padded directly; reading I3)."""
    assert p2.Nx >= p1.Nx and p2.Ny >= p1.Ny and p1.Lz == p2.Lz
    nf = state.shape[0]
    Np1 = p1.Np
    # z: evaluate the series at the new points, per (kx, ky) line
    dz1 = p1.Lz / (p1.Nz - 1)
    z2 = np.arange(p2.Nz) * (p2.Lz / (p2.Nz - 1))
    L1 = Np1 * dz1
    l = np.fft.fftfreq(Np1, 1.0 / Np1)                     # signed integer frequencies
    E = np.exp(2j * np.pi * np.outer(z2, l) / L1)          # [Nz2][N'1]
    if Np1 % 2 == 0:
        E[:, Np1 // 2] = np.cos(np.pi * Np1 * z2 / L1)     # Nyquist as a cosine
    mixed1 = np.einsum("sl,flyx->fsyx", E, state) / Np1    # [nf][Nz2][Ny1][Kx1]
    # x, y: zero padding
    Kx1, Kx2 = p1.Kx, p2.Kx
    mixed2 = np.zeros((nf, p2.Nz, p2.Ny, Kx2), complex)
    scale = (p2.Nx * p2.Ny) / (p1.Nx * p1.Ny)
    ny1 = p1.Ny
    for j1 in range(ny1):
        m = j1 if j1 < ny1 // 2 else j1 - ny1                # signed ky index
        rows = [(m % p2.Ny, 1.0)]
        if ny1 % 2 == 0 and j1 == ny1 // 2 and p2.Ny > ny1:  # coarse Nyquist -> +-N/2, half each
            rows = [((ny1 // 2) % p2.Ny, 0.5), ((-ny1 // 2) % p2.Ny, 0.5)]
        for j2, w in rows:
            blk = mixed1[:, :, j1, :Kx1] * (scale * w)
            if p1.Nx % 2 == 0 and p2.Nx > p1.Nx:
                blk = blk.copy()
                blk[..., Kx1 - 1] *= 0.5                     # coarse x Nyquist (r2c: one side stored)
            mixed2[:, :, j2, :Kx1] += blk
    return z_forward(mixed2, p2)


# ----------------------------------------------------------------------------
# horizontal statistics (Sec. 6 r.m.s. profiles and spectra)
# ----------------------------------------------------------------------------

def profiles(state: np.ndarray, p: Params):
    """Horizontal mean and r.m.s. fluctuation of every field at the Nz
    physical levels, computed in physical space: [nf][Nz] each."""
    phys = to_physical(state, p)
    mean = phys.mean(axis=(-2, -1))
    rms = np.sqrt(((phys - mean[..., None, None]) ** 2).mean(axis=(-2, -1)))
    return mean, rms


def shell_spectrum(state: np.ndarray, p: Params):
    """Horizontal power of every field in shells of |k_perp| (width
    dk = min(2 pi/Lx, 2 pi/Ly), shell j holds j - 1/2 <= |k_perp|/dk < j + 1/2,
    mean mode excluded), averaged over z with the trapezoid rule: sums to the
    z-average of rms^2.  From the physical fields' 2D FFTs (full spectrum)."""
    phys = to_physical(state, p)
    nf = phys.shape[0]
    F = np.fft.fft2(phys, axes=(-2, -1)) / (p.Nx * p.Ny)          # [nf][Nz][Ny][Nx]
    P = np.abs(F) ** 2
    P[..., 0, 0] = 0.0
    kx = 2 * np.pi * np.fft.fftfreq(p.Nx, 1.0 / p.Nx) / p.Lx
    ky = 2 * np.pi * np.fft.fftfreq(p.Ny, 1.0 / p.Ny) / p.Ly
    dk = min(2 * np.pi / p.Lx, 2 * np.pi / p.Ly)
    kmax = math.hypot(math.pi * p.Nx / p.Lx, math.pi * p.Ny / p.Ly)
    ns = int(math.floor(kmax / dk + 0.5)) + 1
    j = np.floor(np.hypot(kx[None, :], ky[:, None]) / dk + 0.5).astype(int)
    wz = np.full(p.Nz, 1.0 / (p.Nz - 1))
    wz[[0, -1]] *= 0.5
    out = np.zeros((nf, ns))
    Pz = np.einsum("fzyx,z->fyx", P, wz)
    for f in range(nf):
        np.add.at(out[f], np.minimum(j, ns - 1).ravel(), Pz[f].ravel())
    return out, dk
