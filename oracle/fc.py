"""FC-Gram continuation and spectral z-derivatives, plain float64.

Follows Sec. 3: the continuation formula (C extension values from the first
and last d samples through the precomputed matrices), the extended periodic
grid of N' = Nz + C points with period L'z = N' dz, the wavenumber vector of
Eq. (k), and Sec. 4.2: derivatives of continued fields are taken by
multiplying the Fourier coefficients by i k.

Readings:
  * dz = Lz / (Nz - 1): both walls are grid points (App. B, the grid
    0 = x_0 < ... < x_{N-1} = 1).
  * Nyquist mode (l = N'/2) is zeroed for odd derivative orders and kept for
    even orders (the paper is silent).
  * The derivative returned is the first Nz samples of the inverse transform.
"""
from __future__ import annotations

import numpy as np

from .fc_tables import mirror


def continuation(f_first: np.ndarray, f_last: np.ndarray, Mr: np.ndarray) -> np.ndarray:
    """The C continuation values from the first and last d samples.

    f_first, f_last: [d, ...] along axis 0.  Returns [C, ...].
    Continuation = M_r f_last + (J_C M_r J_d) f_first   (Sec. 3, App. B eq. Af).
    """
    Ml = mirror(Mr)
    return np.tensordot(Mr, f_last, axes=(1, 0)) + np.tensordot(Ml, f_first, axes=(1, 0))


def extend(f: np.ndarray, Mr: np.ndarray, axis: int = 0) -> np.ndarray:
    """[f; continuation] along ``axis`` (length Nz -> Nz + C), the block form of App. B."""
    f = np.moveaxis(np.asarray(f), axis, 0)
    d = Mr.shape[1]
    c = continuation(f[:d], f[-d:], Mr)
    return np.moveaxis(np.concatenate([f, c], axis=0), 0, axis)


def kz_wavenumbers(Nz: int, C: int, Lz: float) -> np.ndarray:
    """k_l = 2 pi l / L'z in FFT order, L'z = (Nz + C) dz (Eq. (k), shifted index)."""
    Np = Nz + C
    dz = Lz / (Nz - 1)
    return 2 * np.pi * np.fft.fftfreq(Np, d=dz)


def periodic_wavenumbers(N: int, L: float) -> np.ndarray:
    return 2 * np.pi * np.fft.fftfreq(N, d=L / N)


def deriv_factor(k: np.ndarray, order: int) -> np.ndarray:
    """(i k)^order with the Nyquist entry zeroed for odd orders."""
    fac = (1j * k) ** order
    N = k.shape[0]
    if order % 2 == 1 and N % 2 == 0:
        fac = fac.copy()
        fac[N // 2] = 0.0
    return fac


def fc_deriv_z(f: np.ndarray, Lz: float, Mr: np.ndarray, order: int = 1, axis: int = 0) -> np.ndarray:
    """z-derivative of order ``order`` of samples f (Nz along ``axis``) by FC-Gram.

    Continue, DFT of length N' = Nz + C, multiply by (i k)^order, inverse DFT,
    keep the first Nz samples (Sec. 3 and Sec. 4.2).
    """
    f = np.moveaxis(np.asarray(f), axis, 0)
    Nz = f.shape[0]
    C = Mr.shape[0]
    fe = extend(f, Mr, axis=0)
    Fh = np.fft.fft(fe, axis=0)
    k = kz_wavenumbers(Nz, C, Lz)
    fac = deriv_factor(k, order).reshape((-1,) + (1,) * (f.ndim - 1))
    out = np.fft.ifft(Fh * fac, axis=0)[:Nz]
    if np.isrealobj(f):
        out = out.real
    return np.moveaxis(out, 0, axis)


def dense_deriv_operator(Nz: int, C: int, Lz: float, Mr: np.ndarray, order: int) -> np.ndarray:
    """Nz x Nz matrix R . IDFT . diag((ik)^order) . DFT . [I; M] built from explicit
    O(N'^2) sums (no FFT), for brute-force checks on tiny grids."""
    Np = Nz + C
    d = Mr.shape[1]
    E = np.zeros((Np, Nz))
    E[:Nz, :Nz] = np.eye(Nz)
    Ml = mirror(Mr)
    E[Nz:, Nz - d:] += Mr
    E[Nz:, :d] += Ml
    j = np.arange(Np)
    W = np.exp(-2j * np.pi * np.outer(j, j) / Np)  # forward DFT matrix
    Winv = np.conj(W) / Np
    k = kz_wavenumbers(Nz, C, Lz)
    fac = deriv_factor(k, order)
    Dfull = Winv @ (fac[:, None] * W)
    return (Dfull[:Nz] @ E).real
