"""Tolerances shared by the parity tests (derivation in the design notes).

Spectral z-derivatives amplify the rounding of the transformed data by up to
k_max^p (k_max = pi/dz, the largest wavenumber of the continued grid), so
errors are measured relative to |x_ext| k_max^p, where x_ext is the
continued data that enters the transform.  Both the oracle (numpy float64)
and the kernels round at that scale with errors growing like log2 of the
transform length; the bound allows 16 log2(N' + Nz) unit roundoffs.
In float64 the first derivative additionally meets 1e-11 relative L2; the
second derivative's float64 floor grows like (N'/128)^2 (the oracle's own
error vs extended precision is 7.6e-11 at N' = 538), so its relative bound is
1e-11 max(1, (N'/128)^2).
These figures hold for the (d, C) = (5, 25) tables.  The continuation M_r f
cancels terms as large as kappa |f|, kappa = max row sum |M_r| (1.16e4 for
(5, 25), 1.45e6 for (7, 33)), so its rounding, and with it the float64 floor
of every derivative, scales with kappa: other tables get the bounds times
fc_amplification(M_r) = max(1, kappa / 1.16e4).
"""
import numpy as np


def normalized_error(out, ref, xnorm, kmax, order):
    return float(np.linalg.norm(np.asarray(out, dtype=np.float64) - ref) / (xnorm * kmax ** order))


def rel_l2(out, ref):
    return float(np.linalg.norm(np.asarray(out, dtype=np.float64) - ref) / np.linalg.norm(ref))


def norm_bound(dtype, Nz: int = 513, C: int = 25) -> float:
    return 16 * np.log2(2 * Nz + C) * float(np.finfo(dtype).eps)


def rel_bound_f64(order: int, Np: int) -> float:
    return 1e-11 * max(1.0, (Np / 128.0) ** (2 * (order - 1)))


def fc_amplification(Mr) -> float:
    return max(1.0, float(np.abs(np.asarray(Mr)).sum(axis=1).max()) / 11629.26)
