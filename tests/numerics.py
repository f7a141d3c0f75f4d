"""Tolerances shared by the parity tests.

Spectral z-derivatives amplify the rounding of the transformed data by up to
k_max^p (k_max = pi/dz, the largest wavenumber of the continued grid), so
errors are measured relative to |x_ext| k_max^p, where x_ext is the
continued data that enters the transform.  Both the oracle (numpy float64)
and the kernels round at that scale with errors growing like log2 of the
transform length; the bound allows 16 log2(N' + Nz) unit roundoffs.

In float64 both derivatives also meet 1e-11 relative L2 against the oracle up
to N' = 538.  The oracle's own float64 error against the same operator in
extended precision (pinned in tests/test_oracle_fc.py) is about 1e-12 (d/dz)
and 3e-12 (d2/dz2) at N' = 538, and grows with N' (the rounding of the
transform and of the continuation is amplified by k_max and k_max^2): 2e-12
and 8e-12 at N' = 1024.  The kernels evaluate the continuation with
compensated (double-double) sums and stay below 1.1e-12 of the exact result,
so the difference from the oracle is the oracle's own floor; above N' = 538
the bound grows like that floor, (N'/538)^p.

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
    return 1e-11 * max(1.0, (Np / 538.0) ** order)


def fc_amplification(Mr) -> float:
    return max(1.0, float(np.abs(np.asarray(Mr)).sum(axis=1).max()) / 11629.26)
