"""FC-Gram continuation tables, built from the definitions in extended precision.

Follows Sec. 3 (continuation formula and the remark that the tables are
precomputed once) and App. B (matching sets D_r, D_l, the discrete inner
product, the Gram basis from the QR factorisation of the Vandermonde matrix,
oversampled least-squares Fourier continuation with periodicity interval
[1 - delta_r, 2b - (1 - delta_r)], and the block form A f = A_l Q_l^T f_l +
A_r Q_r^T f_r).

Geometry (grid units h = dz, origin at the first right matching point):
  right matching points   t = 0 .. d-1         (samples f_{N-d} .. f_{N-1})
  continuation points     t = d .. d+C-1
  left matching points    t = d+C .. 2d+C-1     (samples f_0 .. f_{d-1} shifted by b)
  Fourier period          P = 2 (d + C)         (= 2b - 2(1 - delta_r) in grid units)

Readings where the paper leaves a choice open ("appropriately selected
bandwidth", "appropriately oversampled"):
  * bandwidth M = floor(2 (d + C) / 3)  (20 for d=5,C=25; 26 for d=7,C=33),
  * oversampling n_os = 20 points per grid interval on both matching intervals,
  * plain least squares (no regularisation), solved by Householder QR at
    60 significant digits.

Because the number of polynomials equals the number of matching points (d),
projecting onto the Gram basis is exact interpolation, so the composite
C x d matrix M_r = A_r Q_r^T does not depend on which basis of the polynomial
space is used.  This oracle therefore fits the d Lagrange polynomials of the
matching nodes directly; the library builds the Gram basis by QR as App. B
describes.  Agreement of the two is a genuine cross-check.

The left-end matrix is the mirror image: M_l = J_C M_r J_d (Sec. 3, the
row-reversal / column-reversal operators in the continuation formula).
"""
from __future__ import annotations

import os
from functools import lru_cache

import numpy as np

N_OS = 20
DPS = 60


def default_bandwidth(d: int, C: int) -> int:
    return (2 * (d + C)) // 3


def _mp():
    import mpmath
    return mpmath


def build_mr_mp(d: int, C: int, M: int | None = None, n_os: int = N_OS, dps: int = DPS,
                basis: str = "lagrange"):
    """Return M_r as a list of C rows of d mpmath numbers.

    basis='lagrange' fits each Lagrange cardinal polynomial of the nodes
    0..d-1; basis='gram' fits the Gram polynomials obtained by QR of the
    Vandermonde matrix (App. B) and multiplies by Q^T.  Both give the same
    matrix in exact arithmetic.
    """
    mp = _mp()
    if M is None:
        M = default_bandwidth(d, C)
    with mp.workdps(dps):
        P = 2 * (d + C)
        ts_r = [mp.mpf(i) / n_os for i in range((d - 1) * n_os + 1)]
        ts_l = [mp.mpf(d + C) + mp.mpf(i) / n_os for i in range((d - 1) * n_os + 1)]
        two_pi_over_P = 2 * mp.pi / P

        def trig_row(t):
            r = [mp.mpf(1)]
            for m in range(1, M + 1):
                a = two_pi_over_P * m * t
                r.append(mp.cos(a))
                r.append(mp.sin(a))
            return r

        A = mp.matrix([trig_row(t) for t in ts_r + ts_l])
        Qa, Ra = mp.qr(A)
        ncol = A.cols

        def lsq(b):
            qtb = Qa.T * b
            x = [mp.mpf(0)] * ncol
            for k in range(ncol - 1, -1, -1):
                s = qtb[k]
                for j in range(k + 1, ncol):
                    s -= Ra[k, j] * x[j]
                x[k] = s / Ra[k, k]
            return x

        cont_rows = [trig_row(mp.mpf(d + j)) for j in range(C)]

        def continuation_of(poly_vals_fn):
            b = mp.matrix([poly_vals_fn(t) for t in ts_r] + [mp.mpf(0)] * len(ts_l))
            x = lsq(b)
            resid = A * mp.matrix(x) - b
            rel = mp.norm(resid) / mp.norm(b)
            return [mp.fsum(xv * rv for xv, rv in zip(x, row)) for row in cont_rows], rel

        cols = []
        resids = []
        if basis == "lagrange":
            for i in range(d):
                def lag(t, i=i):
                    v = mp.mpf(1)
                    for j in range(d):
                        if j != i:
                            v *= (t - j) / mp.mpf(i - j)
                    return v
                col, rel = continuation_of(lag)
                cols.append(col)
                resids.append(rel)
        elif basis == "gram":
            # Vandermonde on the matching nodes, QR -> orthonormal Gram basis values
            V = mp.matrix([[mp.mpf(t) ** p for p in range(d)] for t in range(d)])
            Qv, Rv = mp.qr(V)
            # polynomial coefficients of Gram polynomial k: V c_k = Qv[:, k]
            gram_cols = []
            for k in range(d):
                ck = mp.lu_solve(V, Qv.column(k))
                def gk(t, ck=ck):
                    return mp.fsum(ck[p] * mp.mpf(t) ** p for p in range(d))
                col, rel = continuation_of(gk)
                gram_cols.append(col)
                resids.append(rel)
            # M_r[j, i] = sum_k A[j, k] Q[i, k]
            cols = [[mp.fsum(gram_cols[k][j] * Qv[i, k] for k in range(d)) for j in range(C)]
                    for i in range(d)]
        else:
            raise ValueError(basis)
        Mr = [[cols[i][j] for i in range(d)] for j in range(C)]
        return Mr, resids


def _to_f64(Mr) -> np.ndarray:
    return np.array([[float(v) for v in row] for row in Mr], dtype=np.float64)


def table_path(d: int, C: int, M: int, n_os: int, directory: str) -> str:
    return os.path.join(directory, f"fc_table_d{d}_C{C}_M{M}_os{n_os}.txt")


def write_table(d: int, C: int, directory: str, M: int | None = None, n_os: int = N_OS) -> str:
    """Write M_r (C rows, d columns) to a text file with 25 significant digits."""
    mp = _mp()
    if M is None:
        M = default_bandwidth(d, C)
    Mr, resid = build_mr_mp(d, C, M, n_os)
    path = table_path(d, C, M, n_os, directory)
    with open(path, "w") as fh:
        fh.write(f"# FC-Gram right continuation matrix M_r (C={C} rows, d={d} columns)\n")
        fh.write(f"# bandwidth M={M}, oversampling n_os={n_os}, built at {DPS} digits by oracle.fc_tables\n")
        fh.write(f"# max relative least-squares residual {max(float(r) for r in resid):.3e}\n")
        for row in Mr:
            fh.write(" ".join(mp.nstr(v, 25, min_fixed=-1, max_fixed=-1) for v in row) + "\n")
    return path


def read_table(path: str) -> np.ndarray:
    rows = []
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([float(v) for v in line.split()])
    return np.array(rows, dtype=np.float64)


STORED = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden")


@lru_cache(maxsize=None)
def fc_matrix(d: int, C: int, M: int | None = None, n_os: int = N_OS,
              table_dir: str | None = STORED) -> np.ndarray:
    """float64 M_r (C x d).  Uses a stored table written by ``write_table`` (by
    this module, see tests/golden/make_fc_tables.py) when ``table_dir`` holds
    one, for hosts without mpmath; else builds it."""
    if M is None:
        M = default_bandwidth(d, C)
    if table_dir is not None:
        p = table_path(d, C, M, n_os, table_dir)
        if os.path.exists(p):
            return read_table(p)
    Mr, _ = build_mr_mp(d, C, M, n_os)
    return _to_f64(Mr)


def mirror(Mr: np.ndarray) -> np.ndarray:
    """Left-end matrix M_l = J_C M_r J_d (row and column reversal, Sec. 3)."""
    return Mr[::-1, ::-1].copy()
