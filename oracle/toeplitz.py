"""p2o / p2q map as a block lower-triangular Toeplitz matrix (oracle, FP64).

Test infrastructure only (see the package docstring).

Definition (Sec. "FFT-based Hessian matvecs", Eq. ShiftInvariance): with
time-major vectors m = [m_0; ...; m_{Nt-1}], m_j in R^Nm, and
d = [d_0; ...; d_{Nt-1}], d_i in R^Nd, the discrete p2o map is

    d_i = sum_{j=0}^{i} F_{i-j} m_j,        i = 0 .. Nt-1,

where F_l (l = 0 .. Nt-1, 0-based lag; the paper's F_{l+1,1}) are the blocks
of the first block column.  The p2q map has the same form with Nq rows.
The adjoint is the Euclidean transpose (the paper names F* without a weighted
inner product):

    x_j = sum_{i=j}^{Nt-1} F_{i-j}^T y_i,   j = 0 .. Nt-1.

A block column is given either as an array [Nt, Nrows, Nm] or as a callable
lag -> [Nrows, Nm] (used for operators too large to hold on the host).
"""
from __future__ import annotations

import numpy as np


def _block(Fcol, lag):
    return Fcol(lag) if callable(Fcol) else Fcol[lag]


def dense_p2o(Fcol: np.ndarray) -> np.ndarray:
    """The explicit (Nrows*Nt) x (Nm*Nt) block lower-triangular Toeplitz matrix."""
    Nt, Nr, Nm = Fcol.shape
    F = np.zeros((Nr * Nt, Nm * Nt))
    for i in range(Nt):
        for j in range(i + 1):
            F[i * Nr:(i + 1) * Nr, j * Nm:(j + 1) * Nm] = Fcol[i - j]
    return F


def p2o_apply(Fcol, m: np.ndarray, Nt: int | None = None) -> np.ndarray:
    """d_i = sum_{j<=i} F_{i-j} m_j.   m: [Nt, Nm] -> d: [Nt, Nrows]."""
    Nt = m.shape[0] if Nt is None else Nt
    d = None
    for lag in range(Nt):
        Fl = _block(Fcol, lag)                       # [Nr, Nm]
        if d is None:
            d = np.zeros((Nt, Fl.shape[0]))
        # rows i = lag..Nt-1 receive F_lag m_{i-lag}
        d[lag:] += m[:Nt - lag] @ Fl.T
    return d


def p2o_adjoint(Fcol, y: np.ndarray, Nm: int | None = None) -> np.ndarray:
    """x_j = sum_{i>=j} F_{i-j}^T y_i.   y: [Nt, Nrows] -> x: [Nt, Nm]."""
    Nt = y.shape[0]
    x = None
    for lag in range(Nt):
        Fl = _block(Fcol, lag)
        if x is None:
            x = np.zeros((Nt, Fl.shape[1]))
        # columns j = 0..Nt-1-lag receive F_lag^T y_{j+lag}
        x[:Nt - lag] += y[lag:] @ Fl
    return x


def p2o_apply_entry(block_row, m: np.ndarray, i: int) -> np.ndarray:
    """Row block i of F m computed on its own: sum_{j<=i} F_{i-j}[rows] m_j.

    block_row(lag) -> [nrows, Nm] gives the selected rows of F_lag.
    Returns [nrows].
    """
    acc = 0.0
    for j in range(i + 1):
        acc = acc + block_row(i - j) @ m[j]
    return acc


def p2o_adjoint_entry(block_cols, y: np.ndarray, j: int) -> np.ndarray:
    """Block j of F^T y on selected grid columns: sum_{i>=j} F_{i-j}[:, cols]^T y_i.

    block_cols(lag) -> [Nrows, ncols].  Returns [ncols].
    """
    Nt = y.shape[0]
    acc = 0.0
    for i in range(j, Nt):
        acc = acc + y[i] @ block_cols(i - j)
    return acc
