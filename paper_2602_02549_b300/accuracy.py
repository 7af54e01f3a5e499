"""Error of an emulated product against the exact one, on sampled entries.

Measurement only (used by bench.py): the exact value of sum_h a_ih b_hj is
obtained with error-free transformations (Veltkamp/Dekker splitting gives each
product as p + e exactly, barring overflow and underflow) and math.fsum, which
returns the correctly rounded sum of its arguments.  Valid for the paper's
generator, whose entries stay far from the FP64 overflow and underflow limits.
"""
from __future__ import annotations

import math

import numpy as np

_SPLIT = 134217729.0   # 2^27 + 1


def _two_prod(a: np.ndarray, b: np.ndarray):
    p = a * b
    c = _SPLIT * a
    ah = c - (c - a)
    al = a - ah
    c = _SPLIT * b
    bh = c - (c - b)
    bl = b - bh
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def exact_dot(x: np.ndarray, y: np.ndarray, minus: float = 0.0) -> float:
    """RN(sum x_h y_h - minus), computed exactly and rounded once."""
    p, e = _two_prod(np.asarray(x, np.float64), np.asarray(y, np.float64))
    return math.fsum(np.concatenate([p, e, [-minus]]))


def sampled_errors(A_rows: np.ndarray, B_cols: np.ndarray, C_vals: np.ndarray) -> dict:
    """Errors of C_vals[s] against (A_rows[s] . B_cols[s]) for each sample s.

    Returns the literal relative error max |C - AB| / |AB| (AB != 0), the
    componentwise one max |C - AB| / (|A||B|), the normwise one
    max |C - AB| / max (|A||B|) over the sample, and the sample size.
    """
    err, ab, absab = [], [], []
    for x, y, c in zip(A_rows, B_cols, C_vals):
        err.append(abs(exact_dot(x, y, float(c))))
        ab.append(exact_dot(x, y))
        absab.append(exact_dot(np.abs(x), np.abs(y)))
    err, ab, absab = np.array(err), np.array(ab), np.array(absab)
    nz = ab != 0
    return dict(literal=float((err[nz] / np.abs(ab[nz])).max()) if nz.any() else 0.0,
                componentwise=float((err / np.where(absab > 0, absab, 1)).max()),
                normwise=float(err.max() / absab.max()) if absab.max() > 0 else 0.0,
                samples=int(len(err)))
