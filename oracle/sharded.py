"""Row-sharded Ozaki-II over the ranks of a torch.distributed process group:
Algorithms 1-3 split across devices, with the one exchange step they need.

TEST INFRASTRUCTURE ONLY: part of the CPU oracle.  Only the test suite may
import this module; it shares no code with the GPU library.

Rank r holds a block of consecutive rows of A and all of B, and computes the
same rows of C = OS_II(A, B) (Algorithm 1).  In Algorithm 2:
  * mu'_i, Abar(i, :) and max_h cbar_ih come from row i of A and all of Bbar,
    so mu_i is local to the rank that holds row i;
  * nu'_j and Bbar(:, j) come from column j of B (held by every rank), but
    nu_j needs max_h cbar_hj over ALL m rows, which the ranks hold in pieces.
The exchange is one all-reduce (MAX) of the n integer column maxima of Cbar.
With N chosen by the bound rule (the reading that takes the smallest N whose
N-dependent part of eq. thm:err-2 meets the target; see ozaki2.choose_N), the
rule also needs the maxima over all rows of |A| v and of 2^alpha', and the
per-k maxima over all rows of |A| (for L); they travel in the same buffer: one
all-reduce of n + k + 2 values.  After it, every rank has the unsharded call's
mu (its rows), nu and N, and Algorithm 3 and the inverse scaling are local, so
each rank's rows of C are bit-identical to the unsharded result.
"""
from __future__ import annotations

import numpy as np

from . import ozaki2 as oz
from .constants import constants


def all_reduce_max(buf: np.ndarray, group=None) -> np.ndarray:
    """Elementwise maximum over the ranks (exact for doubles; the integers here
    are below 2^53)."""
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(buf, dtype=np.float64))
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return t.numpy()


def os_ii_rows(A_rows: np.ndarray, B: np.ndarray, N: int = 0, b: int = 64, tau: float = 0.0,
               nmax: int = 20, group=None) -> dict:
    """This rank's rows of OS_II(A, B).  N > 0: fixed N; N == 0: the bound rule
    for target tau with N <= nmax.  Returns C (the rows), mu (the rows), nu, N."""
    A_rows = np.asarray(A_rows, np.float64)
    B = np.asarray(B, np.float64)
    mr, k = A_rows.shape
    n = B.shape[1]
    # Algorithm 2: mu', nu', Abar, Bbar (local; Bbar the same on every rank)
    alpha = oz.floor_log2_absmax(A_rows, axis=1)
    beta = oz.floor_log2_absmax(B, axis=0)
    mu_p = np.where(alpha == oz.INT32_MIN, 0, 5 - alpha.astype(np.int64)).astype(np.int32)
    nu_p = np.where(beta == oz.INT32_MIN, 0, 5 - beta.astype(np.int64)).astype(np.int32)
    Abar = np.empty((mr, k), dtype=np.int8)
    rs, cs = oz._strides(A_rows)
    oz.lib().oz2o_ceil_scaled_abs(mr, k, oz._p(A_rows), rs, cs, oz._p(mu_p), oz._p(Abar))
    BT = B.T
    BbarT = np.empty((n, k), dtype=np.int8)
    rs, cs = oz._strides(BT)
    oz.lib().oz2o_ceil_scaled_abs(n, k, oz._p(BT), rs, cs, oz._p(nu_p), oz._p(BbarT))
    Bbar = np.ascontiguousarray(BbarT.T)
    # Cbar = Abar Bbar for these rows; row maxima complete, column maxima partial
    Cbar = oz.gemm_i8(Abar, Bbar)
    cmax_row = Cbar.max(axis=1) if n else np.zeros(mr, np.int64)
    cmax_col_part = Cbar.max(axis=0) if mr else np.zeros(n, np.int64)
    # what the bound rule needs from all rows
    R = oz.abs_sums(A_rows, 1) if mr else np.zeros(0)
    a2 = oz.pow2_prime(alpha, cmax_row) if mr else np.zeros(0)
    colmaxA = np.abs(A_rows).max(axis=0) if mr else np.zeros(k)
    # the exchange: one all-reduce (MAX) of n + k + 2 values
    buf = np.concatenate([cmax_col_part.astype(np.float64), colmaxA,
                          [float(R.max(initial=0.0)), float(a2.max(initial=0.0))]])
    buf = all_reduce_max(buf, group)
    cmax_col = buf[:n].astype(np.int64)
    if N == 0:
        K = oz.abs_sums(B, 0)
        b2 = oz.pow2_prime(beta, cmax_col)
        L = float(np.max(buf[n:n + k] * np.abs(B).max(axis=1))) if n and k else 0.0
        N, _ = oz.choose_N_from_maxima(float(buf[n + k]), float(K.max(initial=0.0)), float(buf[n + k + 1]),
                                       float(b2.max(initial=0.0)), L, k, tau, nmax, b)
    C = constants(N, b)
    # Dbar = single_up(Cbar) and max commute (single_up is monotone); empty rows -> 1
    drow = oz.single_up(cmax_row)
    dcol = oz.single_up(cmax_col)
    drow = np.where(drow == 0, np.float32(1), drow)
    dcol = np.where(dcol == 0, np.float32(1), dcol)
    mu = (mu_p + oz.exponent_shift(C.c, oz.log2f(drow), C.Pprime)).astype(np.int32)
    nu = (nu_p + oz.exponent_shift(C.c, oz.log2f(dcol), C.Pprime)).astype(np.int32)
    # Algorithm 3 and the inverse scaling, local
    Ap = oz.trunc_scaled_rows(A_rows, mu)
    Bp = np.ascontiguousarray(oz.trunc_scaled_rows(B.T, nu).T)
    r = oz.crt(Ap, Bp, N, b)
    return dict(C=oz.unscale(r["Cpp"], mu, nu, b), mu=mu, nu=nu, N=N)
