"""Seeded synthetic inputs shaped like the paper's test matrices.

This module holds none of the Ozaki-II arithmetic; it only draws matrices, and
both the GPU path (tests, bench) and the CPU oracle take their inputs from it.

Section 5 (Discussion) generates each entry as
    a_ij, b_ij = (rand - 0.5) * exp(randn * phi),
rand uniform in (0, 1], randn standard normal; phi sets the exponent spread.
Here rand = 1 - U[0, 1) and both draws come from NumPy's PCG64 (host) or a
seeded torch generator (device).  FP32 matrices are drawn in FP64 and rounded.
"""
from __future__ import annotations

import numpy as np


def paper_matrix(rows: int, cols: int, phi: float, seed: int, dtype=np.float64) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    u = 1.0 - rng.random((rows, cols))          # (0, 1]
    z = rng.standard_normal((rows, cols))
    a = (u - 0.5) * np.exp(phi * z)
    return a.astype(dtype)


def paper_pair(m: int, n: int, k: int, phi: float, seed: int = 0, dtype=np.float64):
    """A (m x k) with seed `seed`, B (k x n) with seed `seed + 1`."""
    return paper_matrix(m, k, phi, seed, dtype), paper_matrix(k, n, phi, seed + 1, dtype)


def paper_matrix_torch(rows: int, cols: int, phi: float, seed: int, device, dtype=None):
    """The same recipe drawn on a torch device with a seeded torch.Generator."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    u = 1.0 - torch.rand((rows, cols), generator=g, device=device, dtype=torch.float64)
    z = torch.randn((rows, cols), generator=g, device=device, dtype=torch.float64)
    a = (u - 0.5) * torch.exp(phi * z)
    return a if dtype is None else a.to(dtype)


def integer_matrix(rows: int, cols: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Integer-valued FP64 matrix with entries uniform in [lo, hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(lo, hi + 1, size=(rows, cols)).astype(np.float64)


def wide_exponent_matrix(rows: int, cols: int, emin: int, emax: int, seed: int,
                         zero_frac: float = 0.0) -> np.ndarray:
    """Entries +-m * 2^e with m uniform in [1, 2) and e uniform in [emin, emax].

    Covers subnormal (emin < -1022) and huge (emax near 1023) magnitudes.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    m = 1.0 + rng.random((rows, cols))
    e = rng.integers(emin, emax + 1, size=(rows, cols))
    s = np.where(rng.random((rows, cols)) < 0.5, -1.0, 1.0)
    a = s * np.ldexp(m, e)
    if zero_frac > 0:
        a[rng.random((rows, cols)) < zero_frac] = 0.0
    return a


def batched_specs(count: int = 64, seed: int = 0, lo: int = 128, hi: int = 4096):
    """Uneven batch: m, n, k = round(exp(U(ln lo, ln hi))) and phi ~ U(0.5, 4) per problem."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dims = np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=(count, 3)))).astype(int)
    phis = rng.uniform(0.5, 4.0, size=count)
    return [(int(m), int(n), int(k), float(p)) for (m, n, k), p in zip(dims, phis)]
