"""Helpers shared by the GPU tests: run the library on device tensors with every
export switched on, and compare results with the oracle."""
import numpy as np

from paper_2602_02549_b300 import binding as B


def run_gpu(A: np.ndarray, Bm: np.ndarray, N: int = 0, *, fp32: bool = False, target: float = 0.0,
            nmax: int = 0, trans_a: bool = False, trans_b: bool = False, mu_in=None, nu_in=None,
            fast: bool = False):
    """Run the emulated GEMM on cuda:0; returns dict(C, mu, nu, N, W) as numpy.

    A and Bm are the arrays as stored (A^T / B^T when trans_a / trans_b).
    """
    import torch
    dt = torch.float32 if fp32 else torch.float64
    At = torch.tensor(A, dtype=dt, device="cuda")
    Bt = torch.tensor(Bm, dtype=dt, device="cuda")
    m = A.shape[1] if trans_a else A.shape[0]
    n = Bm.shape[0] if trans_b else Bm.shape[1]
    nplanes = N if N else (nmax if nmax else (14 if fp32 else 20))
    mu = torch.full((m,), -99999, dtype=torch.int32, device="cuda")
    nu = torch.full((n,), -99999, dtype=torch.int32, device="cuda")
    nout = torch.zeros(1, dtype=torch.int32, device="cuda")
    W = torch.zeros(nplanes * m * n, dtype=torch.int8, device="cuda")
    kw = dict(n_out=nout, w_out=W)
    if mu_in is not None:
        kw.update(mu_in=torch.tensor(mu_in, dtype=torch.int32, device="cuda"),
                  nu_in=torch.tensor(nu_in, dtype=torch.int32, device="cuda"))
    else:
        kw.update(mu_out=mu, nu_out=nu)
    C = B.matmul(At, Bt, N, target=target, nmax=nmax, trans_a=trans_a, trans_b=trans_b, fast=fast, **kw)
    torch.cuda.synchronize()
    assert B.sync() == 0
    Nused = int(nout.item())
    out = dict(C=C.cpu().numpy().astype(np.float64), N=Nused,
               W=W.cpu().numpy().reshape(nplanes, m, n)[:Nused])
    if mu_in is None:
        out.update(mu=mu.cpu().numpy(), nu=nu.cpu().numpy())
    else:
        out.update(mu=np.asarray(mu_in, np.int32), nu=np.asarray(nu_in, np.int32))
    return out


def ulp_distance(a: np.ndarray, b: np.ndarray, fp32: bool = False) -> np.ndarray:
    """Distance in units in the last place between same-shape float arrays
    (+0 and -0 coincide; distances across a sign change are approximate)."""
    if fp32:
        ia = np.asarray(a, np.float32).view(np.int32).astype(np.int64)
        ib = np.asarray(b, np.float32).view(np.int32).astype(np.int64)
        mask = np.int64(0x7FFFFFFF)
    else:
        ia = np.asarray(a, np.float64).view(np.int64)
        ib = np.asarray(b, np.float64).view(np.int64)
        mask = np.int64(0x7FFFFFFFFFFFFFFF)
    oa = np.where(ia >= 0, ia, -(ia & mask))
    ob = np.where(ib >= 0, ib, -(ib & mask))
    same = (oa >= 0) == (ob >= 0)
    near = np.abs(np.where(same, oa - ob, 0)).astype(np.float64)
    far = np.abs(oa.astype(np.float64)) + np.abs(ob.astype(np.float64))
    return np.where(same, near, far)
