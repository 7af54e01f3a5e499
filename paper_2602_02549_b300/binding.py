"""Python binding of liboz2.so (ctypes): argument marshalling only.

Every step of the emulated GEMM runs in the library's CUDA kernels; this module
turns torch tensors into device pointers, leading dimensions and a stream, and
allocates the workspace through PyTorch's caching allocator.  There is no CPU
fallback: without the built library (python -m paper_2602_02549_b300.build)
or without a CUDA device, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re

from .build import LIB

OZ2_OK, OZ2_EINVAL, OZ2_ERANGE, OZ2_ENOMEM, OZ2_ECUDA, OZ2_ETIMEOUT, OZ2_ENOTSUP = 0, -1, -2, -3, -4, -5, -6
OZ2_ACCURATE, OZ2_FAST, OZ2_TRANS_A, OZ2_TRANS_B = 0, 1, 2, 4
OZ2_CONJ_A, OZ2_CONJ_B = 8, 16
OZ2_COMPONENTWISE = 32
K_MAX, N_MIN, N_MAX = 131072, 2, 49
NPHASES = 7
PHASE_NAMES = ("stats", "quant", "scale_gemm", "exponents", "residues", "gemm", "crt")

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "oz2.h")


class Oz2Error(RuntimeError):
    def __init__(self, status: int, where: str):
        detail = ""
        if status == OZ2_ECUDA:
            line = ctypes.c_int()
            err = lib().oz2_last_error(ctypes.byref(line))
            detail = f" [CUDA error {err} caught at oz2_api.cu:{line.value}]"
        super().__init__(f"{where}: {status_str(status)} ({status}){detail}")
        self.status = status


class oz2_opts(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p),
                ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t),
                ("target", ctypes.c_double),
                ("nmax", ctypes.c_int),
                ("n_out", ctypes.c_void_p),
                ("mu_out", ctypes.c_void_p),
                ("nu_out", ctypes.c_void_p),
                ("mu_in", ctypes.c_void_p),
                ("nu_in", ctypes.c_void_p),
                ("w_out", ctypes.c_void_p),
                ("phase_events", ctypes.c_void_p)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load liboz2.so from the package directory (built in-tree)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing; build it with `python -m paper_2602_02549_b300.build`")
        L = ctypes.CDLL(LIB)
        i, P, sz = ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t
        gemm_args = [i, i, i, P, i, P, i, P, i, i, i]
        for name in ("oz2_gemm", "oz2_sgemm"):
            getattr(L, name).argtypes = gemm_args
            getattr(L, name).restype = i
        for name in ("oz2_gemm_ex", "oz2_sgemm_ex", "oz2_gemm_host", "oz2_sgemm_host"):
            getattr(L, name).argtypes = gemm_args + [ctypes.POINTER(oz2_opts)]
            getattr(L, name).restype = i
        for name in ("oz2_workspace_size", "oz2_host_workspace_size"):
            getattr(L, name).argtypes = [i, i, i, i, i, i]
            getattr(L, name).restype = sz
        L.oz2_k_ranges.argtypes = [i, P, P]
        L.oz2_k_ranges.restype = i
        for name in ("oz2_zgemm", "oz2_cgemm"):
            getattr(L, name).argtypes = gemm_args + [ctypes.POINTER(oz2_opts)]
            getattr(L, name).restype = i
        L.oz2_zworkspace_size.argtypes = [i, i, i, i, i, i]
        L.oz2_zworkspace_size.restype = sz
        L.oz2_sync.argtypes = [P]
        L.oz2_sync.restype = i
        L.oz2_tables.argtypes = [i, i, P, P, P, P]
        L.oz2_tables.restype = i
        L.oz2_check_log2f.argtypes = [P, P]
        L.oz2_check_log2f.restype = i
        L.oz2_status_str.argtypes = [i]
        L.oz2_status_str.restype = ctypes.c_char_p
        L.oz2_version.restype = i
        L.oz2_launch_count.argtypes = []
        L.oz2_launch_count.restype = ctypes.c_longlong
        L.oz2_last_error.argtypes = [P]
        L.oz2_last_error.restype = i
        L.oz2_batched_workspace_size.argtypes = [i, P]
        L.oz2_batched_workspace_size.restype = sz
        L.oz2_gemm_batched.argtypes = [i, P, ctypes.POINTER(oz2_opts)]
        L.oz2_gemm_batched.restype = i
        L.oz2_batched_autotune.argtypes = [i, P, ctypes.POINTER(oz2_opts), ctypes.POINTER(i), P]
        L.oz2_batched_autotune.restype = i
        L.oz2_batched_set_policy.argtypes = [i, P, i]
        L.oz2_batched_set_policy.restype = i
        _lib = L
    return _lib


def header_symbols() -> list[str]:
    """Names of the entry points declared in include/oz2.h."""
    text = open(HEADER).read()
    return re.findall(r"OZ2_API\s+[\w\s\*]+?\b(oz2_\w+)\s*\(", text)


def status_str(status: int) -> str:
    return lib().oz2_status_str(status).decode()


def workspace_size(m: int, n: int, k: int, nmax: int, mode: int = 0, fp32: bool = False) -> int:
    return int(lib().oz2_workspace_size(m, n, k, nmax, mode, int(fp32)))


def host_workspace_size(m: int, n: int, k: int, nmax: int, mode: int = 0, fp32: bool = False) -> int:
    """oz2_host_workspace_size: device bytes of an oz2_gemm_host / oz2_sgemm_host call."""
    return int(lib().oz2_host_workspace_size(m, n, k, nmax, mode, int(fp32)))


def k_ranges(k: int) -> tuple[int, int]:
    """(count, kc): the K ranges a call with this k runs (oz2_k_ranges)."""
    count, kc = ctypes.c_int(), ctypes.c_int()
    rc = lib().oz2_k_ranges(int(k), ctypes.addressof(count), ctypes.addressof(kc))
    if rc:
        raise Oz2Error(rc, "oz2_k_ranges")
    return count.value, kc.value


def tables(N: int, fp32: bool = False) -> dict:
    """The library's own constant tables for N moduli (host-only)."""
    import numpy as np
    s1 = np.zeros(N)
    s2 = np.zeros(N)
    scal = np.zeros(6)
    pp = ctypes.c_float()
    rc = lib().oz2_tables(N, int(fp32), s1.ctypes.data, s2.ctypes.data, scal.ctypes.data, ctypes.addressof(pp))
    if rc:
        raise Oz2Error(rc, "oz2_tables")
    return dict(s1=s1, s2=s2, P1=scal[0], P2=scal[1], Pinv=scal[2], g=scal[3], t=scal[4], gN=scal[5],
                Pprime=np.float32(pp.value))


def wait_selftest(limit_us: int = 20000, stream=None) -> int:
    """oz2_wait_selftest: a bounded device wait that expires on purpose."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    L = lib()
    L.oz2_wait_selftest.argtypes = [ctypes.c_void_p, ctypes.c_uint]
    L.oz2_wait_selftest.restype = ctypes.c_int
    return L.oz2_wait_selftest(ctypes.c_void_p(s.cuda_stream), int(limit_us))


def gemm_timeout_selftest(A, B, C, nmoduli: int, limit_us: int = 5000, *, workspace=None, stream=None) -> int:
    """oz2_gemm_timeout_selftest on float64 CUDA tensors: the emulated GEMM with
    the residue GEMM's loads of one stage left out, so that its bounded waits
    give up after limit_us (the next sync reports OZ2_ETIMEOUT).  Returns the status."""
    import torch
    m, k = A.shape
    n = B.size(1)
    o = oz2_opts()
    s = stream if stream is not None else torch.cuda.current_stream(A.device)
    o.stream = ctypes.c_void_p(s.cuda_stream)
    if workspace is None:
        workspace = torch.empty(workspace_size(m, n, k, nmoduli), dtype=torch.uint8, device=A.device)
    o.workspace = ctypes.c_void_p(workspace.data_ptr())
    o.workspace_bytes = workspace.numel()
    L = lib()
    L.oz2_gemm_timeout_selftest.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p, ctypes.c_int] * 3 + \
        [ctypes.c_int, ctypes.c_uint, ctypes.POINTER(oz2_opts)]
    L.oz2_gemm_timeout_selftest.restype = ctypes.c_int
    with torch.cuda.device(A.device):
        return L.oz2_gemm_timeout_selftest(m, n, k, _ptr(A), _ld(A, "A"), _ptr(B), _ld(B, "B"), _ptr(C),
                                           _ld(C, "C"), int(nmoduli), int(limit_us), ctypes.byref(o))


class oz2_exchange(ctypes.Structure):
    _fields_ = [("cmax_col", ctypes.c_void_p), ("n", ctypes.c_size_t), ("kmax", ctypes.c_void_p),
                ("k", ctypes.c_size_t), ("red", ctypes.c_void_p), ("nred", ctypes.c_size_t)]


def _rows_opts(A, stream, workspace, target, nmax, n_out, mu_out, nu_out):
    import torch
    o = oz2_opts()
    s = stream if stream is not None else torch.cuda.current_stream(A.device)
    o.stream = ctypes.c_void_p(s.cuda_stream)
    o.workspace = ctypes.c_void_p(workspace.data_ptr())
    o.workspace_bytes = workspace.numel()
    o.target = float(target)
    o.nmax = int(nmax)
    o.n_out, o.mu_out, o.nu_out = _ptr(n_out), _ptr(mu_out), _ptr(nu_out)
    return o


def _rows_dims(A, B, mode):
    ta, tb = bool(mode & OZ2_TRANS_A), bool(mode & OZ2_TRANS_B)
    m = A.size(1) if ta else A.size(0)
    k = A.size(0) if ta else A.size(1)
    n = B.size(0) if tb else B.size(1)
    return m, n, k


def gemm_rows_begin(A, B, nmoduli: int = 0, mode: int = 0, *, workspace, target: float = 0.0, nmax: int = 0,
                    stream=None):
    """oz2_gemm_rows_begin on float64 CUDA tensors (this rank's rows of A, all of
    B): returns the three exchange arrays as int32 / int64 tensors that view the
    workspace, to be replaced in place by their element-wise maximum over the
    ranks before gemm_rows_end.  Raises on a non-OK status."""
    import torch
    m, n, k = _rows_dims(A, B, mode)
    o = _rows_opts(A, stream, workspace, target, nmax, None, None, None)
    ex = oz2_exchange()
    L = lib()
    L.oz2_gemm_rows_begin.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p, ctypes.c_int] * 2 + \
        [ctypes.c_int, ctypes.c_int, ctypes.POINTER(oz2_opts), ctypes.POINTER(oz2_exchange)]
    L.oz2_gemm_rows_begin.restype = ctypes.c_int
    with torch.cuda.device(A.device):
        rc = L.oz2_gemm_rows_begin(m, n, k, _ptr(A), _ld(A, "A"), _ptr(B), _ld(B, "B"), int(nmoduli), int(mode),
                                   ctypes.byref(o), ctypes.byref(ex))
    if rc:
        raise Oz2Error(rc, "oz2_gemm_rows_begin")
    base = workspace.data_ptr()

    def view(ptr, count, dtype, size):
        off = ptr - base
        return workspace[off:off + count * size].view(dtype)
    return (view(ex.cmax_col, ex.n, torch.int32, 4), view(ex.kmax, ex.k, torch.int64, 8),
            view(ex.red, ex.nred, torch.int64, 8))


def gemm_rows_end(A, B, C, nmoduli: int = 0, mode: int = 0, *, workspace, target: float = 0.0, nmax: int = 0,
                  stream=None, n_out=None, mu_out=None, nu_out=None) -> int:
    """oz2_gemm_rows_end: this rank's rows of C once the exchange is done.
    Returns the status code."""
    import torch
    m, n, k = _rows_dims(A, B, mode)
    o = _rows_opts(A, stream, workspace, target, nmax, n_out, mu_out, nu_out)
    L = lib()
    L.oz2_gemm_rows_end.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p, ctypes.c_int] * 3 + \
        [ctypes.c_int, ctypes.c_int, ctypes.POINTER(oz2_opts)]
    L.oz2_gemm_rows_end.restype = ctypes.c_int
    with torch.cuda.device(A.device):
        return L.oz2_gemm_rows_end(m, n, k, _ptr(A), _ld(A, "A"), _ptr(B), _ld(B, "B"), _ptr(C), _ld(C, "C"),
                                   int(nmoduli), int(mode), ctypes.byref(o))


def exchange_max(arrays, group=None) -> None:
    """The exchange of a row-sharded call: every array replaced, in place, by
    its element-wise maximum over the ranks of `group` (torch.distributed; NCCL
    on CUDA tensors, gloo on CPU tensors)."""
    import torch.distributed as dist
    for t in arrays:
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)


def matmul_rows(A_rows, B, nmoduli: int = 0, *, target: float = 1e-15, nmax: int = 0, trans_a: bool = False,
                trans_b: bool = False, group=None, out=None, n_out=None):
    """This rank's rows of A @ B when the rows of A are split over the ranks of
    `group` (B whole on every rank): begin, the exchange, end; bit-identical to
    the same rows of the unsharded matmul."""
    import torch
    mode = (OZ2_TRANS_A if trans_a else 0) | (OZ2_TRANS_B if trans_b else 0)
    m, n, k = _rows_dims(A_rows, B, mode)
    nm = nmoduli if nmoduli else (nmax if nmax else 20)
    ws = torch.empty(workspace_size(m, n, k, nm, mode, False), dtype=torch.uint8, device=A_rows.device)
    tgt = target if nmoduli == 0 else 0.0
    arrays = gemm_rows_begin(A_rows, B, nmoduli, mode, workspace=ws, target=tgt, nmax=nmax)
    exchange_max(arrays, group)
    C = out if out is not None else torch.empty((m, n), dtype=torch.float64, device=A_rows.device)
    rc = gemm_rows_end(A_rows, B, C, nmoduli, mode, workspace=ws, target=tgt, nmax=nmax, n_out=n_out)
    if rc:
        raise Oz2Error(rc, "oz2_gemm_rows_end")
    return C


def sum_tables(N: int, fp32: bool = False) -> tuple:
    """The CRT-sum constants as the device holds them: (list of k_l, esum) with
    s_l2 (DGEMM) or s_l1 (SGEMM) = k_l 2^esum (host-only)."""
    k = (ctypes.c_int * (2 * N))()
    e = ctypes.c_int()
    rc = lib().oz2_sum_tables(N, int(fp32), k, ctypes.byref(e))
    if rc:
        raise Oz2Error(rc, "oz2_sum_tables")
    return [k[2 * l + 1] * (1 << 31) + k[2 * l] for l in range(N)], e.value


# --------------------------------------------------------------------------- #
# torch-facing calls
# --------------------------------------------------------------------------- #
def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _ld(t, name):
    if t.dim() != 2:
        raise ValueError(f"{name} must be 2-D")
    if t.stride(1) != 1 and t.size(1) > 1:
        raise ValueError(f"{name} must have unit column stride (row-major)")
    return max(t.stride(0), t.size(1), 1)


def gemm_ex(A, B, C, nmoduli: int = 0, mode: int = 0, *, target: float = 0.0, nmax: int = 0,
            workspace=None, stream=None, n_out=None, mu_out=None, nu_out=None,
            mu_in=None, nu_in=None, w_out=None, phase_events=None) -> int:
    """oz2_gemm_ex / oz2_sgemm_ex on torch CUDA tensors; returns the status code.

    A is m x k (or k x m with OZ2_TRANS_A), B is k x n (or n x k with
    OZ2_TRANS_B), C is m x n; float64 calls oz2_gemm_ex, float32 oz2_sgemm_ex.
    """
    import torch
    fp32 = A.dtype == torch.float32
    if A.dtype not in (torch.float32, torch.float64) or B.dtype != A.dtype or C.dtype != A.dtype:
        raise TypeError("A, B, C must all be float64 or all float32")
    for t, nm in ((A, "A"), (B, "B"), (C, "C")):
        if not t.is_cuda:
            raise ValueError(f"{nm} must be a CUDA tensor (no CPU path)")
    ta, tb = bool(mode & OZ2_TRANS_A), bool(mode & OZ2_TRANS_B)
    m = A.size(1) if ta else A.size(0)
    k = A.size(0) if ta else A.size(1)
    n = B.size(0) if tb else B.size(1)
    kb = B.size(1) if tb else B.size(0)
    if kb != k or tuple(C.shape) != (m, n):
        raise ValueError("shape mismatch")
    o = oz2_opts()
    s = stream if stream is not None else torch.cuda.current_stream(A.device)
    o.stream = ctypes.c_void_p(s.cuda_stream)
    n_eff = nmoduli if nmoduli else (nmax if nmax else (14 if fp32 else 20))
    if workspace is None and m > 0 and n > 0 and k > 0 and n_eff >= 2:
        size = workspace_size(m, n, k, n_eff, mode, fp32)
        if size:
            workspace = torch.empty(size, dtype=torch.uint8, device=A.device)
    if workspace is not None:
        o.workspace = ctypes.c_void_p(workspace.data_ptr())
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    o.target = float(target)
    o.nmax = int(nmax)
    o.n_out, o.mu_out, o.nu_out = _ptr(n_out), _ptr(mu_out), _ptr(nu_out)
    o.mu_in, o.nu_in, o.w_out = _ptr(mu_in), _ptr(nu_in), _ptr(w_out)
    arr = None
    if phase_events is not None:
        # torch.cuda.Event handles, NPHASES + 1 of them, created with timing enabled;
        # torch creates the CUDA event lazily at its first record
        for e in phase_events:
            if not e.cuda_event:
                e.record(s)
        arr = (ctypes.c_void_p * (NPHASES + 1))(*[ctypes.c_void_p(e.cuda_event) for e in phase_events])
        o.phase_events = ctypes.cast(arr, ctypes.c_void_p)
    fn = lib().oz2_sgemm_ex if fp32 else lib().oz2_gemm_ex
    with torch.cuda.device(A.device):
        return fn(m, n, k, _ptr(A), _ld(A, "A"), _ptr(B), _ld(B, "B"), _ptr(C), _ld(C, "C"),
                  nmoduli, mode, ctypes.byref(o))


def gemm_host(A, B, C, nmoduli: int = 0, mode: int = 0, *, target: float = 0.0, nmax: int = 0,
              workspace=None, stream=None, n_out=None, device=None) -> int:
    """oz2_gemm_host / oz2_sgemm_host on torch CPU tensors (pinned or pageable):
    the library copies A and B to the device, runs the emulation on `stream`
    and copies C back.  Shapes as in gemm_ex; `workspace` is a CUDA uint8
    tensor of >= host_workspace_size bytes (allocated here when omitted).
    With pinned tensors C is valid once the stream has completed.  Returns the
    status code."""
    import torch
    fp32 = A.dtype == torch.float32
    if A.dtype not in (torch.float32, torch.float64) or B.dtype != A.dtype or C.dtype != A.dtype:
        raise TypeError("A, B, C must all be float64 or all float32")
    for t, nm in ((A, "A"), (B, "B"), (C, "C")):
        if t.is_cuda:
            raise ValueError(f"{nm} must be a host (CPU) tensor; gemm_ex takes device tensors")
    ta, tb = bool(mode & OZ2_TRANS_A), bool(mode & OZ2_TRANS_B)
    m = A.size(1) if ta else A.size(0)
    k = A.size(0) if ta else A.size(1)
    n = B.size(0) if tb else B.size(1)
    kb = B.size(1) if tb else B.size(0)
    if kb != k or tuple(C.shape) != (m, n):
        raise ValueError("shape mismatch")
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    o = oz2_opts()
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    o.stream = ctypes.c_void_p(s.cuda_stream)
    n_eff = nmoduli if nmoduli else (nmax if nmax else (14 if fp32 else 20))
    if workspace is None and m > 0 and n > 0 and k > 0 and n_eff >= 2:
        size = host_workspace_size(m, n, k, n_eff, mode, fp32)
        if size:
            workspace = torch.empty(size, dtype=torch.uint8, device=dev)
    if workspace is not None:
        o.workspace = ctypes.c_void_p(workspace.data_ptr())
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    o.target = float(target)
    o.nmax = int(nmax)
    o.n_out = _ptr(n_out)
    fn = lib().oz2_sgemm_host if fp32 else lib().oz2_gemm_host
    with torch.cuda.device(dev):
        return fn(m, n, k, _ptr(A), _ld(A, "A"), _ptr(B), _ld(B, "B"), _ptr(C), _ld(C, "C"),
                  nmoduli, mode, ctypes.byref(o))


def matmul(A, B, nmoduli: int = 0, *, target: float = 1e-15, nmax: int = 0, trans_a: bool = False,
           trans_b: bool = False, fast: bool = False, componentwise: bool = False, out=None, **kw):
    """C = A @ B through the Ozaki-II emulation (raises on any non-OK status)."""
    import torch
    m = A.size(1) if trans_a else A.size(0)
    n = B.size(0) if trans_b else B.size(1)
    C = out if out is not None else torch.empty((m, n), dtype=A.dtype, device=A.device)
    mode = (OZ2_FAST if fast else 0) | (OZ2_TRANS_A if trans_a else 0) | (OZ2_TRANS_B if trans_b else 0) | \
        (OZ2_COMPONENTWISE if componentwise else 0)
    rc = gemm_ex(A, B, C, nmoduli, mode, target=target if nmoduli == 0 else 0.0, nmax=nmax, **kw)
    if rc:
        raise Oz2Error(rc, "oz2 gemm")
    return C


def zworkspace_size(m: int, n: int, k: int, nmax: int, mode: int = 0, fp32: bool = False) -> int:
    return int(lib().oz2_zworkspace_size(m, n, k, nmax, mode, int(fp32)))


def zgemm_ex(A, B, C, nmoduli: int = 0, mode: int = 0, *, target: float = 0.0, nmax: int = 0,
             workspace=None, stream=None, n_out=None, mu_out=None, nu_out=None, mu_in=None, nu_in=None) -> int:
    """oz2_zgemm / oz2_cgemm on torch complex CUDA tensors (complex128 / complex64,
    unit column stride); shapes as in gemm_ex.  Returns the status code."""
    import torch
    if A.dtype not in (torch.complex64, torch.complex128) or B.dtype != A.dtype or C.dtype != A.dtype:
        raise TypeError("A, B, C must all be complex128 or all complex64")
    fp32 = A.dtype == torch.complex64
    for t, nm in ((A, "A"), (B, "B"), (C, "C")):
        if not t.is_cuda:
            raise ValueError(f"{nm} must be a CUDA tensor (no CPU path)")
    ta, tb = bool(mode & OZ2_TRANS_A), bool(mode & OZ2_TRANS_B)
    m = A.size(1) if ta else A.size(0)
    k = A.size(0) if ta else A.size(1)
    n = B.size(0) if tb else B.size(1)
    kb = B.size(1) if tb else B.size(0)
    if kb != k or tuple(C.shape) != (m, n):
        raise ValueError("shape mismatch")
    o = oz2_opts()
    s = stream if stream is not None else torch.cuda.current_stream(A.device)
    o.stream = ctypes.c_void_p(s.cuda_stream)
    n_eff = nmoduli if nmoduli else (nmax if nmax else (14 if fp32 else 20))
    if workspace is None and n_eff >= 2:
        size = zworkspace_size(m, n, k, n_eff, mode, fp32)
        if size:
            workspace = torch.empty(size, dtype=torch.uint8, device=A.device)
    if workspace is not None:
        o.workspace = ctypes.c_void_p(workspace.data_ptr())
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    o.target = float(target)
    o.nmax = int(nmax)
    o.n_out, o.mu_out, o.nu_out = _ptr(n_out), _ptr(mu_out), _ptr(nu_out)
    o.mu_in, o.nu_in = _ptr(mu_in), _ptr(nu_in)
    fn = lib().oz2_cgemm if fp32 else lib().oz2_zgemm
    with torch.cuda.device(A.device):
        return fn(m, n, k, _ptr(A), _ld(A, "A"), _ptr(B), _ld(B, "B"), _ptr(C), _ld(C, "C"),
                  nmoduli, mode, ctypes.byref(o))


def zmatmul(A, B, nmoduli: int = 0, *, target: float = 1e-15, nmax: int = 0, trans_a: bool = False,
            trans_b: bool = False, conj_a: bool = False, conj_b: bool = False, fast: bool = False, out=None, **kw):
    """C = op(A) @ op(B) for complex tensors through the emulation (raises on any
    non-OK status); op = transpose and/or conjugate as requested."""
    import torch
    m = A.size(1) if trans_a else A.size(0)
    n = B.size(0) if trans_b else B.size(1)
    C = out if out is not None else torch.empty((m, n), dtype=A.dtype, device=A.device)
    mode = ((OZ2_FAST if fast else 0) | (OZ2_TRANS_A if trans_a else 0) | (OZ2_TRANS_B if trans_b else 0) |
            (OZ2_CONJ_A if conj_a else 0) | (OZ2_CONJ_B if conj_b else 0))
    rc = zgemm_ex(A, B, C, nmoduli, mode, target=target if nmoduli == 0 else 0.0, nmax=nmax, **kw)
    if rc:
        raise Oz2Error(rc, "oz2 complex gemm")
    return C


def launch_count() -> int:
    """Kernels the library has launched in this process so far (oz2_launch_count)."""
    return int(lib().oz2_launch_count())


def sync(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return lib().oz2_sync(ctypes.c_void_p(s.cuda_stream))


def check_log2f(stream=None):
    """Run the assumption-(1) diagnostic; returns (violations, max ratio)."""
    import struct
    import torch
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = lib().oz2_check_log2f(ctypes.c_void_p(s.cuda_stream), ctypes.c_void_p(out.data_ptr()))
    if rc:
        raise Oz2Error(rc, "oz2_check_log2f")
    s.synchronize()
    v = out.cpu().tolist()
    ratio = struct.unpack("<d", struct.pack("<q", v[1]))[0]
    return v[0], ratio


def gemm_noalloc(A, B, C, nmoduli: int = 0, mode: int = 0, *, target: float = 0.0, stream=None) -> int:
    """oz2_gemm_noalloc on float64 torch CUDA tensors (no workspace is passed or
    allocated; the library's fixed device scratch is used).  Returns the status."""
    import torch
    L = lib()
    fn = L.oz2_gemm_noalloc
    fn.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p, ctypes.c_int] * 3 + \
        [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    ta, tb = bool(mode & OZ2_TRANS_A), bool(mode & OZ2_TRANS_B)
    m = A.size(1) if ta else A.size(0)
    k = A.size(0) if ta else A.size(1)
    n = B.size(0) if tb else B.size(1)
    s = stream if stream is not None else torch.cuda.current_stream(A.device)
    with torch.cuda.device(A.device):
        return fn(m, n, k, _ptr(A), _ld(A, "A"), _ptr(B), _ld(B, "B"), _ptr(C), _ld(C, "C"),
                  nmoduli, mode, float(target), ctypes.c_void_p(s.cuda_stream))


class oz2_problem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("n", ctypes.c_int), ("k", ctypes.c_int),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_int),
                ("C", ctypes.c_void_p), ("ldc", ctypes.c_int),
                ("nmoduli", ctypes.c_int), ("target", ctypes.c_double), ("nmax", ctypes.c_int),
                ("mode", ctypes.c_int), ("n_out", ctypes.c_void_p)]


def _problem_array(problems):
    arr = (oz2_problem * len(problems))()
    for q, d in zip(arr, problems):
        A, Bm, C = d["A"], d["B"], d["C"]
        for t in (A, Bm, C):
            if t.dtype.itemsize != 8 or not t.is_cuda:
                raise TypeError("batched problems are float64 CUDA tensors")
        mode = (OZ2_FAST if d.get("fast") else 0) | (OZ2_TRANS_A if d.get("trans_a") else 0) | \
            (OZ2_TRANS_B if d.get("trans_b") else 0) | (OZ2_COMPONENTWISE if d.get("componentwise") else 0)
        q.m = A.size(1) if d.get("trans_a") else A.size(0)
        q.k = A.size(0) if d.get("trans_a") else A.size(1)
        q.n = Bm.size(0) if d.get("trans_b") else Bm.size(1)
        q.A, q.lda = A.data_ptr(), _ld(A, "A")
        q.B, q.ldb = Bm.data_ptr(), _ld(Bm, "B")
        q.C, q.ldc = C.data_ptr(), _ld(C, "C")
        q.nmoduli = int(d.get("nmoduli", 0))
        q.target = float(d.get("target", 0.0))
        q.nmax = int(d.get("nmax", 0))
        q.mode = mode
        q.n_out = d["n_out"].data_ptr() if d.get("n_out") is not None else None
    return arr


def batched_workspace_size(problems) -> int:
    L = lib()
    arr = _problem_array(problems)
    return int(L.oz2_batched_workspace_size(len(problems), ctypes.cast(arr, ctypes.c_void_p)))


def gemm_batched(problems, *, workspace=None, stream=None, phase_events=None) -> int:
    """oz2_gemm_batched on a list of problems, each a dict with float64 CUDA
    tensors A, B, C and optional nmoduli, target, nmax, trans_a, trans_b, fast,
    n_out (device int32[1]).  Returns the status code."""
    import torch
    L = lib()
    arr = _problem_array(problems)
    o = oz2_opts()
    dev = problems[0]["A"].device
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    o.stream = ctypes.c_void_p(s.cuda_stream)
    if workspace is None:
        size = int(L.oz2_batched_workspace_size(len(problems), ctypes.cast(arr, ctypes.c_void_p)))
        workspace = torch.empty(max(size, 256), dtype=torch.uint8, device=dev)
    o.workspace = ctypes.c_void_p(workspace.data_ptr())
    o.workspace_bytes = workspace.numel()
    ev = None
    if phase_events is not None:
        for e in phase_events:
            if not e.cuda_event:
                e.record(s)
        ev = (ctypes.c_void_p * (NPHASES + 1))(*[ctypes.c_void_p(e.cuda_event) for e in phase_events])
        o.phase_events = ctypes.cast(ev, ctypes.c_void_p)
    with torch.cuda.device(dev):
        return L.oz2_gemm_batched(len(problems), ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(o))


def batched_autotune(problems, *, workspace=None, stream=None):
    """oz2_batched_autotune: times the tile policies on this batch and keeps the
    fastest for later gemm_batched calls.  Returns (policy, [ms per policy])."""
    import torch
    L = lib()
    arr = _problem_array(problems)
    o = oz2_opts()
    dev = problems[0]["A"].device
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    o.stream = ctypes.c_void_p(s.cuda_stream)
    if workspace is None:
        workspace = torch.empty(max(batched_workspace_size(problems), 256), dtype=torch.uint8, device=dev)
    o.workspace = ctypes.c_void_p(workspace.data_ptr())
    o.workspace_bytes = workspace.numel()
    pol = ctypes.c_int(-1)
    ms = (ctypes.c_float * 4)()
    with torch.cuda.device(dev):
        rc = L.oz2_batched_autotune(len(problems), ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(o),
                                    ctypes.byref(pol), ctypes.cast(ms, ctypes.c_void_p))
    if rc:
        raise Oz2Error(rc, "oz2_batched_autotune")
    return pol.value, [float(x) for x in ms]


def batched_set_policy(problems, policy: int) -> int:
    """oz2_batched_set_policy: keep tile policy 0, 1 or 2 for this batch's shapes."""
    import torch
    L = lib()
    arr = _problem_array(problems)
    with torch.cuda.device(problems[0]["A"].device):
        return L.oz2_batched_set_policy(len(problems), ctypes.cast(arr, ctypes.c_void_p), int(policy))

