"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/oz2.h declares, rejects bad arguments before touching
CUDA, sizes its workspace, and its independently generated constant tables
equal the oracle's exact ones."""
import ctypes
import subprocess

import numpy as np
import pytest

from oracle.constants import bound_terms, constants
from paper_2602_02549_b300 import binding as B
from paper_2602_02549_b300.build import LIB, build


@pytest.fixture(scope="module")
def lib():
    build()
    return B.lib()


def test_exports_every_declared_symbol(lib):
    names = B.header_symbols()
    assert {"oz2_gemm", "oz2_gemm_ex", "oz2_sgemm", "oz2_sgemm_ex", "oz2_workspace_size", "oz2_sync",
            "oz2_tables", "oz2_status_str", "oz2_version", "oz2_check_log2f"} <= set(names)
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    for n in names:
        assert n in exported, n
        assert hasattr(lib, n)


def test_version_and_status(lib):
    assert lib.oz2_version() >= 100
    assert B.status_str(0) == "OZ2_OK"
    assert "2^17" in B.status_str(B.OZ2_ERANGE)


FAKE = ctypes.c_void_p(0x10000)   # never dereferenced: validation fails first


def call(lib, m=8, n=8, k=8, lda=8, ldb=8, ldc=8, N=14, mode=0, opts=None, A=FAKE, Bp=FAKE, C=FAKE, fp32=False):
    fn = lib.oz2_sgemm_ex if fp32 else lib.oz2_gemm_ex
    return fn(m, n, k, A, lda, Bp, ldb, C, ldc, N, mode, ctypes.byref(opts) if opts else None)


@pytest.mark.parametrize("fp32", [False, True])
def test_argument_validation(lib, fp32):
    E = B.OZ2_EINVAL
    assert call(lib, m=0, fp32=fp32) == E
    assert call(lib, n=-1, fp32=fp32) == E
    assert call(lib, k=0, fp32=fp32) == E
    assert call(lib, lda=7, fp32=fp32) == E
    assert call(lib, ldb=7, fp32=fp32) == E
    assert call(lib, ldc=7, fp32=fp32) == E
    assert call(lib, N=1, fp32=fp32) == E
    assert call(lib, N=50, fp32=fp32) == E
    assert call(lib, mode=8, fp32=fp32) == E
    assert call(lib, A=None, fp32=fp32) == E
    assert call(lib, C=None, fp32=fp32) == E
    # k > 2^17 runs as split-K, which exports no W_l and records no phase events
    K1 = (1 << 17) + 1
    o = B.oz2_opts()
    o.w_out = FAKE
    assert call(lib, k=K1, lda=K1, opts=o, fp32=fp32) == B.OZ2_ENOTSUP
    o = B.oz2_opts()
    o.phase_events = FAKE
    assert call(lib, k=K1, lda=K1, opts=o, fp32=fp32) == B.OZ2_ENOTSUP
    # transposed leading dimensions: A^T is k x m, B^T is n x k
    assert call(lib, m=16, k=8, lda=8, mode=B.OZ2_TRANS_A, ldc=8, fp32=fp32) == E
    assert call(lib, n=16, k=8, ldb=4, ldc=16, mode=B.OZ2_TRANS_B, fp32=fp32) == E
    # N = 0 needs a positive target
    assert call(lib, N=0, fp32=fp32) == E
    o = B.oz2_opts()
    o.target = 0.0
    assert call(lib, N=0, opts=o, fp32=fp32) == E
    o.target, o.nmax = 1e-15, 50
    assert call(lib, N=0, opts=o, fp32=fp32) == E
    # injected exponents: both or neither, and a fixed N
    o = B.oz2_opts()
    o.mu_in = ctypes.c_void_p(0x1000)
    assert call(lib, opts=o, fp32=fp32) == E
    o.nu_in = ctypes.c_void_p(0x2000)
    o.target = 1e-15
    assert call(lib, N=0, opts=o, fp32=fp32) == E


def test_argument_errors_launch_nothing(lib):
    """Argument errors come back before any launch: the library's own kernel
    count does not move."""
    before = B.launch_count()
    assert call(lib, m=0) == B.OZ2_EINVAL
    assert call(lib, ldc=7, fp32=True) == B.OZ2_EINVAL
    assert call(lib, N=50) == B.OZ2_EINVAL
    assert B.launch_count() == before


@pytest.mark.parametrize("fp32", [False, True])
def test_host_arrays_argument_errors(lib, fp32):
    """oz2_gemm_host / oz2_sgemm_host check their arguments as oz2_gemm_ex does,
    before any copy or launch."""
    fn = lib.oz2_sgemm_host if fp32 else lib.oz2_gemm_host
    E = B.OZ2_EINVAL
    before = B.launch_count()

    def host(m=8, n=8, k=8, lda=8, ldb=8, ldc=8, N=14, mode=0, A=FAKE, Bp=FAKE, C=FAKE):
        return fn(m, n, k, A, lda, Bp, ldb, C, ldc, N, mode, None)
    assert host(m=0) == E
    assert host(k=-3) == E
    assert host(lda=7) == E
    assert host(ldb=4, mode=B.OZ2_TRANS_B) == E
    assert host(ldc=7) == E
    assert host(N=50) == E
    assert host(N=0) == E                      # the bound rule needs opts with a target
    assert host(A=None) == E
    assert host(mode=8) == E
    # k beyond 2^17 with per-call exports: refused before any upload
    o = B.oz2_opts()
    o.w_out = ctypes.c_void_p(0x10000)
    K1 = (1 << 17) + 1
    assert fn(8, 8, K1, FAKE, K1, FAKE, 8, FAKE, 8, 14, 0, ctypes.byref(o)) == B.OZ2_ENOTSUP
    assert B.launch_count() == before


def test_host_workspace_size(lib):
    """The device copies of A, B, C (each rounded up to 256 bytes) ahead of the
    emulation's own workspace."""
    r = lambda b: (b + 255) // 256 * 256   # noqa: E731
    for m, n, k, N, fp32 in ((8, 8, 8, 14, False), (100, 37, 1001, 20, False), (33, 65, 17, 9, True),
                             (5, 7, (1 << 17) + 1, 14, False)):
        e = 4 if fp32 else 8
        want = r(e * m * k) + r(e * k * n) + r(e * m * n) + B.workspace_size(m, n, k, N, 0, fp32)
        assert B.host_workspace_size(m, n, k, N, 0, fp32) == want
    assert B.host_workspace_size(0, 8, 8, 14) == 0
    assert B.host_workspace_size(8, 8, 8, 1) == 0


def test_workspace_size(lib):
    assert B.workspace_size(0, 8, 8, 14) == 0
    # k > 2^17: the ranges share one workspace sized for the longest range
    count, kc = B.k_ranges((1 << 17) + 1)
    assert (count, kc) == (2, 65600)
    assert B.workspace_size(8, 8, (1 << 17) + 1, 14) == B.workspace_size(8, 8, kc, 14) > 0
    assert B.workspace_size(8, 8, 8, 1) == 0
    a = B.workspace_size(100, 100, 100, 14)
    b = B.workspace_size(100, 100, 100, 20)
    c = B.workspace_size(1000, 1000, 1000, 20)
    assert 0 < a < b < c
    # dominated by N BF16 residue planes of the padded operands and N INT8 W planes
    m_pad, n_pad, k_pad = 1024, 1024, 1024
    assert c >= 20 * (2 * (m_pad + n_pad) * k_pad + m_pad * n_pad)


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("N", list(range(2, 50)))
def test_tables_match_oracle(lib, N, fp32):
    t = B.tables(N, fp32)
    C = constants(N, 32 if fp32 else 64)
    assert np.array_equal(t["s1"], np.array(C.s1))
    assert np.array_equal(t["s2"], np.array(C.s2))
    assert t["P1"] == C.P1 and t["P2"] == C.P2 and t["Pinv"] == C.Pinv
    assert t["Pprime"] == C.Pprime
    if not fp32:
        assert t["g"] == float(C.g)
    bt = bound_terms(N, 32 if fp32 else 64)
    assert abs(t["t"] / bt["t"] - 1) < 1e-12
    assert abs(t["gN"] / bt["gN"] - 1) < 1e-10


@pytest.mark.parametrize("fp32", [False, True])
def test_sum_tables_exact(lib, fp32):
    # the integer form of the CRT-sum constants reproduces the oracle's doubles
    # exactly, with every integer below 2^62 (the device sums cannot overflow)
    from fractions import Fraction
    for N in range(2, 50):
        k, e = B.sum_tables(N, fp32)
        C = constants(N, 32 if fp32 else 64)
        target = C.s1 if fp32 else C.s2
        for kl, sl in zip(k, target):
            assert 0 <= kl < 1 << 62
            assert Fraction(kl) * Fraction(2) ** e == Fraction(sl)
        assert -1022 <= e and e + 80 <= 1023
    with pytest.raises(B.Oz2Error):
        B.sum_tables(1)


def test_batched_validation_and_workspace(lib):
    P = B.oz2_problem
    good = P(m=8, n=8, k=8, A=0x10000, lda=8, B=0x10000, ldb=8, C=0x10000, ldc=8, nmoduli=14, target=0.0,
             nmax=0, mode=0, n_out=None)
    bad = P(m=8, n=8, k=8, A=0x10000, lda=7, B=0x10000, ldb=8, C=0x10000, ldc=8, nmoduli=14, target=0.0,
            nmax=0, mode=0, n_out=None)
    lib.oz2_gemm_batched.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.oz2_gemm_batched.restype = ctypes.c_int
    lib.oz2_batched_workspace_size.argtypes = [ctypes.c_int, ctypes.c_void_p]
    lib.oz2_batched_workspace_size.restype = ctypes.c_size_t
    arr = (P * 2)(good, bad)
    assert lib.oz2_gemm_batched(2, ctypes.cast(arr, ctypes.c_void_p), None) == B.OZ2_EINVAL
    assert lib.oz2_gemm_batched(-1, None, None) == B.OZ2_EINVAL
    assert lib.oz2_gemm_batched(0, None, None) == 0
    one = (P * 1)(good)
    two = (P * 2)(good, good)
    w1 = lib.oz2_batched_workspace_size(1, ctypes.cast(one, ctypes.c_void_p))
    w2 = lib.oz2_batched_workspace_size(2, ctypes.cast(two, ctypes.c_void_p))
    assert w1 >= B.workspace_size(8, 8, 8, 14) and w2 == 2 * w1


def test_batched_keeps_the_k_limit(lib):
    # split-K is for single calls; a batched problem with k > 2^17 is refused
    P = B.oz2_problem
    K1 = (1 << 17) + 1
    big = P(m=8, n=8, k=K1, A=0x10000, lda=K1, B=0x10000, ldb=8, C=0x10000, ldc=8, nmoduli=14, target=0.0,
            nmax=0, mode=0, n_out=None)
    lib.oz2_gemm_batched.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.oz2_gemm_batched.restype = ctypes.c_int
    lib.oz2_batched_workspace_size.argtypes = [ctypes.c_int, ctypes.c_void_p]
    lib.oz2_batched_workspace_size.restype = ctypes.c_size_t
    arr = (P * 1)(big)
    assert lib.oz2_gemm_batched(1, ctypes.cast(arr, ctypes.c_void_p), None) == B.OZ2_ERANGE
    assert lib.oz2_batched_workspace_size(1, ctypes.cast(arr, ctypes.c_void_p)) == 0


def test_rows_argument_validation(lib):
    # the row-sharded calls reject what they cannot carry before touching CUDA
    lib.oz2_gemm_rows_begin.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p, ctypes.c_int] * 2 + \
        [ctypes.c_int, ctypes.c_int, ctypes.POINTER(B.oz2_opts), ctypes.POINTER(B.oz2_exchange)]
    lib.oz2_gemm_rows_end.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p, ctypes.c_int] * 3 + \
        [ctypes.c_int, ctypes.c_int, ctypes.POINTER(B.oz2_opts)]
    ex = B.oz2_exchange()
    o = B.oz2_opts()
    o.target = 1e-15
    begin = lambda k=8, mode=0, N=0, opts=o, exch=ex: lib.oz2_gemm_rows_begin(   # noqa: E731
        8, 8, k, FAKE, max(k, 8), FAKE, 8, N, mode, ctypes.byref(opts) if opts else None,
        ctypes.byref(exch) if exch else None)
    assert begin(exch=None) == B.OZ2_EINVAL
    assert begin(opts=None) == B.OZ2_EINVAL
    assert begin() == B.OZ2_EINVAL                      # no workspace: it carries the state
    o.workspace = FAKE
    o.workspace_bytes = 1 << 30
    assert begin(k=B.K_MAX + 1) == B.OZ2_ERANGE
    assert begin(mode=B.OZ2_FAST) == B.OZ2_ENOTSUP
    assert begin(mode=B.OZ2_COMPONENTWISE) == B.OZ2_ENOTSUP
    assert lib.oz2_gemm_rows_end(8, 8, 8, FAKE, 8, FAKE, 8, None, 8, 0, 0, ctypes.byref(o)) == B.OZ2_EINVAL
