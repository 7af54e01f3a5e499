"""Complex products on the GPU (oz2_zgemm / oz2_cgemm): each part is a real
emulated product over 2k.  The GPU's per-part (and per-range) N, mu, nu are
injected into the oracle's complex product; real and imaginary parts must agree
to 0 ulp, and each part must meet its Theorem 2 bound against the exact part."""
import numpy as np
import pytest

from paper_2602_02549_b300.inputs import integer_matrix, paper_matrix

from _gpu_util import ulp_distance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2602_02549_b300.build import build
    build()


def cplx(re, im):
    return re.astype(np.float64) + 1j * im.astype(np.float64)


def paper_cplx(r, c, phi, seed, dt=np.float64):
    return cplx(paper_matrix(r, c, phi, seed, dt), paper_matrix(r, c, phi, seed + 1, dt))


def run_z(A, Bm, N=0, *, fp32=False, target=0.0, nmax=0, ta=False, tb=False, ca=False, cb=False, mu_in=None,
          nu_in=None, fast=False):
    import torch
    from paper_2602_02549_b300 import binding as B
    dt = torch.complex64 if fp32 else torch.complex128
    At = torch.tensor(A, dtype=dt, device="cuda")
    Bt = torch.tensor(Bm, dtype=dt, device="cuda")
    m = A.shape[1] if ta else A.shape[0]
    k = A.shape[0] if ta else A.shape[1]
    n = Bm.shape[0] if tb else Bm.shape[1]
    S, _ = B.k_ranges(2 * k)
    nout = torch.zeros(2 * S, dtype=torch.int32, device="cuda")
    kw = dict(n_out=nout)
    if mu_in is None:
        mu = torch.empty(2 * S * m, dtype=torch.int32, device="cuda")
        nu = torch.empty(2 * S * n, dtype=torch.int32, device="cuda")
        kw.update(mu_out=mu, nu_out=nu)
    else:
        kw.update(mu_in=torch.tensor(np.concatenate([np.concatenate(x) for x in mu_in]), dtype=torch.int32,
                                     device="cuda"),
                  nu_in=torch.tensor(np.concatenate([np.concatenate(x) for x in nu_in]), dtype=torch.int32,
                                     device="cuda"))
    C = B.zmatmul(At, Bt, N, target=target, nmax=nmax, trans_a=ta, trans_b=tb, conj_a=ca, conj_b=cb, fast=fast,
                  **kw)
    torch.cuda.synchronize()
    assert B.sync() == 0
    Ns = [int(x) for x in nout.cpu().numpy()]
    out = dict(C=C.cpu().numpy(), S=S, N=(Ns[:S], Ns[S:]))
    if mu_in is None:
        mv = mu.cpu().numpy().reshape(2, S, m)
        nv = nu.cpu().numpy().reshape(2, S, n)
        out["mu"] = ([mv[0, s] for s in range(S)], [mv[1, s] for s in range(S)])
        out["nu"] = ([nv[0, s] for s in range(S)], [nv[1, s] for s in range(S)])
    else:
        out["mu"], out["nu"] = mu_in, nu_in
    return out


def op(X, t, c):
    Y = X.T if t else X
    return np.conj(Y) if c else Y


def check(oracle, Aop, Bop, g, b=64, fast=False):
    r = oracle.os_ii_complex(Aop, Bop, g["N"], b, mu_in=g["mu"], nu_in=g["nu"], fast=fast)
    fp32 = b == 32
    for got, ref in ((g["C"].real, r["C"].real), (g["C"].imag, r["C"].imag)):
        assert ulp_distance(got.astype(np.float64), ref.astype(np.float64), fp32=fp32).max() == 0
    for part, Bp, got in zip(r["parts"], (r["B1"], r["B2"]), (g["C"].real, g["C"].imag)):
        eb = oracle.bound_splitk(r["As"], Bp, part, b)
        err = np.abs(oracle.exact_residual(r["As"], Bp, got.astype(np.float64)))
        assert (err <= eb).all(), f"max ratio {(err / eb).max()}"
    return r


@pytest.mark.parametrize("shape,N", [((40, 36, 300), 14), ((129, 257, 65), 8), ((1, 1, 1), 2)])
def test_zgemm_parity(oracle, shape, N):
    m, n, k = shape
    A, Bm = paper_cplx(m, k, 1.0, m), paper_cplx(k, n, 1.0, n + 50)
    g = run_z(A, Bm, N)
    assert g["N"] == ([N], [N])
    check(oracle, A, Bm, g)


@pytest.mark.parametrize("ta,tb,ca,cb", [(True, False, False, False), (False, True, False, False),
                                         (False, False, True, False), (False, False, False, True),
                                         (True, True, True, True)])
def test_modes(oracle, ta, tb, ca, cb):
    m, n, k = 20, 24, 150
    A = paper_cplx(k, m, 1.0, 1) if ta else paper_cplx(m, k, 1.0, 1)
    Bm = paper_cplx(n, k, 1.0, 3) if tb else paper_cplx(k, n, 1.0, 3)
    g = run_z(A, Bm, 10, ta=ta, tb=tb, ca=ca, cb=cb)
    check(oracle, op(A, ta, ca), op(Bm, tb, cb), g)


def test_bound_rule_and_fast_mode(oracle):
    A, Bm = paper_cplx(64, 48, 2.0, 5), paper_cplx(48, 40, 2.0, 9)
    g = run_z(A, Bm, 0, target=1e-14, nmax=20)
    assert all(2 <= x <= 20 for x in g["N"][0] + g["N"][1])
    check(oracle, A, Bm, g)
    g = run_z(A, Bm, 0, target=1e-14, nmax=20, fast=True)
    check(oracle, A, Bm, g, fast=True)


def test_cgemm(oracle):
    A, Bm = paper_cplx(33, 70, 0.5, 2, np.float32), paper_cplx(70, 17, 0.5, 4, np.float32)
    g = run_z(A, Bm, 7, fp32=True)
    assert g["C"].dtype == np.complex64
    check(oracle, A, Bm, g, b=32)


def test_integer_inputs_exact():
    A = cplx(integer_matrix(15, 400, -7, 7, 1), integer_matrix(15, 400, -7, 7, 2))
    Bm = cplx(integer_matrix(400, 11, -7, 7, 3), integer_matrix(400, 11, -7, 7, 4))
    z = lambda r: ([np.zeros(r, np.int32)], [np.zeros(r, np.int32)])
    g = run_z(A, Bm, 5, mu_in=z(15), nu_in=z(11))
    assert np.array_equal(g["C"], A @ Bm)


def test_long_contraction_runs_split_k(oracle):
    # 2k = 140000 > 2^17: each part runs as two K ranges
    A, Bm = paper_cplx(6, 70000, 1.0, 11), paper_cplx(70000, 5, 1.0, 13)
    g = run_z(A, Bm, 9)
    assert g["S"] == 2 and g["N"] == ([9, 9], [9, 9])
    check(oracle, A, Bm, g)
