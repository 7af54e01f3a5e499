"""Split-K on the GPU (k > 2^17, beyond the paper's assumption of Section 3):
the library runs one emulation per K range and adds the results into C in
range order.  Each range's exponents and N are exported, injected into the
oracle's own split-K (one OS_II per range, FP64 or FP32 additions in the same
order), and the results must agree to 0 ulp; the summed bound (the ranges'
Theorem 2 bounds plus one rounding per addition) must hold against the exact
product."""
import numpy as np
import pytest

from paper_2602_02549_b300.inputs import integer_matrix, paper_pair

from _gpu_util import ulp_distance

pytestmark = pytest.mark.gpu

K_MAX = 1 << 17


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2602_02549_b300.build import build
    build()


def run_splitk(A, Bm, N=0, *, fp32=False, target=0.0, nmax=0, trans_a=False, trans_b=False, mu_in=None,
               nu_in=None):
    """One call through the C ABI; returns C and the per-range N, mu, nu."""
    import torch
    from paper_2602_02549_b300 import binding as B
    dt = torch.float32 if fp32 else torch.float64
    At = torch.tensor(A, dtype=dt, device="cuda")
    Bt = torch.tensor(Bm, dtype=dt, device="cuda")
    m = A.shape[1] if trans_a else A.shape[0]
    k = A.shape[0] if trans_a else A.shape[1]
    n = Bm.shape[0] if trans_b else Bm.shape[1]
    S, _ = B.k_ranges(k)
    nout = torch.zeros(S, dtype=torch.int32, device="cuda")
    kw = dict(n_out=nout)
    if mu_in is None:
        mu = torch.empty(S * m, dtype=torch.int32, device="cuda")
        nu = torch.empty(S * n, dtype=torch.int32, device="cuda")
        kw.update(mu_out=mu, nu_out=nu)
    else:
        kw.update(mu_in=torch.tensor(np.concatenate(mu_in), dtype=torch.int32, device="cuda"),
                  nu_in=torch.tensor(np.concatenate(nu_in), dtype=torch.int32, device="cuda"))
    C = B.matmul(At, Bt, N, target=target, nmax=nmax, trans_a=trans_a, trans_b=trans_b, **kw)
    torch.cuda.synchronize()
    assert B.sync() == 0
    out = dict(C=C.cpu().numpy(), N=[int(x) for x in nout.cpu().numpy()], S=S)
    if mu_in is None:
        out["mu"] = list(mu.cpu().numpy().reshape(S, m))
        out["nu"] = list(nu.cpu().numpy().reshape(S, n))
    else:
        out["mu"], out["nu"] = list(mu_in), list(nu_in)
    return out


def check(oracle, A, Bm, g, b=64):
    """Oracle split-K with the GPU's per-range N, mu, nu: 0 ulp, and the summed bound."""
    A64, B64 = np.asarray(A, np.float64), np.asarray(Bm, np.float64)
    r = oracle.os_ii_splitk(A64, B64, g["N"], b, mu_in=g["mu"], nu_in=g["nu"])
    assert len(r["ranges"]) == g["S"]
    assert ulp_distance(g["C"].astype(np.float64), r["C"].astype(np.float64), fp32=(b == 32)).max() == 0
    for (k0, k1), part in zip(r["ranges"], r["parts"]):
        assert oracle.lemma0_holds(part["Ap"], part["Bp"], part["N"])
    eb = oracle.bound_splitk(A64, B64, r, b)
    err = np.abs(oracle.exact_residual(A64, B64, g["C"].astype(np.float64)))
    assert (err <= eb).all(), f"max ratio {(err / eb).max()}"
    return r


@pytest.mark.parametrize("k,N", [(K_MAX + 37, 9), (2 * K_MAX, 14), (2 * K_MAX + 1, 5)])
def test_dgemm_fixed_N(oracle, k, N):
    A, Bm = paper_pair(24, 20, k, 1.0, seed=k % 97)
    g = run_splitk(A, Bm, N)
    assert g["S"] == len(oracle.splitk_ranges(k)) and g["N"] == [N] * g["S"]
    check(oracle, A, Bm, g)


def test_dgemm_bound_rule(oracle):
    # three ranges, each choosing its own N for target / 3
    k, tau, nmax = 3 * K_MAX - 5, 1e-15, 20
    A, Bm = paper_pair(24, 20, k, 1.0, seed=4)
    g = run_splitk(A, Bm, 0, target=tau, nmax=nmax)
    assert g["S"] == 3
    for (k0, k1), Ng in zip(oracle.splitk_ranges(k), g["N"]):
        As, Bs = np.ascontiguousarray(A[:, k0:k1]), np.ascontiguousarray(Bm[k0:k1])
        s = oracle.scaling(As, Bs, 14)
        _, info = oracle.choose_N(As, Bs, s["alpha"], s["beta"], s["cmax_row"], s["cmax_col"], tau / 3, nmax)
        rat = info["ratios"]
        assert rat[Ng] <= tau / 3 * (1 + 1e-9) or Ng == nmax
        if Ng > 2:
            assert rat[Ng - 1] > tau / 3 * (1 - 1e-9)
    r = check(oracle, A, Bm, g)
    # the N-dependent target holds for the sum: normwise error well inside tau
    exact_abs = np.abs(A) @ np.abs(Bm)
    err = np.abs(oracle.exact_residual(A, Bm, g["C"]))
    assert err.max() / exact_abs.max() <= tau
    assert len(r["parts"]) == 3


def test_integer_inputs_exact():
    # mu = nu = 0 injected keeps A' = A; at N = 5 every range is exact and the
    # FP64 additions of integers below 2^53 are too
    k = 2 * K_MAX + 3
    A = integer_matrix(17, k, -4, 4, seed=1)
    Bm = integer_matrix(k, 9, -4, 4, seed=2)
    from paper_2602_02549_b300 import binding as B
    S, _ = B.k_ranges(k)
    g = run_splitk(A, Bm, 5, mu_in=[np.zeros(17, np.int32)] * S, nu_in=[np.zeros(9, np.int32)] * S)
    assert g["S"] == 3
    assert np.array_equal(g["C"], (A.astype(np.int64) @ Bm.astype(np.int64)).astype(np.float64))


def test_sgemm(oracle):
    k = K_MAX + 513
    A, Bm = paper_pair(33, 17, k, 0.5, seed=8, dtype=np.float32)
    g = run_splitk(A, Bm, 7, fp32=True)
    assert g["C"].dtype == np.float32
    check(oracle, A, Bm, g, b=32)


@pytest.mark.parametrize("ta,tb", [(True, False), (False, True), (True, True)])
def test_transposes(oracle, ta, tb):
    k = K_MAX + 100
    A, Bm = paper_pair(12, 10, k, 1.0, seed=6)
    g = run_splitk(np.ascontiguousarray(A.T) if ta else A, np.ascontiguousarray(Bm.T) if tb else Bm, 6,
                   trans_a=ta, trans_b=tb)
    check(oracle, A, Bm, g)


def test_autograd_long_contraction():
    # forward k = 140000 (two ranges); the backward products have short k
    import torch
    from paper_2602_02549_b300.autograd import oz2_matmul
    A, Bm = paper_pair(8, 6, 140000, 1.0, seed=9)
    At = torch.tensor(A, device="cuda", requires_grad=True)
    Bt = torch.tensor(Bm, device="cuda", requires_grad=True)
    T = torch.tensor(np.random.default_rng(0).standard_normal((8, 6)), device="cuda")
    loss = ((oz2_matmul(At, Bt) - T) ** 2).sum()
    loss.backward()
    Ar = torch.tensor(A, device="cuda", requires_grad=True)
    Br = torch.tensor(Bm, device="cuda", requires_grad=True)
    ref = ((Ar @ Br - T) ** 2).sum()
    ref.backward()
    assert abs(loss.item() - ref.item()) <= 1e-12 * abs(ref.item())
    for g, h in ((At.grad, Ar.grad), (Bt.grad, Br.grad)):
        assert ((g - h).abs().max() / h.abs().max()).item() <= 1e-13
