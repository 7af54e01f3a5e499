"""GPU parity of the componentwise N rule (OZ2_COMPONENTWISE): the N the
library picks meets the oracle's criterion (choose_N_componentwise: the
N-dependent part of eq. thm:err-1 at most tau L_ij on every entry) and N - 1
does not, up to the FP32 rounding of the device's ratio maxima; the product
then equals the plain call at that N bit for bit, in single and batched calls."""
import numpy as np
import pytest

from paper_2602_02549_b300.inputs import paper_pair

pytestmark = pytest.mark.gpu

SLACK = 1e-5          # the device's ratio maxima are FP32 upper bounds (a few ulp)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2602_02549_b300.build import build
    build()


def oracle_rule(oracle, A, B, tau, nmax, fast=False):
    s = oracle.scaling(A, B, 14, fast=fast)
    return oracle.choose_N_componentwise(A, B, s["alpha"], s["beta"], s["cmax_row"], s["cmax_col"], tau, nmax)


def check_N(N, info, tau, nmax):
    r = info["ratios"]
    if N == nmax and not r[N] <= tau * (1 + SLACK):
        return all(v > tau * (1 - SLACK) for v in r.values())
    return r[N] <= tau * (1 + SLACK) and (N == 2 or r[N - 1] > tau * (1 - SLACK))


CASES = [(200, 300, 700, 0.5, 1e-15), (257, 129, 2050, 1.0, 1e-12), (64, 520, 300, 0.5, 1e-8),
         (300, 200, 1100, 4.0, 1e-15), (130, 140, 5000, 1.0, 1e-15)]


@pytest.mark.parametrize("fast", [False, True])
@pytest.mark.parametrize("case", CASES)
def test_componentwise_N_matches_oracle(oracle, case, fast):
    import torch
    from paper_2602_02549_b300 import binding as B
    m, n, k, phi, tau = case
    A, Bm = paper_pair(m, n, k, phi, seed=m + k)
    At, Bt = torch.tensor(A, device="cuda"), torch.tensor(Bm, device="cuda")
    nout = torch.zeros(1, dtype=torch.int32, device="cuda")
    C = B.matmul(At, Bt, 0, target=tau, nmax=30, fast=fast, componentwise=True, n_out=nout)
    torch.cuda.synchronize()
    assert B.sync() == 0
    N = int(nout.item())
    _, info = oracle_rule(oracle, A, Bm, tau, 30, fast)
    assert check_N(N, info, tau, 30), (N, info["ratios"])
    ref = B.matmul(At, Bt, N, fast=fast)
    torch.cuda.synchronize()
    assert torch.equal(C, ref)


def test_componentwise_needs_the_bound_rule():
    import torch
    from paper_2602_02549_b300 import binding as B
    A = torch.ones((4, 4), dtype=torch.float64, device="cuda")
    C = torch.empty((4, 4), dtype=torch.float64, device="cuda")
    assert B.gemm_ex(A, A, C, 14, B.OZ2_COMPONENTWISE) == B.OZ2_EINVAL


def test_componentwise_batched_equals_single_calls(oracle):
    import torch
    from paper_2602_02549_b300 import binding as B
    probs, singles = [], []
    for i, (m, n, k, phi) in enumerate([(150, 270, 400, 0.5), (300, 90, 1300, 1.0), (64, 64, 64, 0.5)]):
        A, Bm = paper_pair(m, n, k, phi, seed=40 + i)
        At, Bt = torch.tensor(A, device="cuda"), torch.tensor(Bm, device="cuda")
        probs.append(dict(A=At, B=Bt, C=torch.empty((m, n), dtype=torch.float64, device="cuda"), nmoduli=0,
                          target=1e-13, nmax=30, componentwise=True,
                          n_out=torch.zeros(1, dtype=torch.int32, device="cuda")))
        singles.append(B.matmul(At, Bt, 0, target=1e-13, nmax=30, componentwise=True))
    assert B.gemm_batched(probs) == 0
    torch.cuda.synchronize()
    assert B.sync() == 0
    for q, ref in zip(probs, singles):
        assert torch.equal(q["C"], ref)
