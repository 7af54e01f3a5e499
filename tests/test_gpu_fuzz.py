"""GPU parity on seeded random cases: shapes with ragged tiles, N from 2 to 49,
both precisions, transposes and fast mode, each checked against the CPU oracle
with the GPU's exponents injected (W_l bit-exact, C within 2 ulp, Theorem 2's
bound on every entry) - the combinations the fixed cases do not enumerate.
"""
import numpy as np
import pytest

from paper_2602_02549_b300.inputs import paper_pair

from _gpu_util import run_gpu
from test_gpu_parity import check_against_oracle

pytestmark = pytest.mark.gpu


def _cases(count=24, seed=2026):
    rng = np.random.default_rng(seed)
    out = []
    for c in range(count):
        m = int(rng.integers(1, 300))
        n = int(rng.integers(1, 300))
        k = int(rng.integers(1, 2100))
        N = int(rng.integers(2, 50))
        b = 32 if rng.random() < 0.3 else 64
        phi = float(rng.choice([0.5, 1.0, 2.0, 4.0]))
        ta, tb = bool(rng.random() < 0.3), bool(rng.random() < 0.3)
        fast = bool(rng.random() < 0.25)
        out.append((c, m, n, k, N, b, phi, ta, tb, fast))
    return out


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2602_02549_b300.build import build
    build()


@pytest.mark.parametrize("case", _cases(), ids=lambda c: "c%d_m%d_n%d_k%d_N%d_b%d" % c[:6])
def test_random_case(oracle, case):
    c, m, n, k, N, b, phi, ta, tb, fast = case
    dt = np.float64 if b == 64 else np.float32
    A, Bm = paper_pair(m, n, k, phi, seed=1000 + c, dtype=dt)
    As = np.ascontiguousarray(A.T) if ta else A
    Bs = np.ascontiguousarray(Bm.T) if tb else Bm
    g = run_gpu(As, Bs, N, fp32=(b == 32), trans_a=ta, trans_b=tb, fast=fast)
    assert g["N"] == N
    check_against_oracle(oracle, A.astype(np.float64), Bm.astype(np.float64), g, b=b)
