"""Batched calls on seeded random batches: ragged shapes (rows shorter than a
warp, single columns, k past a K segment), transposes, fast mode, fixed and
bound-chosen N, under every tile policy and from a workspace full of NaN bytes.
Every problem of a batch must give the N and the bits of C of its own
oz2_gemm_ex call (the single calls are checked against the oracle elsewhere)."""
import numpy as np
import pytest

from paper_2602_02549_b300.inputs import paper_matrix

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2602_02549_b300.build import build
    build()


def _batch(seed):
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(int(rng.integers(5, 17))):
        m = int(rng.choice([int(rng.integers(1, 9)), int(rng.integers(1, 700))]))
        n = int(rng.choice([int(rng.integers(1, 9)), int(rng.integers(1, 700))]))
        k = int(rng.choice([int(rng.integers(1, 70)), int(rng.integers(1, 3000))]))
        fixed = rng.random() < 0.4
        specs.append(dict(m=m, n=n, k=k, phi=float(rng.choice([0.5, 1.0, 2.0, 4.0])),
                          N=int(rng.integers(2, 31)) if fixed else 0,
                          tau=0.0 if fixed else float(rng.choice([1e-10, 1e-14, 1e-15])),
                          fast=bool(rng.random() < 0.25), ta=bool(rng.random() < 0.3),
                          tb=bool(rng.random() < 0.3)))
    return specs


def _problems(specs, seed):
    import torch
    probs = []
    for i, s in enumerate(specs):
        A = paper_matrix(s["m"], s["k"], s["phi"], seed + 2 * i)
        Bm = paper_matrix(s["k"], s["n"], s["phi"], seed + 2 * i + 1)
        probs.append(dict(A=torch.tensor(np.ascontiguousarray(A.T) if s["ta"] else A, device="cuda"),
                          B=torch.tensor(np.ascontiguousarray(Bm.T) if s["tb"] else Bm, device="cuda"),
                          C=torch.full((s["m"], s["n"]), float("nan"), dtype=torch.float64, device="cuda"),
                          nmoduli=s["N"], target=s["tau"], nmax=30 if s["N"] == 0 else 0, fast=s["fast"],
                          trans_a=s["ta"], trans_b=s["tb"],
                          n_out=torch.zeros(1, dtype=torch.int32, device="cuda")))
    return probs


def _single(q):
    import torch
    from paper_2602_02549_b300 import binding as B
    C = torch.empty_like(q["C"])
    nout = torch.zeros(1, dtype=torch.int32, device="cuda")
    mode = (B.OZ2_FAST if q["fast"] else 0) | (B.OZ2_TRANS_A if q["trans_a"] else 0) | \
        (B.OZ2_TRANS_B if q["trans_b"] else 0)
    assert B.gemm_ex(q["A"], q["B"], C, q["nmoduli"], mode, target=q["target"], nmax=q["nmax"], n_out=nout) == 0
    return int(nout.item()), C


@pytest.mark.parametrize("seed", [11, 12, 13, 14, 15, 16])
def test_random_batch_equals_single_calls(seed):
    import torch
    from paper_2602_02549_b300 import binding as B
    specs = _batch(seed)
    probs = _problems(specs, 100 * seed)
    refs = [_single(q) for q in probs]
    for policy in (0, 1, 2):
        assert B.batched_set_policy(probs, policy) == 0
        ws = torch.full((B.batched_workspace_size(probs),), 0xFF, dtype=torch.uint8, device="cuda")
        for q in probs:
            q["C"].fill_(float("nan"))
            q["n_out"].zero_()
        assert B.gemm_batched(probs, workspace=ws) == 0
        torch.cuda.synchronize()
        assert B.sync() == 0
        for i, (q, (N, C)) in enumerate(zip(probs, refs)):
            assert int(q["n_out"].item()) == N, (policy, i, specs[i])
            assert torch.equal(q["C"], C), (policy, i, specs[i])
