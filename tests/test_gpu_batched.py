"""Batched emulated DGEMM: every problem of one oz2_gemm_batched call must be
bit-identical to oz2_gemm_ex on the same problem (same exponents, same N), and
the call must capture into a CUDA graph and replay correctly."""
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


SPECS = [  # m, n, k, phi, nmoduli, target, fast, trans_a, trans_b
    (128, 256, 64, 0.5, 14, 0.0, False, False, False),
    (300, 200, 1500, 1.0, 0, 1e-14, False, False, False),
    (33, 65, 17, 2.0, 8, 0.0, False, True, False),
    (513, 129, 700, 4.0, 0, 1e-12, False, False, True),
    (1, 1, 1, 1.0, 5, 0.0, False, False, False),
    (777, 333, 2049, 1.0, 0, 1e-15, False, False, False),
    (250, 260, 300, 1.0, 17, 0.0, True, False, False),
    (64, 1000, 900, 2.0, 0, 1e-14, True, True, True),
    (1200, 40, 80, 0.5, 20, 0.0, False, False, False),
    (90, 91, 4100, 1.0, 0, 1e-15, False, False, False),
]


def make_problems(seed0=0):
    import torch
    probs = []
    for i, (m, n, k, phi, N, tau, fast, ta, tb) in enumerate(SPECS):
        A = paper_matrix(m, k, phi, seed0 + 2 * i)
        Bm = paper_matrix(k, n, phi, seed0 + 2 * i + 1)
        As = np.ascontiguousarray(A.T) if ta else A
        Bs = np.ascontiguousarray(Bm.T) if tb else Bm
        probs.append(dict(A=torch.tensor(As, device="cuda"), B=torch.tensor(Bs, device="cuda"),
                          C=torch.full((m, n), float("nan"), dtype=torch.float64, device="cuda"),
                          nmoduli=N, target=tau, nmax=30 if N == 0 else 0, fast=fast, trans_a=ta, trans_b=tb,
                          n_out=torch.zeros(1, dtype=torch.int32, device="cuda")))
    return probs


def single_reference(q):
    import torch
    from paper_2602_02549_b300 import binding as B
    C = torch.empty_like(q["C"])
    nout = torch.zeros(1, dtype=torch.int32, device="cuda")
    mode = (B.OZ2_FAST if q["fast"] else 0) | (B.OZ2_TRANS_A if q["trans_a"] else 0) | \
        (B.OZ2_TRANS_B if q["trans_b"] else 0)
    assert B.gemm_ex(q["A"], q["B"], C, q["nmoduli"], mode, target=q["target"], nmax=q["nmax"], n_out=nout) == 0
    return C, nout


def test_batched_equals_single_calls():
    import torch
    from paper_2602_02549_b300 import binding as B
    probs = make_problems()
    assert B.gemm_batched(probs) == 0
    torch.cuda.synchronize()
    assert B.sync() == 0
    for q in probs:
        C, nout = single_reference(q)
        torch.cuda.synchronize()
        assert int(q["n_out"].item()) == int(nout.item())
        assert torch.equal(q["C"], C)


def test_batched_graph_capture_and_replay():
    import torch
    from paper_2602_02549_b300 import binding as B
    probs = make_problems()
    ws = torch.empty(B.batched_workspace_size(probs), dtype=torch.uint8, device="cuda")
    assert B.gemm_batched(probs, workspace=ws) == 0          # first call outside capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        assert B.gemm_batched(probs, workspace=ws, stream=s) == 0
    for seed in (100, 200):
        fresh = make_problems(seed)
        for q, f in zip(probs, fresh):
            q["A"].copy_(f["A"])
            q["B"].copy_(f["B"])
            q["C"].fill_(float("nan"))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        for q in probs:
            C, nout = single_reference(q)
            torch.cuda.synchronize()
            assert torch.equal(q["C"], C) and int(q["n_out"].item()) == int(nout.item())


@pytest.mark.parametrize("policy", [1, 2])
def test_tile_policies_equal_single_calls(policy):
    # 128 x 128 tiles (all problems, or the narrow ones) give bit-identical results
    import torch
    from paper_2602_02549_b300 import binding as B
    probs = make_problems(7)
    assert B.batched_set_policy(probs, policy) == 0
    assert B.gemm_batched(probs) == 0
    torch.cuda.synchronize()
    assert B.sync() == 0
    for q in probs:
        C, nout = single_reference(q)
        torch.cuda.synchronize()
        assert int(q["n_out"].item()) == int(nout.item())
        assert torch.equal(q["C"], C)
    assert B.batched_set_policy(probs, 0) == 0


def test_autotune_keeps_a_policy_and_results():
    import torch
    from paper_2602_02549_b300 import binding as B
    probs = make_problems(11)
    policy, ms = B.batched_autotune(probs)
    assert policy in (0, 1, 2, 3)
    assert len(ms) == 4 and all(t > 0 for t in ms)
    assert ms[policy] == min(ms)
    for q in probs:
        q["C"].fill_(float("nan"))
    assert B.gemm_batched(probs) == 0          # runs with the kept policy
    torch.cuda.synchronize()
    assert B.sync() == 0
    for q in probs:
        C, nout = single_reference(q)
        torch.cuda.synchronize()
        assert torch.equal(q["C"], C)
    assert B.batched_set_policy(probs, 5) == B.OZ2_EINVAL


def test_more_problems_than_one_group():
    # 70 problems: one group of 64 and one of 6, launched one after the other
    # on the same workspace layout; every problem bit-identical to its single
    # call, also under the autotuner's kept policy
    import torch
    from paper_2602_02549_b300 import binding as B
    rng = np.random.default_rng(70)
    probs = []
    for i in range(70):
        m, n, k = (int(v) for v in rng.integers(1, 200, size=3))
        Bm = paper_matrix(k, n, 1.0, 3 * i + 1)
        probs.append(dict(A=torch.tensor(paper_matrix(m, k, 1.0, 3 * i), device="cuda"),
                          B=torch.tensor(np.ascontiguousarray(Bm.T) if i % 4 == 0 else Bm, device="cuda"),
                          C=torch.full((m, n), float("nan"), dtype=torch.float64, device="cuda"),
                          nmoduli=0 if i % 3 else 12, target=1e-14 if i % 3 else 0.0, nmax=30 if i % 3 else 0,
                          fast=i % 5 == 0, trans_a=False, trans_b=i % 4 == 0,
                          n_out=torch.zeros(1, dtype=torch.int32, device="cuda")))
    refs = [single_reference(q) for q in probs]
    for tuned in (False, True):
        if tuned:
            B.batched_autotune(probs)
        for q in probs:
            q["C"].fill_(float("nan"))
        assert B.gemm_batched(probs) == 0
        torch.cuda.synchronize()
        assert B.sync() == 0
        for q, (C, nout) in zip(probs, refs):
            assert int(q["n_out"].item()) == int(nout.item())
            assert torch.equal(q["C"], C)


def test_batched_benchmark_set(oracle):
    # the batched benchmark's 64 problems (m, n, k log-uniform in [128, 4096],
    # phi ~ U(0.5, 4), tau = 1e-14): autotuned tiles, graph-captured call, each
    # problem bit-identical to its single call; sampled entries of four
    # problems against the oracle with the single call's exponents
    import torch
    from paper_2602_02549_b300 import binding as B
    from paper_2602_02549_b300.inputs import batched_specs, paper_matrix_torch
    dev = torch.device("cuda", 0)
    probs = []
    for i, (m, n, k, phi) in enumerate(batched_specs(64, 0)):
        probs.append(dict(A=paper_matrix_torch(m, k, phi, 2 * i, dev), B=paper_matrix_torch(k, n, phi, 2 * i + 1, dev),
                          C=torch.full((m, n), float("nan"), dtype=torch.float64, device=dev), nmoduli=0,
                          target=1e-14, nmax=30, fast=False, trans_a=False, trans_b=False,
                          n_out=torch.zeros(1, dtype=torch.int32, device=dev)))
    ws = torch.empty(B.batched_workspace_size(probs), dtype=torch.uint8, device=dev)
    B.batched_autotune(probs, workspace=ws)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        assert B.gemm_batched(probs, workspace=ws, stream=s) == 0
    for q in probs:
        q["C"].fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert B.sync() == 0
    rng = np.random.default_rng(3)
    checked = 0
    for idx, q in enumerate(probs):
        m, n = q["C"].shape
        C = torch.empty_like(q["C"])
        nout = torch.zeros(1, dtype=torch.int32, device=dev)
        mu = torch.empty(m, dtype=torch.int32, device=dev)
        nu = torch.empty(n, dtype=torch.int32, device=dev)
        assert B.gemm_ex(q["A"], q["B"], C, 0, 0, target=1e-14, nmax=30, n_out=nout, mu_out=mu, nu_out=nu) == 0
        torch.cuda.synchronize()
        assert int(q["n_out"].item()) == int(nout.item())
        assert torch.equal(q["C"], C)
        if idx % 16 == 0:
            ii = np.sort(rng.choice(m, size=min(m, 8), replace=False))
            jj = np.sort(rng.choice(n, size=min(n, 8), replace=False))
            A_rows = q["A"][ii].cpu().numpy()
            B_cols = q["B"][:, jj].cpu().numpy()
            ref = oracle.os_ii_block(A_rows, B_cols, mu.cpu().numpy()[ii], nu.cpu().numpy()[jj], int(nout.item()))
            got = C.cpu().numpy()[np.ix_(ii, jj)]
            assert np.abs(got.view(np.int64) - ref.view(np.int64)).max() <= 2
            checked += 1
    assert checked == 4
