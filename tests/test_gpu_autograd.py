"""Differentiable emulated GEMM (torch.autograd.Function with a hand-written
backward through the same emulated path)."""
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


def test_gradcheck_against_finite_differences():
    # FP64 central differences of the emulated forward vs the emulated backward
    import torch
    from paper_2602_02549_b300.autograd import Oz2Matmul
    g = torch.Generator().manual_seed(0)
    A = torch.randn(7, 5, dtype=torch.float64, generator=g).cuda().requires_grad_()
    B = torch.randn(5, 6, dtype=torch.float64, generator=g).cuda().requires_grad_()
    assert torch.autograd.gradcheck(lambda a, b: Oz2Matmul.apply(a, b, 20), (A, B), eps=1e-6, atol=1e-8,
                                    rtol=1e-6)


# the last shape is the autograd benchmark's (A 4096 x 2048, B 2048 x 1024)
@pytest.mark.parametrize("shape", [(130, 70, 90), (300, 257, 129), (4096, 2048, 1024)])
def test_loss_gradient_matches_fp64(shape):
    # loss = ||A B - T||_F^2: dA = 2 (AB - T) B^T, dB = 2 A^T (AB - T)
    import torch
    from paper_2602_02549_b300.autograd import oz2_matmul
    m, k, n = shape
    A = torch.tensor(paper_matrix(m, k, 1.0, 1), device="cuda", requires_grad=True)
    B = torch.tensor(paper_matrix(k, n, 1.0, 2), device="cuda", requires_grad=True)
    T = torch.tensor(paper_matrix(m, n, 1.0, 3), device="cuda")
    loss = ((oz2_matmul(A, B, 0, 1e-15) - T) ** 2).sum()
    loss.backward()
    with torch.no_grad():
        R = A @ B - T
        dA = 2 * R @ B.t()
        dB = 2 * A.t() @ R
        ref_loss = (R ** 2).sum()
    assert abs(loss.item() - ref_loss.item()) <= 1e-12 * ref_loss.item()
    # normwise agreement at the level of FP64 GEMM rounding
    for got, ref in ((A.grad, dA), (B.grad, dB)):
        err = (got - ref).abs().max().item()
        scale = ref.abs().max().item()
        assert err <= 1e-13 * scale, (err, scale)


@pytest.mark.parametrize("nmoduli", [14, 0])
@pytest.mark.parametrize("both", [True, False])
def test_backward_uses_transposed_operands_exactly(nmoduli, both):
    # the backward products (one batched call when both gradients are wanted,
    # single calls otherwise) equal direct emulated calls on materialised
    # transposes, bit for bit; nmoduli = 0: each product's own bound-chosen N
    import torch
    from paper_2602_02549_b300 import binding as Bd
    from paper_2602_02549_b300.autograd import oz2_matmul
    A = torch.tensor(paper_matrix(64, 48, 1.0, 4), device="cuda", requires_grad=True)
    B = torch.tensor(paper_matrix(48, 80, 4.0, 5), device="cuda", requires_grad=both)
    dC = torch.tensor(paper_matrix(64, 80, 2.0, 6), device="cuda")
    oz2_matmul(A, B, nmoduli, 1e-15).backward(dC)
    with torch.no_grad():
        dA = Bd.matmul(dC, B.t().contiguous(), nmoduli, target=1e-15)
        dB = Bd.matmul(A.t().contiguous(), dC, nmoduli, target=1e-15)
    assert torch.equal(A.grad, dA)
    if both:
        assert torch.equal(B.grad, dB)
    else:
        assert B.grad is None


def test_call_from_another_host_thread():
    # a host thread that has only made runtime calls must still work (the
    # tensor-map encoding is a driver call that needs a current context)
    import threading
    import torch
    from paper_2602_02549_b300 import binding as Bd
    A = torch.tensor(paper_matrix(40, 30, 1.0, 7), device="cuda")
    B = torch.tensor(paper_matrix(30, 20, 1.0, 8), device="cuda")
    ref = Bd.matmul(A, B, 14)
    out = {}

    def work():
        out["C"] = Bd.matmul(A, B, 14)
        torch.cuda.synchronize()

    t = threading.Thread(target=work)
    t.start()
    t.join()
    assert torch.equal(out["C"], ref)


def test_backward_single_calls_beyond_k_max():
    # dB = A^T dC has the inner dimension m; with m just above 2^17 the
    # two-problem batched backward (k <= 2^17 per problem) cannot take it, so
    # both gradients come from single calls, dB through split-K.  Each equals a
    # direct emulated call on the materialised transpose, bit for bit.
    import torch
    from paper_2602_02549_b300 import binding as Bd
    from paper_2602_02549_b300.autograd import oz2_matmul
    m, k, n = Bd.K_MAX + 3, 8, 3
    A = torch.tensor(paper_matrix(m, k, 1.0, 11), device="cuda", requires_grad=True)
    B = torch.tensor(paper_matrix(k, n, 1.0, 12), device="cuda", requires_grad=True)
    dC = torch.tensor(paper_matrix(m, n, 1.0, 13), device="cuda")
    oz2_matmul(A, B, 0, 1e-15).backward(dC)
    with torch.no_grad():
        dA = Bd.matmul(dC, B.t().contiguous(), 0, target=1e-15)
        dB = Bd.matmul(A.t().contiguous(), dC, 0, target=1e-15)
        ref = A.detach().t() @ dC
    assert torch.equal(A.grad, dA)
    assert torch.equal(B.grad, dB)
    assert ((B.grad - ref).abs().max() <= 1e-13 * ref.abs().max()).item()
