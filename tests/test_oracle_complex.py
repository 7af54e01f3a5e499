"""Pins of the oracle's complex products (an extension: the paper's analysis
covers real GEMM).  A complex product is two real ones over 2k:
Re(AB) = [Re A, Im A][Re B; -Im B], Im(AB) = [Re A, Im A][Im B; Re B].

* the identity itself, exactly, on integer-valued complex matrices;
* integer inputs with A' = A, B' = B (mu = nu = 0) at N = 5 come out exact;
* Theorem 2's bound holds per part against the exact real and imaginary parts;
* at N = 20 the result matches numpy's complex product to rounding level, and a
  planted sign mistake in the parts (on the CPU) is caught by these checks.
"""
import numpy as np
import pytest

from paper_2602_02549_b300.inputs import integer_matrix, paper_matrix


def cplx(re, im):
    return re.astype(np.float64) + 1j * im.astype(np.float64)


def int_cplx(r, c, seed, lo=-6, hi=6):
    return cplx(integer_matrix(r, c, lo, hi, seed), integer_matrix(r, c, lo, hi, seed + 1))


def test_parts_identity_exact(oracle):
    A, B = int_cplx(7, 11, 1), int_cplx(11, 5, 3)
    As, B1, B2 = oracle.complex_parts(A, B)
    IA = As.astype(np.int64)
    ref_re = A.real.astype(np.int64) @ B.real.astype(np.int64) - A.imag.astype(np.int64) @ B.imag.astype(np.int64)
    ref_im = A.real.astype(np.int64) @ B.imag.astype(np.int64) + A.imag.astype(np.int64) @ B.real.astype(np.int64)
    assert np.array_equal(IA @ B1.astype(np.int64), ref_re)
    assert np.array_equal(IA @ B2.astype(np.int64), ref_im)


def test_integer_inputs_exact(oracle):
    A, B = int_cplx(9, 300, 5), int_cplx(300, 7, 7)
    z = ([np.zeros(9, np.int32)], [np.zeros(9, np.int32)]), ([np.zeros(7, np.int32)], [np.zeros(7, np.int32)])
    r = oracle.os_ii_complex(A, B, 5, mu_in=z[0], nu_in=z[1])
    assert np.array_equal(r["C"], A @ B)


@pytest.mark.parametrize("b", [64, 32])
def test_bound_per_part(oracle, b):
    dt = np.float64 if b == 64 else np.float32
    A = cplx(paper_matrix(12, 400, 1.0, 1, dt), paper_matrix(12, 400, 1.0, 2, dt))
    B = cplx(paper_matrix(400, 9, 1.0, 3, dt), paper_matrix(400, 9, 1.0, 4, dt))
    r = oracle.os_ii_complex(A, B, 12 if b == 64 else 7, b)
    for part, Bp in zip(r["parts"], (r["B1"], r["B2"])):
        eb = oracle.bound_splitk(r["As"], Bp, part, b)
        err = np.abs(oracle.exact_residual(r["As"], Bp, part["C"].astype(np.float64)))
        assert (err <= eb).all()


def test_high_N_matches_numpy_and_catches_a_sign_mistake(oracle):
    A = cplx(paper_matrix(10, 256, 0.5, 5), paper_matrix(10, 256, 0.5, 6))
    B = cplx(paper_matrix(256, 8, 0.5, 7), paper_matrix(256, 8, 0.5, 8))
    r = oracle.os_ii_complex(A, B, 20)
    ref = A @ B
    scale = (np.abs(A) @ np.abs(B)).max()
    assert np.abs(r["C"] - ref).max() <= 1e-15 * scale
    # planted: +Im B in the real part's operand
    As, B1, _ = oracle.complex_parts(A, B)
    wrong = oracle.os_ii(As, np.vstack([B.real, B.imag]), 20)["C"]
    assert np.abs(wrong - ref.real).max() > 1e-3 * scale
