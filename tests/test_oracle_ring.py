"""Pins of the oracle's ring arithmetic in Z_{2^32}[X]/(X^N + 1).

Each product routine is checked against something other than itself: a product
worked by hand, sympy's polynomial remainder, and ring identities."""
import numpy as np
import pytest
import sympy

import oracle
import synth

M32 = 1 << 32


def test_schoolbook_by_hand_n4():
    # (1 + 2X + 3X^2 + 4X^3)(5 + 6X + 7X^2 + 8X^3): full product coefficients
    # 5, 16, 34, 60, 61, 52, 32 (degrees 0..6); X^4 = -1 folds degree 4+d onto d with a
    # minus sign: [5 - 61, 16 - 52, 34 - 32, 60] = [-56, -36, 2, 60].
    out = oracle.poly_mul_schoolbook([1, 2, 3, 4], [5, 6, 7, 8])
    assert out.tolist() == [M32 - 56, M32 - 36, 2, 60]


@pytest.mark.parametrize("N", [8, 16])
def test_schoolbook_vs_sympy(N):
    X = sympy.symbols("X")
    mod = sympy.Poly(X**N + 1, X)
    a = synth.uniform_u32(3, 100 + N, N)
    b = synth.uniform_u32(3, 200 + N, N)
    pa = sympy.Poly([int(v) for v in a[::-1]], X)
    pb = sympy.Poly([int(v) for v in b[::-1]], X)
    r = (pa * pb).rem(mod)
    coeffs = [int(c) % M32 for c in reversed(r.all_coeffs())]
    coeffs += [0] * (N - len(coeffs))
    assert oracle.poly_mul_schoolbook(a, b).tolist() == coeffs


@pytest.mark.parametrize("N", [4, 16, 32, 64, 256, 1024])
def test_karatsuba_equals_schoolbook(N):
    for trial in range(3):
        a = synth.uniform_u32(5, 10 * N + trial, N)
        b = synth.uniform_u32(6, 10 * N + trial, N)
        np.testing.assert_array_equal(oracle.poly_mul_karatsuba(a, b), oracle.poly_mul_schoolbook(a, b))


def test_karatsuba_small_signed_digits_times_torus():
    # The blind rotation multiplies digit polynomials in [-512, 511] by torus
    # polynomials; check that shape explicitly against an exact integer convolution.
    N = 1024
    d = (synth.uniform_u32(8, 1, N) % 1024).astype(np.int64) - 512
    b = synth.uniform_u32(8, 2, N).astype(np.int64)
    full = np.zeros(2 * N, dtype=object)
    for i in range(N):
        full[i:i + N] += int(d[i]) * b.astype(object)
    ref = [(int(full[j]) - int(full[j + N])) % M32 for j in range(N)]
    got = oracle.poly_mul_karatsuba((d % M32).astype(np.uint32), b.astype(np.uint32))
    assert got.tolist() == ref


def test_monomial_identities():
    N = 64
    v = synth.uniform_u32(9, 1, N)
    # X^N = -1, X^(2N) = 1.
    neg = (M32 - v.astype(np.int64)) % M32
    np.testing.assert_array_equal(oracle.poly_mul_monomial(v, N), neg.astype(np.uint32))
    np.testing.assert_array_equal(oracle.poly_mul_monomial(v, 2 * N), v)
    # X^e v equals the product with the polynomial X^e (e < N), and X^a X^b = X^(a+b).
    for e in (1, 5, N - 1):
        mono = np.zeros(N, np.uint32)
        mono[e] = 1
        np.testing.assert_array_equal(oracle.poly_mul_monomial(v, e), oracle.poly_mul_schoolbook(mono, v))
    for a_, b_ in ((3, 70), (100, 29), (127, 127)):
        lhs = oracle.poly_mul_monomial(oracle.poly_mul_monomial(v, a_), b_)
        np.testing.assert_array_equal(lhs, oracle.poly_mul_monomial(v, a_ + b_))
    # Coefficient 0 of X^(-k) v is v_k for k < N (the rotation direction the test
    # vector of the blind rotation relies on).
    for k in (0, 1, 17, N - 1):
        assert oracle.poly_mul_monomial(v, 2 * N - k)[0] == v[k]
