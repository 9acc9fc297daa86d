"""Pins of the oracle's gadget decomposition, key-switch digits and modulus switch."""
from fractions import Fraction

import numpy as np

import oracle
import synth

M32 = 1 << 32


def _signed(x):
    x %= M32
    return x - M32 if x >= M32 // 2 else x


def test_gadget_digits_recompose_within_two():
    xs = list(synth.uniform_u32(21, 1, 4000)) + [0, 1, 2, 3, M32 - 1, M32 // 2, M32 // 2 - 1, 1 << 30, 3 << 30]
    for x in xs:
        d = oracle.gadget_digits(int(x), lg=3, Bgbit=10)
        assert all(-512 <= int(v) <= 511 for v in d)
        rec = sum(int(d[p]) * (1 << (32 - 10 * (p + 1))) for p in range(3))
        assert abs(_signed(int(x) - rec)) <= 2


def test_gadget_digits_of_zero_and_exact_multiples():
    assert oracle.gadget_digits(0).tolist() == [0, 0, 0]
    # Multiples of 2^2 are reproduced exactly (the closed-form bootstrap relies on it).
    for x in (1 << 30, 3 << 30, 4, 12345 << 2):
        d = oracle.gadget_digits(x)
        rec = sum(int(d[p]) * (1 << (32 - 10 * (p + 1))) for p in range(3))
        assert (rec - x) % M32 == 0


def test_ks_digits_recompose_within_half_ulp():
    for x in list(synth.uniform_u32(22, 1, 4000)) + [0, M32 - 1, (1 << 15) - 1, 1 << 15]:
        v = oracle.ks_digits(int(x), t=8, basebit=2)
        assert all(0 <= int(d) <= 3 for d in v)
        rec = sum(int(v[j]) << (30 - 2 * j) for j in range(8))
        assert abs(_signed(int(x) - rec)) <= 1 << 15


def test_modswitch_is_round_half_up_to_2N():
    N = 1024
    for x in list(synth.uniform_u32(23, 1, 2000)) + [0, (1 << 20) - 1, 1 << 20, M32 - 1, M32 - (1 << 20)]:
        exact = Fraction(int(x) * 2 * N, M32)
        want = int(exact + Fraction(1, 2)) % (2 * N)  # floor(x + 1/2) for x >= 0
        assert oracle.modswitch(int(x), N) == want
