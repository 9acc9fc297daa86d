"""The exactness argument of the GPU product engine, checked on the CPU from the constants the
CUDA sources compile with (no GPU, no oracle): the two NTT primes, the lazy-reduction bounds
of the forward transform and the multiply-accumulate, and the centred CRT range that makes
every negacyclic product mod 2^32 exact."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N, LG, BG = 1024, 3, 1 << 10


def _const(name: str) -> int:
    src = open(os.path.join(ROOT, "paper_2407_19871_gb300", "csrc", "common.cuh")).read()
    m = re.search(rf"constexpr\s+uint32_t\s+{name}\s*=\s*(\d+)u?;", src)
    assert m, name
    return int(m.group(1))


PRIMES = [_const("PRIME0"), _const("PRIME1")]


@pytest.mark.parametrize("p", PRIMES)
def test_primes_support_negacyclic_length_1024(p):
    sympy = pytest.importorskip("sympy")
    assert sympy.isprime(p)
    assert (p - 1) % (2 * N) == 0                     # a primitive 2N-th root of unity psi exists
    g = next(g for g in range(2, 100) if pow(g, (p - 1) // 2, p) == p - 1)
    psi = pow(g, (p - 1) // (2 * N), p)
    assert pow(psi, N, p) == p - 1                    # psi^N = -1: the negacyclic twist


@pytest.mark.parametrize("p", PRIMES)
def test_lazy_forward_transform_and_mac_fit_their_words(p):
    """Inputs in [0, 2p) grow by at most 2p per Cooley-Tukey stage: after log2 N = 10 stages
    they stay below 22p, which must fit 32 bits.  The multiply-accumulate adds (k+1) lg = 6
    products of a transformed digit (< 22p) and a key word (< p) in 64 bits; its Montgomery
    reduction (T + m p) / 2^32 then lies below 7p, still a 32-bit value."""
    assert 22 * p < 2 ** 32
    T = 6 * (22 * p - 1) * (p - 1)
    assert T < 2 ** 64
    assert (T + (2 ** 32 - 1) * p) // 2 ** 32 < 7 * p < 2 ** 32
    # A lazy Shoup product y w - floor(y w' / 2^32) p of y < 2^32 lies in [0, 2p).
    assert 2 * p < 2 ** 32


@pytest.mark.parametrize("p", PRIMES)
def test_split_kernel_per_product_reduction_bounds(p):
    """The split blind rotation reduces each product on its own: x < 22p and a key word < p give
    x k < 22 p^2 < 2^32 p, so the Montgomery result lies in [0, 2p); the 6 digit rows' results
    summed in shared memory stay below 12p < 2^32."""
    assert 22 * p * p < 2 ** 32 * p
    assert ((22 * p - 1) * (p - 1) + (2 ** 32 - 1) * p) // 2 ** 32 < 2 * p
    assert 6 * 2 * p < 2 ** 32


def test_centred_crt_range_covers_every_product():
    """|sum_r sum_j d * b| <= (k+1) lg * N * (Bg/2) * 2^31 with digits in [-Bg/2, Bg/2) and
    key words centred in [-2^31, 2^31): the two-prime product must exceed twice that bound so
    the centred lift is the exact integer, whose residue mod 2^32 is the torus result."""
    p0, p1 = PRIMES
    bound = 2 * LG * N * (BG // 2) * 2 ** 31
    assert p0 * p1 > 2 * bound
    assert p0 != p1
