"""Inputs that drive the external product of the blind rotation to the edge of its exactness
argument (TFHE's external product, J. Cryptology 2020, which the paper's EvalGate in Section 2.2
defers to).

One CMux step adds sum_r dig_r(X) * BSK_i[r](X) to the accumulator, a negacyclic product whose
integer coefficients are bounded by (k+1) lg N (Bg/2) 2^31 = 6 * 1024 * 512 * 2^31 ~ 2^52.6 when
digits lie in [-512, 511] and key words are read centred in [-2^31, 2^31).  Random keys and
ciphertexts only reach about 2^46.  The crafted case below reaches 3 * 2^50 ~ 2^51.6:

* every bootstrapping-key word is 0x80000000 (centred -2^31);
* the test vector is mu = 0x3FEFFBFF, so that 2 mu + OFF = 2^32: a body difference of 2 mu
  decomposes into the digits -512, -512, -512;
* a mask or body word of 2^31 switches to 1024 = N, and X^N = -1, so with bbar = 1024 the
  accumulator starts at (0, -v) and a step with abar_i = 1024 has D = -2 ACC = (0, 2 mu).

Each body digit row is then the constant polynomial -512, and the product of two constant
polynomials has coefficient k = (2k + 2 - N) d b: up to N * 512 * 2^31 = 2^50 per row, three rows
per component.  Every such sum is 0 mod 2^32, so the accumulator keeps (0, -mu) step after step
and every step with abar_i = 1024 sits at the edge.  Variants add random low bits to the key
words (values still within 2^24 of -2^31), which makes the results non-trivial mod 2^32 while the
first step stays near the edge.

Test infrastructure only: shared by the CPU check that the case reaches the edge and the GPU
parity tests that run it.
"""
from __future__ import annotations

import numpy as np

import synth

MU_EDGE = 0x3FEFFBFF
HALF = 1 << 31


def crafted_bsk(p, low_bits: int = 0, seed: int = 0) -> np.ndarray:
    """[n][2 lg][2][N] key words 0x80000000, plus uniform low bits below 2^low_bits."""
    bsk = np.full((p.n, 2 * p.lg, 2, p.N), HALF, np.uint32)
    if low_bits:
        r = synth.uniform_u32(seed, 950, bsk.size).reshape(bsk.shape)
        bsk |= r & np.uint32((1 << low_bits) - 1)
    return bsk


def crafted_lwes(p, count: int, seed: int = 0) -> np.ndarray:
    """count LWE samples with b = 2^31.  Sample 0 has a_0 = 2^31 and every other mask word 0 (one
    edge step); sample 1 has every mask word 2^31 (n edge steps); later samples draw each mask
    word from {0, 2^31} (a random subset of edge steps)."""
    lwe = np.zeros((count, p.n + 1), np.uint32)
    lwe[:, p.n] = HALF
    if count > 0:
        lwe[0, 0] = HALF
    if count > 1:
        lwe[1, :p.n] = HALF
    if count > 2:
        pick = synth.bits(seed, 951, (count - 2) * p.n).reshape(count - 2, p.n)
        lwe[2:, :p.n] = pick.astype(np.uint32) * np.uint32(HALF)
    return lwe
