"""The crafted edge case of the external product (tests/crt_edge.py), on the CPU: it reaches
the magnitudes that decide the GPU engine's exactness, and the oracle's blind rotation gives
its closed form on it.  TFHE's external product (J. Cryptology 2020), to which the paper's
EvalGate (Section 2.2) defers."""
import os
import re

import numpy as np

import oracle
import synth
from crt_edge import HALF, MU_EDGE, crafted_bsk, crafted_lwes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _prime(name: str) -> int:
    src = open(os.path.join(ROOT, "paper_2407_19871_gb300", "csrc", "common.cuh")).read()
    return int(re.search(rf"constexpr\s+uint32_t\s+{name}\s*=\s*(\d+)u?;", src).group(1))


def _negacyclic_int(d: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Exact integer negacyclic product of two int64 polynomials (|coefficients| small enough
    that every partial sum fits int64)."""
    N = len(d)
    full = np.convolve(d, b)              # degree 2N - 2, exact in int64 here
    out = full[:N].copy()
    out[:N - 1] -= full[N:]
    return out


def _centred(w: np.ndarray) -> np.ndarray:
    return w.astype(np.int64) - ((w.astype(np.int64) >> 31) << 32)


def test_first_step_reaches_the_crt_edge():
    """Sample 0 (a_0 = b = 2^31) under the all-0x80000000 key: the integer sum of the first
    external product peaks at 3 * 2^50 ~ 2^51.6, within the design bound 6 * 1024 * 512 * 2^31
    and the centred CRT range p0 p1 / 2, and far above the ~2^46 random inputs reach."""
    p = synth.DEFAULT
    bsk = crafted_bsk(p)
    lwe = crafted_lwes(p, 1)[0]
    abar = [oracle.modswitch(int(x), p.N) for x in lwe]
    assert abar[0] == p.N and abar[p.n] == p.N and not any(abar[1:p.n])
    # ACC = (0, X^-N v) = (0, -mu); D = X^N ACC - ACC = -2 ACC = (0, 2 mu).
    d_body = oracle.gadget_digits((2 * MU_EDGE) & 0xFFFFFFFF, p.lg, p.Bgbit)
    d_mask = oracle.gadget_digits(0, p.lg, p.Bgbit)
    assert d_body.tolist() == [-512] * p.lg and d_mask.tolist() == [0] * p.lg
    peak = 0
    for comp in range(2):
        s = np.zeros(p.N, np.int64)
        for r in range(2 * p.lg):
            dig = (d_mask if r < p.lg else d_body)[r % p.lg]
            s += _negacyclic_int(np.full(p.N, dig, np.int64), _centred(bsk[0, r, comp]))
        # closed form of constant polynomials: coefficient k = lg (2k + 2 - N) d b
        k = np.arange(p.N, dtype=np.int64)
        assert np.array_equal(s, p.lg * (2 * k + 2 - p.N) * (-512) * (-HALF))
        peak = max(peak, int(np.abs(s).max()))
    assert peak == 3 * 2 ** 50
    assert peak > 2 ** 51.5
    bound = 2 * p.lg * p.N * 512 * 2 ** 31
    assert peak <= bound
    assert peak < _prime("PRIME0") * _prime("PRIME1") // 2


def test_low_bit_variant_stays_near_the_edge():
    """Key words within 2^24 of -2^31: the first step's sums still exceed 2^51.5."""
    p = synth.DEFAULT
    bsk = crafted_bsk(p, low_bits=24, seed=3)
    d = np.full(p.N, -512, np.int64)
    s = sum(_negacyclic_int(d, _centred(bsk[0, r, 1])) for r in range(p.lg, 2 * p.lg))
    assert np.abs(s).max() > 2 ** 51.5


def test_oracle_closed_form_on_the_edge_case():
    """Every edge step adds a multiple of 2^40 to each coefficient, i.e. 0 mod 2^32, so the
    accumulator stays (0, -mu) through all n steps: the extracted sample is exactly
    (0, ..., 0, -mu).  The oracle's exact products must reproduce this on samples with one,
    all and a random subset of edge steps."""
    p = synth.DEFAULT
    keys = oracle.Keys(p, np.zeros(p.n, np.uint8), np.zeros(p.N, np.uint8), crafted_bsk(p),
                       np.zeros(1, np.uint32))
    lwe = crafted_lwes(p, 3, seed=5)
    ext = oracle.bootstrap_extract(keys, lwe, mu=MU_EDGE)
    assert not ext[:, :p.N].any()
    assert (ext[:, p.N] == (1 << 32) - MU_EDGE).all()
