"""Seeded synthetic inputs shared by the CPU oracle, the GPU tests and the benchmark.

This module only draws random numbers and lays out plaintext workloads.  It holds
none of the TFHE arithmetic: no encryption, no key assembly, no polynomial product,
no gate logic.  Every random number the method consumes (secret key bits, masks,
Gaussian noise) is drawn here and handed to both implementations as an input, so
the oracle and the CUDA path see identical randomness in the same process.

Generator: SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used in counter mode: draw i of stream (seed, s)
is mix64(base(seed, s) + (i + 1) * GAMMA).  Being counter based, any slice of a
stream can be regenerated without generating its prefix.

Gaussian noise: Box-Muller on two 53-bit uniforms in (0, 1]; the real sample z*sigma
is scaled by 2^32 and rounded half away from zero to a torus32 integer (mod 2^32).
Noise is a standard deviation on the torus, as in the paper's Encrypt (Section 2.2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream ids: one independent SplitMix64 stream per purpose.
STREAM_LWE_KEY = 1
STREAM_RLWE_KEY = 2
STREAM_BSK_MASK = 3
STREAM_BSK_NOISE = 4
STREAM_KSK_MASK = 5
STREAM_KSK_NOISE = 6
STREAM_ENC_MASK = 16
STREAM_ENC_NOISE = 17
STREAM_PLAIN = 32


@dataclass(frozen=True)
class Params:
    """TFHE parameter set (ring degree N, LWE dimension n, gadget and key-switch bases)."""

    n: int = 630
    N: int = 1024
    k: int = 1
    Bgbit: int = 10
    lg: int = 3
    basebit: int = 2
    t: int = 8
    sigma_lwe: float = 2.0 ** -15
    sigma_rlwe: float = 2.0 ** -25


DEFAULT = Params()


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _base(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.array([(int(seed) * 0x100000001B3 + int(stream)) & (2**64 - 1)], dtype=np.uint64)
        return _mix64(s + GAMMA)[0]


def splitmix64(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+count-1 of stream (seed, stream) as uint64."""
    base = _base(seed, stream)
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        return _mix64(base + idx * GAMMA)


def uniform_u32(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform torus32 values: the low 32 bits of each draw."""
    return (splitmix64(seed, stream, count, offset) & np.uint64(0xFFFFFFFF)).astype(np.uint32)


def bits(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform bits (the top bit of each draw) as uint8."""
    return (splitmix64(seed, stream, count, offset) >> np.uint64(63)).astype(np.uint8)


def gaussian_t32(seed: int, stream: int, count: int, sigma: float, offset: int = 0) -> np.ndarray:
    """Discretised Gaussian torus32 noise with standard deviation sigma (torus units)."""
    if sigma == 0.0 or count == 0:
        return np.zeros(count, dtype=np.uint32)
    d = splitmix64(seed, stream, 2 * count, 2 * offset)
    u = ((d >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)  # (0, 1]
    u1, u2 = u[0::2], u[1::2]
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
    x = z * sigma * 4294967296.0
    r = np.sign(x) * np.floor(np.abs(x) + 0.5)
    return (r.astype(np.int64) & 0xFFFFFFFF).astype(np.uint32)


@dataclass
class KeyDraws:
    """All randomness a key generation consumes.

    s:          [n] LWE secret key bits.
    S:          [N] TRLWE secret key bits (k = 1).
    bsk_mask:   [n][(k+1)*lg][N] uniform mask polynomial of each TRGSW row.
    bsk_noise:  [n][(k+1)*lg][N] Gaussian noise polynomial of each row (sigma_rlwe).
    ksk_mask:   [N][t][2^basebit][n] uniform LWE masks of the key-switching key.
    ksk_noise:  [N][t][2^basebit] Gaussian noise of each key-switching sample (sigma_lwe).
    """

    params: Params
    s: np.ndarray
    S: np.ndarray
    bsk_mask: np.ndarray
    bsk_noise: np.ndarray
    ksk_mask: np.ndarray
    ksk_noise: np.ndarray


def key_draws(seed: int, p: Params = DEFAULT, *, noiseless: bool = False,
              zero_masks: bool = False) -> KeyDraws:
    """Key randomness for seed.  noiseless sets all noise to 0; zero_masks sets all
    masks to 0 (with noiseless this gives the trivial keys whose bootstrap has a
    closed form)."""
    rows = (p.k + 1) * p.lg
    B = 1 << p.basebit
    s = bits(seed, STREAM_LWE_KEY, p.n)
    S = bits(seed, STREAM_RLWE_KEY, p.N)
    nb = p.n * rows * p.N
    nk = p.N * p.t * B
    if zero_masks:
        bm = np.zeros(nb, np.uint32)
        km = np.zeros(nk * p.n, np.uint32)
    else:
        bm = uniform_u32(seed, STREAM_BSK_MASK, nb)
        km = uniform_u32(seed, STREAM_KSK_MASK, nk * p.n)
    sr = 0.0 if noiseless else p.sigma_rlwe
    sl = 0.0 if noiseless else p.sigma_lwe
    bn = gaussian_t32(seed, STREAM_BSK_NOISE, nb, sr)
    kn = gaussian_t32(seed, STREAM_KSK_NOISE, nk, sl)
    return KeyDraws(p, s, S, bm.reshape(p.n, rows, p.N), bn.reshape(p.n, rows, p.N),
                    km.reshape(p.N, p.t, B, p.n), kn.reshape(p.N, p.t, B))


@dataclass
class LweDraws:
    """Randomness of `count` LWE encryptions: masks [count][n], noise [count]."""

    mask: np.ndarray
    noise: np.ndarray


def lwe_draws(seed: int, count: int, p: Params = DEFAULT, *, offset: int = 0,
              noiseless: bool = False, stream: int = STREAM_ENC_MASK) -> LweDraws:
    m = uniform_u32(seed, stream, count * p.n, offset * p.n).reshape(count, p.n)
    e = gaussian_t32(seed, stream + 1, count, 0.0 if noiseless else p.sigma_lwe, offset)
    return LweDraws(m, e)


# ----------------------------------------------------------------------------
# Plaintext workload recipes (no encryption here).
# ----------------------------------------------------------------------------

def int_to_bits(v: int, l: int) -> np.ndarray:
    """Bits of the l-bit two's-complement pattern of v, least significant first."""
    v &= (1 << l) - 1
    return np.array([(v >> i) & 1 for i in range(l)], dtype=np.uint8)


def nand_pairs(seed: int, count: int) -> tuple[np.ndarray, np.ndarray]:
    """Uniform plaintext bit pairs for the gate-bootstrapping microbenchmark."""
    b = bits(seed, STREAM_PLAIN, 2 * count)
    return b[0::2].copy(), b[1::2].copy()


@dataclass
class CityQuery:
    """One query of the city-batch workload: point (x, y), one box, one service."""

    x: int
    y: int
    box: tuple[int, int, int, int]  # X1, X2, Y1, Y2
    service: np.ndarray  # [m] bits, least significant first


def city_batch(seed: int, count: int, l: int = 32, m: int = 256) -> list[CityQuery]:
    """Box bounds uniform in [0, 2^l) sorted (lo < hi); half of the points uniform
    inside the box, the other half uniform in the box widened by its own width on each
    side (clamped to [0, 2^l)) and outside it; m uniform service bits."""
    L = 1 << l
    out: list[CityQuery] = []
    draws = splitmix64(seed, STREAM_PLAIN, 16 * count)
    svc = bits(seed, STREAM_PLAIN + 1, count * m).reshape(count, m)
    pos = 0

    def nxt() -> int:
        nonlocal pos
        v = int(draws[pos]) ; pos += 1
        return v

    def bound_pair() -> tuple[int, int]:
        while True:
            a, b = nxt() % L, nxt() % L
            if a != b:
                return (min(a, b), max(a, b))

    for q in range(count):
        (x1, x2), (y1, y2) = bound_pair(), bound_pair()
        inside = (q % 2) == 0

        def coord(lo: int, hi: int) -> int:
            if inside:
                return lo + nxt() % (hi - lo)
            w = hi - lo
            a, b = max(0, lo - w), min(L, hi + w)
            outer = (lo - a) + (b - hi)
            if outer == 0:
                return lo + nxt() % (hi - lo)
            r = nxt() % outer
            return a + r if r < lo - a else hi + (r - (lo - a))

        x = coord(x1, x2)
        y = coord(y1, y2)
        out.append(CityQuery(x, y, (x1, x2, y1, y2), svc[q].copy()))
    return out


@dataclass
class MultiBoxQuery:
    x: int
    y: int
    l: int
    boxes: list[tuple[int, int, int, int]]
    services: np.ndarray  # [B_x][m]


def multibox_batch(seed: int, count: int, m: int = 512, max_boxes: int = 128,
                   widths: tuple[int, ...] = (16, 24, 32)) -> list[MultiBoxQuery]:
    """Uneven workload: per query B_x ~ U{1..max_boxes}, l ~ U(widths), bounds uniform
    sorted pairs, point uniform in [0, 2^l)^2, m uniform service bits per box."""
    out: list[MultiBoxQuery] = []
    d = splitmix64(seed, STREAM_PLAIN, count * (4 + 4 * max_boxes + 8))
    pos = 0
    for q in range(count):
        bx = 1 + int(d[pos]) % max_boxes
        l = widths[int(d[pos + 1]) % len(widths)]
        L = 1 << l
        x, y = int(d[pos + 2]) % L, int(d[pos + 3]) % L
        pos += 4
        boxes = []
        for _ in range(bx):
            a, b, c, e = (int(d[pos + i]) % L for i in range(4))
            pos += 4
            boxes.append((min(a, b), max(a, b), min(c, e), max(c, e)))
        svc = bits(seed, STREAM_PLAIN + 2 + q, bx * m).reshape(bx, m)
        out.append(MultiBoxQuery(x, y, l, boxes, svc))
    return out
