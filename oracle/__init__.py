"""CPU TFHE oracle -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg (and its
`--impl reference` arm) may import this package.  The product path (the CUDA
library and its binding) never loads it.

This package wraps tfhe_oracle.c (plain C, compiled with gcc, OpenMP over
independent gates) through ctypes and adds the circuit layer in plain Python
(circuits.py).  It shares no code with the CUDA path; the only module both sides
use is `synth`, which draws the random numbers and holds no TFHE arithmetic.

Paper passages followed (LocPIR, arXiv 2407.19871):
  * encoding f(m) = m/4 - 1/8, Encrypt, Decrypt: Section 2.2 (TFHE bullet list);
  * HomAND = Bootstrap((0, -1/8) + c1 + c2): Section 2.2, EvalGate;
  * the other gates follow the standard TFHE gate constructions the paper defers to.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

from synth import KeyDraws, LweDraws, Params

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tfhe_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

NAND, AND, OR, XOR, XNOR, NOT, MUX = range(7)
OP_NAMES = {"NAND": NAND, "AND": AND, "OR": OR, "XOR": XOR, "XNOR": XNOR, "NOT": NOT, "MUX": MUX}

EIGHTH = 1 << 29  # 1/8 on the torus


def build(force: bool = False) -> str:
    """Compile tfhe_oracle.c into liboracle.so next to it (gcc, -O3, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def lib() -> ctypes.CDLL:
    """The oracle library.  ORACLE_LIB, when set, names a prebuilt copy to load instead; the
    mutation tests use it to run the pins against deliberately broken builds."""
    global _lib
    if _lib is None:
        L = ctypes.CDLL(os.environ.get("ORACLE_LIB") or build())
        c_int, c_size, c_u32 = ctypes.c_int, ctypes.c_size_t, ctypes.c_uint32
        sig = {
            "or_poly_mul_schoolbook": (None, [c_int, _u32p, _u32p, _u32p]),
            "or_poly_mul_karatsuba": (None, [c_int, _u32p, _u32p, _u32p]),
            "or_poly_mul_monomial": (None, [c_int, _u32p, c_int, _u32p]),
            "or_gadget_digits": (None, [c_int, c_int, c_u32, _i32p]),
            "or_ks_digits": (None, [c_int, c_int, c_u32, _u32p]),
            "or_modswitch": (c_u32, [c_u32, c_int]),
            "or_lwe_phase": (None, [c_int, c_size, _u8p, _u32p, _u32p]),
            "or_lwe_encrypt": (None, [c_int, c_size, _u8p, _u32p, _u32p, _u32p, _u32p]),
            "or_keygen_bsk": (None, [c_int, c_int, c_int, c_int, _u8p, _u8p, _u32p, _u32p, _u32p]),
            "or_keygen_ksk": (None, [c_int, c_int, c_int, c_int, _u8p, _u8p, _u32p, _u32p, _u32p]),
            "or_blind_rotate": (None, [c_int, c_int, c_int, c_int, _u32p, _u32p, c_u32, _u32p]),
            "or_sample_extract": (None, [c_int, _u32p, _u32p]),
            "or_key_switch": (None, [c_int, c_int, c_int, c_int, _u32p, _u32p, _u32p]),
            "or_gate_batch": (c_int, [c_int, c_int, c_int, c_int, c_int, c_int, _u32p, _u32p, c_int,
                                      _u32p, _u32p, _u32p, _u32p, c_size, c_int]),
            "or_bootstrap_extract_batch": (None, [c_int, c_int, c_int, c_int, _u32p, _u32p, c_u32,
                                                  _u32p, c_size, c_int]),
            "or_max_threads": (c_int, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def threads() -> int:
    return int(lib().or_max_threads())


def _u32(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint32))


# ---------------------------------------------------------------------------
# Ring and decomposition primitives.
# ---------------------------------------------------------------------------

def poly_mul_schoolbook(a, b) -> np.ndarray:
    a, b = _u32(a), _u32(b)
    out = np.empty_like(a)
    lib().or_poly_mul_schoolbook(len(a), a, b, out)
    return out


def poly_mul_karatsuba(a, b) -> np.ndarray:
    a, b = _u32(a), _u32(b)
    out = np.empty_like(a)
    lib().or_poly_mul_karatsuba(len(a), a, b, out)
    return out


def poly_mul_monomial(v, e: int) -> np.ndarray:
    v = _u32(v)
    out = np.empty_like(v)
    lib().or_poly_mul_monomial(len(v), v, int(e), out)
    return out


def gadget_digits(x: int, lg: int = 3, Bgbit: int = 10) -> np.ndarray:
    d = np.zeros(lg, np.int32)
    lib().or_gadget_digits(lg, Bgbit, int(x) & 0xFFFFFFFF, d)
    return d


def ks_digits(x: int, t: int = 8, basebit: int = 2) -> np.ndarray:
    v = np.zeros(t, np.uint32)
    lib().or_ks_digits(t, basebit, int(x) & 0xFFFFFFFF, v)
    return v


def modswitch(x: int, N: int = 1024) -> int:
    return int(lib().or_modswitch(int(x) & 0xFFFFFFFF, N))


# ---------------------------------------------------------------------------
# Keys, encryption, decryption.
# ---------------------------------------------------------------------------

@dataclass
class Keys:
    params: Params
    s: np.ndarray    # [n] uint8
    S: np.ndarray    # [N] uint8
    bsk: np.ndarray  # [n][2 lg][2][N] uint32 (coefficient domain)
    ksk: np.ndarray  # [N][t][2^basebit][n+1] uint32


def keygen_bsk(d: KeyDraws) -> np.ndarray:
    p = d.params
    bsk = np.empty((p.n, 2 * p.lg, 2, p.N), np.uint32)
    lib().or_keygen_bsk(p.n, p.N, p.lg, p.Bgbit, d.s, d.S, _u32(d.bsk_mask), _u32(d.bsk_noise), bsk)
    return bsk


def keygen_ksk(d: KeyDraws) -> np.ndarray:
    p = d.params
    B = 1 << p.basebit
    ksk = np.empty((p.N, p.t, B, p.n + 1), np.uint32)
    lib().or_keygen_ksk(p.n, p.N, p.t, p.basebit, d.s, d.S, _u32(d.ksk_mask), _u32(d.ksk_noise), ksk)
    return ksk


def keygen(d: KeyDraws) -> Keys:
    """KeyGen (Section 2.2): LWE key s, TRLWE key S, bootstrapping and key-switching keys."""
    return Keys(d.params, d.s, d.S, keygen_bsk(d), keygen_ksk(d))


def encode(bits) -> np.ndarray:
    """f(m) = m/4 - 1/8 as torus32: 1 -> 2^29, 0 -> -2^29."""
    b = np.asarray(bits, dtype=np.uint8)
    return np.where(b != 0, EIGHTH, (1 << 32) - EIGHTH).astype(np.uint32)


def encrypt_mu(s: np.ndarray, mu, draws: LweDraws) -> np.ndarray:
    """(a, <a, s> + e + mu) for each message mu (torus32), masks/noise from draws."""
    mu = _u32(np.atleast_1d(mu))
    cnt, n = draws.mask.shape
    assert cnt == len(mu) and n == len(s)
    out = np.empty((cnt, n + 1), np.uint32)
    lib().or_lwe_encrypt(n, cnt, np.ascontiguousarray(s, np.uint8), _u32(draws.mask),
                         _u32(draws.noise), mu, out)
    return out


def encrypt(s: np.ndarray, bits, draws: LweDraws) -> np.ndarray:
    """Encrypt (Section 2.2) each bit with the encoding f."""
    return encrypt_mu(s, encode(np.atleast_1d(bits)), draws)


def zero_samples(s: np.ndarray, draws: LweDraws) -> np.ndarray:
    """Zero-phase samples (a, <a, s> + e) the client sends with its public key (Algorithm 1's
    inputs: b = a K + e)."""
    return encrypt_mu(s, np.zeros(draws.mask.shape[0], np.uint32), draws)


def preprocess(zero: np.ndarray, bits) -> np.ndarray:
    """Algorithm 1 (Preprocess): S_i[j] + ct_ij, i.e. add the plaintext encoding (0, f(bit))
    of each service bit to the client's zero-phase sample."""
    out = _u32(np.atleast_2d(zero)).copy()
    out[:, -1] = (out[:, -1].astype(np.uint64) + encode(np.atleast_1d(bits)).astype(np.uint64)) & 0xFFFFFFFF
    return out


def trivial(bit: int, n: int) -> np.ndarray:
    """Noiseless, maskless sample (0, f(bit))."""
    c = np.zeros(n + 1, np.uint32)
    c[n] = encode([bit])[0]
    return c


def phase(s: np.ndarray, ct) -> np.ndarray:
    ct = _u32(np.atleast_2d(ct))
    n = ct.shape[1] - 1
    out = np.empty(ct.shape[0], np.uint32)
    lib().or_lwe_phase(n, ct.shape[0], np.ascontiguousarray(s, np.uint8), ct, out)
    return out


def decrypt(s: np.ndarray, ct) -> np.ndarray:
    """Decrypt (Section 2.2): round the phase to +-1/8 and invert f; as int32 the
    phase is positive for 1 (a phase of exactly 0 decodes to 0)."""
    return (phase(s, ct).view(np.int32) > 0).astype(np.uint8)


# ---------------------------------------------------------------------------
# Bootstrapping steps and gates.
# ---------------------------------------------------------------------------

def blind_rotate(p: Params, bsk: np.ndarray, bar, mu: int = EIGHTH) -> np.ndarray:
    bar = _u32(bar)
    acc = np.empty((2, p.N), np.uint32)
    lib().or_blind_rotate(p.n, p.N, p.lg, p.Bgbit, _u32(bsk), bar, mu & 0xFFFFFFFF, acc)
    return acc


def sample_extract(acc: np.ndarray) -> np.ndarray:
    acc = _u32(acc)
    N = acc.shape[-1]
    out = np.empty(N + 1, np.uint32)
    lib().or_sample_extract(N, acc, out)
    return out


def key_switch(p: Params, ksk: np.ndarray, ext) -> np.ndarray:
    ext = _u32(ext)
    out = np.empty(p.n + 1, np.uint32)
    lib().or_key_switch(p.n, p.N, p.t, p.basebit, _u32(ksk), ext, out)
    return out


def bootstrap_extract(keys: Keys, lwe, mu: int = EIGHTH, nthreads: int | None = None) -> np.ndarray:
    """Mod switch + blind rotation + sample extraction of pre-combined LWEs [count][n+1]."""
    p = keys.params
    lwe = _u32(np.atleast_2d(lwe))
    out = np.empty((lwe.shape[0], p.N + 1), np.uint32)
    lib().or_bootstrap_extract_batch(p.n, p.N, p.lg, p.Bgbit, _u32(keys.bsk), lwe, mu, out,
                                     lwe.shape[0], nthreads or threads())
    return out


def gate_batch(keys: Keys, op: int, a, b=None, c=None, nthreads: int | None = None) -> np.ndarray:
    """Evaluate independent gates; out = op(a, b) or, for MUX, a ? b : c."""
    p = keys.params
    a = _u32(np.atleast_2d(a))
    b = a if b is None else _u32(np.atleast_2d(b))
    c = a if c is None else _u32(np.atleast_2d(c))
    out = np.empty_like(a)
    rc = lib().or_gate_batch(p.n, p.N, p.lg, p.Bgbit, p.t, p.basebit, _u32(keys.bsk), _u32(keys.ksk),
                             int(op), a, b, c, out, a.shape[0], nthreads or threads())
    if rc != 0:
        raise ValueError(f"oracle gate_batch failed ({rc})")
    return out
