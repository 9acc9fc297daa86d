"""Pins of the oracle's client side: encoding, Encrypt/Decrypt, key structure, sizes.

Phases are recomputed here with independent numpy arithmetic (exact integer dot
products and convolutions), not with the oracle's own routines."""
import json
import math
import os

import numpy as np

import oracle
import synth

M32 = 1 << 32
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _negacyclic_exact(a, b):
    N = len(a)
    full = np.convolve(np.asarray(a, dtype=object), np.asarray(b, dtype=object))
    full = np.concatenate([full, np.zeros(2 * N - len(full), dtype=object)])
    return np.array([(int(full[j]) - int(full[j + N])) % M32 for j in range(N)], dtype=np.uint64)


def test_encoding_is_m_over_4_minus_one_eighth():
    # f(m) = m/4 - 1/8 (Section 2.2): 1 -> 1/8, 0 -> -1/8 = 7/8.
    assert oracle.encode([1, 0]).tolist() == [M32 // 8, M32 - M32 // 8]


def test_encrypt_phase_is_message_plus_noise(keys):
    p = keys.params
    bits = synth.bits(31, 1, 64)
    dr = synth.lwe_draws(31, 64)
    ct = oracle.encrypt(keys.s, bits, dr)
    s64 = keys.s.astype(np.uint64)
    dot = (ct[:, :p.n].astype(np.uint64) * s64).sum(axis=1) % M32
    ph = (ct[:, p.n].astype(np.uint64) - dot) % M32
    want = (oracle.encode(bits).astype(np.uint64) + dr.noise.astype(np.uint64)) % M32
    np.testing.assert_array_equal(ph, want)
    np.testing.assert_array_equal(oracle.decrypt(keys.s, ct), bits)
    # Masks are the drawn uniform values.
    np.testing.assert_array_equal(ct[:, :p.n], dr.mask)


def test_decrypt_needs_error_below_one_sixteenth(keys):
    # Decrypt rounds to the nearest of +-1/8, correct iff |e| < 1/16 (Section 2.2).
    n = keys.params.n
    for bit in (0, 1):
        for e in (-(M32 // 16) + 1, M32 // 16 - 1):
            c = oracle.trivial(bit, n)
            c[n] = (int(c[n]) + e) % M32
            assert oracle.decrypt(keys.s, c)[0] == bit


def test_noise_has_requested_stddev():
    e = synth.gaussian_t32(41, 1, 200000, 2.0 ** -15).view(np.int32).astype(np.float64) / M32
    assert abs(e.mean()) < 5 * 2.0 ** -15 / math.sqrt(200000)
    assert abs(e.std() / 2.0 ** -15 - 1) < 0.01


def test_bsk_rows_encrypt_key_bits(keys):
    """Row r = c lg + p of BSK_i has phase e_r - s_i g_p S(X) (c = 0: the gadget term sits
    in the mask) or e_r + s_i g_p (c = 1: in the body), g_p = 2^(32 - 10(p+1))."""
    p = keys.params
    d = synth.key_draws(0)
    S = keys.S.astype(np.uint64)
    for i in (0, 1, 317, p.n - 1):
        for r in range(2 * p.lg):
            a = keys.bsk[i, r, 0].astype(np.uint64)
            b = keys.bsk[i, r, 1].astype(np.uint64)
            ph = (b - _negacyclic_exact(a, S)) % M32
            c, q = divmod(r, p.lg)
            g = int(keys.s[i]) << (32 - 10 * (q + 1))
            want = d.bsk_noise[i, r].astype(np.uint64).copy()
            if c == 0:
                want = (want - (g * S) % M32) % M32
            else:
                want[0] = (int(want[0]) + g) % M32
            np.testing.assert_array_equal(ph, want)


def test_ksk_samples_encrypt_scaled_key_bits(keys):
    p = keys.params
    d = synth.key_draws(0)
    s64 = keys.s.astype(np.uint64)
    for i in (0, 5, p.N - 1):
        for j in range(p.t):
            for v in range(4):
                row = keys.ksk[i, j, v].astype(np.uint64)
                ph = (int(row[p.n]) - int((row[:p.n] * s64).sum())) % M32
                want = (int(d.ksk_noise[i, j, v]) + v * int(keys.S[i]) * (1 << (32 - 2 * (j + 1)))) % M32
                assert ph == want


def test_ciphertext_sizes_match_paper():
    g = json.load(open(os.path.join(GOLD, "sizes.json")))
    kib = lambda n, count: count * (n + 1) * 4 / 1024
    n80, n128 = g["n"]["lambda80"], g["n"]["lambda128"]
    # The paper truncates these sizes to the printed digits.
    assert math.floor(kib(n80, 1) * 100) / 100 == g["tlwe_kb"]["lambda80"]
    assert math.floor(kib(n80, 81)) == g["samples81_kb"]["lambda80"]
    assert math.floor(kib(n128, 81)) == g["samples81_kb"]["lambda128"]
    for lam, n in (("lambda80", n80), ("lambda128", n128)):
        for l, kb in g["gps_kb"][lam].items():
            got = kib(n, int(l))
            assert math.floor(got * 10) / 10 == kb or math.floor(got) == kb
    assert synth.DEFAULT.n == n128


def test_preprocess_alg1_phase_and_decryption(keys):
    """Algorithm 1: the zero-phase sample plus (0, f(bit)) has phase f(bit) + e exactly and
    decrypts to the bit."""
    n, cnt = keys.params.n, 40
    bits = synth.bits(81, 1, cnt)
    dr = synth.lwe_draws(81, cnt)
    zero = oracle.zero_samples(keys.s, dr)
    ph0 = oracle.phase(keys.s, zero)
    np.testing.assert_array_equal(ph0, dr.noise)  # phase 0 + e
    ct = oracle.preprocess(zero, bits)
    want = (oracle.encode(bits).astype(np.uint64) + dr.noise.astype(np.uint64)) % M32
    np.testing.assert_array_equal(oracle.phase(keys.s, ct), want)
    np.testing.assert_array_equal(oracle.decrypt(keys.s, ct), bits)
    np.testing.assert_array_equal(ct[:, :n], zero[:, :n])
