"""Pins of the oracle's bootstrap: closed forms under trivial keys, extraction and
key switching against independent arithmetic, noise against the TFHE variance
bound, and gate truth tables."""
import math

import numpy as np
import pytest

import oracle
import synth

M32 = 1 << 32


def _rot(v, e, N):
    """X^e v by index arithmetic (independent of the oracle's routine)."""
    out = np.zeros(N, dtype=np.int64)
    for i in range(N):
        d = (i + e) % (2 * N)
        if d < N:
            out[d] += int(v[i])
        else:
            out[d - N] -= int(v[i])
    return (out % M32).astype(np.uint32)


def _ms(x, N=1024):
    return ((int(x) + (1 << 20)) % M32) >> 21


def test_blind_rotate_closed_form_trivial_keys(keys_trivial):
    """With noiseless, maskless keys every external product is exact, so the
    accumulator ends at (0, X^(-phi) v), phi = bar_n - sum_i bar_i s_i mod 2N."""
    p = keys_trivial.params
    s = keys_trivial.s
    for trial in range(3):
        lwe = synth.uniform_u32(51, trial, p.n + 1)
        bar = np.array([_ms(x) for x in lwe], np.uint32)
        phi = (int(bar[p.n]) - sum(int(bar[i]) * int(s[i]) for i in range(p.n))) % (2 * p.N)
        acc = oracle.blind_rotate(p, keys_trivial.bsk, bar)
        v = np.full(p.N, 1 << 29, np.uint32)
        np.testing.assert_array_equal(acc[0], np.zeros(p.N, np.uint32))
        np.testing.assert_array_equal(acc[1], _rot(v, (2 * p.N - phi) % (2 * p.N), p.N))


def test_sample_extract_phase_is_coefficient_zero(keys):
    """Phase of the extracted N-LWE under S equals coefficient 0 of b - a S."""
    N = keys.params.N
    acc = np.stack([synth.uniform_u32(52, 1, N), synth.uniform_u32(52, 2, N)])
    ext = oracle.sample_extract(acc)
    S = keys.S.astype(np.int64)
    # (a S)_0 = a_0 S_0 - sum_{j>=1} a_{N-j} S_j
    aS0 = int(acc[0, 0]) * int(S[0]) - sum(int(acc[0, N - j]) * int(S[j]) for j in range(1, N))
    want = (int(acc[1, 0]) - aS0) % M32
    got = (int(ext[N]) - sum(int(ext[j]) * int(S[j]) for j in range(N))) % M32
    assert got == want


def test_key_switch_closed_form_trivial_ksk(keys_trivial):
    """Maskless, noiseless KSK: the output is (0, b' - sum_i S_i round16(a'_i))."""
    p = keys_trivial.params
    ext = synth.uniform_u32(53, 1, p.N + 1)
    out = oracle.key_switch(p, keys_trivial.ksk, ext)
    assert not out[:p.n].any()
    r16 = lambda x: ((((int(x) + (1 << 15)) % M32) >> 16) << 16) % M32
    want = (int(ext[p.N]) - sum(r16(ext[i]) * int(keys_trivial.S[i]) for i in range(p.N))) % M32
    assert int(out[p.n]) == want


def test_key_switch_phase_error_bounded(keys):
    """KS keeps the phase within the rounding and key noise it adds (loose 6-sigma bound)."""
    p = keys.params
    ext = synth.uniform_u32(54, 1, p.N + 1)
    out = oracle.key_switch(p, keys.ksk, ext)
    ph_in = (int(ext[p.N]) - sum(int(ext[i]) * int(keys.S[i]) for i in range(p.N))) % M32
    ph_out = int(oracle.phase(keys.s, out)[0])
    err = ((ph_out - ph_in + M32 // 2) % M32 - M32 // 2) / M32
    sd = math.sqrt(p.N * p.t * p.sigma_lwe ** 2 + p.N / 2 * (2.0 ** -16) ** 2 / 12)
    assert abs(err) < 6 * sd + p.N * 2.0 ** -17


@pytest.mark.parametrize("op", ["NAND", "AND", "OR", "XOR", "XNOR"])
def test_gate_closed_form_trivial_keys(keys_trivial, op):
    """Under trivial keys a gate output is exactly (0, +-1/8), + iff the switched
    phase of the pre-combined sample lies in [0, N)."""
    p = keys_trivial.params
    cnt = 4
    a = oracle.encrypt(keys_trivial.s, [0, 0, 1, 1], synth.lwe_draws(55, cnt, noiseless=True))
    b = oracle.encrypt(keys_trivial.s, [0, 1, 0, 1], synth.lwe_draws(56, cnt, noiseless=True))
    out = oracle.gate_batch(keys_trivial, oracle.OP_NAMES[op], a, b)
    truth = {"NAND": [1, 1, 1, 0], "AND": [0, 0, 0, 1], "OR": [0, 1, 1, 1], "XOR": [0, 1, 1, 0], "XNOR": [1, 0, 0, 1]}[op]
    for g in range(cnt):
        assert not out[g, :p.n].any()
        assert int(out[g, p.n]) == (1 << 29 if truth[g] else M32 - (1 << 29))


def test_gate_truth_tables_noiseless_keys(keys_noiseless):
    ka = keys_noiseless
    A = [0, 0, 1, 1]
    B = [0, 1, 0, 1]
    a = oracle.encrypt(ka.s, A, synth.lwe_draws(57, 4))
    b = oracle.encrypt(ka.s, B, synth.lwe_draws(58, 4))
    table = {"NAND": [1, 1, 1, 0], "AND": [0, 0, 0, 1], "OR": [0, 1, 1, 1], "XOR": [0, 1, 1, 0], "XNOR": [1, 0, 0, 1]}
    for name, want in table.items():
        got = oracle.decrypt(ka.s, oracle.gate_batch(ka, oracle.OP_NAMES[name], a, b))
        assert got.tolist() == want, name
    assert oracle.decrypt(ka.s, oracle.gate_batch(ka, oracle.NOT, a)).tolist() == [1, 1, 0, 0]
    sel = [0, 0, 0, 0, 1, 1, 1, 1]
    x1 = [0, 0, 1, 1, 0, 0, 1, 1]
    x0 = [0, 1, 0, 1, 0, 1, 0, 1]
    cs = oracle.encrypt(ka.s, sel, synth.lwe_draws(59, 8))
    c1 = oracle.encrypt(ka.s, x1, synth.lwe_draws(60, 8))
    c0 = oracle.encrypt(ka.s, x0, synth.lwe_draws(61, 8))
    got = oracle.decrypt(ka.s, oracle.gate_batch(ka, oracle.MUX, cs, c1, c0))
    assert got.tolist() == [x1[i] if sel[i] else x0[i] for i in range(8)]


@pytest.mark.slow
def test_bootstrap_noise_variance_within_tfhe_bound(keys):
    """Output phase error of NAND bootstraps: mean ~ 0, variance between half the
    expected external-product + key-switch variance and the worst-case bound
    (TFHE, J. Cryptology 2020: Var_BR = n (k+1) lg N E[d^2] sigma_rlwe^2,
    E[d^2] ~ Bg^2/12 expected, (Bg/2)^2 worst case; Var_KS = N t sigma_lwe^2)."""
    p = keys.params
    cnt = 64
    A = synth.bits(62, 1, cnt)
    B = synth.bits(62, 2, cnt)
    a = oracle.encrypt(keys.s, A, synth.lwe_draws(63, cnt))
    b = oracle.encrypt(keys.s, B, synth.lwe_draws(64, cnt))
    out = oracle.gate_batch(keys, oracle.NAND, a, b)
    truth = 1 - (A & B)
    ph = oracle.phase(keys.s, out).astype(np.int64)
    ideal = np.where(truth == 1, 1 << 29, M32 - (1 << 29))
    err = (((ph - ideal + M32 // 2) % M32) - M32 // 2) / M32
    Bg = 1 << p.Bgbit
    base = p.n * (p.k + 1) * p.lg * p.N * p.sigma_rlwe ** 2
    var_ks = p.N * p.t * p.sigma_lwe ** 2
    expected = base * Bg ** 2 / 12 + var_ks
    bound = base * (Bg / 2) ** 2 + var_ks + p.N * (2.0 ** -16) ** 2 / 12
    var = float(np.mean(err ** 2))
    assert abs(err.mean()) < 4 * math.sqrt(bound / cnt)
    assert 0.5 * expected < var < bound
    assert (oracle.decrypt(keys.s, out) == truth).all()
