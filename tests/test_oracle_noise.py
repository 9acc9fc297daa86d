"""Statistical pins of the oracle's noise against TFHE's variance formulas (Chillotti et al.,
J. Cryptology 2020: external product and key switch), over more than 10^4 samples each.

Every coefficient j of a blind-rotated accumulator carries its own external-product error, with
the same law as coefficient 0 (the one a gate extracts), so one blind rotation yields N = 1024
samples.  The ideal accumulator is exactly X^-phi v (phi the rounded phase), so each error is
known without decrypting a gate.  The expected variances, with E[d^2] = Bg^2 / 12 for uniform
gadget digits:
  blind rotation: Var_BR = n (k+1) lg N (Bg^2 / 12) sigma_rlwe^2   (2^-11.70 here)
  key switch:     digits v in {0, 1, 2, 3} (uniform, not centred) select key rows whose noise
                  is fixed per key, so a key switch adds a key-dependent offset
                  -sum_{i,j} (e_ij1 + e_ij2 + e_ij3) / 4 plus a zero-mean error of variance
                  Var_KS = N t (9/16) sigma_lwe^2 + |S| 2^-32 / 12   (2^-17.8); averaged over
                  keys the mean square is N t (3/4) sigma_lwe^2, below the N t sigma_lwe^2
                  that counts every digit as non-zero
  gate output:    Var_BR + Var_KS;  MUX output: 2 Var_BR + Var_KS   (u1 + u2 before the switch)
"""
import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.slow
M32 = 1 << 32


def _centred(x) -> np.ndarray:
    x = np.asarray(x, np.int64) % M32
    return np.where(x >= M32 // 2, x - M32, x)


def _negacyclic(a: np.ndarray, S: np.ndarray) -> np.ndarray:
    """(a S) mod (X^N + 1) mod 2^32 for a binary S, by exact int64 convolution (numpy only)."""
    N = len(a)
    full = np.convolve(np.asarray(a, np.int64), np.asarray(S, np.int64))
    out = full[:N].copy()
    out[:N - 1] -= full[N:]
    return out % M32


def _ideal_acc(p, bar, s, mu):
    """Phase of X^-phi v with v_j = mu: coefficient j is mu when j + phi mod 2N < N, else -mu."""
    phi = (int(bar[p.n]) - sum(int(bar[i]) * int(s[i]) for i in range(p.n))) % (2 * p.N)
    j = np.arange(p.N)
    return np.where((j + phi) % (2 * p.N) < p.N, mu, M32 - mu).astype(np.int64)


def _acc_errors(keys, lwes, mu=oracle.EIGHTH):
    """Blind-rotate each LWE (oracle, one thread per call) and return, per input, the N
    coefficient errors of the accumulator's phase under S as fractions of the torus
    ([count][N]), the accumulators, and their ideal phases X^-phi v ([count][N], int64)."""
    p = keys.params
    bars = [np.array([oracle.modswitch(int(x), p.N) for x in lwe], np.uint32) for lwe in lwes]
    with ThreadPoolExecutor(max_workers=oracle.threads()) as ex:
        accs = list(ex.map(lambda b: oracle.blind_rotate(p, keys.bsk, b, mu), bars))
    errs, ideals = [], []
    for bar, acc in zip(bars, accs):
        ph = (acc[1].astype(np.int64) - _negacyclic(acc[0], keys.S)) % M32
        ideal = _ideal_acc(p, bar, keys.s, mu)
        errs.append(_centred(ph - ideal) / M32)
        ideals.append(ideal)
    return np.array(errs), accs, np.array(ideals)


def _extract(acc, j):
    """N-LWE (a', b') under S whose phase is coefficient j of the accumulator's phase:
    (a S)_j = sum_{k<=j} a_{j-k} S_k - sum_{k>j} a_{N+j-k} S_k."""
    a = acc[0].astype(np.int64)
    N = len(a)
    k = np.arange(N)
    ap = np.where(k <= j, a[(j - k) % N], -a[(N + j - k) % N]) % M32
    return np.concatenate([ap, [int(acc[1][j])]]).astype(np.uint32)


def _expected(p, S=None):
    Bg = 1 << p.Bgbit
    base = p.n * (p.k + 1) * p.lg * p.N * p.sigma_rlwe ** 2
    var_br = base * Bg ** 2 / 12
    bound_br = base * (Bg / 2) ** 2
    ones = p.N / 2 if S is None else int(np.sum(S))
    var_ks = p.N * p.t * (9 / 16) * p.sigma_lwe ** 2 + ones * 2.0 ** -32 / 12
    return var_br, bound_br, var_ks


def _ks_offset(keys) -> float:
    """The key switch's key-dependent mean error, from the key-switching key's own noise: each
    row KSK[i][j][v] has phase v S_i 2^(32 - 2(j+1)) + e_ijv under s; a digit v is uniform in
    {0..3} (v = 0 reads no row), so the mean error is -sum_{i,j} (e_ij1 + e_ij2 + e_ij3) / 4."""
    p = keys.params
    rows = keys.ksk[:, :, 1:, :].reshape(-1, p.n + 1)
    ph = oracle.phase(keys.s, rows).astype(np.int64).reshape(p.N, p.t, 3)
    i = np.arange(p.N)[:, None, None]
    j = np.arange(p.t)[None, :, None]
    v = np.arange(1, 4)[None, None, :]
    msg = (v * keys.S[i].astype(np.int64) << (32 - 2 * (j + 1))) % M32
    e = _centred(ph - msg) / M32
    return -float(e.sum()) / 4


def test_blind_rotation_noise_over_16k_coefficients(keys):
    """16 blind rotations x 1024 coefficients: mean ~ 0, variance within 10% of Var_BR (the
    sample variance of 16,384 near-independent errors has a relative spread of ~1%), and below
    the worst-case (Bg/2)^2 bound."""
    p = keys.params
    lwes = synth.uniform_u32(70, 1, 16 * (p.n + 1)).reshape(16, p.n + 1)
    errs, _, _ = _acc_errors(keys, lwes)
    e = errs.reshape(-1)
    var_br, bound_br, _ = _expected(p)
    var = float(np.mean(e ** 2))
    assert abs(float(e.mean())) < 4 * math.sqrt(var_br / e.size)
    assert 0.9 * var_br < var < 1.1 * var_br, (var, var_br)
    assert var < bound_br
    # Gaussian shape: the fourth moment of a normal sample is 3 var^2.
    assert 2.7 < float(np.mean(e ** 4)) / var ** 2 < 3.3


def test_key_switch_noise_over_4096_samples(keys):
    """4,096 random N-LWE samples under S with known phase: the key switch adds an error of
    variance Var_KS (within 10%)."""
    p = keys.params
    cnt = 4096
    ext = synth.uniform_u32(71, 1, cnt * (p.N + 1)).reshape(cnt, p.N + 1)
    phase_in = (ext[:, p.N].astype(np.int64) - (ext[:, :p.N].astype(np.int64) @ keys.S.astype(np.int64))) % M32
    with ThreadPoolExecutor(max_workers=oracle.threads()) as ex:
        outs = np.stack(list(ex.map(lambda x: oracle.key_switch(p, keys.ksk, x), ext)))
    phase_out = oracle.phase(keys.s, outs).astype(np.int64)
    e = _centred(phase_out - phase_in) / M32
    _, _, var_ks = _expected(p, keys.S)
    var = float(np.var(e))
    assert abs(float(e.mean()) - _ks_offset(keys)) < 4 * math.sqrt(var_ks / cnt)
    assert 0.9 * var_ks < var < 1.1 * var_ks, (var, var_ks)


def test_mux_output_noise_over_4096_extractions(keys):
    """MUX output = KS((0, 1/8) + u1 + u2): both halves' accumulators, every coefficient j
    extracted, summed, shifted by 1/8 and key-switched.  4 MUX x 1024 coefficients: the output
    error has variance 2 Var_BR + Var_KS (within 10%), i.e. about twice a two-input gate's."""
    p = keys.params
    nmux = 4
    lwes = synth.uniform_u32(72, 1, 2 * nmux * (p.n + 1)).reshape(2 * nmux, p.n + 1)
    _, accs, ideals = _acc_errors(keys, lwes)
    var_br, _, var_ks = _expected(p, keys.S)
    samples, want_phase = [], []
    for m in range(nmux):
        for j in range(p.N):
            u = (_extract(accs[2 * m], j).astype(np.int64) + _extract(accs[2 * m + 1], j).astype(np.int64)) % M32
            u[p.N] = (u[p.N] + oracle.EIGHTH) % M32
            samples.append(u.astype(np.uint32))
            want_phase.append(int(ideals[2 * m, j]) + int(ideals[2 * m + 1, j]) + oracle.EIGHTH)
    with ThreadPoolExecutor(max_workers=oracle.threads()) as ex:
        outs = np.stack(list(ex.map(lambda x: oracle.key_switch(p, keys.ksk, x), samples)))
    post = oracle.phase(keys.s, outs).astype(np.int64)
    ideal_phase = np.array(want_phase, np.int64)
    e = _centred(post - ideal_phase) / M32
    var = float(np.var(e))
    want = 2 * var_br + var_ks
    assert abs(float(e.mean()) - _ks_offset(keys)) < 4 * math.sqrt(want / e.size)
    assert 0.9 * want < var < 1.1 * want, (var, want)


def test_chained_mux_decisions(keys):
    """A chain t <- MUX(sel_i, t, c_i) of 6 MUX gates (the comparator's pattern, Algorithm 2)
    through the oracle's gates: every intermediate output decrypts to the plaintext MUX and its
    phase error stays within 6 standard deviations of the MUX output law."""
    p = keys.params
    var_br, _, var_ks = _expected(p)
    sd = math.sqrt(2 * var_br + var_ks)
    sel = synth.bits(73, 1, 6)
    cs = synth.bits(73, 2, 6)
    t_bit = 0
    t = oracle.trivial(0, p.n)[None, :]
    es = oracle.encrypt(keys.s, sel, synth.lwe_draws(74, 6))
    ec = oracle.encrypt(keys.s, cs, synth.lwe_draws(75, 6))
    for i in range(6):
        t = oracle.gate_batch(keys, oracle.MUX, es[i:i + 1], t, ec[i:i + 1])
        t_bit = t_bit if sel[i] else int(cs[i])
        assert int(oracle.decrypt(keys.s, t)[0]) == t_bit
        ph = int(oracle.phase(keys.s, t)[0])
        ideal = oracle.EIGHTH if t_bit else M32 - oracle.EIGHTH
        err = abs(int(_centred([ph - ideal])[0])) / M32
        assert err < 6 * sd
