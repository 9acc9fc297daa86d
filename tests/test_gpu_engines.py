"""The tensor-core alternative engines (Toeplitz GEMM blind rotation in bf16 and int8 limbs,
one-hot int8 GEMM key switch) through the C-ABI: every output word equals the oracle's, as
for the default engines, and switching engines back and forth changes no bit."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same, empty_dev, to_dev, to_host

pytestmark = pytest.mark.gpu

EIGHTH = 1 << 29


@pytest.fixture
def engines_ctx(gpu_ctx):
    yield gpu_ctx
    gpu_ctx.lp_set_engines(0, 0)   # leave the shared context on its defaults


def _random_lwes(seed, count, n):
    return synth.uniform_u32(seed, 902, count * (n + 1)).reshape(count, n + 1)


@pytest.mark.parametrize("br", [1, 2])
@pytest.mark.parametrize("count", [1, 6])
def test_tensor_blind_rotation_matches_oracle(engines_ctx, keys, br, count):
    p = keys.params
    lwe = _random_lwes(31 + count + 10 * br, count, p.n)
    engines_ctx.lp_set_engines(br, 0)
    ext = empty_dev(count, p.N + 1)
    engines_ctx.lp_bootstrap_extract(to_dev(lwe), EIGHTH, ext, count)
    engines_ctx.lp_sync()
    assert_same(to_host(ext), oracle.bootstrap_extract(keys, lwe), f"engine {br} bootstrap_extract")


def test_tensor_blind_rotation_zero_steps(engines_ctx, keys):
    """Inputs whose mod-switched mask is all zero: every CMux multiplies a zero difference
    (the NTT engine skips these steps; the GEMM engine computes them)."""
    p = keys.params
    lwe = np.zeros((3, p.n + 1), np.uint32)
    lwe[:, p.n] = [0, 1 << 30, 3 << 30]
    want = oracle.bootstrap_extract(keys, lwe)
    for br in (1, 2):
        engines_ctx.lp_set_engines(br, 0)
        ext = empty_dev(3, p.N + 1)
        engines_ctx.lp_bootstrap_extract(to_dev(lwe), EIGHTH, ext, 3)
        engines_ctx.lp_sync()
        assert_same(to_host(ext), want, f"engine {br} zero steps")


@pytest.mark.parametrize("count", [1, 19])
def test_onehot_key_switch_matches_oracle(engines_ctx, keys, count):
    p = keys.params
    ext = synth.uniform_u32(77 + count, 903, count * (p.N + 1)).reshape(count, p.N + 1)
    engines_ctx.lp_set_engines(0, 1)
    out = empty_dev(count, p.n + 1)
    engines_ctx.lp_key_switch(to_dev(ext), out, count)
    engines_ctx.lp_sync()
    want = np.stack([oracle.key_switch(p, keys.ksk, ext[g]) for g in range(count)])
    assert_same(to_host(out), want, "one-hot key_switch")


@pytest.mark.parametrize("op", [oracle.NAND, oracle.XOR, oracle.MUX])
def test_gates_all_engine_pairs_agree(engines_ctx, keys, op):
    """A gate batch (MUX: two rotations per gate, summed in the key switch) is bit-identical
    under every (blind rotation, key switch) engine pair and equals the oracle."""
    p = keys.params
    count = 5
    bits = synth.bits(12, 3, 3 * count).reshape(3, count)
    cts = [oracle.encrypt(keys.s, bits[k], synth.lwe_draws(12, count, offset=k * count)) for k in range(3)]
    want = oracle.gate_batch(keys, op, cts[0], cts[1], cts[2] if op == oracle.MUX else None)
    for br in (0, 1, 2):
        for ks in (0, 1):
            engines_ctx.lp_set_engines(br, ks)
            out = empty_dev(count, p.n + 1)
            engines_ctx.lp_gate_batch(op, to_dev(cts[0]), to_dev(cts[1]),
                                      to_dev(cts[2]) if op == oracle.MUX else None, out, count)
            engines_ctx.lp_sync()
            assert_same(to_host(out), want, f"op {op} engines ({br}, {ks})")


def test_unknown_engine_is_rejected(engines_ctx):
    from paper_2407_19871_gb300.locpir import LocpirError
    with pytest.raises(LocpirError):
        engines_ctx.lp_set_engines(7, 0)
    with pytest.raises(LocpirError):
        engines_ctx.lp_set_engines(0, 2)


@pytest.mark.parametrize("variant", [3, 4, 5, 6])
def test_ntt_variants_match_oracle(engines_ctx, keys, variant):
    """The batched (4 ciphertexts per CTA), split (12 warps per ciphertext), paired (two CTAs per
    ciphertext) and quad (four CTAs per ciphertext) NTT kernels, forced, on one full group plus
    a ragged one."""
    p = keys.params
    lwe = _random_lwes(61 + variant, 7, p.n)
    engines_ctx.lp_set_engines(variant, 0)
    ext = empty_dev(7, p.N + 1)
    engines_ctx.lp_bootstrap_extract(to_dev(lwe), EIGHTH, ext, 7)
    engines_ctx.lp_sync()
    assert_same(to_host(ext), oracle.bootstrap_extract(keys, lwe), f"variant {variant}")


def test_split_kernel_beyond_one_wave(engines_ctx, keys):
    """More ciphertexts than SMs, forced split: CTAs loop over several ciphertexts each.  The
    split and batched kernels agree on every word, and sampled rows equal the oracle's."""
    import torch
    p = keys.params
    count = 2 * torch.cuda.get_device_properties(0).multi_processor_count + 5
    lwe = _random_lwes(63, count, p.n)
    outs = {}
    for variant in (3, 4):
        engines_ctx.lp_set_engines(variant, 0)
        ext = empty_dev(count, p.N + 1)
        engines_ctx.lp_bootstrap_extract(to_dev(lwe), EIGHTH, ext, count)
        engines_ctx.lp_sync()
        outs[variant] = to_host(ext)
    assert_same(outs[4], outs[3], "split vs batched")
    rows = [0, count // 2, count - 1]
    assert_same(outs[4][rows], oracle.bootstrap_extract(keys, lwe[rows]), "split vs oracle (sampled rows)")


def test_autotune_sets_a_crossing_and_keeps_bits(gpu_ctx, keys):
    """lp_autotune picks a multiple of the SM count in [1, 4] per SM; a gate batch afterwards
    is still bit-identical to the oracle."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    w = gpu_ctx.lp_autotune()
    assert w % sms == 0 and sms <= w <= 4 * sms
    p = keys.params
    bits = synth.bits(13, 1, 10).reshape(2, 5)
    a = oracle.encrypt(keys.s, bits[0], synth.lwe_draws(13, 5))
    b = oracle.encrypt(keys.s, bits[1], synth.lwe_draws(13, 5, offset=5))
    out = empty_dev(5, p.n + 1)
    gpu_ctx.lp_gate_batch(oracle.AND, to_dev(a), to_dev(b), None, out, 5)
    gpu_ctx.lp_sync()
    assert_same(to_host(out), oracle.gate_batch(keys, oracle.AND, a, b, None), "after autotune")
